// Steps 1-2 of the path (§2): per-track FC network and the per-event slice histogram,
// plus the first UNet convolution (1 -> 16 channels, k5) and its 2:1 max-pool, fused so
// that the histogram never leaves shared memory on its way into the UNet.
//
// A persistent grid walks the events, one event at a time per CTA (§3: each event is
// processed by one thread block); per event:
//   a. validate the event's offsets; bypass it (flag = 1, histogram of zeros) when they
//      are negative, decreasing or past the feature arrays, or the event holds more
//      than max_tracks tracks;
//   b. slice index per track, s = floor((z + 100) / 10) in float32 round-to-nearest;
//      a track is dropped when a feature is not finite or s is outside [0, 40);
//   c. stable counting sort of the valid tracks by slice (integer work only), with the
//      boundary tracks' second slices (§3) when the boundary width is non-zero;
//   d. hidden layers 1-5 of the FC net, one thread per track, in chunks of 256 sorted
//      tracks, into a shared-memory tile of h5 vectors;
//   e. output layer + histogram, bin-parallel: the thread owning bin j of slice s computes
//      softplus(W6[j] . h5 + b6[j]) for each of the slice's tracks in sorted (= input)
//      order and adds it to bin 100 s + j sequentially, so the order depends only on the
//      event's own track list: results are bitwise reproducible and identical alone or
//      in any batch. No float atomics.
//   f. e1 = LeakyReLU(conv_k5(hist)), p1 = maxpool2(e1), stored in the form's precision.
#include "front_common.cuh"

namespace pvf {
namespace {

using namespace front;

constexpr int kThreads = 256;
constexpr int kChunk = 256;               // tracks per FC chunk = threads
constexpr int kHPitch = kFcHidden + 1;    // 33: conflict-free per-track rows

struct FrontSmem {
    // byte offsets into dynamic shared memory
    static constexpr size_t fc = 0;                                   // kFcFloats floats
    static constexpr size_t enc1 = fc + sizeof(float) * kFcFloats;    // 6 c0 floats
    static constexpr size_t hist = (enc1 + sizeof(float) * kEnc1FloatsMax + 15) / 16 * 16;
    static constexpr size_t h5 = hist + sizeof(float) * kBins;        // kChunk x 33
    static constexpr size_t cnt = h5 + sizeof(float) * kChunk * kHPitch;  // 41 ints
    static constexpr size_t seg = cnt + sizeof(int) * 48;             // 41 ints
    static constexpr size_t run = seg + sizeof(int) * 48;             // 40 ints
    static constexpr size_t sorted = run + sizeof(int) * 48;          // uint16 [entries]
    __host__ __device__ static size_t slices(int entries) { return sorted + 2 * (size_t)((entries + 7) / 8 * 8); }
    __host__ __device__ static size_t total(int max_tracks, float edge) {
        return slices(front_entries(max_tracks, edge)) + (size_t)max_tracks + 16;
    }
};

// Hidden layers 1-5 of the FC net for one track; writes h5 (32 floats) to h_row.
__device__ __forceinline__ void fc_hidden(const float *__restrict__ W, const float x[kFcInPad],
                                          float *h_row) {
    float h[kFcHidden], g[kFcHidden];
    {
        const float *w1 = W + fc_w_off(0);
        const float *b1 = W + fc_b_off(0);
#pragma unroll
        for (int o = 0; o < kFcHidden; ++o) {
            const float4 *wr = reinterpret_cast<const float4 *>(w1 + o * kFcInPad);
            float acc = b1[o];
#pragma unroll
            for (int i4 = 0; i4 < kFcInPad / 4; ++i4) {
                float4 w = wr[i4];
                acc = fmaf(w.x, x[4 * i4 + 0], acc);
                acc = fmaf(w.y, x[4 * i4 + 1], acc);
                acc = fmaf(w.z, x[4 * i4 + 2], acc);
                acc = fmaf(w.w, x[4 * i4 + 3], acc);
            }
            h[o] = leaky(acc);
        }
    }
#pragma unroll
    for (int l = 1; l < 5; ++l) {
        const float *wl = W + fc_w_off(l);
        const float *bl = W + fc_b_off(l);
#pragma unroll
        for (int o = 0; o < kFcHidden; ++o) {
            const float4 *wr = reinterpret_cast<const float4 *>(wl + o * kFcHidden);
            float acc = bl[o];
#pragma unroll
            for (int i4 = 0; i4 < kFcHidden / 4; ++i4) {
                float4 w = wr[i4];
                acc = fmaf(w.x, h[4 * i4 + 0], acc);
                acc = fmaf(w.y, h[4 * i4 + 1], acc);
                acc = fmaf(w.z, h[4 * i4 + 2], acc);
                acc = fmaf(w.w, h[4 * i4 + 3], acc);
            }
            g[o] = leaky(acc);
        }
#pragma unroll
        for (int o = 0; o < kFcHidden; ++o) h[o] = g[o];
    }
#pragma unroll
    for (int o = 0; o < kFcHidden; ++o) h_row[o] = h[o];
}

// ENC1 = false: steps a-e only (the histogram), nothing written to e1/p1.
// EDGE: boundary tracks fill a second slice (a.edge > 0).
// C0: UNet base width of the e1 / p1 tensors written here (16, or 32 in this float32 form).
// IV: e1 / p1 in the per-interval layout (kSlices windowed sequences per event).
template <int PREC, bool ENC1, bool EDGE, int C0, bool IV = false>
__global__ void __launch_bounds__(kThreads) k_front(FrontArgs a) {
    using T = typename Elem<PREC>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    float *sfc = reinterpret_cast<float *>(smem + FrontSmem::fc);
    float *senc = reinterpret_cast<float *>(smem + FrontSmem::enc1);
    float *shist = reinterpret_cast<float *>(smem + FrontSmem::hist);
    float *sh5 = reinterpret_cast<float *>(smem + FrontSmem::h5);
    int *scnt = reinterpret_cast<int *>(smem + FrontSmem::cnt);
    int *sseg = reinterpret_cast<int *>(smem + FrontSmem::seg);
    int *srun = reinterpret_cast<int *>(smem + FrontSmem::run);
    uint16_t *ssorted = reinterpret_cast<uint16_t *>(smem + FrontSmem::sorted);
    uint8_t *sslice = smem + FrontSmem::slices(EDGE ? 2 * a.max_tracks : a.max_tracks);

    const int tid = threadIdx.x;
    if constexpr (ENC1)
        for (int i = tid; i < 6 * C0; i += kThreads) senc[i] = a.enc1[i];
    if (!a.hist_in)
        for (int i = tid; i < kFcFloats; i += kThreads) sfc[i] = a.fc[i];
    __syncthreads();

    // persistent: the CTA walks the launch's events (weights loaded once above)
    for (int e = blockIdx.x; e < a.n_events; e += gridDim.x) {
        const int ge = a.ev_base + e;
        if (a.hist_in) {
            const float *src = a.hist_in + (size_t)ge * kBins;
            for (int i = tid; i < kBins; i += kThreads) shist[i] = src[i];
        } else {
            // ---- a-c. validate, slice per track, stable sort by slice
            for (int i = tid; i < kBins; i += kThreads) shist[i] = 0.0f;
            int64_t t0;
            int nvalid;
            validate_sort<kThreads, EDGE>(a, ge, tid, scnt, sseg, srun, ssorted, sslice, t0, nvalid);

            // ---- d/e. hidden layers per track, then output layer + per-bin sequential sums
            const float *w6t = sfc + fc_w_off(5);
            const float *b6 = sfc + fc_b_off(5);
            const int grp = tid / kFcOut, j = tid % kFcOut;   // two groups of 100 bin threads
            for (int c0 = 0; c0 < nvalid; c0 += kChunk) {
                const int r = c0 + tid;
                if (r < nvalid) {
                    const int en = ssorted[r];
                    float x[kFcInPad];
                    track_features(a, t0 + entry_track<EDGE>(en), entry_slice<EDGE>(en, sslice), x);
                    fc_hidden(sfc, x, sh5 + tid * kHPitch);
                }
                __syncthreads();
                if (grp < 2) {
                    float w[kFcHidden];
#pragma unroll
                    for (int i = 0; i < kFcHidden; ++i) w[i] = w6t[i * kFcOut + j];
                    const float bj = b6[j];
                    const int c1 = min(c0 + kChunk, nvalid);
                    for (int s = grp; s < kSlices; s += 2) {
                        const int lo = max(sseg[s], c0), hi = min(sseg[s + 1], c1);
                        if (lo >= hi) continue;
                        float acc = shist[s * kSliceBins + j];
                        for (int rr = lo; rr < hi; ++rr) {
                            const float *hr = sh5 + (rr - c0) * kHPitch;
                            float o = bj;
#pragma unroll
                            for (int i = 0; i < kFcHidden; ++i) o = fmaf(w[i], hr[i], o);
                            acc = __fadd_rn(acc, softplus_f(o));
                        }
                        shist[s * kSliceBins + j] = acc;
                    }
                }
                __syncthreads();
            }
        }
        __syncthreads();

        if (a.hist_out) {
            float4 *dst = reinterpret_cast<float4 *>(a.hist_out + (size_t)ge * kBins);
            const float4 *src = reinterpret_cast<const float4 *>(shist);
            for (int i = tid; i < kBins / 4; i += kThreads) dst[i] = src[i];
        }

        if constexpr (ENC1 && IV) enc1_pool_windows_f32<kThreads, C0>(a, e, tid, shist, senc);
        else if constexpr (ENC1) enc1_pool<T, kThreads, false, C0>(a, e, tid, shist, senc);
        __syncthreads();                   // shist and the sort arrays are reused next event
    }
}

// Persistent grid: as many CTAs as the shared memory lets reside (at most two per SM,
// the register limit at 256 threads), capped by the number of events.
template <int PREC, bool ENC1, bool EDGE, int C0, bool IV = false>
cudaError_t launch_front_t(const FrontArgs &a, size_t smem, cudaStream_t s) {
    int sms = 0;
    cudaError_t err = current_device_sms(&sms);
    if (err == cudaSuccess) err = prepare_kernel((const void *)k_front<PREC, ENC1, EDGE, C0, IV>, smem, nullptr);
    if (err != cudaSuccess) return err;
    int per_sm = (int)((228 * 1024) / (smem + 1024));
    if (per_sm > 2) per_sm = 2;
    if (a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm) per_sm = a.ctas_per_sm;
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    if (grid > a.n_events) grid = a.n_events;
    k_front<PREC, ENC1, EDGE, C0, IV><<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t front_smem_bytes(int max_tracks, float edge) { return FrontSmem::total(max_tracks, edge); }

cudaError_t launch_front_hist_only(const FrontArgs &a, size_t smem, cudaStream_t s) {
    if (a.n_events <= 0) return cudaSuccess;
    if (a.edge > 0.0f) return cudaErrorInvalidValue;   // the no-allocation path has no boundary tracks
    return launch_front_t<PVF_FP32, false, false, kC0>(a, smem, s);
}

cudaError_t launch_front(const FrontArgs &a, int precision, size_t smem, cudaStream_t s) {
    if (a.n_events <= 0) return cudaSuccess;
    // the tensor-core forms run k_front_tc
    if (precision != PVF_FP32) return cudaErrorInvalidValue;
    if (a.iv) {   // per-interval layout: width 16
        if (a.c0 != kC0) return cudaErrorInvalidValue;
        return a.edge > 0.0f ? launch_front_t<PVF_FP32, true, true, kC0, true>(a, smem, s)
                             : launch_front_t<PVF_FP32, true, false, kC0, true>(a, smem, s);
    }
    if (a.c0 == kC0Max)
        return a.edge > 0.0f ? launch_front_t<PVF_FP32, true, true, kC0Max>(a, smem, s)
                             : launch_front_t<PVF_FP32, true, false, kC0Max>(a, smem, s);
    if (a.c0 != kC0) return cudaErrorInvalidValue;
    return a.edge > 0.0f ? launch_front_t<PVF_FP32, true, true, kC0>(a, smem, s)
                         : launch_front_t<PVF_FP32, true, false, kC0>(a, smem, s);
}

}  // namespace pvf
