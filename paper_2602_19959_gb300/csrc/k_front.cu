// Steps 1-2 of the path (§2): per-track FC network and the per-event slice histogram,
// plus the first UNet convolution (1 -> 16 channels, k5) and its 2:1 max-pool, fused so
// that the histogram never leaves shared memory on its way into the UNet.
//
// One CTA per event (§3: each event maps to one thread block):
//   a. validate the event's offsets; bypass it (flag = 1, histogram of zeros) when they
//      are negative, decreasing or past the feature arrays, or the event holds more
//      than max_tracks tracks;
//   b. slice index per track, s = floor((z + 100) / 10) in float32 round-to-nearest;
//      a track is dropped when a feature is not finite or s is outside [0, 40);
//   c. stable counting sort of the valid tracks by slice (integer work only);
//   d. hidden layers 1-5 of the FC net, one thread per track, in chunks of 256 sorted
//      tracks, into a shared-memory tile of h5 vectors;
//   e. output layer + histogram, bin-parallel: the thread owning bin j of slice s computes
//      softplus(W6[j] . h5 + b6[j]) for each of the slice's tracks in sorted (= input)
//      order and adds it to bin 100 s + j sequentially, so the order depends only on the
//      event's own track list: results are bitwise reproducible and identical alone or
//      in any batch. No float atomics.
//   f. e1 = LeakyReLU(conv_k5(hist)), p1 = maxpool2(e1), stored in the form's precision.
#include "pvf_internal.cuh"

namespace pvf {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 256;               // tracks per FC chunk = threads
constexpr int kHPitch = kFcHidden + 1;    // 33: conflict-free per-track rows

struct FrontSmem {
    // byte offsets into dynamic shared memory
    static constexpr size_t fc = 0;                                   // kFcFloats floats
    static constexpr size_t enc1 = fc + sizeof(float) * kFcFloats;    // kEnc1Floats
    static constexpr size_t hist = (enc1 + sizeof(float) * kEnc1Floats + 15) / 16 * 16;
    static constexpr size_t h5 = hist + sizeof(float) * kBins;        // kChunk x 33
    static constexpr size_t cnt = h5 + sizeof(float) * kChunk * kHPitch;  // 41 ints
    static constexpr size_t seg = cnt + sizeof(int) * 48;             // 41 ints
    static constexpr size_t run = seg + sizeof(int) * 48;             // 40 ints
    static constexpr size_t sorted = run + sizeof(int) * 48;          // uint16 [max_tracks]
    __host__ __device__ static size_t slices(int max_tracks) { return sorted + 2 * (size_t)((max_tracks + 7) / 8 * 8); }
    __host__ __device__ static size_t total(int max_tracks) { return slices(max_tracks) + (size_t)max_tracks + 16; }
};

__device__ __forceinline__ float softplus_f(float x) { return x > 20.0f ? x : log1pf(expf(x)); }

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

// Slice of a float32 z (round-to-nearest add and divide); -1 when outside [0, 40).
__device__ __forceinline__ int slice_of(float z) {
    float q = __fdiv_rn(__fadd_rn(z, 100.0f), 10.0f);
    if (!(q >= 0.0f && q < 40.0f)) return -1;
    return (int)floorf(q);
}

// Stores the 16 channels of storage row `row` of event e: channel-last float32 rows for
// the FP32 form, plane-major rows (two bf16 planes / one e4m3 plane) otherwise.
template <class T>
__device__ __forceinline__ void store_row16(void *base, int64_t e, int64_t rows_e, int64_t row,
                                            const float v[kC0], float inv_scale) {
    if constexpr (sizeof(T) == 4) {
        float4 *d = reinterpret_cast<float4 *>(reinterpret_cast<float *>(base) + (e * rows_e + row) * kC0);
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (sizeof(T) == 2) {
        uint4 pk[2];
        __nv_bfloat162 *b = reinterpret_cast<__nv_bfloat162 *>(pk);
#pragma unroll
        for (int i = 0; i < 8; ++i) b[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        unsigned char *cb = reinterpret_cast<unsigned char *>(base);
        *reinterpret_cast<uint4 *>(cb + planar_off(e, 0, 2, rows_e, row)) = pk[0];
        *reinterpret_cast<uint4 *>(cb + planar_off(e, 1, 2, rows_e, row)) = pk[1];
    } else {
        uint4 pk;
        __nv_fp8_e4m3 *b = reinterpret_cast<__nv_fp8_e4m3 *>(&pk);
#pragma unroll
        for (int i = 0; i < 16; ++i) b[i] = __nv_fp8_e4m3(v[i] * inv_scale);
        unsigned char *cb = reinterpret_cast<unsigned char *>(base);
        *reinterpret_cast<uint4 *>(cb + planar_off(e, 0, 1, rows_e, row)) = pk;
    }
}

template <class T>
__device__ __forceinline__ void zero_row16(void *base, int64_t e, int64_t rows_e, int64_t row) {
    float z[kC0];
#pragma unroll
    for (int i = 0; i < kC0; ++i) z[i] = 0.0f;
    store_row16<T>(base, e, rows_e, row, z, 1.0f);
}

// ENC1 = false: steps a-e only (the histogram), nothing written to e1/p1.
template <int PREC, bool ENC1 = true>
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
    uint8_t *sslice = smem + FrontSmem::slices(a.max_tracks);

    const int tid = threadIdx.x;
    const int e = blockIdx.x;
    const int ge = a.ev_base + e;

    if constexpr (ENC1)
        for (int i = tid; i < kEnc1Floats; i += kThreads) senc[i] = a.enc1[i];

    if (a.hist_in) {
        const float *src = a.hist_in + (size_t)ge * kBins;
        for (int i = tid; i < kBins; i += kThreads) shist[i] = src[i];
    } else {
        // ---- a. validate
        const int64_t t0 = a.offsets[ge], t1 = a.offsets[ge + 1];
        const bool bypass = t0 < 0 || t1 < t0 || t1 > a.n_tracks || (t1 - t0) > a.max_tracks;
        const int n = bypass ? 0 : (int)(t1 - t0);
        if (tid == 0) {
            a.ev_flag[ge] = bypass ? 1 : 0;
            if (bypass) raise_status(a.status, PVF_WARN_EVENTS_SKIPPED);
        }
        for (int i = tid; i < kFcFloats; i += kThreads) sfc[i] = a.fc[i];
        for (int i = tid; i < kBins; i += kThreads) shist[i] = 0.0f;
        if (tid < 48) { scnt[tid] = 0; srun[tid] = 0; }
        __syncthreads();

        // ---- b. slice per track (integer counts through shared atomics: exact)
        for (int t = tid; t < n; t += kThreads) {
            const int64_t gt = t0 + t;
            bool finite = true;
#pragma unroll
            for (int k = 0; k < kFeatures; ++k) finite &= isfinite(a.feat[k][gt]);
            const int s = finite ? slice_of(a.feat[2][gt]) : -1;
            sslice[t] = s < 0 ? 255 : (uint8_t)s;
            if (s >= 0) atomicAdd(&scnt[s], 1);
        }
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int s = 0; s < kSlices; ++s) { sseg[s] = acc; acc += scnt[s]; }
            sseg[kSlices] = acc;
        }
        __syncthreads();

        // ---- c. stable ranks by slice: warp 0 walks the tracks in input order
        if (tid < 32) {
            const unsigned lane = tid;
            for (int base = 0; base < n; base += 32) {
                const int t = base + lane;
                const int s = t < n ? sslice[t] : 255;
                const unsigned peers = __match_any_sync(0xffffffffu, s);
                const unsigned lower = peers & ((1u << lane) - 1u);
                int before = 0;
                if (s != 255) before = srun[s];
                __syncwarp();
                if (s != 255) {
                    ssorted[sseg[s] + before + __popc(lower)] = (uint16_t)t;
                    if (lower == 0) srun[s] = before + __popc(peers);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        const int nvalid = sseg[kSlices];

        // ---- d/e. hidden layers per track, then output layer + per-bin sequential sums
        const float *w6t = sfc + fc_w_off(5);
        const float *b6 = sfc + fc_b_off(5);
        const int grp = tid / kFcOut, j = tid % kFcOut;   // two groups of 100 bin threads
        for (int c0 = 0; c0 < nvalid; c0 += kChunk) {
            const int r = c0 + tid;
            if (r < nvalid) {
                const int t = ssorted[r];
                const int64_t gt = t0 + t;
                const int s = sslice[t];
                float x[kFcInPad];
#pragma unroll
                for (int k = 0; k < kFeatures; ++k) x[k] = a.feat[k][gt];
                x[2] = __fsub_rn(x[2], -100.0f + 10.0f * (float)s);   // slice-relative z (exact offset)
#pragma unroll
                for (int k = kFeatures; k < kFcInPad; ++k) x[k] = 0.0f;
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

    if constexpr (!ENC1) return;
    // ---- f. e1 = LeakyReLU(conv_k5(hist) + b), p1 = maxpool2(e1)
    const int64_t rows1 = padded_rows(kBins), rows2 = padded_rows(kBins / 2);
    const float inv = a.e1_inv_scale;
    float vmax = 0.0f;
    for (int q = tid; q < kBins / 2; q += kThreads) {
        float hv[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int p = 2 * q + k - 2;
            hv[k] = (p >= 0 && p < kBins) ? shist[p] : 0.0f;
        }
        float v0[kC0], v1[kC0], vp[kC0];
#pragma unroll
        for (int co = 0; co < kC0; ++co) {
            float a0 = senc[5 * kC0 + co], a1 = a0;
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                a0 = fmaf(senc[t * kC0 + co], hv[t], a0);
                a1 = fmaf(senc[t * kC0 + co], hv[t + 1], a1);
            }
            v0[co] = leaky(a0);
            v1[co] = leaky(a1);
            vp[co] = fmaxf(v0[co], v1[co]);
            vmax = fmaxf(vmax, fmaxf(fabsf(v0[co]), fabsf(v1[co])));
        }
        store_row16<T>(a.e1, e, rows1, 2 * q + kPad, v0, inv);
        store_row16<T>(a.e1, e, rows1, 2 * q + 1 + kPad, v1, inv);
        store_row16<T>(a.p1, e, rows2, q + kPad, vp, inv);
    }
    if (a.amax) {   // calibration: integer max on the float bits (order-independent)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if ((tid & 31) == 0) atomicMax(reinterpret_cast<int *>(a.amax), __float_as_int(vmax));
    }
    if (tid < 4) {
        const int r = tid < 2 ? tid : kBins + tid;             // rows 0,1 and L+2, L+3
        zero_row16<T>(a.e1, e, rows1, r);
        const int rp = tid < 2 ? tid : kBins / 2 + tid;
        zero_row16<T>(a.p1, e, rows2, rp);
    }
}

}  // namespace

size_t front_smem_bytes(int max_tracks) { return FrontSmem::total(max_tracks); }

cudaError_t launch_front_hist_only(const FrontArgs &a, size_t smem, cudaStream_t s) {
    if (a.n_events <= 0) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(k_front<PVF_FP32, false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_front<PVF_FP32, false><<<a.n_events, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_front(const FrontArgs &a, int precision, size_t smem, cudaStream_t s) {
    if (a.n_events <= 0) return cudaSuccess;
    dim3 grid(a.n_events), block(kThreads);
    cudaError_t err = cudaSuccess;
    switch (precision) {
    case PVF_FP32:
        err = cudaFuncSetAttribute(k_front<PVF_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) k_front<PVF_FP32><<<grid, block, smem, s>>>(a);
        break;
    case PVF_BF16:
        err = cudaFuncSetAttribute(k_front<PVF_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) k_front<PVF_BF16><<<grid, block, smem, s>>>(a);
        break;
    default:
        err = cudaFuncSetAttribute(k_front<PVF_FP8_E4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) k_front<PVF_FP8_E4M3><<<grid, block, smem, s>>>(a);
        break;
    }
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace pvf
