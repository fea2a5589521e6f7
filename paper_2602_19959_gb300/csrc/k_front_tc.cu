// Steps 1-2 of the path (§2) for the tensor-core forms: the per-track FC network on
// tcgen05 (bf16 operands, fp32 accumulation in TMEM), the deterministic histogram, and
// enc1 + pool. A persistent grid (two CTAs per SM) walks the events, one event at a time
// per CTA (§3: each event is processed by one thread block), so weights and TMEM are set
// up once per CTA rather than once per event.
//
// Per tile of 128 slice-sorted tracks (one track per TMEM lane / thread; two tiles per
// pass, one per warpgroup, sharing each layer's MMA round trip):
//   X [128 x 16] (nine features, feature 2 slice-relative, zero padded) ->
//   5 x { MMA (N = 32) -> TMEM -> bias + LeakyReLU -> bf16 -> H [128 x 32] } ->
//   MMA (N = 112, 100 used) -> TMEM -> bias + softplus (fp32) -> staging tile (25
//   columns at a time) ->
//   per-bin sums in a fixed two-level order: within each 32-row chunk of the sorted
//   tracks a slice segment's outputs are added in order, then the chunk partials are
//   added in row order to hist[100 s + j].
// The layers are dependent, so the tile runs MMA and epilogue in lockstep; one thread
// issues the MMAs, every wait on their completion is bounded. The histogram order
// depends only on the event's own track list (chunks are counted from the event's first
// sorted track), so results are identical alone and in any batch.
#include "front_common.cuh"
#include "tc_ptx.cuh"

namespace pvf {
namespace {

using namespace front;
using namespace tc;

constexpr int kT = 256;                 // threads: two warpgroups, one 128-row tile each
constexpr int kRows = 128;              // tile rows = TMEM lanes
constexpr int kN6 = kFcN6;              // 100 outputs padded to a multiple of 16
constexpr int kQ = 25;                  // output columns per staging pass (4 passes)
constexpr int kTmemCols = 256;          // tile g uses columns [128 g, 128 g + 112)

struct TcSmem {
    static constexpr size_t img = 0;                                   // kFcImgBytes
    static constexpr size_t bias = img + kFcImgBytes;                  // kFcBTotal floats
    static constexpr size_t enc1 = bias + sizeof(float) * kFcBTotal;   // kEnc1Floats
    static constexpr size_t x = (enc1 + sizeof(float) * kEnc1Floats + 127) / 128 * 128;  // 2 tiles x 2 planes
    static constexpr size_t h = x + 2 * 2 * kRows * 16;                // 2 tiles x 4 planes
    static constexpr size_t hist = h + 2 * 4 * kRows * 16;
    static constexpr size_t stage = hist + sizeof(float) * kBins;      // 2 tiles x 128 x 25 floats
    static constexpr size_t cnt = stage + sizeof(float) * 2 * kRows * kQ;
    static constexpr size_t seg = cnt + sizeof(int) * 48;
    static constexpr size_t run = seg + sizeof(int) * 48;
    static constexpr size_t bar = (run + sizeof(int) * 48 + 15) / 16 * 16;   // mbarrier + slot + flag
    static constexpr size_t sorted = bar + 32;
    __host__ __device__ static size_t slices(int mt) { return sorted + 2 * (size_t)((mt + 7) / 8 * 8); }
    __host__ __device__ static size_t total(int mt) { return slices(mt) + (size_t)mt + 16; }
};

__device__ __forceinline__ uint4 pack8_bf16(const float *v) {
    uint4 r;
    __nv_bfloat162 *b = reinterpret_cast<__nv_bfloat162 *>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    return r;
}

// Per pass of up to two 128-track tiles (warpgroup g owns tile g, one row per thread):
// six dependent layers, each one MMA round trip for both tiles, then the output layer
// in four 25-column passes through a staging tile and the ordered per-bin sums.
template <int PREC>
__global__ void __launch_bounds__(kT, 2) k_front_tc(FrontArgs a) {
    using T = typename Elem<PREC>::T;
    extern __shared__ __align__(128) unsigned char smem[];
    float *sbias = reinterpret_cast<float *>(smem + TcSmem::bias);
    float *senc = reinterpret_cast<float *>(smem + TcSmem::enc1);
    float *shist = reinterpret_cast<float *>(smem + TcSmem::hist);
    float *sstage = reinterpret_cast<float *>(smem + TcSmem::stage);
    int *scnt = reinterpret_cast<int *>(smem + TcSmem::cnt);
    int *sseg = reinterpret_cast<int *>(smem + TcSmem::seg);
    int *srun = reinterpret_cast<int *>(smem + TcSmem::run);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + TcSmem::bar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + TcSmem::bar + 8);
    volatile int *never = reinterpret_cast<volatile int *>(smem + TcSmem::bar + 12);
    uint16_t *ssorted = reinterpret_cast<uint16_t *>(smem + TcSmem::sorted);
    uint8_t *sslice = smem + TcSmem::slices(a.max_tracks);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = warp >> 2;                       // tile of this warpgroup
    const int m = tid & (kRows - 1);               // row within the tile = TMEM lane
    const uint32_t lane_field = (uint32_t)((warp & 3) * 32) << 16;

    // once per CTA: enc1 weights, FC operand images and biases, barrier, TMEM
    for (int i = tid; i < kEnc1Floats; i += kT) senc[i] = a.enc1[i];
    if (!a.hist_in) {
        for (int i = tid; i < kFcImgBytes / 16; i += kT)
            reinterpret_cast<uint4 *>(smem + TcSmem::img)[i] = reinterpret_cast<const uint4 *>(a.fc_img)[i];
        for (int i = tid; i < kFcBTotal; i += kT) sbias[i] = a.fc[kFcWTotal + i];
        fence_proxy_async_smem();          // weight image -> visible to the tensor core
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        *never = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t img = smem_u32(smem + TcSmem::img);
    const uint32_t sx = smem_u32(smem + TcSmem::x), sh = smem_u32(smem + TcSmem::h);
    unsigned char *xbuf = smem + TcSmem::x + (size_t)g * 2 * kRows * 16;
    unsigned char *hbuf = smem + TcSmem::h + (size_t)g * 4 * kRows * 16;
    const uint32_t dcol = tmem + lane_field + (uint32_t)(g * 128);
    bool failed = false;
    uint32_t phase = 0;

    // persistent: the CTA walks the launch's events
    for (int e = blockIdx.x; e < a.n_events; e += gridDim.x) {
        const int ge = a.ev_base + e;
        if (a.hist_in) {
            const float *src = a.hist_in + (size_t)ge * kBins;
            for (int i = tid; i < kBins; i += kT) shist[i] = src[i];
            __syncthreads();
        } else {
            for (int i = tid; i < kBins; i += kT) shist[i] = 0.0f;
            int64_t t0;
            int nvalid;
            validate_sort<kT>(a, ge, tid, scnt, sseg, srun, ssorted, sslice, t0, nvalid);
            if (failed) nvalid = 0;        // a timed-out MMA ends the tensor-core work
            for (int c0 = 0; c0 < nvalid && !failed; c0 += 2 * kRows) {
                const int ntile = nvalid - c0 > kRows ? 2 : 1;
                const bool active = g < ntile;         // warpgroup has a tile in this pass
                const int r = c0 + g * kRows + m;
                const bool live = r < nvalid;
                if (active) {   // X row: the track's features in bf16, zero rows past the event
                    float x[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) x[k] = 0.0f;
                    if (live) {
                        const int t = ssorted[r];
                        track_features(a, t0 + t, sslice[t], x);
                    }
                    *reinterpret_cast<uint4 *>(xbuf + (0 * kRows + m) * 16) = pack8_bf16(x);
                    *reinterpret_cast<uint4 *>(xbuf + (1 * kRows + m) * 16) = pack8_bf16(x + 8);
                }
                fence_proxy_async_smem();
                tc_fence_before();
                __syncthreads();
                for (int l = 0; l < 6 && !failed; ++l) {
                    tc_fence_after();
                    if (tid == 0) {
                        for (int tg = 0; tg < ntile; ++tg) {
                            const uint32_t d = tmem + (uint32_t)(tg * 128);
                            if (l == 0) {
                                mma_bf16(d, smem_desc(sx + tg * 2 * kRows * 16, kRows * 16, 128),
                                         smem_desc(img, kFcHidden * 16, 128), idesc_f32acc(kRows, kFcHidden, 1), 0);
                            } else {
                                const int n = l < 5 ? kFcHidden : kN6;
                                const uint32_t w = img + fc_img_off(l);
                                const uint32_t ha = sh + tg * 4 * kRows * 16;
#pragma unroll
                                for (int kb = 0; kb < 2; ++kb)
                                    mma_bf16(d, smem_desc(ha + 2 * kb * kRows * 16, kRows * 16, 128),
                                             smem_desc(w + 2 * kb * n * 16, n * 16, 128),
                                             idesc_f32acc(kRows, n, 1), kb);
                            }
                        }
                        mma_commit(bar);
                    }
                    const bool ok = mbar_wait(bar, phase, never);
                    phase ^= 1;
                    if (__syncthreads_or(!ok)) { failed = true; break; }
                    tc_fence_after();
                    if (l < 5) {
                        if (active) {
                            float v[32];
                            tmem_ld16(dcol, *reinterpret_cast<float(*)[16]>(v));
                            tmem_ld16(dcol + 16, *reinterpret_cast<float(*)[16]>(v + 16));
                            const float *b = sbias + l * kFcHidden;
#pragma unroll
                            for (int o = 0; o < kFcHidden; ++o) v[o] = leaky(v[o] + b[o]);
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                *reinterpret_cast<uint4 *>(hbuf + (k * kRows + m) * 16) = pack8_bf16(v + 8 * k);
                        }
                        fence_proxy_async_smem();
                        tc_fence_before();
                        __syncthreads();
                        continue;
                    }
                    // output layer: four passes of 25 columns through the staging tile
                    const float *b6 = sbias + 5 * kFcHidden;
                    const int c1 = min(c0 + 2 * kRows, nvalid);
#pragma unroll 1
                    for (int q = 0; q < kFcOut / kQ; ++q) {
                        if (active) {
                            float v[32];
                            tmem_ld16(dcol + q * kQ, *reinterpret_cast<float(*)[16]>(v));
                            tmem_ld16(dcol + q * kQ + 16, *reinterpret_cast<float(*)[16]>(v + 16));
                            if (live) {
                                float *row = sstage + ((size_t)g * kRows + m) * kQ;
#pragma unroll
                                for (int j = 0; j < kQ; ++j) row[j] = softplus_f(v[j] + b6[q * kQ + j]);
                            }
                        }
                        tc_fence_before();
                        __syncthreads();
                        // per-bin sums in a fixed two-level order: thread (column j, chunk k)
                        // adds the rows of each slice segment inside its 32-row chunk in
                        // order and leaves the chunk's partial in the segment's last row of
                        // the chunk; then each (slice, column) adds its chunks' partials in
                        // row order to the histogram
                        const int nrow = c1 - c0;
                        if (tid < 8 * kQ) {
                            const int j = tid % kQ, k = tid / kQ;
                            const int r0 = 32 * k, r1 = min(r0 + 32, nrow);
                            // from the slice of the chunk's first row to the last one it holds
                            for (int s = r0 < r1 ? sslice[ssorted[c0 + r0]] : kSlices;
                                 s < kSlices && sseg[s] - c0 < r1; ++s) {
                                const int lo = max(sseg[s] - c0, r0), hi = min(sseg[s + 1] - c0, r1);
                                if (lo >= hi) continue;
                                float acc = sstage[(size_t)lo * kQ + j];
                                for (int rr = lo + 1; rr < hi; ++rr) acc = __fadd_rn(acc, sstage[(size_t)rr * kQ + j]);
                                sstage[(size_t)(hi - 1) * kQ + j] = acc;
                            }
                        }
                        __syncthreads();
                        for (int it = tid; it < kSlices * kQ; it += kT) {
                            const int s = it / kQ, j = it % kQ;
                            const int lo = max(sseg[s] - c0, 0), hi = min(sseg[s + 1] - c0, nrow);
                            if (lo >= hi) continue;
                            float acc = shist[s * kSliceBins + q * kQ + j];
                            for (int k = lo / 32; k <= (hi - 1) / 32; ++k)
                                acc = __fadd_rn(acc, sstage[(size_t)(min(hi, 32 * (k + 1)) - 1) * kQ + j]);
                            shist[s * kSliceBins + q * kQ + j] = acc;
                        }
                        __syncthreads();
                    }
                }
            }
            if (failed) {
                for (int i = tid; i < kBins; i += kT) shist[i] = 0.0f;
                if (tid == 0) raise_status(a.status, PVF_ERR_TIMEOUT);
            }
            __syncthreads();
        }
        if (a.hist_out) {
            float4 *dst = reinterpret_cast<float4 *>(a.hist_out + (size_t)ge * kBins);
            const float4 *src = reinterpret_cast<const float4 *>(shist);
            for (int i = tid; i < kBins / 4; i += kT) dst[i] = src[i];
        }
        enc1_pool<T, kT>(a, e, tid, shist, senc);
        __syncthreads();                   // shist and the sort arrays are reused next event
    }
    if (failed && tid == 0) {
        // the last MMAs still complete before TMEM is released
        mma_commit(bar);
        const uint64_t tw = globaltimer();
        while (!mbar_try_wait(bar, phase)) if (globaltimer() - tw > kWaitLimitNs) break;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

template <int PREC>
cudaError_t launch_front_tc_t(const FrontArgs &a, cudaStream_t s) {
    // persistent grid: as many CTAs as fit on the GPU at once (shared memory allows two
    // per SM, which also fill the 512 TMEM columns), each walking events
    static size_t configured = 0;
    static int grid_cap = 0;
    const size_t smem = TcSmem::total(a.max_tracks);
    if (smem > configured) {
        cudaError_t err = cudaFuncSetAttribute(k_front_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        configured = smem;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid_cap = (sms > 0 ? sms : 1) * 2;
    }
    const int per_sm = (int)((228 * 1024) / (smem + 1024));
    int grid = grid_cap / 2 * (per_sm < 2 ? (per_sm < 1 ? 1 : per_sm) : 2);
    if (grid > a.n_events) grid = a.n_events;
    k_front_tc<PREC><<<grid, kT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_front_tc(const FrontArgs &a, int precision, cudaStream_t s) {
    if (a.n_events <= 0) return cudaSuccess;
    return precision == PVF_BF16 ? launch_front_tc_t<PVF_BF16>(a, s) : launch_front_tc_t<PVF_FP8_E4M3>(a, s);
}

}  // namespace pvf
