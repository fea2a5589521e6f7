// Steps 1-2 of the path (§2) for the tensor-core forms: the per-track FC network on
// tcgen05 (bf16 operands, fp32 accumulation in TMEM), the deterministic histogram, and
// enc1 + pool, one CTA per event (§3: each event maps to one thread block).
//
// Per tile of 128 slice-sorted tracks (one track per TMEM lane / thread):
//   X [128 x 16] (nine features, feature 2 slice-relative, zero padded) ->
//   5 x { MMA (N = 32) -> TMEM -> bias + LeakyReLU -> bf16 -> H [128 x 32] } ->
//   MMA (N = 112, 100 used) -> TMEM -> bias + softplus (fp32) -> staging tile ->
//   per-bin sums: the thread owning bin j adds, for each slice segment of the tile, the
//   segment's outputs in sorted (= input) order to hist[100 s + j].
// The layers are dependent, so the tile runs MMA and epilogue in lockstep; one thread
// issues the MMAs, every wait on their completion is bounded. The histogram order
// depends only on the event's own track list, as in the float32 form.
#include "front_common.cuh"
#include "tc_ptx.cuh"

namespace pvf {
namespace {

using namespace front;
using namespace tc;

constexpr int kT = 128;                 // threads = tile rows = TMEM lanes
constexpr int kN6 = 112;                // 100 outputs padded to a multiple of 16
constexpr int kStagePitch = kFcOut + 1; // 101: conflict-free rows and columns
constexpr int kTmemCols = 128;

struct TcSmem {
    static constexpr size_t img = 0;                                   // kFcImgBytes
    static constexpr size_t bias = img + kFcImgBytes;                  // kFcBTotal floats
    static constexpr size_t enc1 = bias + sizeof(float) * kFcBTotal;   // kEnc1Floats
    static constexpr size_t x = (enc1 + sizeof(float) * kEnc1Floats + 127) / 128 * 128;  // 2 planes
    static constexpr size_t h = x + 2 * kT * 16;                       // 4 planes
    static constexpr size_t hist = h + 4 * kT * 16;
    static constexpr size_t stage = hist + sizeof(float) * kBins;      // kT x 101 floats
    static constexpr size_t cnt = stage + sizeof(float) * kT * kStagePitch;
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

template <int PREC>
__global__ void __launch_bounds__(kT) k_front_tc(FrontArgs a) {
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
    const int e = blockIdx.x, ge = a.ev_base + e;
    const uint32_t lane_field = (uint32_t)(warp * 32) << 16;

    for (int i = tid; i < kEnc1Floats; i += kT) senc[i] = a.enc1[i];
    if (tid == 0) {
        mbar_init(bar, 1);
        *never = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    bool failed = false;
    uint32_t phase = 0;

    if (a.hist_in) {
        const float *src = a.hist_in + (size_t)ge * kBins;
        for (int i = tid; i < kBins; i += kT) shist[i] = src[i];
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    } else {
        for (int i = tid; i < kFcImgBytes / 16; i += kT)
            reinterpret_cast<uint4 *>(smem + TcSmem::img)[i] = reinterpret_cast<const uint4 *>(a.fc_img)[i];
        for (int i = tid; i < kFcBTotal; i += kT) sbias[i] = a.fc[kFcWTotal + i];
        for (int i = tid; i < kBins; i += kT) shist[i] = 0.0f;
        fence_proxy_async_smem();          // weight image -> visible to the tensor core
        tc_fence_before();
        int64_t t0;
        int nvalid;
        validate_sort<kT>(a, ge, tid, scnt, sseg, srun, ssorted, sslice, t0, nvalid);
        tc_fence_after();
        const uint32_t tmem = *tmem_slot;
        const uint32_t img = smem_u32(smem + TcSmem::img);
        const uint32_t sx = smem_u32(smem + TcSmem::x), sh = smem_u32(smem + TcSmem::h);
        unsigned char *hbuf = smem + TcSmem::h;

        for (int c0 = 0; c0 < nvalid && !failed; c0 += kT) {
            const int r = c0 + tid;
            const bool live = r < nvalid;
            {   // X tile row: the track's features in bf16, zero rows past the event
                float x[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) x[k] = 0.0f;
                if (live) {
                    const int t = ssorted[r];
                    track_features(a, t0 + t, sslice[t], x);
                }
                *reinterpret_cast<uint4 *>(smem + TcSmem::x + (0 * kT + tid) * 16) = pack8_bf16(x);
                *reinterpret_cast<uint4 *>(smem + TcSmem::x + (1 * kT + tid) * 16) = pack8_bf16(x + 8);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            for (int l = 0; l < 6; ++l) {
                tc_fence_after();
                if (tid == 0) {
                    if (l == 0) {
                        mma_bf16(tmem, smem_desc(sx, kT * 16, 128), smem_desc(img, kFcHidden * 16, 128),
                                 idesc_f32acc(kT, kFcHidden, 1), 0);
                    } else {
                        const int n = l < 5 ? kFcHidden : kN6;
                        const uint32_t w = img + fc_img_off(l);
#pragma unroll
                        for (int kb = 0; kb < 2; ++kb)
                            mma_bf16(tmem, smem_desc(sh + 2 * kb * kT * 16, kT * 16, 128),
                                     smem_desc(w + 2 * kb * n * 16, n * 16, 128),
                                     idesc_f32acc(kT, n, 1), kb);
                    }
                    mma_commit(bar);
                }
                const bool ok = mbar_wait(bar, phase, never);
                phase ^= 1;
                if (__syncthreads_or(!ok)) { failed = true; break; }
                tc_fence_after();
                if (l < 5) {
                    float v[32];
                    tmem_ld16(tmem + lane_field, *reinterpret_cast<float(*)[16]>(v));
                    tmem_ld16(tmem + lane_field + 16, *reinterpret_cast<float(*)[16]>(v + 16));
                    const float *b = sbias + l * kFcHidden;
#pragma unroll
                    for (int o = 0; o < kFcHidden; ++o) v[o] = leaky(v[o] + b[o]);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        *reinterpret_cast<uint4 *>(hbuf + (k * kT + tid) * 16) = pack8_bf16(v + 8 * k);
                    fence_proxy_async_smem();
                    tc_fence_before();
                    __syncthreads();
                } else {
                    const float *b6 = sbias + 5 * kFcHidden;
#pragma unroll 1
                    for (int c = 0; c < kN6; c += 16) {
                        float v[16];
                        tmem_ld16(tmem + lane_field + c, v);
                        if (live) {
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (c + j < kFcOut) sstage[tid * kStagePitch + c + j] = softplus_f(v[j] + b6[c + j]);
                        }
                    }
                    tc_fence_before();
                    __syncthreads();
                    if (tid < kFcOut) {
                        const int j = tid;
                        const int c1 = min(c0 + kT, nvalid);
                        for (int s = 0; s < kSlices; ++s) {
                            const int lo = max(sseg[s], c0), hi = min(sseg[s + 1], c1);
                            if (lo >= hi) continue;
                            float acc = shist[s * kSliceBins + j];
                            for (int rr = lo; rr < hi; ++rr) acc = __fadd_rn(acc, sstage[(rr - c0) * kStagePitch + j]);
                            shist[s * kSliceBins + j] = acc;
                        }
                    }
                    __syncthreads();
                }
            }
        }
        if (failed) {
            // the last MMAs still complete before TMEM is released
            if (tid == 0) {
                raise_status(a.status, PVF_ERR_TIMEOUT);
                mma_commit(bar);
                const uint64_t tw = globaltimer();
                while (!mbar_try_wait(bar, phase)) if (globaltimer() - tw > kWaitLimitNs) break;
            }
            for (int i = tid; i < kBins; i += kT) shist[i] = 0.0f;
        }
        __syncthreads();
    }

    if (a.hist_out) {
        float4 *dst = reinterpret_cast<float4 *>(a.hist_out + (size_t)ge * kBins);
        const float4 *src = reinterpret_cast<const float4 *>(shist);
        for (int i = tid; i < kBins / 4; i += kT) dst[i] = src[i];
    }
    enc1_pool<T, kT>(a, e, tid, shist, senc);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tmem_slot, kTmemCols);
}

}  // namespace

cudaError_t launch_front_tc(const FrontArgs &a, int precision, cudaStream_t s) {
    if (a.n_events <= 0) return cudaSuccess;
    const size_t smem = TcSmem::total(a.max_tracks);
    cudaError_t err;
    if (precision == PVF_BF16) {
        err = cudaFuncSetAttribute(k_front_tc<PVF_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) k_front_tc<PVF_BF16><<<a.n_events, kT, smem, s>>>(a);
    } else {
        err = cudaFuncSetAttribute(k_front_tc<PVF_FP8_E4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) k_front_tc<PVF_FP8_E4M3><<<a.n_events, kT, smem, s>>>(a);
    }
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace pvf
