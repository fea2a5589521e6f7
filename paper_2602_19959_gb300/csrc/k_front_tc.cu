// Steps 1-2 of the path (§2) for the tensor-core forms: the per-track FC network on
// tcgen05 (16-bit operands: f16 in the FP16 form, bf16 in the BF16 and FP8 forms; fp32
// accumulation in TMEM), the deterministic histogram, and
// enc1 + pool. A persistent grid (up to four 128-thread CTAs per SM, which fill the 512
// TMEM columns) walks the events, one event at a time per CTA (§3: each event is
// processed by one thread block), so weights and TMEM are set up once per CTA rather
// than once per event.
//
// Per pass of up to 128 slice-sorted tracks (one track per TMEM lane / thread in the
// hidden layers):
//   X [128 x 16] (nine features, feature 2 slice-relative, zero padded) ->
//   5 x { MMA (M = 128 tracks, N = 32) -> TMEM -> bias + LeakyReLU -> 16-bit ->
//         H [128 x 32] } ->
//   output layer as the transposed product Out^T = W6^T H^T (one MMA, M = 128 output
//   lanes, N = tracks of the pass), so TMEM lane = output bin and column = sorted track ->
//   each thread adds bias + softplus of its bin over the tracks in sorted order, flushing
//   a slice's running sum into hist[100 s + j] when the slice's segment ends (and at the
//   pass's last track).
// Every bin is thus summed in one fixed order that depends only on the event's own
// sorted track list: results are identical alone and in any batch. One thread issues the
// MMAs; every wait on their completion is bounded.
#include "front_common.cuh"
#include "tc_ptx.cuh"

namespace pvf {
namespace {

using namespace front;
using namespace tc;

constexpr int kT = 128;                 // threads: one warpgroup
constexpr int kRows = 128;              // tile rows = TMEM lanes = tracks per pass
constexpr int kPlane = kRows * 16;      // bytes of one K-major plane of X or H
constexpr int kTmemCols = 128;          // hidden layers: columns [0, 32); output: [0, N)

struct TcSmem {
    static constexpr size_t img = 0;                                   // kFcImgBytes
    static constexpr size_t bias = img + kFcImgBytes;                  // kFcBTotal floats
    static constexpr size_t enc1 = bias + sizeof(float) * kFcBTotal;   // kEnc1Floats
    static constexpr size_t x = (enc1 + sizeof(float) * kEnc1FloatsMax + 127) / 128 * 128;  // 2 planes x 128 rows
    static constexpr size_t h = x + 2 * kPlane;                        // 4 planes x 128 rows
    static constexpr size_t hist = h + 4 * kPlane;
    static constexpr size_t cnt = hist + sizeof(float) * kBins;
    static constexpr size_t seg = cnt + sizeof(int) * 48;
    static constexpr size_t run = seg + sizeof(int) * 48;
    static constexpr size_t bar = (run + sizeof(int) * 48 + 15) / 16 * 16;   // mbarrier, TMEM slot, flag, next event
    static constexpr size_t sorted = bar + 32;
    __host__ __device__ static size_t slices(int ne) { return sorted + 2 * (size_t)((ne + 7) / 8 * 8); }
    __host__ __device__ static size_t total(int mt, float edge) {
        return slices(front_entries(mt, edge)) + (size_t)mt + 16;
    }
};

// FC operand type of each form and its tcgen05 kind::f16 format code (0 = f16, 1 = bf16).
template <int PREC> struct FcOp {
    using T = __nv_bfloat16;
    static constexpr uint32_t FMT = 1;
};
template <> struct FcOp<PVF_FP16> {
    using T = __half;
    static constexpr uint32_t FMT = 0;
};

// softplus(x) = max(x, 0) + log(1 + u), u = exp(-|x|) in (0, 1], for the tensor-core forms
// (their FC operands are 16-bit): the hardware exp2/log2 approximations give it in a few
// instructions with an absolute error of a few 1e-7. Below x = -15 the value is u itself
// (log(1 + u) = u to 1e-7 relative), which keeps tiny terms positive instead of rounding
// 1 + u to 1.
__device__ __forceinline__ float softplus_tc(float x) {
    const float u = __expf(-fabsf(x));
    const float l = fmaf(__log2f(1.0f + u), 0.69314718f, fmaxf(x, 0.0f));
    return x < -15.0f ? u : l;
}

// EDGE: boundary tracks fill a second slice (a.edge > 0); without them the sort and the
// entry decoding compile to the one-slice form.
template <int PREC, bool EDGE>
__global__ void __launch_bounds__(kT, 4) k_front_tc(FrontArgs a) {
    using T = typename Elem<PREC>::T;
    using FT = typename FcOp<PREC>::T;
    constexpr uint32_t FMT = FcOp<PREC>::FMT;
    extern __shared__ __align__(128) unsigned char smem[];
    float *sbias = reinterpret_cast<float *>(smem + TcSmem::bias);
    float *senc = reinterpret_cast<float *>(smem + TcSmem::enc1);
    float *shist = reinterpret_cast<float *>(smem + TcSmem::hist);
    int *scnt = reinterpret_cast<int *>(smem + TcSmem::cnt);
    int *sseg = reinterpret_cast<int *>(smem + TcSmem::seg);
    int *srun = reinterpret_cast<int *>(smem + TcSmem::run);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + TcSmem::bar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + TcSmem::bar + 8);
    volatile int *never = reinterpret_cast<volatile int *>(smem + TcSmem::bar + 12);
    int *snext = reinterpret_cast<int *>(smem + TcSmem::bar + 16);   // the CTA's next event
    uint16_t *ssorted = reinterpret_cast<uint16_t *>(smem + TcSmem::sorted);
    uint8_t *sslice = smem + TcSmem::slices(EDGE ? 2 * a.max_tracks : a.max_tracks);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = tid;                             // row of the pass = TMEM lane
    const uint32_t lane_field = (uint32_t)(warp * 32) << 16;
    // output layer: this thread's TMEM lane holds output o (-1: a zero row)
    const int o_bin = lane < kFcOutPerWarp ? warp * kFcOutPerWarp + lane : -1;

    // once per CTA: enc1 weights, FC operand images and biases, barrier, TMEM
    for (int i = tid; i < 6 * a.c0; i += kT) senc[i] = a.enc1[i];   // W[t][co] then b, c0 channels
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
    // launched in stream order (its inputs come from the caller); lets the next kernel
    // start its prologue while this one runs
    grid_dep_launch();
    const uint32_t img = smem_u32(smem + TcSmem::img);
    const uint32_t sx = smem_u32(smem + TcSmem::x), sh = smem_u32(smem + TcSmem::h);
    unsigned char *xrow = smem + TcSmem::x + (size_t)m * 16;   // + plane * kPlane
    unsigned char *hrow = smem + TcSmem::h + (size_t)m * 16;
    const uint32_t dcol = tmem + lane_field;
    const float b6 = o_bin >= 0 ? sbias[5 * kFcHidden + o_bin] : 0.0f;
    bool failed = false;
    uint32_t phase = 0;

    // a device-side count is read here (features and offsets come from the caller, in
    // stream order) and copied to device memory for the kernels after this one
    const int n_ev = launch_events(a.n_dyn, a.ev_base, a.n_events);
    if (a.n_dyn_copy && blockIdx.x == 0 && tid == 0)
        *a.n_dyn_copy = *reinterpret_cast<const volatile int32_t *>(a.n_dyn);

    // persistent: the CTA walks the launch's events, its first one blockIdx.x, then the
    // next unclaimed one (a global ticket: CTAs that finish early take more events, and
    // each event is still computed whole by one CTA, so results do not depend on which)
    for (int e = blockIdx.x; e < n_ev;) {
        const int ge = a.ev_base + e;
        if (a.hist_in) {
            const float *src = a.hist_in + (size_t)ge * kBins;
            for (int i = tid; i < kBins; i += kT) shist[i] = src[i];
            __syncthreads();
        } else {
            for (int i = tid; i < kBins; i += kT) shist[i] = 0.0f;
            int64_t t0;
            int nvalid;
            validate_sort<kT, EDGE>(a, ge, tid, scnt, sseg, srun, ssorted, sslice, t0, nvalid);
            if (failed) nvalid = 0;        // a timed-out MMA ends the tensor-core work
            for (int c0 = 0; c0 < nvalid && !failed; c0 += kRows) {
                const int r = c0 + m;
                const bool live = r < nvalid;
                {   // X row: the track's features in 16 bits, zero rows past the event
                    float x[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) x[k] = 0.0f;
                    if (live) {
                        const int en = ssorted[r];
                        track_features(a, t0 + entry_track<EDGE>(en), entry_slice<EDGE>(en, sslice), x);
                    }
                    *reinterpret_cast<uint4 *>(xrow) = pack8<FT>(x);
                    *reinterpret_cast<uint4 *>(xrow + kPlane) = pack8<FT>(x + 8);
                }
                fence_proxy_async_smem();
                tc_fence_before();
                __syncthreads();
                const int nrow = min(nvalid - c0, kRows);
                const int n6 = (nrow + 15) / 16 * 16;          // output MMA: N = tracks, rounded
                for (int l = 0; l < 6 && !failed; ++l) {
                    tc_fence_after();
                    if (tid == 0) {
                        if (l == 0) {
                            mma_f16(tmem, smem_desc(sx, kPlane, 128), smem_desc(img, kFcHidden * 16, 128),
                                    idesc_f32acc(kRows, kFcHidden, FMT), 0);
                        } else if (l < 5) {
                            const uint32_t w = img + fc_img_off(l);
#pragma unroll
                            for (int kb = 0; kb < 2; ++kb)
                                mma_f16(tmem, smem_desc(sh + 2 * kb * kPlane, kPlane, 128),
                                        smem_desc(w + 2 * kb * kFcHidden * 16, kFcHidden * 16, 128),
                                        idesc_f32acc(kRows, kFcHidden, FMT), kb);
                        } else {   // Out^T [128 lanes x n6] = W6^T (A) x H^T (B = H, K-major)
                            const uint32_t w = img + fc_img_off(5);
#pragma unroll
                            for (int kb = 0; kb < 2; ++kb)
                                mma_f16(tmem, smem_desc(w + 2 * kb * kFcM6 * 16, kFcM6 * 16, 128),
                                        smem_desc(sh + 2 * kb * kPlane, kPlane, 128),
                                        idesc_f32acc(kFcM6, n6, FMT), kb);
                        }
                        mma_commit(bar);
                    }
                    const bool ok = mbar_wait(bar, phase, never);
                    phase ^= 1;
                    if (__syncthreads_or(!ok)) { failed = true; break; }
                    tc_fence_after();
                    if (l < 5) {
                        float v[32];
                        tmem_ld16(dcol, *reinterpret_cast<float(*)[16]>(v));
                        tmem_ld16(dcol + 16, *reinterpret_cast<float(*)[16]>(v + 16));
                        const float *b = sbias + l * kFcHidden;
#pragma unroll
                        for (int o = 0; o < kFcHidden; ++o) v[o] = leaky(v[o] + b[o]);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            *reinterpret_cast<uint4 *>(hrow + k * kPlane) = pack8<FT>(v + 8 * k);
                        fence_proxy_async_smem();
                        tc_fence_before();
                        __syncthreads();
                        continue;
                    }
                    // output layer: this thread adds its bin over the pass's tracks in order,
                    // 32 at a time, flushing slice s's running sum when its segment ends
                    float acc = 0.0f;
                    int s = entry_slice<EDGE>(ssorted[c0], sslice);
                    int send = sseg[s + 1] - c0;               // first pass row past slice s
#pragma unroll 1
                    for (int col = 0; col < nrow; col += 32) {
                        float v[32];
                        tmem_ld32(tmem + lane_field + (uint32_t)col, v);
#pragma unroll
                        for (int t = 0; t < 32; ++t) v[t] = softplus_tc(v[t] + b6);
                        if (col + 32 <= min(nrow, send)) {     // one slice throughout
#pragma unroll
                            for (int t = 0; t < 32; ++t) acc = __fadd_rn(acc, v[t]);
                            continue;
                        }
                        // several segments in this chunk: one branch-free masked pass per
                        // segment, in row order (adding zeros leaves the sum bit-identical,
                        // and the loop body stays small enough for the instruction cache;
                        // an unrolled loop with a flush per segment end measured slower)
                        const int cnt = min(32, nrow - col);
                        int t0 = 0;
#pragma unroll 1
                        while (t0 < cnt) {
                            const int t1 = min(cnt, send - col);
                            const uint32_t hi = t1 >= 32 ? 0xFFFFFFFFu : ((1u << t1) - 1u);
                            const uint32_t msk = hi & ~((1u << t0) - 1u);
#pragma unroll
                            for (int t = 0; t < 32; ++t) acc = __fadd_rn(acc, ((msk >> t) & 1u) ? v[t] : 0.0f);
                            if (t1 < cnt) {                    // slice s ends at row col + t1
                                if (o_bin >= 0) {
                                    float *hp = shist + s * kSliceBins + o_bin;
                                    *hp = __fadd_rn(*hp, acc);
                                }
                                acc = 0.0f;
                                s = entry_slice<EDGE>(ssorted[c0 + col + t1], sslice);
                                send = sseg[s + 1] - c0;
                            }
                            t0 = t1;
                        }
                    }
                    if (o_bin >= 0) {   // the pass's last segment (its slice may continue next pass)
                        float *hp = shist + s * kSliceBins + o_bin;
                        *hp = __fadd_rn(*hp, acc);
                    }
                    tc_fence_before();
                    __syncthreads();
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
        if (a.iv) enc1_pool<T, kT, true, kC0, true>(a, e, tid, shist, senc);
        else if (a.c0 == kC0Max) enc1_pool<T, kT, false, kC0Max>(a, e, tid, shist, senc);   // the wide network
        else enc1_pool<T, kT>(a, e, tid, shist, senc);
        if (tid == 0) *snext = a.ev_ctr ? (int)gridDim.x + atomicAdd(a.ev_ctr, 1) : e + (int)gridDim.x;
        __syncthreads();                   // shist and the sort arrays are reused next event
        e = *snext;
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
    if (a.ev_ctr && tid == 0) {   // the last CTA to finish resets the tickets for the next launch
        __threadfence();
        if (atomicAdd(a.ev_ctr + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(a.ev_ctr, 0);
            atomicExch(a.ev_ctr + 1, 0);
        }
    }
}

}  // namespace

// Persistent grid: the schedule's CTAs per SM (0 = 4, which fill the SM's 512 TMEM
// columns), as shared memory allows, each walking events.
template <int PREC, bool EDGE>
cudaError_t launch_front_tc_k(const FrontArgs &a, cudaStream_t s) {
    const size_t smem = TcSmem::total(a.max_tracks, a.edge);
    int sms = 0;
    cudaError_t err = current_device_sms(&sms);
    if (err == cudaSuccess) err = prepare_kernel((const void *)k_front_tc<PREC, EDGE>, smem, nullptr);
    if (err != cudaSuccess) return err;
    int per_sm = (int)((228 * 1024) / (smem + 1024));
    if (per_sm > 4) per_sm = 4;
    if (a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm) per_sm = a.ctas_per_sm;
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    if (grid > a.n_events) grid = a.n_events;
    k_front_tc<PREC, EDGE><<<grid, kT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_front_tc_t(const FrontArgs &a, cudaStream_t s) {
    return a.edge > 0.0f ? launch_front_tc_k<PREC, true>(a, s) : launch_front_tc_k<PREC, false>(a, s);
}

cudaError_t launch_front_tc(const FrontArgs &a, int precision, cudaStream_t s) {
    if (a.n_events <= 0) return cudaSuccess;
    if ((a.c0 != kC0 && a.c0 != kC0Max) || (a.iv && a.c0 != kC0)) return cudaErrorInvalidValue;
    switch (precision) {
    case PVF_BF16: return launch_front_tc_t<PVF_BF16>(a, s);
    case PVF_FP16: return launch_front_tc_t<PVF_FP16>(a, s);
    case PVF_FP8_E4M3: return launch_front_tc_t<PVF_FP8_E4M3>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pvf
