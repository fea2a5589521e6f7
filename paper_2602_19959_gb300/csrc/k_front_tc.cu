// Steps 1-2 of the path (§2) for the tensor-core forms: the per-track FC network on
// tcgen05 (16-bit operands: f16 in the FP16 form, bf16 in the BF16 and FP8 forms; fp32
// accumulation in TMEM), the deterministic histogram, and
// enc1 + pool. A persistent grid walks the events, one event at a time per CTA (§3: each
// event is processed by one thread block), so weights and TMEM are set up once per CTA
// rather than once per event. Two shapes: NT = 128 threads (one warpgroup, passes of 128
// tracks, 128 TMEM columns; up to four CTAs per SM, for large launches) or NT = 256 (two
// warpgroups, passes of 256 tracks, 256 columns; up to two per SM, for small ones).
//
// Per pass of up to NT slice-sorted tracks (NT / 128 tiles of 128 rows, one per
// warpgroup, one track per TMEM lane / thread in the hidden layers):
//   X [NT x 16] (nine features, feature 2 slice-relative, zero padded) ->
//   5 x { MMA per tile (M = 128 tracks, N = 32) -> TMEM -> bias + LeakyReLU -> 16-bit ->
//         H [NT x 32] } ->
//   output layer as the transposed product Out^T = W6^T H^T (one MMA, M = 128 output
//   lanes, N = tracks of the pass), so TMEM lane = output bin and column = sorted track ->
//   each thread adds bias + softplus of its bin over the tracks in sorted order, flushing
//   a slice's running sum into hist[100 s + j] when the slice's segment ends.
// With two warpgroups, warpgroup 0 takes the pass's first 128 tracks and warpgroup 1 the
// rest; warpgroup 1 adds its first segment's partial after warpgroup 0 has added its own.
// A bin's sum is thus split into partials at every multiple of 128 sorted tracks and
// inside a partial runs in sorted order, in both shapes: every bin is summed in one fixed
// order that depends only on the event's own sorted track list, so results are identical
// alone, in any batch and under either shape. One thread issues the MMAs; every wait on
// their completion is bounded.
#include "front_common.cuh"
#include "tc_ptx.cuh"

namespace pvf {
namespace {

using namespace front;
using namespace tc;

constexpr int kRows = 128;              // tile rows = TMEM lanes

// NT threads = NT / 128 warpgroups, one 128-row tile each; a pass holds NT tracks.
// TMEM: NT columns (hidden layers: tile g at column 128 g; output layer: [0, N)).
template <int NT> struct TcSmem {
    static constexpr int kPlane = NT * 16;   // bytes of one K-major plane of X or H
    static constexpr size_t img = 0;                                   // kFcImgBytes
    static constexpr size_t bias = img + kFcImgBytes;                  // kFcBTotal floats
    static constexpr size_t enc1 = bias + sizeof(float) * kFcBTotal;   // kEnc1Floats
    static constexpr size_t x = (enc1 + sizeof(float) * kEnc1FloatsMax + 127) / 128 * 128;  // 2 planes x NT rows
    static constexpr size_t h = x + 2 * kPlane;                        // 4 planes x NT rows
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
template <int PREC, bool EDGE, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_front_tc(FrontArgs a) {
    static_assert(NT == 128 || NT == 256, "one or two warpgroups");
    using TcSmem = pvf::TcSmem<NT>;
    constexpr int kT = NT, kPass = NT, kPlane = TcSmem::kPlane, kTmemCols = NT;
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
    const int g = warp >> 2;                       // tile of this warpgroup
    const int m = tid & (kRows - 1);               // row within the tile = TMEM lane
    const uint32_t lane_field = (uint32_t)((warp & 3) * 32) << 16;
    // output layer: this thread's TMEM lane holds output o (-1: a zero row)
    const int o_bin = lane < kFcOutPerWarp ? (warp & 3) * kFcOutPerWarp + lane : -1;

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
    unsigned char *xrow = smem + TcSmem::x + (size_t)(g * kRows + m) * 16;   // + plane * kPlane
    unsigned char *hrow = smem + TcSmem::h + (size_t)(g * kRows + m) * 16;
    const uint32_t dcol = tmem + lane_field + (uint32_t)(g * 128);
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
            for (int c0 = 0; c0 < nvalid && !failed; c0 += kPass) {
                const int ntile = NT == 128 ? 1 : (nvalid - c0 > kRows ? 2 : 1);
                const bool active = g < ntile;         // warpgroup has a tile in this pass
                const int r = c0 + g * kRows + m;
                const bool live = r < nvalid;
                if (active) {   // X row: the track's features in 16 bits, zero rows past the event
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
                const int nrow = min(nvalid - c0, kPass);
                const int n6 = (nrow + 15) / 16 * 16;          // output MMA: N = tracks, rounded
                for (int l = 0; l < 6 && !failed; ++l) {
                    tc_fence_after();
                    if (tid == 0) {
                        if (l == 0) {
                            for (int tg = 0; tg < ntile; ++tg)
                                mma_f16(tmem + (uint32_t)(tg * 128), smem_desc(sx + tg * kRows * 16, kPlane, 128),
                                        smem_desc(img, kFcHidden * 16, 128), idesc_f32acc(kRows, kFcHidden, FMT), 0);
                        } else if (l < 5) {
                            const uint32_t w = img + fc_img_off(l);
                            for (int tg = 0; tg < ntile; ++tg) {
#pragma unroll
                                for (int kb = 0; kb < 2; ++kb)
                                    mma_f16(tmem + (uint32_t)(tg * 128),
                                            smem_desc(sh + tg * kRows * 16 + 2 * kb * kPlane, kPlane, 128),
                                            smem_desc(w + 2 * kb * kFcHidden * 16, kFcHidden * 16, 128),
                                            idesc_f32acc(kRows, kFcHidden, FMT), kb);
                            }
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
                        if (active) {
                            float v[32];
                            tmem_ld16(dcol, *reinterpret_cast<float(*)[16]>(v));
                            tmem_ld16(dcol + 16, *reinterpret_cast<float(*)[16]>(v + 16));
                            const float *b = sbias + l * kFcHidden;
#pragma unroll
                            for (int o = 0; o < kFcHidden; ++o) v[o] = leaky(v[o] + b[o]);
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                *reinterpret_cast<uint4 *>(hrow + k * kPlane) = pack8<FT>(v + 8 * k);
                        }
                        fence_proxy_async_smem();
                        tc_fence_before();
                        __syncthreads();
                        continue;
                    }
                    // output layer: warpgroup g adds its bin over pass rows [cb, ce) in order
                    const int half = min(nrow, kRows);
                    const int cb = g == 0 ? 0 : half, ce = g == 0 ? min(half, nrow) : nrow;
                    float acc = 0.0f, held = 0.0f;
                    int held_s = -1;
                    if (cb < ce) {
                        int s = entry_slice<EDGE>(ssorted[c0 + cb], sslice);
                        int send = sseg[s + 1] - c0;           // first pass row past slice s
                        bool hold = NT == 256 && g == 1;       // warpgroup 1 holds its first segment
#pragma unroll 1
                        for (int col = cb; col < ce; col += 32) {
                            float v[32];
                            tmem_ld32(tmem + lane_field + (uint32_t)col, v);
#pragma unroll
                            for (int t = 0; t < 32; ++t) v[t] = softplus_tc(v[t] + b6);
                            if (col + 32 <= min(ce, send)) {   // one slice throughout
#pragma unroll
                                for (int t = 0; t < 32; ++t) acc = __fadd_rn(acc, v[t]);
                                continue;
                            }
                            // several segments in this chunk: one branch-free masked pass per
                            // segment, in row order (adding zeros leaves the sum bit-identical,
                            // and the loop body stays small enough for the instruction cache)
                            const int cnt = min(32, ce - col);
                            int t0 = 0;
#pragma unroll 1
                            while (t0 < cnt) {
                                const int t1 = min(cnt, send - col);
                                const uint32_t hi = t1 >= 32 ? 0xFFFFFFFFu : ((1u << t1) - 1u);
                                const uint32_t msk = hi & ~((1u << t0) - 1u);
#pragma unroll
                                for (int t = 0; t < 32; ++t) acc = __fadd_rn(acc, ((msk >> t) & 1u) ? v[t] : 0.0f);
                                if (t1 < cnt) {                // slice s ends at row col + t1
                                    if (hold) { held = acc; held_s = s; hold = false; }
                                    else if (o_bin >= 0) {
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
                        if (hold) { held = acc; held_s = s; }
                        else if (o_bin >= 0) {
                            float *hp = shist + s * kSliceBins + o_bin;
                            *hp = __fadd_rn(*hp, acc);
                        }
                    }
                    tc_fence_before();
                    __syncthreads();
                    if (held_s >= 0 && o_bin >= 0) {
                        float *hp = shist + held_s * kSliceBins + o_bin;
                        *hp = __fadd_rn(*hp, held);
                    }
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
        if (tid == 0) {
            int next = e + (int)gridDim.x;
            if (a.ev_ctr) {
                // one ticket per processed event: the ticket n_ev - 1 is the launch's last,
                // and its taker resets the counter for the next launch (CTAs without an
                // event never touch it)
                const int k = atomicAdd(a.ev_ctr, 1);
                if (k == n_ev - 1) atomicExch(a.ev_ctr, 0);
                next = (int)gridDim.x + k;
            }
            *snext = next;
        }
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
}

}  // namespace

template <int PREC, bool EDGE, int NT>
cudaError_t launch_front_tc_k(const FrontArgs &a, int per_sm, cudaStream_t s) {
    // persistent grid: up to per_sm CTAs per SM, as shared memory allows (NT TMEM columns
    // each: 512 / NT CTAs fill an SM's 512 columns), each walking events
    const size_t smem = TcSmem<NT>::total(a.max_tracks, a.edge);
    int sms = 0;
    cudaError_t err = current_device_sms(&sms);
    if (err == cudaSuccess) err = prepare_kernel((const void *)k_front_tc<PREC, EDGE, NT>, smem, nullptr);
    if (err != cudaSuccess) return err;
    const int fit = (int)((228 * 1024) / (smem + 1024));
    if (per_sm > fit) per_sm = fit;
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    if (grid > a.n_events) grid = a.n_events;
    k_front_tc<PREC, EDGE, NT><<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

// CTAs per SM (the schedule's value): 1 or 2 run the two-warpgroup shape, 3 or 4 (and
// larger values, clamped) the one-warpgroup shape. 0: a launch of at most four events per
// SM (a serving batch) takes two 256-thread CTAs per SM, which halve each event's latency;
// a larger one four 128-thread CTAs per SM, which process more events at once. The
// shapes give bit-identical results.
template <int PREC, bool EDGE>
cudaError_t launch_front_tc_e(const FrontArgs &a, cudaStream_t s) {
    int per_sm = a.ctas_per_sm;
    if (per_sm <= 0) {
        int sms = 0;
        const cudaError_t err = current_device_sms(&sms);
        if (err != cudaSuccess) return err;
        per_sm = a.n_events <= 4 * sms ? 2 : 4;
    }
    if (per_sm <= 2) return launch_front_tc_k<PREC, EDGE, 256>(a, per_sm, s);
    return launch_front_tc_k<PREC, EDGE, 128>(a, per_sm > 4 ? 4 : per_sm, s);
}

template <int PREC>
cudaError_t launch_front_tc_t(const FrontArgs &a, cudaStream_t s) {
    return a.edge > 0.0f ? launch_front_tc_e<PREC, true>(a, s) : launch_front_tc_e<PREC, false>(a, s);
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
