// End of step 3 and step 4 of the path (§2): the final c0 -> 1 channel k5 convolution
// (float32 in every form) and heuristic peak finding on its output.
//
// A persistent grid of 256-thread CTAs walks the events, one event at a time per CTA:
//   1. f[p] = b + sum_t sum_ci W[t][ci] d1[p + t - 2][ci]  (the logit; prob = sigmoid(f)),
//      kept in shared memory, optionally copied out;
//   2. local-maximum rule with a fixed threshold in place of the paper's learned ones:
//      bin i is a PV iff p[i] > 0.01, p[i] > p[j] for the 5 bins on its left and
//      p[i] >= p[j] for the 5 bins on its right (clipped at the ends). Because sigmoid
//      is strictly increasing these decisions are taken exactly on f (the threshold
//      becomes ln(0.01 / 0.99)), which avoids the float32 saturation of sigmoid
//      (which rounds to 1 for f > 16.6) turning distinct maxima into ties;
//   3. z = centroid over bins [i - 3, i + 3] with weights p[j] = sigmoid(f[j]);
//   4. ordered compaction: each thread owns 16 consecutive bins and tests them in
//      registers (a 16-bit candidate mask); a block-wide exclusive scan of
//      the per-thread counts gives each PV its slot, so PVs are written in ascending z
//      without atomics. The true count is always reported.
#include "pvf_internal.cuh"

namespace pvf {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;    // kThreads * kPerThread >= kBins
// ln(0.01 / 0.99) rounded to float
constexpr float kThrLogit = -4.59511985013459f;

// Loads channels [16 g, 16 g + 16) of storage row `row` of event e of the channel-last
// float32 tensor d1 with C0 channels.
template <int C0>
__device__ __forceinline__ void load_seg16_f32(const void *base, int64_t e, int64_t rows_e, int64_t row,
                                               int g, float v[16]) {
    const float4 *s = reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(base) +
                                                       (e * rows_e + row) * C0 + 16 * g);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float4 x = s[i];
        v[4 * i] = x.x; v[4 * i + 1] = x.y; v[4 * i + 2] = x.z; v[4 * i + 3] = x.w;
    }
}

__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

// CONV: the logit comes from the final conv over d1 (the float32 form, base width C0);
// otherwise it is read from a.logit_in. Without the conv the kernel fits eight CTAs per SM.
// IV: d1 is in the per-interval layout; bin 100 s + j is position j + kIvPad of interval
// s's sequence.
template <bool CONV, int C0, bool IV = false>
__global__ void __launch_bounds__(kThreads, CONV ? 2 : 8) k_tail(TailArgs a) {
    __shared__ __align__(16) float sf[kThreads * kPerThread];
    __shared__ float sw[kFinalFloatsMax];
    __shared__ int swarp[kThreads / 32];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if constexpr (CONV) {
        for (int i = tid; i < 5 * C0 + 1; i += kThreads) sw[i] = a.final_w[i];
        __syncthreads();
    }
    // the logits (or d1) are the previous kernel's output (dependent launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // persistent: the CTA walks the launch's events
    const int n_ev = launch_events(a.n_dyn, a.ev_base, a.n_events);
    for (int e = blockIdx.x; e < n_ev; e += gridDim.x) {
        const int ge = a.ev_base + e;
        if constexpr (!CONV) {
            const float *src = a.logit_in + (size_t)(ge - a.logit_in_base) * kBins;
            for (int p = tid; p < kBins; p += kThreads) sf[p] = src[p];
        } else {
            const int64_t rows1 = padded_rows(IV ? kIvLen : kBins);
            for (int p = tid; p < kBins; p += kThreads) {
                float acc = sw[5 * C0];
                // sequence and position of bin p (storage row x + t = position x + t - 2)
                const int64_t seq = IV ? (int64_t)e * kSlices + p / kSliceBins : e;
                const int x = IV ? p % kSliceBins + kIvPad : p;
#pragma unroll
                for (int t = 0; t < 5; ++t) {
#pragma unroll 1
                    for (int g = 0; g < C0 / 16; ++g) {
                        float v[16];
                        load_seg16_f32<C0>(a.d1, seq, rows1, x + t, g, v);
#pragma unroll
                        for (int ci = 0; ci < 16; ++ci) acc = fmaf(sw[t * C0 + 16 * g + ci], v[ci], acc);
                    }
                }
                sf[p] = acc;
            }
        }
        __syncthreads();
        if (a.logit_out) {
            float *dst = a.logit_out + (size_t)ge * kBins;
            for (int p = tid; p < kBins; p += kThreads) dst[p] = sf[p];
        }
        if (a.pv_count) {
            const bool bypass = a.ev_flag && a.ev_flag[ge] != 0;
            // ---- candidate flags: thread tid owns bins [16 tid, 16 tid + 16). It loads them with
            //      their +-5 neighbours (bins 16 tid - 8 .. 16 tid + 23, 16-byte loads) into
            //      registers and tests each bin there; bins outside [0, kBins) read as -inf, which
            //      no finite logit fails (the same as not comparing clipped neighbours).
            static_assert(kBins % 4 == 0 && kPerThread == 16 && kPeakHalfWin <= 8, "flag window");
            const int i0 = tid * kPerThread;
            unsigned mask = 0;
            if (!bypass && i0 < kBins) {
                const float ninf = __int_as_float(0xff800000);
                const float4 *s4 = reinterpret_cast<const float4 *>(sf);
                float w[kPerThread + 16];
#pragma unroll
                for (int k = 0; k < (kPerThread + 16) / 4; ++k) {
                    const int j = i0 - 8 + 4 * k;
                    const float4 x = (j >= 0 && j + 3 < kBins) ? s4[j >> 2] : make_float4(ninf, ninf, ninf, ninf);
                    w[4 * k] = x.x; w[4 * k + 1] = x.y; w[4 * k + 2] = x.z; w[4 * k + 3] = x.w;
                }
#pragma unroll
                for (int b = 0; b < kPerThread; ++b) {
                    const float fi = w[b + 8];
                    bool c = i0 + b < kBins && fi > kThrLogit;
#pragma unroll
                    for (int d = 1; d <= kPeakHalfWin; ++d) c = c && fi > w[b + 8 - d] && fi >= w[b + 8 + d];
                    mask |= (unsigned)c << b;
                }
            }
            const int cnt = __popc(mask);
            // ---- block exclusive scan of cnt
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) swarp[warp] = incl;
            __syncthreads();
            int wbase = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) {
                const int v = swarp[w];
                if (w < warp) wbase += v;
                total += v;
            }
            int idx = wbase + incl - cnt;
            float *zout = a.pv_z + (size_t)ge * a.max_pv;
            while (mask) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1;
                if (idx < a.max_pv) {
                    const int i = i0 + k;
                    float num = 0.0f, den = 0.0f;
#pragma unroll
                    for (int d = -kCentroidHalf; d <= kCentroidHalf; ++d) {
                        const int j = i + d;
                        if (j < 0 || j >= kBins) continue;
                        const float pj = sigmoid_f(sf[j]);
                        num = fmaf(pj, (float)d, num);
                        den += pj;
                    }
                    // z = zc(i) + 0.1 * (sum p_j (j - i) / sum p_j), zc(i) = -100 + (i + 0.5) * 0.1
                    zout[idx] = fmaf((float)i + 0.5f + num / den, kBinW, kZLo);
                }
                ++idx;
            }
            if (tid == 0) {
                a.pv_count[ge] = bypass ? -1 : total;
                if (!bypass && total > a.max_pv) raise_status(a.status, PVF_WARN_TRUNCATED);
            }
        }
        __syncthreads();                       // sf and swarp are reused next event
    }
}

}  // namespace

cudaError_t launch_tail(const TailArgs &a, int precision, cudaStream_t s) {
    if (a.n_events <= 0) return cudaSuccess;
    // persistent grid of resident CTAs (their launch bounds fix the registers: two per SM
    // with the final conv, eight without), each walking events
    int sms = 0;
    const cudaError_t err = current_device_sms(&sms);
    if (err != cudaSuccess) return err;
    int per_sm = a.logit_in ? 8 : 2;
    if (a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm) per_sm = a.ctas_per_sm;
    dim3 grid(a.n_events < per_sm * sms ? a.n_events : per_sm * sms), block(kThreads);
    if (a.logit_in) return launch_pdl(k_tail<false, kC0>, grid, block, 0, s, a);
    // the final conv runs here in the FP32 form only (the tensor-core forms run it in
    // dec1's epilogue and pass logits)
    if (precision != PVF_FP32) return cudaErrorInvalidValue;
    if (a.iv) {
        if (a.c0 != kC0) return cudaErrorInvalidValue;
        k_tail<true, kC0, true><<<grid, block, 0, s>>>(a);
    } else if (a.c0 == kC0Max) k_tail<true, kC0Max><<<grid, block, 0, s>>>(a);
    else if (a.c0 == kC0) k_tail<true, kC0><<<grid, block, 0, s>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace pvf
