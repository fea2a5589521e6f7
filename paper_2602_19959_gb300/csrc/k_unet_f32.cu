// Step 3 of the path (§2, UNet-style 1D CNN) in plain float32 on CUDA cores: the
// "plain FP32 GPU form" that the tensor-core forms are measured against.
//
// Layers (positions L, channels):   enc2 16->32 @2000 (+pool)   enc3 32->64 @1000 (+pool)
//   enc4 64->128 @500   up3 128->64 @500->1000   dec3 [64+64]->64 @1000
//   up2 64->32 @1000->2000   dec2 [32+32]->32 @2000   up1 32->16 @2000->4000
//   dec1 [16+16]->16 @4000. Every conv is k5 with zero "same" padding, every conv and
// ConvT is followed by LeakyReLU(0.01); the skip concat is [upsampled, skip] and is
// read in place from the two tensors (never materialised); the 2:1 max-pool is taken in
// the producing conv's epilogue.
//
// Each CTA computes a tile of TP positions x all C_out channels of one event; each
// thread owns an 8 x 8 register block (8 consecutive positions x 8 channels). Inputs
// are staged through shared memory in chunks of 16 channels (transposed to
// [channel][position] so a thread's 12 halo'd inputs are three aligned float4 loads);
// the weights of the chunk sit next to them as [tap][channel][C_out]. The sum over
// (channel chunk, channel, tap) runs in a fixed order: results are deterministic.
#include "pvf_internal.cuh"

namespace pvf {
namespace {

constexpr int kKC = 16;   // input channels per shared-memory chunk

// KC input channels per shared-memory chunk (8 where 16 would exceed the 48 KB of static
// shared memory: the wide variant's 128- and 256-channel layers).
template <int CA, int CB, int COUT, int TP, bool POOL, int KC = kKC>
__global__ void __launch_bounds__((TP / 8) * (COUT / 8))
k_conv5_f32(const float *__restrict__ inA, const float *__restrict__ inB,
            const float *__restrict__ W, const float *__restrict__ bias,
            float *__restrict__ out, float *__restrict__ outp, int L) {
    constexpr int CIN = CA + CB;
    constexpr int NCG = COUT / 8, NPG = TP / 8, NT = NCG * NPG;
    constexpr int XR = TP + 4;              // halo'd rows of the tile
    constexpr int XP = TP + 8;              // shared pitch (multiple of 4 floats)
    static_assert(CA % KC == 0 && CB % KC == 0 && KC % 4 == 0, "channel chunks must not straddle");
    constexpr int Q = KC / 4;               // float4 per halo'd row of a chunk
    __shared__ __align__(16) float xs[KC][XP];
    __shared__ __align__(16) float ws[5][KC][COUT];

    const int tid = threadIdx.x;
    const int cg = tid % NCG, pg = tid / NCG;
    const int e = blockIdx.y;
    const int p0 = blockIdx.x * TP;
    const int64_t rowsE = padded_rows(L);

    float acc[8][8];
#pragma unroll
    for (int qi = 0; qi < 8; ++qi) {
        const float b = bias[cg * 8 + qi];
#pragma unroll
        for (int pi = 0; pi < 8; ++pi) acc[pi][qi] = b;
    }

    for (int kc = 0; kc < CIN; kc += KC) {
        const bool fromA = kc < CA;
        const int C = fromA ? CA : CB;
        const int coff = fromA ? kc : kc - CA;
        const float *src = (fromA ? inA : inB) + (size_t)e * rowsE * C + coff;
        // tile row r <-> event row p0 - 2 + r <-> storage row p0 + r
        for (int idx = tid; idx < XR * Q; idx += NT) {
            const int r = idx / Q, c4 = idx % Q;
            const int64_t srow = (int64_t)p0 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (srow < rowsE) v = *reinterpret_cast<const float4 *>(src + srow * C + 4 * c4);
            xs[4 * c4 + 0][r] = v.x;
            xs[4 * c4 + 1][r] = v.y;
            xs[4 * c4 + 2][r] = v.z;
            xs[4 * c4 + 3][r] = v.w;
        }
        for (int idx = tid; idx < 5 * KC * COUT / 4; idx += NT) {
            const int t = idx / (KC * COUT / 4), rem = idx % (KC * COUT / 4);
            const int k = rem / (COUT / 4), c4 = rem % (COUT / 4);
            reinterpret_cast<float4 *>(&ws[t][k][0])[c4] =
                reinterpret_cast<const float4 *>(W + ((size_t)t * CIN + kc + k) * COUT)[c4];
        }
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < KC; ++k) {
            float xv[12];
            const float4 *xr = reinterpret_cast<const float4 *>(&xs[k][pg * 8]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float4 v = xr[i];
                xv[4 * i] = v.x; xv[4 * i + 1] = v.y; xv[4 * i + 2] = v.z; xv[4 * i + 3] = v.w;
            }
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                const float4 *wr = reinterpret_cast<const float4 *>(&ws[t][k][cg * 8]);
                const float4 wa = wr[0], wb = wr[1];
                const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int pi = 0; pi < 8; ++pi)
#pragma unroll
                    for (int qi = 0; qi < 8; ++qi) acc[pi][qi] = fmaf(xv[pi + t], wv[qi], acc[pi][qi]);
            }
        }
        __syncthreads();
    }

    float *ob = out + (size_t)e * rowsE * COUT;
#pragma unroll
    for (int pi = 0; pi < 8; ++pi) {
        const int p = p0 + pg * 8 + pi;
        if (p < L) {
            float4 *d = reinterpret_cast<float4 *>(ob + (size_t)(p + kPad) * COUT + cg * 8);
            d[0] = make_float4(leaky(acc[pi][0]), leaky(acc[pi][1]), leaky(acc[pi][2]), leaky(acc[pi][3]));
            d[1] = make_float4(leaky(acc[pi][4]), leaky(acc[pi][5]), leaky(acc[pi][6]), leaky(acc[pi][7]));
        }
    }
    if constexpr (POOL) {
        const int Lp = L / 2;
        float *pb = outp + (size_t)e * padded_rows(Lp) * COUT;
#pragma unroll
        for (int pi = 0; pi < 8; pi += 2) {
            const int p = p0 + pg * 8 + pi;
            if (p + 1 < L) {
                float v[8];
#pragma unroll
                for (int qi = 0; qi < 8; ++qi) v[qi] = fmaxf(leaky(acc[pi][qi]), leaky(acc[pi + 1][qi]));
                float4 *d = reinterpret_cast<float4 *>(pb + (size_t)(p / 2 + kPad) * COUT + cg * 8);
                d[0] = make_float4(v[0], v[1], v[2], v[3]);
                d[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
        }
    }
    // pad rows of this event: written by the first and the last tile
    // (a single tile is both: it writes both sides)
    const bool first = blockIdx.x == 0, last = blockIdx.x == gridDim.x - 1;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        if (!(side == 0 ? first : last)) continue;
        const int base = side == 0 ? 0 : L + kPad;
        for (int i = tid; i < 2 * COUT; i += NT) ob[(size_t)base * COUT + i] = 0.0f;
        if constexpr (POOL) {
            const int Lp = L / 2;
            float *pb = outp + (size_t)e * padded_rows(Lp) * COUT;
            const int pbase = side == 0 ? 0 : Lp + kPad;
            for (int i = tid; i < 2 * COUT; i += NT) pb[(size_t)pbase * COUT + i] = 0.0f;
        }
    }
}

// ConvTranspose1d k2 s2 + LeakyReLU: out[2i + r][co] = lrelu(b[co] + sum_ci W[ci][r][co] in[i][ci]).
// A GEMM per event with M = input positions, N = 2 * C_out (column n = r * C_out + co).
template <int CIN, int COUT, int TP>
__global__ void __launch_bounds__((TP / 8) * (2 * COUT / 8))
k_convT_f32(const float *__restrict__ in, const float *__restrict__ W,
            const float *__restrict__ bias, float *__restrict__ out, int Lin) {
    constexpr int N = 2 * COUT;
    constexpr int NCG = N / 8, NPG = TP / 8, NT = NCG * NPG;
    constexpr int XP = TP + 4;
    __shared__ __align__(16) float xs[kKC][XP];
    __shared__ __align__(16) float ws[kKC][N];

    const int tid = threadIdx.x;
    const int cg = tid % NCG, pg = tid / NCG;
    const int e = blockIdx.y;
    const int p0 = blockIdx.x * TP;
    const int64_t rowsIn = padded_rows(Lin);
    const int Lout = 2 * Lin;
    const int64_t rowsOut = padded_rows(Lout);
    const int rr = (cg * 8) / COUT;        // phase r of this thread's columns
    const int co0 = (cg * 8) % COUT;

    float acc[8][8];
#pragma unroll
    for (int qi = 0; qi < 8; ++qi) {
        const float b = bias[co0 + qi];
#pragma unroll
        for (int pi = 0; pi < 8; ++pi) acc[pi][qi] = b;
    }
    const float *src = in + (size_t)e * rowsIn * CIN;
    for (int kc = 0; kc < CIN; kc += kKC) {
        for (int idx = tid; idx < TP * (kKC / 4); idx += NT) {
            const int r = idx >> 2, c4 = idx & 3;
            const int p = p0 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p < Lin) v = *reinterpret_cast<const float4 *>(src + (size_t)(p + kPad) * CIN + kc + 4 * c4);
            xs[4 * c4 + 0][r] = v.x;
            xs[4 * c4 + 1][r] = v.y;
            xs[4 * c4 + 2][r] = v.z;
            xs[4 * c4 + 3][r] = v.w;
        }
        for (int idx = tid; idx < kKC * N / 4; idx += NT) {
            const int k = idx / (N / 4), c4 = idx % (N / 4);
            reinterpret_cast<float4 *>(&ws[k][0])[c4] =
                reinterpret_cast<const float4 *>(W + (size_t)(kc + k) * N)[c4];
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kKC; ++k) {
            const float4 *xr = reinterpret_cast<const float4 *>(&xs[k][pg * 8]);
            const float4 xa = xr[0], xb = xr[1];
            const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            const float4 *wr = reinterpret_cast<const float4 *>(&ws[k][cg * 8]);
            const float4 wa = wr[0], wb = wr[1];
            const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int pi = 0; pi < 8; ++pi)
#pragma unroll
                for (int qi = 0; qi < 8; ++qi) acc[pi][qi] = fmaf(xv[pi], wv[qi], acc[pi][qi]);
        }
        __syncthreads();
    }
    float *ob = out + (size_t)e * rowsOut * COUT;
#pragma unroll
    for (int pi = 0; pi < 8; ++pi) {
        const int i = p0 + pg * 8 + pi;
        if (i < Lin) {
            float4 *d = reinterpret_cast<float4 *>(ob + (size_t)(2 * i + rr + kPad) * COUT + co0);
            d[0] = make_float4(leaky(acc[pi][0]), leaky(acc[pi][1]), leaky(acc[pi][2]), leaky(acc[pi][3]));
            d[1] = make_float4(leaky(acc[pi][4]), leaky(acc[pi][5]), leaky(acc[pi][6]), leaky(acc[pi][7]));
        }
    }
    const bool first = blockIdx.x == 0, last = blockIdx.x == gridDim.x - 1;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {   // a single tile is both first and last
        if (!(side == 0 ? first : last)) continue;
        const int base = side == 0 ? 0 : Lout + kPad;
        for (int i = tid; i < 2 * COUT; i += NT) ob[(size_t)base * COUT + i] = 0.0f;
    }
}

template <int CA, int CB, int COUT, int TP, bool POOL, int KC = kKC>
cudaError_t conv5(const void *a, const void *b, const float *W, const float *bias, void *out,
                  void *outp, int L, int n, cudaStream_t s) {
    dim3 grid((L + TP - 1) / TP, n), block((TP / 8) * (COUT / 8));
    k_conv5_f32<CA, CB, COUT, TP, POOL, KC><<<grid, block, 0, s>>>(
        (const float *)a, (const float *)b, W, bias, (float *)out, (float *)outp, L);
    return cudaGetLastError();
}

template <int CIN, int COUT, int TP>
cudaError_t convT(const void *in, const float *W, const float *bias, void *out, int Lin, int n,
                  cudaStream_t s) {
    dim3 grid((Lin + TP - 1) / TP, n), block((TP / 8) * (2 * COUT / 8));
    k_convT_f32<CIN, COUT, TP><<<grid, block, 0, s>>>((const float *)in, W, bias, (float *)out, Lin);
    return cudaGetLastError();
}

// The layer sequence for base width C (levels C, 2C, 4C, 8C). Tiles halve as the channel
// counts double, so every CTA keeps (TP / 8) x (C_out / 8) = 128 threads; in the wide
// variant the 2C-, 4C- and 8C-input convolutions stage 8 channels per chunk so that their
// weights fit the 48 KB of static shared memory (enc4 at C = 32: 40 KB).
template <int C>
cudaError_t run_f32(const ConvF32Weights &w, const UnetBuffers &b, int n, cudaStream_t s,
                    const ProfHook *prof) {
    constexpr int KW = C > kC0 ? 8 : kKC;
    cudaError_t err;
#define PVF_TRY(name, x) do { ProfScope ps_(prof, name, s); err = (x); if (err != cudaSuccess) return err; } while (0)
    // each tensor is packed in its slot with its own per-event stride (L + 4) * C
    PVF_TRY("enc2", (conv5<C, 0, 2 * C, 256 * 16 / C, true>(b.s0, nullptr, w.w[0], w.b[0], b.e2, b.s1, 2000, n, s)));
    PVF_TRY("enc3", (conv5<2 * C, 0, 4 * C, 128 * 16 / C, true, KW>(b.s1, nullptr, w.w[1], w.b[1], b.e3, b.s0, 1000, n, s)));
    PVF_TRY("enc4", (conv5<4 * C, 0, 8 * C, 64 * 16 / C, false, KW>(b.s0, nullptr, w.w[2], w.b[2], b.deep, nullptr, 500, n, s)));
    PVF_TRY("up3", (convT<8 * C, 4 * C, 64 * 16 / C>(b.deep, w.uw[0], w.ub[0], b.up, 500, n, s)));
    PVF_TRY("dec3", (conv5<4 * C, 4 * C, 4 * C, 128 * 16 / C, false, KW>(b.up, b.e3, w.w[3], w.b[3], b.deep, nullptr, 1000, n, s)));
    PVF_TRY("up2", (convT<4 * C, 2 * C, 128 * 16 / C>(b.deep, w.uw[1], w.ub[1], b.up, 1000, n, s)));
    PVF_TRY("dec2", (conv5<2 * C, 2 * C, 2 * C, 256 * 16 / C, false>(b.up, b.e2, w.w[4], w.b[4], b.deep, nullptr, 2000, n, s)));
    PVF_TRY("up1", (convT<2 * C, C, 256 * 16 / C>(b.deep, w.uw[2], w.ub[2], b.up, 2000, n, s)));
    PVF_TRY("dec1", (conv5<C, C, C, 512 * 16 / C, false>(b.up, b.e1, w.w[5], w.b[5], b.deep, nullptr, 4000, n, s)));
#undef PVF_TRY
    return cudaSuccess;
}

// The per-interval layout: kSlices sequences of kIvLen bins per event (104, 52, 26, 13
// positions per level), each layer one small tile per sequence (32 threads per CTA).
template <int C>
cudaError_t run_f32_iv(const ConvF32Weights &w, const UnetBuffers &b, int n, cudaStream_t s,
                       const ProfHook *prof) {
    constexpr int L1 = kIvLen, L2 = L1 / 2, L3 = L1 / 4, L4 = L1 / 8;
    const int ns = n * kSlices;                  // at most 64000 (the plan caps the chunk)
    cudaError_t err;
#define PVF_TRY(name, x) do { ProfScope ps_(prof, name, s); err = (x); if (err != cudaSuccess) return err; } while (0)
    PVF_TRY("enc2", (conv5<C, 0, 2 * C, 64, true>(b.s0, nullptr, w.w[0], w.b[0], b.e2, b.s1, L2, ns, s)));
    PVF_TRY("enc3", (conv5<2 * C, 0, 4 * C, 32, true>(b.s1, nullptr, w.w[1], w.b[1], b.e3, b.s0, L3, ns, s)));
    PVF_TRY("enc4", (conv5<4 * C, 0, 8 * C, 16, false>(b.s0, nullptr, w.w[2], w.b[2], b.deep, nullptr, L4, ns, s)));
    PVF_TRY("up3", (convT<8 * C, 4 * C, 16>(b.deep, w.uw[0], w.ub[0], b.up, L4, ns, s)));
    PVF_TRY("dec3", (conv5<4 * C, 4 * C, 4 * C, 32, false>(b.up, b.e3, w.w[3], w.b[3], b.deep, nullptr, L3, ns, s)));
    PVF_TRY("up2", (convT<4 * C, 2 * C, 32>(b.deep, w.uw[1], w.ub[1], b.up, L3, ns, s)));
    PVF_TRY("dec2", (conv5<2 * C, 2 * C, 2 * C, 64, false>(b.up, b.e2, w.w[4], w.b[4], b.deep, nullptr, L2, ns, s)));
    PVF_TRY("up1", (convT<2 * C, C, 64>(b.deep, w.uw[2], w.ub[2], b.up, L2, ns, s)));
    PVF_TRY("dec1", (conv5<C, C, C, 128, false>(b.up, b.e1, w.w[5], w.b[5], b.deep, nullptr, L1, ns, s)));
#undef PVF_TRY
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_unet_f32(const ConvF32Weights &w, const UnetBuffers &b, int n, bool iv, cudaStream_t s,
                            const ProfHook *prof) {
    if (n <= 0) return cudaSuccess;
    if (iv) {
        if (w.c0 != kC0 || n * kSlices > 65535) return cudaErrorInvalidValue;
        return run_f32_iv<kC0>(w, b, n, s, prof);
    }
    if (w.c0 == kC0) return run_f32<kC0>(w, b, n, s, prof);
    if (w.c0 == kC0Max) return run_f32<kC0Max>(w, b, n, s, prof);
    return cudaErrorInvalidValue;
}

}  // namespace pvf
