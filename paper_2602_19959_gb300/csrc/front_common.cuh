// Device code shared by the front kernels (k_front.cu: CUDA-core FC for the FP32 form and
// the static-scratch histogram; k_front_tc.cu: tcgen05 FC for the BF16 and FP8 forms):
// event validation, the stable slice sort, and enc1 + pool with its stores.
#pragma once

#include "pvf_internal.cuh"

namespace pvf {
namespace front {

__device__ __forceinline__ float softplus_f(float x) { return x > 20.0f ? x : log1pf(expf(x)); }

// Slice of a float32 z (round-to-nearest add and divide); -1 when outside [0, 40).
__device__ __forceinline__ int slice_of(float z) {
    float q = __fdiv_rn(__fadd_rn(z, 100.0f), 10.0f);
    if (!(q >= 0.0f && q < 40.0f)) return -1;
    return (int)floorf(q);
}

// Stores the 16 channels of storage row `row` of event e: channel-last float32 rows for
// the FP32 form, plane-major rows (two 16-bit planes / one e4m3 plane) otherwise.
template <class T>
__device__ __forceinline__ void store_row16(void *base, int64_t e, int64_t rows_e, int64_t row,
                                            const float v[kC0], float inv_scale) {
    if constexpr (sizeof(T) == 4) {
        float4 *d = reinterpret_cast<float4 *>(reinterpret_cast<float *>(base) + (e * rows_e + row) * kC0);
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (sizeof(T) == 2) {
        unsigned char *cb = reinterpret_cast<unsigned char *>(base);
        *reinterpret_cast<uint4 *>(cb + planar_off(e, 0, 2, rows_e, row)) = pack8<T>(v);
        *reinterpret_cast<uint4 *>(cb + planar_off(e, 1, 2, rows_e, row)) = pack8<T>(v + 8);
    } else {
        uint4 pk;
        pack_e4m3<16>(v, inv_scale, reinterpret_cast<uint32_t *>(&pk));
        unsigned char *cb = reinterpret_cast<unsigned char *>(base);
        *reinterpret_cast<uint4 *>(cb + planar_off(e, 0, 1, rows_e, row)) = pk;
    }
}

// Channels [16 g, 16 g + 16) of storage row `row` of event e in a plane-major tensor of C0
// channels (16-bit: planes 2 g and 2 g + 1 of C0 / 8; e4m3: plane g of C0 / 16).
template <class T, int C0>
__device__ __forceinline__ void store_seg16_pm(void *base, int64_t e, int64_t rows_e, int64_t row, int g,
                                               const float v[16], float inv_scale) {
    unsigned char *cb = reinterpret_cast<unsigned char *>(base);
    if constexpr (sizeof(T) == 2) {
        *reinterpret_cast<uint4 *>(cb + planar_off(e, 2 * g, C0 / 8, rows_e, row)) = pack8<T>(v);
        *reinterpret_cast<uint4 *>(cb + planar_off(e, 2 * g + 1, C0 / 8, rows_e, row)) = pack8<T>(v + 8);
    } else {
        uint4 pk;
        pack_e4m3<16>(v, inv_scale, reinterpret_cast<uint32_t *>(&pk));
        *reinterpret_cast<uint4 *>(cb + planar_off(e, g, C0 / 16, rows_e, row)) = pk;
    }
}

template <class T>
__device__ __forceinline__ void zero_row16(void *base, int64_t e, int64_t rows_e, int64_t row) {
    float z[kC0];
#pragma unroll
    for (int i = 0; i < kC0; ++i) z[i] = 0.0f;
    store_row16<T>(base, e, rows_e, row, z, 1.0f);
}

// Sorted entries: bits 0-13 hold the track's index within the event, bits 14-15 the
// slice the entry fills relative to the track's own: 0 its own, 1 the slice below, 2 the
// slice above (the second slice of a boundary track, §3). sslice[t] holds the track's own
// slice in bits 0-5 and that tag in bits 6-7; 255 marks a dropped track.
// Without boundary tracks (EDGE = false) an entry is the track index and sslice[t] its
// slice: the kernels are then instantiated without any of this decoding.
constexpr int kEntTrack = 0x3FFF;
template <bool EDGE>
__device__ __forceinline__ int entry_track(int en) {
    return EDGE ? (en & kEntTrack) : en;
}
template <bool EDGE>
__device__ __forceinline__ int entry_slice(int en, const uint8_t *sslice) {
    if constexpr (!EDGE) {
        return sslice[en];
    } else {
        const int d = en >> 14;
        return (int)(sslice[en & kEntTrack] & 63u) - (d & 1) + (d >> 1);
    }
}

// Steps a-c for event ge: validation (bypass flag), slice per track, stable counting
// sort by slice. On return (after a block barrier) ssorted[0..nvalid) holds the event's
// entries grouped by slice, sseg[s]..sseg[s+1] bounding slice s: within a slice, first
// the slice's own valid tracks in input order, then the boundary tracks of the two
// neighbouring slices that also fill it (a.edge > 0), in input order. A valid track of
// slice s whose slice-relative z (float32) is below a.edge also fills s - 1 (s > 0); one
// at or above a.edge_hi = 10 - a.edge also fills s + 1 (s < 39).
// EDGE = false: no boundary tracks (a.edge is 0). scnt/srun must hold 48 ints each.
// Every thread of the block must call this.
template <int NT, bool EDGE>
__device__ __forceinline__ void validate_sort(const FrontArgs &a, int ge, int tid, int *scnt, int *sseg,
                                              int *srun, uint16_t *ssorted, uint8_t *sslice,
                                              int64_t &t0_out, int &nvalid_out) {
    const int src = a.ev_index ? a.ev_index[ge] : ge;      // gathered events: store index
    const int64_t t0 = a.offsets[src], t1 = a.offsets[src + 1];
    const bool bypass = t0 < 0 || t1 < t0 || t1 > a.n_tracks || (t1 - t0) > a.max_tracks;
    const int n = bypass ? 0 : (int)(t1 - t0);
    if (tid == 0) {
        a.ev_flag[ge] = bypass ? 1 : 0;
        if (bypass) raise_status(a.status, PVF_WARN_EVENTS_SKIPPED);
    }
    if (tid < 48) { scnt[tid] = 0; srun[tid] = 0; }
    __syncthreads();
    // slice per track (integer counts through shared atomics: exact)
    for (int t = tid; t < n; t += NT) {
        const int64_t gt = t0 + t;
        bool finite = true;
#pragma unroll
        for (int k = 0; k < kFeatures; ++k) finite &= isfinite(a.feat[k][gt]);
        const float z = a.feat[2][gt];
        const int s = finite ? slice_of(z) : -1;
        int tag = 0;
        if (s >= 0) {
            atomicAdd(&scnt[s], 1);
            if constexpr (EDGE) {
                const float zr = __fsub_rn(z, -100.0f + 10.0f * (float)s);   // as feature 2
                if (s > 0 && zr < a.edge) tag = 1;
                else if (s < kSlices - 1 && zr >= a.edge_hi) tag = 2;
                if (tag) atomicAdd(&scnt[s - (tag & 1) + (tag >> 1)], 1);
            }
        }
        sslice[t] = s < 0 ? 255 : (uint8_t)(s | (tag << 6));
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int s = 0; s < kSlices; ++s) { sseg[s] = acc; acc += scnt[s]; }
        sseg[kSlices] = acc;
    }
    __syncthreads();
    // stable ranks by slice: warp 0 walks the tracks in input order, once for their own
    // slices and once more for the second slices of boundary tracks
    if (tid < 32) {
        const unsigned lane = tid;
#pragma unroll 1
        for (int pass = 0; pass < (EDGE ? 2 : 1); ++pass) {
            for (int base = 0; base < n; base += 32) {
                const int t = base + lane;
                int s = 255, en = t;
                if constexpr (!EDGE) {
                    if (t < n) s = sslice[t];
                } else if (t < n && sslice[t] != 255) {
                    const int own = sslice[t] & 63, tag = sslice[t] >> 6;
                    if (pass == 0) {
                        s = own;
                    } else if (tag) {
                        s = own - (tag & 1) + (tag >> 1);
                        en = t | (tag << 14);
                    }
                }
                const unsigned peers = __match_any_sync(0xffffffffu, s);
                const unsigned lower = peers & ((1u << lane) - 1u);
                int before = 0;
                if (s != 255) before = srun[s];
                __syncwarp();
                if (s != 255) {
                    ssorted[sseg[s] + before + __popc(lower)] = (uint16_t)en;
                    if (lower == 0) srun[s] = before + __popc(peers);
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    t0_out = t0;
    nvalid_out = sseg[kSlices];
}

// The nine features of track gt with feature 2 made slice-relative (exact offset).
__device__ __forceinline__ void track_features(const FrontArgs &a, int64_t gt, int s, float x[kFcInPad]) {
#pragma unroll
    for (int k = 0; k < kFeatures; ++k) x[k] = a.feat[k][gt];
    x[2] = __fsub_rn(x[2], -100.0f + 10.0f * (float)s);
#pragma unroll
    for (int k = kFeatures; k < kFcInPad; ++k) x[k] = 0.0f;
}

// Stores channels [8 h, 8 h + 8) of storage row `row` of event e: half a channel-last
// float32 row, one of the two 16-bit planes, or half of the e4m3 plane's 16-byte row.
template <class T>
__device__ __forceinline__ void store_half8(void *base, int64_t e, int64_t rows_e, int64_t row, int h,
                                            const float v[8], float inv_scale) {
    if constexpr (sizeof(T) == 4) {
        float4 *d = reinterpret_cast<float4 *>(reinterpret_cast<float *>(base) + (e * rows_e + row) * kC0 + 8 * h);
        d[0] = make_float4(v[0], v[1], v[2], v[3]);
        d[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else if constexpr (sizeof(T) == 2) {
        *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(base) + planar_off(e, h, 2, rows_e, row)) =
            pack8<T>(v);
    } else {
        uint2 pk;
        pack_e4m3<8>(v, inv_scale, reinterpret_cast<uint32_t *>(&pk));
        *reinterpret_cast<uint2 *>(reinterpret_cast<unsigned char *>(base) + planar_off(e, 0, 1, rows_e, row) + 8 * h) = pk;
    }
}

// Step f: e1 = LeakyReLU(conv_k5(hist) + b), p1 = maxpool2(e1), stored in the form's
// precision with the pad rows zeroed; calibration (AMAX) folds max |e1| into a.amax[0].
// Thread tid owns channels [8 h, 8 h + 8), h = tid & 1, of every position pair it takes,
// so its 40 weights and 8 biases stay in registers and the loop reads only the histogram
// from shared memory; the two threads of a pair write the two halves of each row.
// IV: the per-interval layout of the tensor-core forms: e1 and p1 hold the event's kSlices
// sequences end to end, each the conv of the interval's kIvLen-bin window (its bins with
// kIvPad zero bins on each side), two zero rows before each sequence and two after the
// last (neighbouring sequences share the two between them).
template <class T, int NT, bool AMAX, bool IV = false>
__device__ __forceinline__ void enc1_pool_t(const FrontArgs &a, int e, int tid, const float *shist,
                                            const float *senc) {
    static_assert(NT % 2 == 0, "thread pairs");
    constexpr int S1 = kIvLen + kPad, S2 = kIvLen / 2 + kPad;   // rows per sequence
    const int64_t rows1 = IV ? (int64_t)kSlices * S1 + kPad : padded_rows(kBins);
    const int64_t rows2 = IV ? (int64_t)kSlices * S2 + kPad : padded_rows(kBins / 2);
    constexpr int NQ = IV ? kSlices * (kIvLen / 2) : kBins / 2;         // position pairs
    const float inv = a.e1_inv_scale;
    const int h = tid & 1;
    float w[5][8], bias[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int t = 0; t < 5; ++t) w[t][j] = senc[t * kC0 + 8 * h + j];
        bias[j] = senc[5 * kC0 + 8 * h + j];
    }
    float vmax = 0.0f;
#pragma unroll 2   // two position pairs in flight per thread: front 81.6 -> 79.5 us (FP16)
    for (int qi = tid >> 1; qi < NQ; qi += NT / 2) {
        // the pair's sequence (IV) and first position; e1 rows r1, r1 + 1, p1 row r2
        const int sq = IV ? qi / (kIvLen / 2) : 0, q = IV ? qi % (kIvLen / 2) : qi;
        const int64_t r1 = (int64_t)sq * S1 * IV + 2 * q + kPad, r2 = (int64_t)sq * S2 * IV + q + kPad;
        float hv[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if constexpr (IV) {
                const int b = 2 * q + k - 2 - kIvPad;    // bin of the interval at window position
                hv[k] = (b >= 0 && b < kSliceBins) ? shist[sq * kSliceBins + b] : 0.0f;
            } else {
                const int p = 2 * q + k - 2;
                hv[k] = (p >= 0 && p < kBins) ? shist[p] : 0.0f;
            }
        }
        float v0[8], v1[8], vp[8];
        // channel pairs (j, j + 1) as one packed two-lane FMA (each lane an fmaf, in the
        // same tap order): half the FMA instructions, identical results
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            float2 a0 = make_float2(bias[j], bias[j + 1]), a1 = a0;
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                const float2 wt = make_float2(w[t][j], w[t][j + 1]);
                a0 = __ffma2_rn(wt, make_float2(hv[t], hv[t]), a0);
                a1 = __ffma2_rn(wt, make_float2(hv[t + 1], hv[t + 1]), a1);
            }
            v0[j] = leaky(a0.x); v0[j + 1] = leaky(a0.y);
            v1[j] = leaky(a1.x); v1[j + 1] = leaky(a1.y);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            vp[j] = fmaxf(v0[j], v1[j]);
            if constexpr (AMAX) vmax = fmaxf(vmax, fmaxf(fabsf(v0[j]), fabsf(v1[j])));
        }
        store_half8<T>(a.e1, e, rows1, r1, h, v0, inv);
        store_half8<T>(a.e1, e, rows1, r1 + 1, h, v1, inv);
        store_half8<T>(a.p1, e, rows2, r2, h, vp, inv);
    }
    if constexpr (AMAX) {   // calibration: integer max on the float bits (order-independent)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if ((tid & 31) == 0) atomicMax(reinterpret_cast<int *>(a.amax), __float_as_int(vmax));
    }
    if constexpr (IV) {     // the two rows before each sequence and the two after the last
        for (int idx = tid; idx < (kSlices + 1) * 2; idx += NT) {
            const int sq = idx >> 1, k = idx & 1;
            zero_row16<T>(a.e1, e, rows1, (int64_t)sq * S1 + k);
            zero_row16<T>(a.p1, e, rows2, (int64_t)sq * S2 + k);
        }
    } else if (tid < 4) {
        const int r = tid < 2 ? tid : kBins + tid;             // rows 0,1 and L+2, L+3
        zero_row16<T>(a.e1, e, rows1, r);
        const int rp = tid < 2 ? tid : kBins / 2 + tid;
        zero_row16<T>(a.p1, e, rows2, rp);
    }
}

// Channels [16 g, 16 g + 16) of storage row `row` of event e in a channel-last float32
// tensor of C0 channels.
template <int C0>
__device__ __forceinline__ void store_seg16_f32(void *base, int64_t e, int64_t rows_e, int64_t row, int g,
                                                const float v[16]) {
    float4 *d = reinterpret_cast<float4 *>(reinterpret_cast<float *>(base) + (e * rows_e + row) * C0 + 16 * g);
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// Step f with the weights read from shared memory per position pair, for the float32 front,
// whose FC registers leave no room for them (same arithmetic, same order). senc holds
// W[t][co] (5 C0 floats) then b[co]; the C0 channels are produced 16 at a time. A width
// above 16 exists only in the float32 form.
template <class T, int NT, bool AMAX, int C0>
__device__ __forceinline__ void enc1_pool_shared_t(const FrontArgs &a, int e, int tid, const float *shist,
                                                   const float *senc) {
    static_assert(C0 % 16 == 0, "16-channel segments");
    const int64_t rows1 = padded_rows(kBins), rows2 = padded_rows(kBins / 2);
    const float inv = a.e1_inv_scale;
    float vmax = 0.0f;
    for (int q = tid; q < kBins / 2; q += NT) {
        float hv[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int p = 2 * q + k - 2;
            hv[k] = (p >= 0 && p < kBins) ? shist[p] : 0.0f;
        }
#pragma unroll 1
        for (int g = 0; g < C0 / 16; ++g) {
            float v0[16], v1[16], vp[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int co = 16 * g + j;
                float a0 = senc[5 * C0 + co], a1 = a0;
#pragma unroll
                for (int t = 0; t < 5; ++t) {
                    a0 = fmaf(senc[t * C0 + co], hv[t], a0);
                    a1 = fmaf(senc[t * C0 + co], hv[t + 1], a1);
                }
                v0[j] = leaky(a0);
                v1[j] = leaky(a1);
                vp[j] = fmaxf(v0[j], v1[j]);
                if constexpr (AMAX) vmax = fmaxf(vmax, fmaxf(fabsf(v0[j]), fabsf(v1[j])));
            }
            if constexpr (C0 == kC0) {
                store_row16<T>(a.e1, e, rows1, 2 * q + kPad, v0, inv);
                store_row16<T>(a.e1, e, rows1, 2 * q + 1 + kPad, v1, inv);
                store_row16<T>(a.p1, e, rows2, q + kPad, vp, inv);
            } else if constexpr (sizeof(T) == 4) {
                store_seg16_f32<C0>(a.e1, e, rows1, 2 * q + kPad, g, v0);
                store_seg16_f32<C0>(a.e1, e, rows1, 2 * q + 1 + kPad, g, v1);
                store_seg16_f32<C0>(a.p1, e, rows2, q + kPad, g, vp);
            } else {   // the wide network in the tensor-core forms: plane-major segments
                store_seg16_pm<T, C0>(a.e1, e, rows1, 2 * q + kPad, g, v0, inv);
                store_seg16_pm<T, C0>(a.e1, e, rows1, 2 * q + 1 + kPad, g, v1, inv);
                store_seg16_pm<T, C0>(a.p1, e, rows2, q + kPad, g, vp, inv);
            }
        }
    }
    if constexpr (AMAX) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if ((tid & 31) == 0) atomicMax(reinterpret_cast<int *>(a.amax), __float_as_int(vmax));
    }
    if (tid < 4) {
        const int r = tid < 2 ? tid : kBins + tid;
        const int rp = tid < 2 ? tid : kBins / 2 + tid;
        if constexpr (C0 == kC0) {
            zero_row16<T>(a.e1, e, rows1, r);
            zero_row16<T>(a.p1, e, rows2, rp);
        } else {
            float z[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) z[i] = 0.0f;
            for (int g = 0; g < C0 / 16; ++g) {
                if constexpr (sizeof(T) == 4) {
                    store_seg16_f32<C0>(a.e1, e, rows1, r, g, z);
                    store_seg16_f32<C0>(a.p1, e, rows2, rp, g, z);
                } else {
                    store_seg16_pm<T, C0>(a.e1, e, rows1, r, g, z, 1.0f);
                    store_seg16_pm<T, C0>(a.p1, e, rows2, rp, g, z, 1.0f);
                }
            }
        }
    }
}

// Step f in the per-interval layout (float32 form): e1 and p1 hold kSlices sequences per
// event (sequence e * kSlices + s = interval s), each the conv of the interval's kIvLen-bin
// window -- the interval's bins with kIvPad zero bins on each side -- with zero padding
// beyond the window, as each interval runs the UNet on its own. Same arithmetic per
// position as enc1_pool_shared_t.
template <int NT, int C0>
__device__ __forceinline__ void enc1_pool_windows_f32(const FrontArgs &a, int e, int tid, const float *shist,
                                                      const float *senc) {
    constexpr int Q = kIvLen / 2;                 // position pairs per window
    const int64_t rows1 = padded_rows(kIvLen), rows2 = padded_rows(kIvLen / 2);
    for (int idx = tid; idx < kSlices * Q; idx += NT) {
        const int s = idx / Q, q = idx % Q;
        const int64_t seq = (int64_t)e * kSlices + s;
        float hv[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int b = 2 * q + k - 2 - kIvPad;     // bin of the interval at window position 2q + k - 2
            hv[k] = (b >= 0 && b < kSliceBins) ? shist[s * kSliceBins + b] : 0.0f;
        }
#pragma unroll 1
        for (int g = 0; g < C0 / 16; ++g) {
            float v0[16], v1[16], vp[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int co = 16 * g + j;
                float a0 = senc[5 * C0 + co], a1 = a0;
#pragma unroll
                for (int t = 0; t < 5; ++t) {
                    a0 = fmaf(senc[t * C0 + co], hv[t], a0);
                    a1 = fmaf(senc[t * C0 + co], hv[t + 1], a1);
                }
                v0[j] = leaky(a0);
                v1[j] = leaky(a1);
                vp[j] = fmaxf(v0[j], v1[j]);
            }
            store_seg16_f32<C0>(a.e1, seq, rows1, 2 * q + kPad, g, v0);
            store_seg16_f32<C0>(a.e1, seq, rows1, 2 * q + 1 + kPad, g, v1);
            store_seg16_f32<C0>(a.p1, seq, rows2, q + kPad, g, vp);
        }
    }
    // the pad rows of every window: 0, 1 and L + 2, L + 3
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.0f;
    for (int idx = tid; idx < kSlices * 4; idx += NT) {
        const int s = idx >> 2, k = idx & 3;
        const int64_t seq = (int64_t)e * kSlices + s;
        const int r = k < 2 ? k : kIvLen + k, rp = k < 2 ? k : kIvLen / 2 + k;
        for (int g = 0; g < C0 / 16; ++g) {
            store_seg16_f32<C0>(a.e1, seq, rows1, r, g, z);
            store_seg16_f32<C0>(a.p1, seq, rows2, rp, g, z);
        }
    }
}

// REGW: weights in registers (tensor-core front, width 16) or read from shared memory
// (float32 front, width C0).
template <class T, int NT, bool REGW = true, int C0 = kC0, bool IV = false>
__device__ __forceinline__ void enc1_pool(const FrontArgs &a, int e, int tid, const float *shist,
                                          const float *senc) {
    if constexpr (REGW) {
        static_assert(C0 == kC0, "register weights for width 16");
        if (a.amax) enc1_pool_t<T, NT, true, IV>(a, e, tid, shist, senc);
        else enc1_pool_t<T, NT, false, IV>(a, e, tid, shist, senc);
    } else {
        if (a.amax) enc1_pool_shared_t<T, NT, true, C0>(a, e, tid, shist, senc);
        else enc1_pool_shared_t<T, NT, false, C0>(a, e, tid, shist, senc);
    }
}

}  // namespace front
}  // namespace pvf
