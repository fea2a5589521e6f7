// Internal definitions shared by the libpvf CUDA translation units.
//
// Data layout in the device pool (all offsets planned once at pvf_create):
//   * weights, converted from the float32 master blob into per-kernel layouts;
//   * per-event state: a bypass flag per event, the histogram rows when requested;
//   * UNet activations for one chunk of events, channel-last with two zero pad rows on
//     each side of every event: element (event e, position p, channel c) of a tensor
//     with L positions and C channels sits at row e * (L + 4) + p + 2, column c.
//     Producers write their own pad rows, so buffers can be reused by later layers.
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "pvf.h"

namespace pvf {

// Geometry of the method (§2): 400 mm region, 40 slices (intervals) of 100 bins.
constexpr int kBins = 4000;
constexpr int kSlices = 40;
constexpr int kSliceBins = 100;
constexpr int kFeatures = 9;
constexpr int kFcHidden = 32;
constexpr int kFcOut = 100;
constexpr int kFcInPad = 12;   // layer-1 input padded to a multiple of 4 floats
constexpr int kC0 = 16;        // UNet base width; levels have 16, 32, 64, 128 channels
constexpr int kC0Max = 32;     // widest variant (float32 form only): 32, 64, 128, 256
// Per-interval layout (float32 form): each interval is a sequence of kIvLen bins, its
// kSliceBins bins with kIvPad zero bins on each side (the fewest that survive 3 poolings).
constexpr int kIvPad = 2;
constexpr int kIvLen = kSliceBins + 2 * kIvPad;
static_assert(kIvLen % 8 == 0, "three 2:1 poolings");
constexpr int kPad = 2;        // zero rows on each side of an event (k5 "same" padding)
constexpr float kZLo = -100.0f;
constexpr float kBinW = 0.1f;
constexpr float kThreshold = 0.01f;
constexpr int kPeakHalfWin = 5;
constexpr int kCentroidHalf = 3;

// FC weights in float32. Layers 1-5: W[out][in] row-major, layer 1 padded to 12 inputs;
// layer 6 transposed, W6T[in][out] (bin-parallel output layer); then all biases.
constexpr int kFcW1 = kFcHidden * kFcInPad;          // 384
constexpr int kFcWH = kFcHidden * kFcHidden;         // 1024
constexpr int kFcW6 = kFcOut * kFcHidden;            // 3200
constexpr int kFcWTotal = kFcW1 + 4 * kFcWH + kFcW6; // 7680
constexpr int kFcBTotal = 5 * kFcHidden + kFcOut;    // 260
constexpr int kFcFloats = kFcWTotal + kFcBTotal;     // 7940

// Offsets inside the packed FC block (floats).
__host__ __device__ constexpr int fc_w_off(int l) {
    return l == 0 ? 0 : (l < 5 ? kFcW1 + (l - 1) * kFcWH : kFcW1 + 4 * kFcWH);
}
__host__ __device__ constexpr int fc_b_off(int l) {
    return kFcWTotal + (l < 5 ? l * kFcHidden : 5 * kFcHidden);
}

// FC weights of the tensor-core forms: bf16 images of K-major tcgen05 operands (planes of
// 8 inputs x rows x 16 bytes). Layers 1-5 are B operands with N = 32 rows (layer 1:
// K = 16, nine features then zeros; layers 2-5: K = 32). Layer 6 is the A operand of the
// transposed product (outputs on TMEM lanes): M = 128 rows, K = 32, output o on row
// 32 (o / 25) + o % 25 so that each warp's lane quarter holds 25 outputs; other rows zero.
constexpr int kFcM6 = 128;
constexpr int kFcOutPerWarp = 25;
__host__ __device__ constexpr int fc6_row(int o) { return 32 * (o / kFcOutPerWarp) + o % kFcOutPerWarp; }
constexpr int kFcImgW1 = 2 * kFcHidden * 16;
constexpr int kFcImgWH = 4 * kFcHidden * 16;
constexpr int kFcImgW6 = 4 * kFcM6 * 16;
constexpr int kFcImgBytes = kFcImgW1 + 4 * kFcImgWH + kFcImgW6;   // 17408
__host__ __device__ constexpr int fc_img_off(int l) {
    return l == 0 ? 0 : (l < 5 ? kFcImgW1 + (l - 1) * kFcImgWH : kFcImgW1 + 4 * kFcImgWH);
}

// enc1 (1 -> 16, k5) in float32: W[t][co] then b[co].
constexpr int kEnc1Floats = 5 * kC0 + kC0;
constexpr int kEnc1FloatsMax = 6 * kC0Max;
// final (16 -> 1, k5) in float32: W[t][ci] then b.
constexpr int kFinalFloats = 5 * kC0 + 1;
constexpr int kFinalFloatsMax = 5 * kC0Max + 1;

// Device status word values are pvf_status codes; kernels raise them with atomicMax
// (an integer maximum: order-independent).
__device__ __forceinline__ void raise_status(int32_t *word, int32_t s) {
    if (word) atomicMax(word, s);
}

__device__ __forceinline__ float leaky(float x) { return x > 0.0f ? x : 0.01f * x; }

// Storage element of an activation tensor for each precision form.
template <int PREC> struct Elem;
template <> struct Elem<PVF_FP32> { using T = float; };
template <> struct Elem<PVF_BF16> { using T = __nv_bfloat16; };
template <> struct Elem<PVF_FP8_E4M3> { using T = __nv_fp8_e4m3; };
template <> struct Elem<PVF_FP16> { using T = __half; };

// The 16-bit tensor-core forms (tcgen05 kind::f16 with bf16 or f16 operands).
__host__ __device__ constexpr bool is16(int prec) { return prec == PVF_BF16 || prec == PVF_FP16; }

// Two floats rounded to nearest even as one 32-bit pair of T (lo in the low half). The
// f16 conversion saturates to the largest finite value, +-65504, and keeps NaN.
template <class T> __device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&b);
}
template <> __device__ __forceinline__ uint32_t pack2<__half>(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
// 8 floats as one 16-byte row of T.
template <class T> __device__ __forceinline__ uint4 pack8(const float *v) {
    return make_uint4(pack2<T>(v[0], v[1]), pack2<T>(v[2], v[3]), pack2<T>(v[4], v[5]), pack2<T>(v[6], v[7]));
}

template <class T> __device__ __forceinline__ T to_elem(float v, float inv_scale);
template <> __device__ __forceinline__ float to_elem<float>(float v, float) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_elem<__nv_bfloat16>(float v, float) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half to_elem<__half>(float v, float) {
    return __ushort_as_half((unsigned short)(pack2<__half>(v, 0.0f) & 0xFFFFu));
}
template <> __device__ __forceinline__ __nv_fp8_e4m3 to_elem<__nv_fp8_e4m3>(float v, float inv) {
    return __nv_fp8_e4m3(v * inv);   // saturating round-to-nearest-even
}
template <class T> __device__ __forceinline__ float from_elem(T v, float scale);
template <> __device__ __forceinline__ float from_elem<float>(float v, float) { return v; }
template <> __device__ __forceinline__ float from_elem<__nv_bfloat16>(__nv_bfloat16 v, float) {
    return __bfloat162float(v);
}
template <> __device__ __forceinline__ float from_elem<__half>(__half v, float) {
    return __half2float(v);
}
template <> __device__ __forceinline__ float from_elem<__nv_fp8_e4m3>(__nv_fp8_e4m3 v, float s) {
    return float(v) * s;
}

// Events one launch processes. Without a device-side count (n_dyn null) that is the
// launch's n_events. With one, *n_dyn is the event count of the whole call, read at run
// time (so a captured graph serves any count up to its capacity), and the launch, which
// covers events [base, base + n_events) of the call, processes the part below that count.
// The word is written before the launch (by the host or by an earlier kernel of the
// stream), so a volatile load sees the current value.
__device__ __forceinline__ int launch_events(const int32_t *n_dyn, int base, int n_events) {
    if (!n_dyn) return n_events;
    const int n = *reinterpret_cast<const volatile int32_t *>(n_dyn) - base;
    return n < 0 ? 0 : (n > n_events ? n_events : n);
}

// Rows per event of a padded activation tensor with L positions.
__host__ __device__ __forceinline__ int64_t padded_rows(int L) { return (int64_t)L + 2 * kPad; }

// Plane-major layout of the tensor-core forms: a tensor with C channels is stored as
// C / PW planes of 16-byte rows (PW = 16 / element size channels per row):
//   byte offset of (event e, plane k, storage row r) = ((e * P + k) * rows_per_event + r) * 16
// so a plane of an event is one contiguous run of rows, which a single bulk copy moves
// into the shared-memory operand layout of tcgen05.
__host__ __device__ __forceinline__ size_t planar_off(int64_t e, int k, int planes, int64_t rows_e,
                                                      int64_t row) {
    return ((size_t)(e * planes + k) * (size_t)rows_e + (size_t)row) * 16;
}

// e4m3 codes of v[0..N) * inv_scale packed four to a word (v[4 i] in the low byte of
// out[i]), two per conversion instruction (round to nearest even, saturating to the
// largest finite value, as __nv_fp8_e4m3(float)).
template <int N>
__device__ __forceinline__ void pack_e4m3(const float *v, float inv_scale, uint32_t *out) {
    static_assert(N % 4 == 0, "whole words");
#pragma unroll
    for (int i = 0; i < N; i += 4) {
        const __nv_fp8x2_storage_t lo =
            __nv_cvt_float2_to_fp8x2(make_float2(v[i] * inv_scale, v[i + 1] * inv_scale), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t hi =
            __nv_cvt_float2_to_fp8x2(make_float2(v[i + 2] * inv_scale, v[i + 3] * inv_scale), __NV_SATFINITE,
                                     __NV_E4M3);
        out[i / 4] = (uint32_t)lo | ((uint32_t)hi << 16);
    }
}

// ---------------------------------------------------------------- kernel arguments

struct FrontArgs {
    const float *feat[kFeatures];
    const int32_t *offsets;      // global offsets array (n_total_events + 1)
    int64_t n_tracks;            // length of every feature array
    int32_t n_events;            // events in this launch
    int32_t ev_base;             // global index of the launch's first event
    int32_t max_tracks;          // per-event cap
    int32_t c0;                  // UNet base width (16, or 32 in the float32 form)
    int32_t iv;                  // per-interval layout: e1 / p1 as kSlices sequences per event
    float edge;                  // boundary-track width in mm (0: every track in one slice)
    float edge_hi;               // 10 - edge, rounded to float
    const float *fc;             // packed FC block (kFcFloats); its biases serve both forms
    const unsigned char *fc_img; // tensor-core forms: bf16 FC operand images (kFcImgBytes)
    const float *enc1;           // kEnc1Floats
    const float *hist_in;        // non-null: skip steps 1-2, read histograms (global rows)
    float *hist_out;             // nullable, global rows [ev_base + e]
    void *e1;                    // chunk-local padded [n][4004][16]
    void *p1;                    // chunk-local padded [n][2004][16]
    float e1_inv_scale;          // fp8 only: 1 / scale of e1/p1
    float *amax;                 // calibration: max |e1| into amax[0], or null
    int32_t *ev_flag;            // global [max_events]: 1 = bypassed
    int32_t *status;
    const int32_t *ev_index;     // nullable: event e of the call is event ev_index[e] of the
                                 // offsets array (a gather from a larger event store)
    const int32_t *n_dyn;        // nullable: device-side event count of the call (any memory
                                 // the device reads; see launch_events)
    int32_t *n_dyn_copy;         // with n_dyn: pool word that receives *n_dyn, which the
                                 // later kernels of the call read from device memory
    int32_t ctas_per_sm;         // launch schedule: 0 = as many as fit
    int32_t *ev_ctr;             // tensor-core front: the next-event ticket, a pool word
                                 // that is zero between launches; null: static stride
};

struct TailArgs {
    const void *d1;              // chunk-local padded [n][4004][c0], or null for logit_in
    const float *logit_in;       // non-null: peaks only, read logits
    int32_t logit_in_base;       // event index of logit_in's first row (0: global rows)
    float d1_scale;              // fp8 only
    const float *final_w;        // 5 c0 + 1 floats: W[t][ci], then b
    int32_t c0;                  // width of d1 (16, or 32 in the float32 form)
    int32_t iv;                  // per-interval layout: d1 holds kSlices sequences per event
    int32_t n_events;
    int32_t ev_base;
    const int32_t *ev_flag;      // nullable (all events valid)
    float *logit_out;            // nullable, global rows
    float *pv_z;                 // global [n_total][max_pv]
    int32_t *pv_count;           // global [n_total]
    int32_t max_pv;
    int32_t *status;
    const int32_t *n_dyn;        // nullable: device-side event count of the call
    int32_t ctas_per_sm;         // launch schedule: 0 = as many as fit
};

// Optional per-launch timing hook: begin/end bracket one kernel launch on stream s.
struct ProfHook {
    void (*begin)(void *ctx, const char *name, cudaStream_t s);
    void (*end)(void *ctx, cudaStream_t s);
    void *ctx;
};
struct ProfScope {
    const ProfHook *h;
    cudaStream_t s;
    ProfScope(const ProfHook *hook, const char *name, cudaStream_t st) : h(hook), s(st) {
        if (h) h->begin(h->ctx, name, s);
    }
    ~ProfScope() { if (h) h->end(h->ctx, s); }
};

// Launch with programmatic stream serialization: the kernel may start while the previous
// kernel of the stream finishes; it must call griddepcontrol.wait before reading that
// kernel's output, and triggers its own dependents only after that wait, so at most two
// kernels share the GPU and the earlier one is always fully resident.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Per-device launch set-up (csrc/launch_setup.cu), thread-safe: the SM count of the
// current device, and a kernel's attributes on the current device with its dynamic
// shared-memory limit raised to at least smem_bytes there (once per kernel and device).
cudaError_t current_device_sms(int *sms);
cudaError_t prepare_kernel(const void *kernel, size_t smem_bytes, cudaFuncAttributes *attr);

// Host-side launchers (defined in the kernel translation units).
cudaError_t launch_front(const FrontArgs &a, int precision, size_t smem_bytes, cudaStream_t s);
// Sorted (track, slice) entries an event may hold: boundary tracks (§3) fill a second
// slice, so up to two per track when the boundary width is non-zero.
__host__ __device__ __forceinline__ int front_entries(int max_tracks, float edge) {
    return edge > 0.0f ? 2 * max_tracks : max_tracks;
}
size_t front_smem_bytes(int max_tracks, float edge);
// Steps 1-2 + enc1 with the FC on tcgen05 (BF16 and FP8 forms).
cudaError_t launch_front_tc(const FrontArgs &a, int precision, cudaStream_t s);
// Steps 1-2 only (validate, sort, FC, histogram into a.hist_out), float32; e1/p1 unused.
cudaError_t launch_front_hist_only(const FrontArgs &a, size_t smem_bytes, cudaStream_t s);
// Reads a "PVFW" blob and writes the packed float32 FC block (kFcFloats floats) to out.
pvf_status pack_fc_from_blob(const void *blob, size_t bytes, float *out);
cudaError_t launch_tail(const TailArgs &a, int precision, cudaStream_t s);

struct ConvF32Weights {
    int c0;                       // base width: 16 or 32
    const float *w[6], *b[6];     // enc2, enc3, enc4, dec3, dec2, dec1: W[5][Cin][Cout]
    const float *uw[3], *ub[3];   // up3, up2, up1: W[Cin][2][Cout]
};
// Activation slots of one chunk of events, assigned by liveness (layer order: front,
// enc2, enc3, enc4, up3, dec3, up2, dec2, up1, dec1, tail):
//   big slots (kBigElems per event):   e1 | e2 | e3 | deep = e4, d3, d2, d1 | up = u3, u2, u1
//   small slots (kSmallElems per event): s0 = p1, p3 | s1 = p2
// (for base width 16; a width-32 network doubles both)
// Inside its slot a tensor is packed with its own per-event stride (L + 4) * C, which is
// never larger than the slot's per-event size.
constexpr int64_t kBigElems = 504 * 128;    // largest of (L + 4) * C over the big tensors
constexpr int64_t kSmallElems = 504 * 64;   // largest over p1, p2, p3
struct UnetBuffers {
    void *e1, *e2, *e3, *deep, *up, *s0, *s1;
    float *logits;   // tensor-core forms: final-conv output of the chunk, [n][4000]
};
// iv: per-interval layout (kSlices sequences of kIvLen bins per event).
cudaError_t launch_unet_f32(const ConvF32Weights &w, const UnetBuffers &b, int n_events, bool iv,
                            cudaStream_t s, const ProfHook *prof);

}  // namespace pvf

// Plan values of a handle, for the host runtime in other translation units.
int pvf_handle_max_pv(const pvf_handle *h);
int pvf_handle_max_events(const pvf_handle *h);
int pvf_handle_precision(const pvf_handle *h);
// A dynamic-count graph (pvf_graph_create_dynamic) whose event e is event ev_index[e] of a
// larger store (tracks and store_offsets index the store; ev_index and n_events are read
// on the device at each launch). For the serving loop.
// (C linkage, not exported: the library is built with hidden visibility.)
extern "C" pvf_status graph_create_gather(pvf_handle *h, const pvf_tracks_soa *store,
                                          const int32_t *store_offsets, const int32_t *ev_index,
                                          const int32_t *n_events, int32_t max_n_events, float *pv_z,
                                          int32_t *pv_count, pvf_graph **out);
