// Interface of the tensor-core (tcgen05) forms of the UNet: weight packing at creation
// and the per-chunk launch sequence.
#pragma once

#include <vector>

#include "pvf_internal.cuh"

namespace pvf {

// A float32 master layer as read from the weight blob (PyTorch layouts).
struct LayerF32 {
    const float *w, *b;
    uint32_t shape[3];
};

// FP8 per-tensor activation scales (value = stored e4m3 x scale). The two halves of a
// skip concat feed one accumulator column, so they share a scale:
enum {
    kScaleL1 = 0,   // e1, p1, u1 (level 1, 16 channels)
    kScaleL2 = 1,   // e2, p2, u2
    kScaleL3 = 2,   // e3, p3, u3
    kScaleE4 = 3,   // e4 (shared-memory operand of the fused up3 GEMM)
    kScaleD3 = 4,   // d3 (operand of the fused up2 GEMM)
    kScaleD2 = 5,   // d2 (operand of the fused up1 GEMM)
    kScaleD1 = 6,   // d1 (input of the final conv)
    kNumScales = 7
};

// Device pointers of the packed tensor-core weights inside the pool.
struct TcNet {
    int precision;
    const void *w[9];        // enc2, enc3, enc4, dec3, dec2, dec1, up3, up2, up1 (packed)
    const float *b[9];       // biases, float32
    const float *wscale[9];  // per-accumulator-column dequantisation scales (fp8)
    float act_scale[PVF_N_ACT_SCALES];
    const float *final_w;    // final conv (float32, W[t][ci] then b)
    const unsigned char *fc_img;   // bf16 FC operand images (kFcImgBytes)
    float *amax;             // calibration capture (kNumScales floats) or null
    int32_t *status;         // device status word
    int32_t *sched;          // 6 x 2 tile-scheduler counters (zero between launches)
    int32_t ctas_per_sm[6];  // launch schedule per conv kernel (0 = as many as fit)
    int32_t iv;              // per-interval layout (kSlices sequences per event)
    int32_t c0;              // UNet base width (16, or 32: the wide network)
};

size_t tc_weight_bytes(int precision, int c0);
bool tc_supported(int precision);
// Packs the 9 tensor-core layers into host bytes destined for dev_base (offsets are
// computed for that device address) and fills net with the device pointers.
bool tc_pack_weights(int precision, const std::vector<LayerF32> &layers, const float *act_scale,
                     std::vector<unsigned char> &out, TcNet *net, unsigned char *dev_base);
// n_dyn (nullable): device-side event count of the call, of which this launch covers
// events [dyn_base, dyn_base + n_events) (see launch_events).
cudaError_t launch_unet_tc(const TcNet &net, const UnetBuffers &b, int n_events, const int32_t *n_dyn,
                           int dyn_base, cudaStream_t s, const ProfHook *prof);
// Tests of the bounded waits: the enc2 kernel with its MMA thread waiting stall_us on a
// barrier that nothing arrives on (it records PVF_ERR_TIMEOUT and unwinds).
cudaError_t launch_stall_test_tc(const TcNet &net, const UnetBuffers &b, int n_events, uint32_t stall_us,
                                 cudaStream_t s);

}  // namespace pvf
