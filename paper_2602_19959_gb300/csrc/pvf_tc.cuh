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

// Device pointers of the packed tensor-core weights inside the pool.
struct TcNet {
    int precision;
    const void *w[9];        // enc2, enc3, enc4, dec3, dec2, dec1, up3, up2, up1 (packed)
    const float *b[9];       // biases, float32
    const float *wscale[9];  // fp8: per-output-channel weight scales (null for bf16)
    float in_scale[9];       // fp8: per-tensor scale of each layer's input
    float out_inv_scale[9];  // fp8: 1 / scale of each layer's stored output
};

size_t tc_weight_bytes(int precision);
bool tc_supported(int precision);
// Packs the 9 tensor-core layers into host bytes destined for dev_base (offsets are
// computed for that device address) and fills net with the device pointers.
bool tc_pack_weights(int precision, const std::vector<LayerF32> &layers, const float *act_scale,
                     std::vector<unsigned char> &out, TcNet *net, unsigned char *dev_base);
cudaError_t launch_unet_tc(const TcNet &net, const UnetBuffers &b, int n_events, cudaStream_t s,
                           const ProfHook *prof);

}  // namespace pvf
