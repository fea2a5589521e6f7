// Tensor-core (tcgen05) forms of the UNet: placeholder until the kernels land.
#include "pvf_tc.cuh"

namespace pvf {

size_t tc_weight_bytes(int) { return 0; }
bool tc_supported(int) { return false; }
bool tc_pack_weights(int, const std::vector<LayerF32> &, const float *, std::vector<unsigned char> &,
                     TcNet *, unsigned char *) {
    return false;
}
cudaError_t launch_unet_tc(const TcNet &, const UnetBuffers &, int, cudaStream_t, const ProfHook *) {
    return cudaErrorNotSupported;
}

}  // namespace pvf
