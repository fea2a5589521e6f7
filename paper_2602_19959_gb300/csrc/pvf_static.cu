// pvf_histogram_static: steps 1-2 of the path for callers that cannot allocate device
// memory. The kernel's scratch (the packed float32 FC weights and the per-event bypass
// flags) lives in a fixed array compiled into the library instead of a caller's pool.
#include <mutex>
#include <vector>

#include "pvf_internal.cuh"

namespace pvf {
namespace {

constexpr int kStaticMaxEvents = 4096;    // events per call
constexpr int kStaticMaxTracks = 2048;    // tracks per event; larger events are bypassed
constexpr size_t kOffFlags = 0;                                       // int32 [kStaticMaxEvents]
constexpr size_t kOffFc = kOffFlags + sizeof(int32_t) * kStaticMaxEvents;  // float [kFcFloats]
constexpr size_t kScratchBytes = (kOffFc + sizeof(float) * kFcFloats + 255) / 256 * 256;
static_assert(kScratchBytes == 48384, "size stated in include/pvf.h");

// Held by every GPU that loads the library, until the process exits. In host code this
// name is only a stand-in for the symbol, never a device address.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_dev[kMaxDevices];   // device address of g_scratch, per device
std::mutex g_scratch_mu;

// Device address of g_scratch on the current device, looked up once per device.
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_scratch);
        if (err != cudaSuccess) return err;
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace pvf

using namespace pvf;

extern "C" pvf_status pvf_histogram_static(const void *weights_blob, size_t blob_bytes,
                                           const pvf_tracks_soa *tracks, const int32_t *offsets,
                                           int32_t n_events, float *out_hist, int32_t *out_bypass,
                                           pvf_stream_t stream_) {
    if (n_events < 0 || n_events > kStaticMaxEvents) return PVF_ERR_INVALID_ARG;
    if (!tracks || tracks->n_tracks < 0) return PVF_ERR_INVALID_ARG;
    for (int k = 0; k < PVF_N_FEATURES; ++k)
        if (!tracks->f[k] || reinterpret_cast<uintptr_t>(tracks->f[k]) % 4) return PVF_ERR_INVALID_ARG;
    if (!offsets || reinterpret_cast<uintptr_t>(offsets) % 4 || !out_hist ||
        reinterpret_cast<uintptr_t>(out_hist) % 16 ||
        (out_bypass && reinterpret_cast<uintptr_t>(out_bypass) % 4))
        return PVF_ERR_INVALID_ARG;
    std::vector<float> fc(kFcFloats);
    const pvf_status st = pack_fc_from_blob(weights_blob, blob_bytes, fc.data());
    if (st != PVF_OK) return st;
    if (n_events == 0) return PVF_OK;

    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return PVF_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    // this call's weights overwrite the previous call's; the flags are written per event
    // by the kernel before they are read, so nothing needs clearing. The copy is from
    // pageable memory (this entry point allocates nothing, pinned staging included): the
    // runtime stages it before returning, which may wait for work queued on the stream.
    if (cudaMemcpyAsync(base + kOffFc, fc.data(), sizeof(float) * kFcFloats, cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return PVF_ERR_CUDA;
    FrontArgs a{};
    for (int k = 0; k < kFeatures; ++k) a.feat[k] = tracks->f[k];
    a.n_tracks = tracks->n_tracks;
    a.offsets = offsets;
    a.n_events = n_events;
    a.ev_base = 0;
    a.max_tracks = kStaticMaxTracks;
    a.fc = reinterpret_cast<const float *>(base + kOffFc);
    a.hist_out = out_hist;
    a.e1_inv_scale = 1.0f;
    a.ev_flag = out_bypass ? out_bypass : reinterpret_cast<int32_t *>(base + kOffFlags);
    a.status = nullptr;
    if (launch_front_hist_only(a, front_smem_bytes(kStaticMaxTracks, 0.0f), s) != cudaSuccess)
        return PVF_ERR_CUDA;
    return PVF_OK;
}
