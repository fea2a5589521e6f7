// Per-device launch set-up of the library's kernels.
//
// A kernel's dynamic shared-memory limit (cudaFuncAttributeMaxDynamicSharedMemorySize)
// is a property of the kernel on one device: raising it on device 0 leaves it at the
// default on device 1. The SM count that sizes the persistent grids is also a property
// of the device. Both are cached here per (kernel, device) and per device, behind a
// mutex, so that handles on different devices and calls from different threads each
// see the set-up of their own current device.
#include <map>
#include <mutex>
#include <utility>

#include "pvf_internal.cuh"

namespace pvf {
namespace {

struct KernelState {
    size_t smem_limit = 0;       // largest dynamic shared memory set so far on this device
    cudaFuncAttributes attr{};
};

std::mutex g_mu;
std::map<int, int> g_sms;                                        // device -> SM count
std::map<std::pair<const void *, int>, KernelState> g_kernels;   // (kernel, device)

}  // namespace

cudaError_t current_device_sms(int *sms) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_sms.find(dev);
    if (it == g_sms.end()) {
        int n = 0;
        err = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (err != cudaSuccess) return err;
        it = g_sms.emplace(dev, n > 0 ? n : 1).first;
    }
    *sms = it->second;
    return cudaSuccess;
}

cudaError_t prepare_kernel(const void *kernel, size_t smem_bytes, cudaFuncAttributes *attr) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lock(g_mu);
    auto key = std::make_pair(kernel, dev);
    auto it = g_kernels.find(key);
    if (it == g_kernels.end()) {
        KernelState ks;
        err = cudaFuncGetAttributes(&ks.attr, kernel);
        if (err != cudaSuccess) return err;
        it = g_kernels.emplace(key, ks).first;
    }
    KernelState &ks = it->second;
    if (smem_bytes > ks.smem_limit) {
        err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (err != cudaSuccess) return err;
        ks.smem_limit = smem_bytes;
    }
    if (attr) *attr = ks.attr;
    return cudaSuccess;
}

}  // namespace pvf
