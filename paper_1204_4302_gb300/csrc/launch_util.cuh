// Host-side launch helpers shared by the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace demag {
namespace {

// Opt in to more than 48 KB of dynamic shared memory, once per kernel and
// device (the cache is per template argument, i.e. per kernel).
int sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

template <auto Kern>
cudaError_t allow_smem(size_t bytes)
{
    // Opt the kernel in to the device's whole per-block shared memory once per
    // device (launch sizes can differ from call to call); the occupancy still
    // follows the size each launch asks for.
    const auto kern = Kern;
    static int done_for = -1;
    static size_t limit = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (done_for != dev) {
        int optin = 0;
        cudaFuncAttributes fa;
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        const size_t dyn = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        if (dyn > 48 * 1024 &&
            (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) != cudaSuccess)
            return e;
        limit = dyn > 48 * 1024 ? dyn : 48 * 1024;
        done_for = dev;
    }
    return bytes <= limit ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace
}  // namespace demag
