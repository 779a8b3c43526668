// Allocation-free energy reduction: E = -(mu0/2) V sum M.H from a field the
// caller already has, with the per-block partial sums kept in a fixed device
// array that belongs to the library instead of memory obtained per call.
//
// Who needs it: callers that may not call cudaMalloc / cudaFree at the point
// where they want the energy. Examples are code running while a stream is
// being captured into a CUDA graph in the global capture mode (allocation
// calls are illegal there), hosts whose device memory is handed out only by
// their own pool allocator, and tight integrator loops where an allocation
// (which can synchronise the device) is not acceptable. The regular energy
// path needs a plan, whose creation allocates; this entry point needs none.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "demag.h"

namespace {

// Capacity of the fixed partial-sum array: one double per block of
// kValuesPerBlock values, so at most kMaxPartials * kValuesPerBlock values
// (3 components x cells) per call.
constexpr int kMaxPartials = 65536;  // 512 KB of device memory per GPU
constexpr int kThreads = 256;
constexpr int kValuesPerBlock = kThreads * 32;
constexpr int kMaxDevices = 64;
constexpr double kMu0 = 4e-7 * 3.14159265358979323846;

// Shared by every call on a device and kept until the process exits. Every
// call writes each slot it later reads, so nothing needs clearing between
// calls; two calls that run at the same time on the GPU (e.g. on two
// streams) write the same slots and race.
static __device__ __align__(256) double g_partials[kMaxPartials];

std::mutex g_lock;
double *g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx[kMaxDevices] = {0};

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_dot_partials(const T *__restrict__ M, const T *__restrict__ H, int64_t n, double *__restrict__ partials)
{
    __shared__ double red[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kValuesPerBlock;
    const int64_t end = base + kValuesPerBlock < n ? base + kValuesPerBlock : n;
    double s = 0.0;
    for (int64_t i = base + threadIdx.x; i < end; i += kThreads) s += (double)M[i] * (double)H[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kThreads)
k_sum_partials(const double *__restrict__ partials, int count, double factor, double *__restrict__ E)
{
    // Neumaier-compensated sum per thread, then a compensated pairwise tree.
    __shared__ double ss[kThreads], sc[kThreads];
    double s = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < count; i += kThreads) {
        const double v = partials[i];
        const double t = s + v;
        c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const double a = ss[threadIdx.x], b = ss[threadIdx.x + w];
            const double t = a + b;
            const double e = fabs(a) >= fabs(b) ? (a - t) + b : (b - t) + a;
            ss[threadIdx.x] = t;
            sc[threadIdx.x] += sc[threadIdx.x + w] + e;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = factor * (ss[0] + sc[0]);
}

// Identity of the current device's context (the driver's 64-bit context
// id, unique for the life of the process), so that an address looked up in
// a context that has since been destroyed (cudaDeviceReset) is never reused.
// 0 when the driver entry points are unavailable: then the address is looked
// up again on every call.
using CtxGetCurrent = int (*)(void **);
using CtxGetId = int (*)(void *, unsigned long long *);

unsigned long long context_id()
{
    static CtxGetCurrent get_current = nullptr;
    static CtxGetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrent>(a);
            get_id = reinterpret_cast<CtxGetId>(b);
        }
    }
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_partials on the current device. The host-side name of
// a __device__ array is only a stand-in and must never reach a kernel; the
// address is looked up once per device and context and cached.
demag_status partials_address(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DEMAG_ERR_CUDA;
    }
    // make the device's primary context current (it is created here after a
    // reset), so that its id can be read
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return DEMAG_ERR_CUDA;
    }
    const unsigned long long ctx = context_id();
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            g_addr[dev] = nullptr;
            return DEMAG_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double *>(p);
        g_ctx[dev] = ctx;
    }
    *out = g_addr[dev];
    return DEMAG_OK;
}

// Device or managed memory reachable from the current device.
bool is_device_ptr(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" demag_status demag_energy_noalloc(int nx, int ny, int nz, double dx, double dy, double dz,
                                             demag_prec prec, const void *M, const void *H, double *E_dev,
                                             void *stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0) || !isfinite(dx) ||
        !isfinite(dy) || !isfinite(dz))
        return DEMAG_ERR_INVALID_ARG;
    if (prec != DEMAG_F32 && prec != DEMAG_F64) return DEMAG_ERR_INVALID_ARG;
    // capacity check before any integer product: 3 nx ny nz in double is
    // exact far beyond the cap, so a huge grid cannot wrap around
    if (3.0 * (double)nx * (double)ny * (double)nz > (double)kMaxPartials * kValuesPerBlock)
        return DEMAG_ERR_UNSUPPORTED;  // beyond the fixed array
    const int64_t n = 3 * (int64_t)nx * ny * nz;
    const int64_t blocks = (n + kValuesPerBlock - 1) / kValuesPerBlock;
    if (!M || !H || !E_dev || ((uintptr_t)M & 15u) || ((uintptr_t)H & 15u) || ((uintptr_t)E_dev & 7u))
        return DEMAG_ERR_INVALID_ARG;
    double *partials = nullptr;
    const demag_status s = partials_address(&partials);
    if (s != DEMAG_OK) return s;
    int dev = -1;
    cudaGetDevice(&dev);
    if (!is_device_ptr(M, dev) || !is_device_ptr(H, dev) || !is_device_ptr(E_dev, dev))
        return DEMAG_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // Launch errors are taken from the launch calls themselves, so an error
    // left pending by unrelated earlier work is neither reported as this
    // call's failure nor cleared from the caller's view.
    const bool clean = cudaPeekAtLastError() == cudaSuccess;
    int64_t nn = n;
    const double factor = -0.5 * kMu0 * dx * dy * dz;
    int count = (int)blocks;
    void *dot_args[] = {(void *)&M, (void *)&H, (void *)&nn, (void *)&partials};
    void *sum_args[] = {(void *)&partials, (void *)&count, (void *)&factor, (void *)&E_dev};
    const void *dot = prec == DEMAG_F32 ? (const void *)k_dot_partials<float> : (const void *)k_dot_partials<double>;
    cudaError_t e = cudaLaunchKernel(dot, dim3((unsigned)blocks), dim3(kThreads), dot_args, 0, st);
    if (e == cudaSuccess) e = cudaLaunchKernel((const void *)k_sum_partials, dim3(1), dim3(kThreads), sum_args, 0, st);
    if (e != cudaSuccess) {
        if (clean) cudaGetLastError();  // clear this call's own launch error only
        return DEMAG_ERR_CUDA;
    }
    return DEMAG_OK;
}
