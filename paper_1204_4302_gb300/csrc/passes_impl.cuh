// Launchers of the field passes: map a runtime transform length onto the
// compile-time kernel instantiations of fft_engine.cuh. Included once per
// element type (passes_f32.cu, passes_f64.cu).
#pragma once
#include "fft_engine.cuh"
#include "plan.h"

namespace demag {

namespace {

// Opt in to more than 48 KB of dynamic shared memory, once per kernel and
// device (the cache is per template argument, i.e. per kernel).
template <auto Kern>
cudaError_t allow_smem(size_t bytes)
{
    const auto kern = Kern;
    static int done_for = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (done_for == dev) return cudaSuccess;
    if (bytes > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
    }
    done_for = dev;
    return cudaSuccess;
}

template <typename T>
__global__ void k_x1_fwd(XIn<T> a, int64_t n, typename Cplx<T>::type *__restrict__ out)
{
    using C = typename Cplx<T>::type;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cmk<C>(a.in[i] * a.wscalar * cell_weight(a.wcell, (int)i, a.rows_per_comp, 1, 0), (T)0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_x1_inv(const typename Cplx<T>::type *__restrict__ in, int64_t n, XOut<T> o)
{
    const T g = o.gdev ? (T)(*o.gdev) : (T)1;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T h = in[i].x * o.scale;
        const T w = cell_weight(o.wcell, (int)i, o.rows_per_comp, 1, 0);
        if (o.out) o.out[i] = h * o.oscale * g * w;
        if (o.partials) acc += (double)(o.mscale * w * o.Mref[i] * h);
    }
    if (o.partials) block_partial<256>(acc, o.partials);
}

}  // namespace

#define DEMAG_FOR_EACH_L(M) \
    M(1) M(2) M(4) M(8) M(16) M(32) M(64) M(128) M(256) M(512) M(1024)

template <typename T>
cudaError_t Passes<T>::x_fwd(int L, const XIn<T> &a, int nrows, int nvalid, C *out, int64_t out_rs,
                             const C *twx, cudaStream_t st)
{
    if (nrows <= 0) return cudaSuccess;
#define DEMAG_CASE(LL)                                                                        \
    case LL: {                                                                                \
        if constexpr (LL <= 512) {                                                            \
            using S = TileShape<T, LL>;                                                       \
            const size_t sm = swsize(LL * S::TC) * sizeof(C);                                 \
            cudaError_t e = allow_smem<k_x_fwd<T, LL>>(sm);                                   \
            if (e != cudaSuccess) return e;                                                   \
            const int grid = (nrows + S::TC - 1) / S::TC;                                     \
            k_x_fwd<T, LL><<<grid, S::NT, sm, st>>>(a, nrows, nvalid, out, out_rs, twx); \
            return cudaGetLastError();                                                        \
        } else {                                                                              \
            return cudaErrorInvalidValue;                                                     \
        }                                                                                     \
    }
    switch (L) { DEMAG_FOR_EACH_L(DEMAG_CASE) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
}

template <typename T>
int Passes<T>::x_blocks(int L, int nrows)
{
    const int tc = (Tile<T>::NT * Tile<T>::EPT) / L;
    return (nrows + tc - 1) / tc;
}

template <typename T>
cudaError_t Passes<T>::x_inv(int L, const C *in, int64_t in_rs, int nrows, int nvalid, const XOut<T> &o,
                             const C *twx, cudaStream_t st)
{
    if (nrows <= 0) return cudaSuccess;
#define DEMAG_CASE(LL)                                                                        \
    case LL: {                                                                                \
        if constexpr (LL <= 512) {                                                            \
            using S = TileShape<T, LL>;                                                       \
            const size_t sm = swsize(LL * S::TC) * sizeof(C);                                 \
            cudaError_t e = allow_smem<k_x_inv<T, LL>>(sm);                                   \
            if (e != cudaSuccess) return e;                                                   \
            const int grid = (nrows + S::TC - 1) / S::TC;                                     \
            k_x_inv<T, LL><<<grid, S::NT, sm, st>>>(in, in_rs, nrows, nvalid, o, twx);           \
            return cudaGetLastError();                                                        \
        } else {                                                                              \
            return cudaErrorInvalidValue;                                                     \
        }                                                                                     \
    }
    switch (L) { DEMAG_FOR_EACH_L(DEMAG_CASE) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
}

template <typename T>
cudaError_t Passes<T>::col(int L, bool inv, const C *in, C *out, int ncols, int width, int64_t iss,
                           int64_t irs, int nin, int64_t oss, int64_t ors, int nout, const C *tw,
                           int twstride, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
#define DEMAG_CASE(LL)                                                                        \
    case LL: {                                                                                \
        using S = TileShape<T, LL>;                                                           \
        const size_t sm = swsize(LL * S::TC) * sizeof(C);                                     \
        const int grid = (ncols + S::TC - 1) / S::TC;                                         \
        if (inv) {                                                                            \
            cudaError_t e = allow_smem<k_col_fft<T, LL, true>>(sm);                           \
            if (e != cudaSuccess) return e;                                                   \
            k_col_fft<T, LL, true><<<grid, S::NT, sm, st>>>(in, out, ncols, width, iss, irs, nin, \
                                                           oss, ors, nout, tw, twstride);     \
        } else {                                                                              \
            cudaError_t e = allow_smem<k_col_fft<T, LL, false>>(sm);                          \
            if (e != cudaSuccess) return e;                                                   \
            k_col_fft<T, LL, false><<<grid, S::NT, sm, st>>>(in, out, ncols, width, iss, irs, nin, \
                                                            oss, ors, nout, tw, twstride);    \
        }                                                                                     \
        return cudaGetLastError();                                                            \
    }
    switch (L) { DEMAG_FOR_EACH_L(DEMAG_CASE) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
}

template <typename T>
cudaError_t Passes<T>::zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
                             int nrows, const T *nhat, int Py, int Kx, const C *tw, int twstride,
                             cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
#define DEMAG_CASE(LL)                                                                        \
    case LL: {                                                                                \
        using Sh = TileShape<T, LL>;                                                          \
        const size_t sm = 3 * swsize(LL * Sh::TC) * sizeof(C);                                \
        cudaError_t e = allow_smem<k_z_conv<T, LL>>(sm);                                      \
        if (e != cudaSuccess) return e;                                                       \
        const int grid = (ncols + Sh::TC - 1) / Sh::TC;                                       \
        k_z_conv<T, LL><<<grid, Sh::NT, sm, st>>>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, \
                                                 tw, twstride);                               \
        return cudaGetLastError();                                                            \
    }
    switch (L) { DEMAG_FOR_EACH_L(DEMAG_CASE) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
}

template <typename T>
cudaError_t Passes<T>::x1_fwd(const XIn<T> &a, int64_t n, C *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_x1_fwd<T><<<grid, 256, 0, st>>>(a, n, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Passes<T>::x1_inv(const C *in, int64_t n, const XOut<T> &o, int nblocks, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_x1_inv<T><<<nblocks, 256, 0, st>>>(in, n, o);
    return cudaGetLastError();
}

}  // namespace demag
