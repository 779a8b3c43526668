// Launchers of the field passes: map a runtime transform length onto the
// compile-time kernel instantiations of fft_engine.cuh. Included once per
// element type (passes_f32.cu, passes_f64.cu).
#pragma once
#include "fft2.cuh"
#include "fft_engine.cuh"
#include <string.h>

#include <algorithm>

#include "launch_util.cuh"
#include "plan.h"
#include "sp.cuh"
#include "xpipe.cuh"
#include "zws.cuh"

namespace demag {

namespace {

bool pow2_len(int L) { return L > 0 && (L & (L - 1)) == 0; }

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
    if (o.partials) block_partial<256>(acc, o.partials, blockIdx.x);
}

}  // namespace

#define DEMAG_FOR_EACH_L(M) \
    M(1) M(2) M(4) M(8) M(16) M(32) M(64) M(128) M(256) M(512) M(1024)

namespace {
// Resident CTAs per SM of a kernel at a given dynamic shared-memory size
// (cached per kernel for the last size asked).
template <auto Kern>
int resident_ctas(int threads, size_t smem)
{
    static size_t last = (size_t)-1;
    static int occ = 1;
    if (smem != last) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, Kern, threads, smem) != cudaSuccess || o < 1) o = 1;
        occ = o;
        last = smem;
    }
    return occ;
}

template <typename T, int L>
cudaError_t x_fwd_pipe(const XIn<T> &a, int nrows, int nvalid, typename Cplx<T>::type *out, int64_t out_rs,
                       const typename Cplx<T>::type *twx, cudaStream_t st)
{
    using S = XShape<T, L>;
    const size_t sm = XPipeSmem<T, L, T>::bytes(S::TR * nvalid);
    cudaError_t e = allow_smem<k_x_fwd_tma<T, L>>(sm);
    if (e != cudaSuccess) return e;
    const int ntiles = (nrows + S::TR - 1) / S::TR;
    const int cap = sm_count() * resident_ctas<k_x_fwd_tma<T, L>>(S::NT, sm);
    k_x_fwd_tma<T, L><<<ntiles < cap ? ntiles : cap, S::NT, sm, st>>>(a.in, a.wscalar, nrows, nvalid, out, out_rs,
                                                                      twx, ntiles);
    return cudaGetLastError();
}

template <typename T, int L, bool P1>
cudaError_t x_inv_pipe(const typename Cplx<T>::type *in, int in_rs, int nrows, int nvalid, const XOut<T> &o,
                       const typename Cplx<T>::type *twx, cudaStream_t st)
{
    using S = XShape<T, L>;
    const size_t sm = 2 * xinv_slot_bytes<T, L>(in_rs) + 2 * sizeof(uint64_t);
    cudaError_t e = allow_smem<k_x_inv_tma<T, L, P1>>(sm);
    if (e != cudaSuccess) return e;
    const int ntiles = (nrows + S::TR - 1) / S::TR;
    const int cap = sm_count() * resident_ctas<k_x_inv_tma<T, L, P1>>(S::NT, sm);
    k_x_inv_tma<T, L, P1><<<ntiles < cap ? ntiles : cap, S::NT, sm, st>>>(in, in_rs, nrows, nvalid, o, twx, ntiles);
    return cudaGetLastError();
}
}  // namespace

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, through the runtime's entry-point lookup
// (no link against the driver library). nullptr if unavailable.
EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Map of the y pass input: nslabs slabs of nin rows of width complex values
// (row pitch irs, slab pitch iss complex), seen as reals; box 2 TC reals x BR
// rows x 1 slab. Cached for the last arguments (one per element type and L).
template <typename T, int L>
bool y_input_map(CUtensorMap *out, const typename Cplx<T>::type *in, int width, int nin, int nslabs, int64_t irs,
                 int64_t iss, int BR)
{
    static CUtensorMap cache;
    static const void *k_in = nullptr;
    static int64_t k_key[6] = {0, 0, 0, 0, 0, 0};
    const int64_t key[6] = {width, nin, nslabs, irs, iss, BR};
    if (k_in == in && memcmp(key, k_key, sizeof key) == 0) {
        *out = cache;
        return true;
    }
    EncodeTiled enc = encoder();
    if (!enc) return false;
    using C = typename Cplx<T>::type;
    constexpr int TC = Col3Shape<T, L>::TC;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * width, (cuuint64_t)nin, (cuuint64_t)nslabs};
    const cuuint64_t strides[2] = {(cuuint64_t)irs * sizeof(C), (cuuint64_t)iss * sizeof(C)};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * TC), (cuuint32_t)BR, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    if (enc(&cache, dt, 3, const_cast<void *>(static_cast<const void *>(in)), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        k_in = nullptr;
        return false;
    }
    k_in = in;
    memcpy(k_key, key, sizeof key);
    *out = cache;
    return true;
}

// Pipelined pruned forward column pass (TMA tensor copies); returns
// cudaErrorNotSupported when the arguments do not allow it (caller falls back).
template <typename T, int L>
cudaError_t col_fwd_tma(const typename Cplx<T>::type *in, typename Cplx<T>::type *out, int ncols, int width,
                        int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, const typename Cplx<T>::type *tw,
                        int twstride, cudaStream_t st)
{
    using C = typename Cplx<T>::type;
    using S = Col3Shape<T, L>;
    if (width <= 0 || ncols % width != 0 || nin < 1 || 2 * nin > L) return cudaErrorNotSupported;
    if (((uintptr_t)in & 15) || (irs * (int64_t)sizeof(C)) % 16 || (iss * (int64_t)sizeof(C)) % 16)
        return cudaErrorNotSupported;
    const int nslabs = ncols / width;
    const int BR = nin <= 256 ? nin : 256;
    const int nb = (nin + BR - 1) / BR;
    CUtensorMap map;
    if (!y_input_map<T, L>(&map, in, width, nin, nslabs, irs, iss, BR)) return cudaErrorNotSupported;
    const size_t ex = ((size_t)swsize(L * S::TC) * sizeof(C) + 127) / 128 * 128;
    const size_t inb = ((size_t)nb * BR * S::TC * sizeof(C) + 127) / 128 * 128;
    const size_t sm = 128 + ex + 2 * inb + 2 * sizeof(uint64_t);
    if (sm > 227 * 1024) return cudaErrorNotSupported;  // e.g. FP64 at L = 1024 with more than 256 rows
    cudaError_t e = allow_smem<k_col_tma_fwd<T, L>>(sm);
    if (e != cudaSuccess) return e;
    const int ntiles = ((width + S::TC - 1) / S::TC) * nslabs;
    const int cap = sm_count() * resident_ctas<k_col_tma_fwd<T, L>>(S::NT, sm);
    k_col_tma_fwd<T, L><<<ntiles < cap ? ntiles : cap, S::NT, sm, st>>>(map, out, width, nslabs, nin, BR, nb, oss,
                                                                         ors, tw, twstride);
    return cudaGetLastError();
}
}  // namespace

namespace {
// Map of the z pass input S2 [3][nz][Py][Kxp] complex seen as reals: dims
// (2 Kx, Py, nz, 3), box (2 TC, 1, nz, 3): one copy per tile. Cached for the
// last arguments (one per element type and L).
template <typename T, int L>
bool z_input_map(CUtensorMap *out, const typename Cplx<T>::type *S, int Kx, int Py, int nz, int64_t ss, int64_t rs,
                 int64_t cs)
{
    static CUtensorMap cache;
    static const void *k_S = nullptr;
    static int64_t k_key[6] = {0, 0, 0, 0, 0, 0};
    const int64_t key[6] = {Kx, Py, nz, ss, rs, cs};
    if (k_S == S && memcmp(key, k_key, sizeof key) == 0) {
        *out = cache;
        return true;
    }
    EncodeTiled enc = encoder();
    if (!enc) return false;
    using C = typename Cplx<T>::type;
    constexpr int TC = ZShape<T, L, ZTmaV<L>::V>::TC;
    const cuuint64_t dims[4] = {(cuuint64_t)2 * Kx, (cuuint64_t)Py, (cuuint64_t)nz, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)ss * sizeof(C), (cuuint64_t)rs * sizeof(C), (cuuint64_t)cs * sizeof(C)};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * TC), 1, (cuuint32_t)nz, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    if (enc(&cache, dt, 4, const_cast<void *>(static_cast<const void *>(S)), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        k_S = nullptr;
        return false;
    }
    k_S = S;
    memcpy(k_key, key, sizeof key);
    *out = cache;
    return true;
}

template <typename T, int L>
cudaError_t zconv_tma(typename Cplx<T>::type *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                      const T *nhat, int Py, int Kx, const typename Cplx<T>::type *tw, int twstride, cudaStream_t st)
{
    using C = typename Cplx<T>::type;
    using Sh = ZShape<T, L, ZTmaV<L>::V>;
    if (twstride != 1 || width != Kx || ncols != Py * Kx || nrows < 1 || 2 * nrows > L || cs != (int64_t)nrows * rs ||
        ((uintptr_t)S & 15) || (ss * (int64_t)sizeof(C)) % 16 || (rs * (int64_t)sizeof(C)) % 16)
        return cudaErrorNotSupported;
    CUtensorMap map;
    if (!z_input_map<T, L>(&map, S, Kx, Py, nrows, ss, rs, cs)) return cudaErrorNotSupported;
    const size_t stg = ((size_t)3 * nrows * Sh::TC * sizeof(C) + 127) / 128 * 128;
    const size_t sm = 128 + stg + 3 * swsize(L * Sh::TC) * sizeof(C) + (L / 2 + 1) * 6 * Sh::TC * sizeof(T) + 8;
    if (sm > 227 * 1024) return cudaErrorNotSupported;
    cudaError_t e = allow_smem<k_z_conv_tma<T, L>>(sm);
    if (e != cudaSuccess) return e;
    const int ntr = (Kx + Sh::TC - 1) / Sh::TC;
    const int ntiles = ntr * Py;
    const int cap = sm_count();
    k_z_conv_tma<T, L><<<ntiles < cap ? ntiles : cap, Sh::NT, sm, st>>>(map, S, Kx, Py, ss, rs, cs, nrows, nhat, tw,
                                                                         ntr, ntiles);
    return cudaGetLastError();
}
template <typename T, int L>
cudaError_t sp_zconv_tma(typename Cplx<T>::type *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
                         int nrows, int nout, const T *that, int Py, int Kx, const typename Cplx<T>::type *tw,
                         const typename Cplx<T>::type *phx, const typename Cplx<T>::type *phy,
                         const typename Cplx<T>::type *phz, cudaStream_t st)
{
    using C = typename Cplx<T>::type;
    using Sh = ZShape<T, L, 0>;
    if (width != Kx || ncols != Py * Kx || nrows < 1 || 2 * nrows > L || cs != (int64_t)nrows * rs ||
        ((uintptr_t)S & 15) || (ss * (int64_t)sizeof(C)) % 16 || (rs * (int64_t)sizeof(C)) % 16)
        return cudaErrorNotSupported;
    CUtensorMap map;
    if (!z_input_map<T, L>(&map, S, Kx, Py, nrows, ss, rs, cs)) return cudaErrorNotSupported;
    const size_t stg = ((size_t)3 * nrows * Sh::TC * sizeof(C) + 127) / 128 * 128;
    const size_t sm = 128 + stg + 3 * swsize(L * Sh::TC) * sizeof(C) +
                      (size_t)(((L / 2 + 1) * 3 * Sh::TC + 1) / 2 * 2) * sizeof(T) + 8;
    if (sm > 227 * 1024) return cudaErrorNotSupported;
    const int ntr = (Kx + Sh::TC - 1) / Sh::TC;
    const int ntiles = ntr * Py;
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    cudaError_t e;
    if (2 * nout <= L) {
        if ((e = allow_smem<k_sp_z_tma<T, L, true>>(sm)) != cudaSuccess) return e;
        k_sp_z_tma<T, L, true><<<grid, Sh::NT, sm, st>>>(map, S, Kx, Py, ss, rs, cs, nrows, nout, that, tw, phx, phy,
                                                          phz, ntr, ntiles);
    } else {
        if ((e = allow_smem<k_sp_z_tma<T, L, false>>(sm)) != cudaSuccess) return e;
        k_sp_z_tma<T, L, false><<<grid, Sh::NT, sm, st>>>(map, S, Kx, Py, ss, rs, cs, nrows, nout, that, tw, phx, phy,
                                                           phz, ntr, ntiles);
    }
    return cudaGetLastError();
}
}  // namespace

namespace {
// Map of S2 [3][nz][Py][Kxp] complex seen as reals for the persistent z pass:
// dims (2 Kx, Py, nz, 3), box (2 TC, 1, nz, 3). Cached for the last arguments.
template <int L, int TC>
bool zws_input_map(CUtensorMap *out, const float2 *S, int Kx, int Py, int nz, int64_t ss, int64_t rs, int64_t cs)
{
    static CUtensorMap cache;
    static const void *k_S = nullptr;
    static int64_t k_key[6] = {0, 0, 0, 0, 0, 0};
    const int64_t key[6] = {Kx, Py, nz, ss, rs, cs};
    if (k_S == S && memcmp(key, k_key, sizeof key) == 0) {
        *out = cache;
        return true;
    }
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)2 * Kx, (cuuint64_t)Py, (cuuint64_t)nz, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)ss * sizeof(float2), (cuuint64_t)rs * sizeof(float2),
                                   (cuuint64_t)cs * sizeof(float2)};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * TC), 1, (cuuint32_t)nz, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(&cache, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(static_cast<const void *>(S)), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        k_S = nullptr;
        return false;
    }
    k_S = S;
    memcpy(k_key, key, sizeof key);
    *out = cache;
    return true;
}

template <int L, int TC, bool EONLY = false, bool FE = false>
cudaError_t zws_launch(float2 *S, int Kx, int Py, int64_t ss, int64_t rs, int64_t cs, int nrows, const float *ntile,
                       const float2 *tw, cudaStream_t st, double *partials = nullptr, int *nparts = nullptr)
{
    using Sh = ZwsShape<L, TC>;
    CUtensorMap map;
    if (!zws_input_map<L, TC>(&map, S, Kx, Py, nrows, ss, rs, cs)) return cudaErrorNotSupported;
    const size_t sm = zws_smem_bytes<L, TC>(nrows);
    if (sm > 227 * 1024) return cudaErrorNotSupported;
    cudaError_t e = allow_smem<k_z_ws<L, TC, EONLY, FE>>(sm);
    if (e != cudaSuccess) return e;
    const int ntx = (Kx + TC - 1) / TC;
    const int ntiles = ntx * Py;
    const int cap = sm_count() * resident_ctas<k_z_ws<L, TC, EONLY, FE>>(Sh::NT, sm);
    int grid = ntiles < cap ? ntiles : cap;
    if (nparts) {  // in: room for per-CTA sums (the persistent loop takes any grid); out: sums written
        if (*nparts > 0 && grid > *nparts) grid = *nparts;
        *nparts = grid;
    }
    k_z_ws<L, TC, EONLY, FE><<<grid, Sh::NT, sm, st>>>(map, S, Kx, Py, ss, rs, cs, nrows, ntile, tw, ntx, ntiles,
                                                       partials);
    return cudaGetLastError();
}

// Arguments the persistent z pass takes (TMA alignment, at most L/2 rows).
bool zws_ok(int L, const void *S, const void *ntile, int nrows, int64_t ss, int64_t rs, int64_t cs, size_t csize)
{
    return (L == 256 || L == 512) && ntile && nrows >= 1 && 2 * nrows <= L && ((uintptr_t)S & 15) == 0 &&
           ((uintptr_t)ntile & 15) == 0 && (ss * (int64_t)csize) % 16 == 0 && (rs * (int64_t)csize) % 16 == 0 &&
           (cs * (int64_t)csize) % 16 == 0;
}
}  // namespace

template <typename T>
size_t Passes<T>::tile_tensor_elems(int L, int Py, int Kx)
{
    if (sizeof(T) != 4 || (L != 256 && L != 512)) return 0;
    return (size_t)(Py / 2 + 1) * zws_ntx4(Kx) * 24 * (L / 2 + 1);  // [hy][ntx4][6][HZ][4]
}

template <typename T>
cudaError_t Passes<T>::tile_tensor(int L, const T *nhat, T *ntile, int Py, int Kx, cudaStream_t st)
{
    const size_t n = tile_tensor_elems(L, Py, Kx);
    if (n == 0) return cudaErrorNotSupported;
    const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 16);
    k_tile_tensor<T><<<grid, 256, 0, st>>>(nhat, ntile, Kx, Py / 2 + 1, L / 2 + 1, zws_ntx4(Kx));
    return cudaGetLastError();
}

template <typename T>
cudaError_t Passes<T>::zconv_ws(int L, C *S, int Kx, int Py, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                const T *ntile, const C *tw, cudaStream_t st, int tc, double *partials, int *nparts)
{
    if constexpr (sizeof(T) != 4) {
        return cudaErrorNotSupported;
    } else {
        if (!zws_ok(L, S, ntile, nrows, ss, rs, cs, sizeof(C))) return cudaErrorNotSupported;
        if (partials) {  // field and spectral energy
            if (L == 256)
                return tc == 4 ? zws_launch<256, 4, false, true>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st, partials, nparts)
                               : zws_launch<256, 8, false, true>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st, partials, nparts);
            return tc == 4 ? zws_launch<512, 4, false, true>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st, partials, nparts)
                           : zws_launch<512, 8, false, true>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st, partials, nparts);
        }
        if (L == 256)
            return tc == 4 ? zws_launch<256, 4>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st)
                           : zws_launch<256, 8>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st);
        return tc == 4 ? zws_launch<512, 4>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st)
                       : zws_launch<512, 8>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st);
    }
}

template <typename T>
cudaError_t Passes<T>::zconv_ws_energy(int L, C *S, int Kx, int Py, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                       const T *ntile, const C *tw, double *partials, int *nparts, cudaStream_t st,
                                       int tc)
{
    if constexpr (sizeof(T) != 4) {
        return cudaErrorNotSupported;
    } else {
        if (!zws_ok(L, S, ntile, nrows, ss, rs, cs, sizeof(C))) return cudaErrorNotSupported;
        if (L == 256)
            return tc == 4 ? zws_launch<256, 4, true>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st, partials, nparts)
                           : zws_launch<256, 8, true>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st, partials, nparts);
        return tc == 4 ? zws_launch<512, 4, true>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st, partials, nparts)
                       : zws_launch<512, 8, true>(S, Kx, Py, ss, rs, cs, nrows, ntile, tw, st, partials, nparts);
    }
}

// Spectral-energy z pass: the 8-point second stage (variant 8) for lengths
// 32..128, as in the field pipeline's fastest form there.
template <int L> constexpr int kZEnergyV = (L >= 32 && L <= 128) ? 8 : 0;

template <typename T>
int Passes<T>::zenergy_blocks(int L, int Py, int Kx)
{
    const int ncols = Py * Kx;
    if (ncols <= 0 || !pow2_len(L) || L > 512) return 0;
    int n;
    if (L <= 16) {
        n = (ncols + Tile2<T>::NT - 1) / Tile2<T>::NT;
    } else {
        int tc;
        switch (L) {
        case 32: tc = ZShape<T, 32, kZEnergyV<32>>::TC; break;
        case 64: tc = ZShape<T, 64, kZEnergyV<64>>::TC; break;
        case 128: tc = ZShape<T, 128, kZEnergyV<128>>::TC; break;
        case 256: tc = ZShape<T, 256, kZEnergyV<256>>::TC; break;
        default: tc = ZShape<T, 512, 0>::TC; break;
        }
        n = (ncols + tc - 1) / tc;
    }
    const int ws = 2 * sm_count();  // the persistent form: at most two CTAs per SM
    return n > ws ? n : ws;
}

template <typename T>
cudaError_t Passes<T>::zconv_energy(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
                                    int nrows, const T *nhat, int Py, int Kx, const C *tw, int twstride,
                                    double *partials, int *nparts, cudaStream_t st)
{
    if (ncols <= 0 || !pow2_len(L) || L > 512 || (L > 1 && 2 * nrows > L)) return cudaErrorNotSupported;
    if (L <= 16) {
        const int grid = (ncols + Tile2<T>::NT - 1) / Tile2<T>::NT;
        *nparts = grid;
#define DEMAG_CASE(LL)                                                                                     \
    case LL:                                                                                               \
        k_z_energy1<T, LL><<<grid, Tile2<T>::NT, 0, st>>>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx,   \
                                                           partials);                                     \
        return cudaGetLastError();
        switch (L) { DEMAG_CASE(1) DEMAG_CASE(2) DEMAG_CASE(4) DEMAG_CASE(8) DEMAG_CASE(16) default: return cudaErrorNotSupported; }
#undef DEMAG_CASE
    }
#define DEMAG_CASE(LL)                                                                                     \
    case LL: {                                                                                             \
        constexpr int V = kZEnergyV<LL>;                                                                   \
        using Sh = ZShape<T, LL, V>;                                                                       \
        const size_t sm = 3 * swsize(LL * Sh::TC) * sizeof(C) + (LL / 2 + 1) * 6 * Sh::TC * sizeof(T);     \
        cudaError_t e = allow_smem<k_z_energy2<T, LL, V>>(sm);                                             \
        if (e != cudaSuccess) return e;                                                                    \
        const int grid = (ncols + Sh::TC - 1) / Sh::TC;                                                    \
        *nparts = grid;                                                                                    \
        k_z_energy2<T, LL, V><<<grid, Sh::NT, sm, st>>>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, \
                                                        twstride, partials);                              \
        return cudaGetLastError();                                                                         \
    }
    switch (L) { DEMAG_CASE(32) DEMAG_CASE(64) DEMAG_CASE(128) DEMAG_CASE(256) DEMAG_CASE(512) default: return cudaErrorNotSupported; }
#undef DEMAG_CASE
}

template <typename T>
int Passes<T>::pipe_error_take()
{
    int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_xpipe_error, sizeof(int)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(g_xpipe_error, &zero, sizeof(int));
    return v;
}

template <typename T>
cudaError_t Passes<T>::x_fwd(int L, const XIn<T> &a, int nrows, int nvalid, C *out, int64_t out_rs,
                             const C *twx, cudaStream_t st, int variant)
{
    if (nrows <= 0) return cudaSuccess;
    if (!pow2_len(L)) return MixedPasses<T>::x_fwd(L, a, nrows, nvalid, out, out_rs, twx, st);
    // pipelined form: rows of the plain field (no per-cell weight) stored back
    // to back, 16-byte multiples, zero-padded half
    if (variant >= 1 && L >= 64 && nvalid <= L && !a.wcell && a.in_rs == nvalid && nvalid % 4 == 0 &&
        ((uintptr_t)a.in & 15) == 0) {
        switch (L) {
        case 64: return x_fwd_pipe<T, 64>(a, nrows, nvalid, out, out_rs, twx, st);
        case 128: return x_fwd_pipe<T, 128>(a, nrows, nvalid, out, out_rs, twx, st);
        case 256: return x_fwd_pipe<T, 256>(a, nrows, nvalid, out, out_rs, twx, st);
        case 512: return x_fwd_pipe<T, 512>(a, nrows, nvalid, out, out_rs, twx, st);
        default: break;
        }
    }
    if (L >= 64) {
#define DEMAG_CASE2(LL)                                                                        \
    case LL: {                                                                                 \
        using S = XShape<T, LL>;                                                               \
        const size_t sm = (size_t)S::TR * S::RS * sizeof(C);                                   \
        const int grid = (nrows + S::TR - 1) / S::TR;                                          \
        if (nvalid <= LL)                                                                      \
            k_x_fwd2<T, LL, true><<<grid, S::NT, sm, st>>>(a, nrows, nvalid, out, out_rs, twx); \
        else                                                                                   \
            k_x_fwd2<T, LL, false><<<grid, S::NT, sm, st>>>(a, nrows, nvalid, out, out_rs, twx); \
        return cudaGetLastError();                                                             \
    }
        switch (L) { DEMAG_CASE2(64) DEMAG_CASE2(128) DEMAG_CASE2(256) DEMAG_CASE2(512) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE2
    }
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
    if (!pow2_len(L)) return MixedPasses<T>::x_blocks(L, nrows);
    int rows_per_cta;
    switch (L) {
    case 64: rows_per_cta = XShape<T, 64>::TR; break;
    case 128: rows_per_cta = XShape<T, 128>::TR; break;
    case 256: rows_per_cta = XShape<T, 256>::TR; break;
    case 512: rows_per_cta = XShape<T, 512>::TR; break;
    default: rows_per_cta = (Tile<T>::NT * Tile<T>::EPT) / L;
    }
    return (nrows + rows_per_cta - 1) / rows_per_cta;
}

template <typename T>
cudaError_t Passes<T>::x_inv(int L, const C *in, int64_t in_rs, int nrows, int nvalid, const XOut<T> &o,
                             const C *twx, cudaStream_t st, int variant)
{
    if (nrows <= 0) return cudaSuccess;
    if (!pow2_len(L)) return MixedPasses<T>::x_inv(L, in, in_rs, nrows, nvalid, o, twx, st);
    if (variant == 2 && L >= 64 && in_rs % 2 == 0 && in_rs <= 2 * L && nvalid <= L + 1 && ((uintptr_t)in & 15) == 0) {
        const bool p1 = nvalid > L;
#define DEMAG_PIPE(LL)                                                                         \
    case LL:                                                                                   \
        return p1 ? x_inv_pipe<T, LL, true>(in, (int)in_rs, nrows, nvalid, o, twx, st)         \
                  : x_inv_pipe<T, LL, false>(in, (int)in_rs, nrows, nvalid, o, twx, st);
        // (L = 512 would hold a whole 32-point stage in registers across the
        // buffer hand-over: one CTA per SM; the one-tile kernel serves it)
        switch (L) { DEMAG_PIPE(64) DEMAG_PIPE(128) DEMAG_PIPE(256) default: break; }
#undef DEMAG_PIPE
    }
    if (L >= 64) {
#define DEMAG_CASE2(LL)                                                                        \
    case LL: {                                                                                 \
        using S = XShape<T, LL>;                                                               \
        const size_t sm = (size_t)S::TR * S::RS * sizeof(C);                                   \
        const int grid = (nrows + S::TR - 1) / S::TR;                                          \
        if (o.partials && o.Mref && nvalid <= LL && nvalid % (16 / sizeof(T)) == 0 &&          \
            o.out_rs % (16 / sizeof(T)) == 0 && ((uintptr_t)o.Mref & 15) == 0) {               \
            const size_t smp = sm + (size_t)S::TR * LL * sizeof(T);                            \
            cudaError_t e = allow_smem<k_x_inv2<T, LL, false, true>>(smp);                     \
            if (e != cudaSuccess) return e;                                                    \
            k_x_inv2<T, LL, false, true><<<grid, S::NT, smp, st>>>(in, in_rs, nrows, nvalid, o, twx); \
        } else if (nvalid <= LL) k_x_inv2<T, LL><<<grid, S::NT, sm, st>>>(in, in_rs, nrows, nvalid, o, twx); \
        else if (nvalid == LL + 1) k_x_inv2<T, LL, true><<<grid, S::NT, sm, st>>>(in, in_rs, nrows, nvalid, o, twx); \
        else return cudaErrorInvalidValue;                                                     \
        return cudaGetLastError();                                                             \
    }
        switch (L) { DEMAG_CASE2(64) DEMAG_CASE2(128) DEMAG_CASE2(256) DEMAG_CASE2(512) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE2
    }
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
template <int L, bool INV, bool PIN, bool POUT, int V>
cudaError_t Passes<T>::col_launch(const C *in, C *out, int ncols, int width, int64_t iss, int64_t irs, int nin,
                                  int64_t oss, int64_t ors, int nout, const C *tw, int twstride,
                                  cudaStream_t st)
{
    using S = ColShape<T, L, V>;
    const size_t sm = swsize(L * S::TC) * sizeof(C);
    cudaError_t e = allow_smem<k_col2<T, L, INV, PIN, POUT, V>>(sm);
    if (e != cudaSuccess) return e;
    const int grid = (ncols + S::TC - 1) / S::TC;
    k_col2<T, L, INV, PIN, POUT, V><<<grid, S::NT, sm, st>>>(in, out, ncols, width, iss, irs, nin, oss, ors, nout,
                                                            tw, twstride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Passes<T>::col(int L, bool inv, const C *in, C *out, int ncols, int width, int64_t iss,
                           int64_t irs, int nin, int64_t oss, int64_t ors, int nout, const C *tw,
                           int twstride, cudaStream_t st, int variant)
{
    if (ncols <= 0) return cudaSuccess;
    if (!pow2_len(L))
        return MixedPasses<T>::col(L, inv, in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride, st);
    if (L <= 16) {
        // one thread per column
        const int grid = (ncols + Tile2<T>::NT - 1) / Tile2<T>::NT;
#define DEMAG_CASE(LL)                                                                         \
    case LL:                                                                                   \
        if (inv)                                                                               \
            k_col1<T, LL, true><<<grid, Tile2<T>::NT, 0, st>>>(in, out, ncols, width, iss, irs, nin, oss, ors, nout); \
        else                                                                                   \
            k_col1<T, LL, false><<<grid, Tile2<T>::NT, 0, st>>>(in, out, ncols, width, iss, irs, nin, oss, ors, nout); \
        return cudaGetLastError();
        switch (L) { DEMAG_CASE(1) DEMAG_CASE(2) DEMAG_CASE(4) DEMAG_CASE(8) DEMAG_CASE(16) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
    }
    // the zero padding halves the input (forward) or the output (inverse)
    const bool pin = 2 * nin <= L, pout = 2 * nout <= L;
    // variant 3: forward by the TMA pipeline, inverse as variant 2
    if (variant == 3 && !inv && pin && nout == L && (L == 512 || L == 1024)) {
        const cudaError_t e = L == 512 ? col_fwd_tma<T, 512>(in, out, ncols, width, iss, irs, nin, oss, ors, tw, twstride, st)
                                       : col_fwd_tma<T, 1024>(in, out, ncols, width, iss, irs, nin, oss, ors, tw, twstride, st);
        if (e != cudaErrorNotSupported) return e;
    }
    if (variant == 3) variant = 2;
    if (variant == 2 && (L == 512 || L == 1024) && (pin || pout) && !(pin && inv) && !(pout && !inv)) {
#define DEMAG_C3(LL)                                                                                    \
    if (L == LL) {                                                                                      \
        using S3 = Col3Shape<T, LL>;                                                                    \
        const size_t sm3 = swsize(LL * S3::TC) * sizeof(C);                                             \
        const int grid3 = (ncols + S3::TC - 1) / S3::TC;                                                \
        cudaError_t e3;                                                                                 \
        if (inv) {                                                                                      \
            e3 = allow_smem<k_col3<T, LL, true, false, true>>(sm3);                                     \
            if (e3 != cudaSuccess) return e3;                                                           \
            k_col3<T, LL, true, false, true><<<grid3, S3::NT, sm3, st>>>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride); \
        } else {                                                                                        \
            e3 = allow_smem<k_col3<T, LL, false, true, false>>(sm3);                                    \
            if (e3 != cudaSuccess) return e3;                                                           \
            k_col3<T, LL, false, true, false><<<grid3, S3::NT, sm3, st>>>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride); \
        }                                                                                               \
        return cudaGetLastError();                                                                      \
    }
        DEMAG_C3(512)
        DEMAG_C3(1024)
#undef DEMAG_C3
    }
    // variant 1 (swapped radix order) exists for the pruned field passes
#define DEMAG_CASE(LL)                                                                         \
    case LL:                                                                                   \
        if (!inv && pin) return variant == 1 ? col_launch<LL, false, true, false, 1>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride, st) \
                                             : col_launch<LL, false, true, false, 0>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride, st); \
        if (inv && pout) return variant == 1 ? col_launch<LL, true, false, true, 1>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride, st) \
                                             : col_launch<LL, true, false, true, 0>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride, st); \
        if (inv) return col_launch<LL, true, false, false, 0>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride, st); \
        return col_launch<LL, false, false, false, 0>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride, st);
    switch (L) { DEMAG_CASE(32) DEMAG_CASE(64) DEMAG_CASE(128) DEMAG_CASE(256) DEMAG_CASE(512) DEMAG_CASE(1024) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
}

template <typename T>
template <int L, int V>
cudaError_t Passes<T>::zconv_launch(C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                    const T *nhat, int Py, int Kx, const C *tw, int twstride, cudaStream_t st)
{
    using Sh = ZShape<T, L, V>;
    const size_t sm = 3 * swsize(L * Sh::TC) * sizeof(C) + (L / 2 + 1) * 6 * Sh::TC * sizeof(T);
    cudaError_t e = allow_smem<k_z_conv2<T, L, V>>(sm);
    if (e != cudaSuccess) return e;
    const int grid = (ncols + Sh::TC - 1) / Sh::TC;
    k_z_conv2<T, L, V><<<grid, Sh::NT, sm, st>>>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride);
    return cudaGetLastError();
}

template <typename T>
template <int L>
cudaError_t Passes<T>::zconv_pipe(C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                  const T *nhat, int Py, int Kx, const C *tw, int twstride, cudaStream_t st)
{
    using Sh = ZShape<T, L, 0>;
    const size_t sm = 3 * swsize(L * Sh::TC) * sizeof(C) + 3 * (L / 2) * Sh::TC * sizeof(C) +
                      (L / 2 + 1) * 6 * Sh::TC * sizeof(T);
    if (sm > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem<k_z_conv3<T, L>>(sm);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    const int ntiles = (ncols + Sh::TC - 1) / Sh::TC;
    const int grid = ntiles < sms ? ntiles : sms;
    k_z_conv3<T, L><<<grid, Sh::NT, sm, st>>>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, ntiles);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Passes<T>::zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
                             int nrows, const T *nhat, int Py, int Kx, const C *tw, int twstride,
                             cudaStream_t st, int variant)
{
    if (ncols > 0 && !pow2_len(L))
        return MixedPasses<T>::zconv(L, S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
    if (variant == 5 && ncols > 0 && 2 * nrows <= L) {
        cudaError_t e = cudaErrorNotSupported;
        switch (L) {
        case 32: e = zconv_tma<T, 32>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st); break;
        case 64: e = zconv_tma<T, 64>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st); break;
        case 128: e = zconv_tma<T, 128>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st); break;
        case 256: e = zconv_tma<T, 256>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st); break;
        case 512: e = zconv_tma<T, 512>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st); break;
        default: break;
        }
        if (e != cudaErrorNotSupported) return e;
        variant = 0;
    }
    if (variant == 3 && ncols > 0 && 2 * nrows <= L) {
        switch (L) {
        case 64: return zconv_pipe<64>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
        case 128: return zconv_pipe<128>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
        case 256: return zconv_pipe<256>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
        case 512: return zconv_pipe<512>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
        default: variant = 0;
        }
    }
    if (ncols <= 0) return cudaSuccess;
    if (2 * nrows > L && L > 1) return cudaErrorInvalidValue;  // the z pass always has padding
    if (L <= 16) {
        const int grid = (ncols + Tile2<T>::NT - 1) / Tile2<T>::NT;
#define DEMAG_CASE(LL)                                                                         \
    case LL:                                                                                   \
        k_z_conv1<T, LL><<<grid, Tile2<T>::NT, 0, st>>>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx); \
        return cudaGetLastError();
        switch (L) { DEMAG_CASE(1) DEMAG_CASE(2) DEMAG_CASE(4) DEMAG_CASE(8) DEMAG_CASE(16) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
    }
    if (L == 1024) {
        // three length-1024 columns do not fit the two-stage register layout
        using Sh = TileShape<T, 1024>;
        const size_t sm = 3 * swsize(1024 * Sh::TC) * sizeof(C);
        cudaError_t e = allow_smem<k_z_conv<T, 1024>>(sm);
        if (e != cudaSuccess) return e;
        const int grid = (ncols + Sh::TC - 1) / Sh::TC;
        k_z_conv<T, 1024><<<grid, Sh::NT, sm, st>>>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride);
        return cudaGetLastError();
    }
#define DEMAG_CASE(LL)                                                                         \
    case LL:                                                                                   \
        return variant == 1 ? zconv_launch<LL, 1>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st) \
             : variant == 2 ? zconv_launch<LL, 2>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st) \
             : variant == 4 ? zconv_launch<LL, 4>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st) \
                            : zconv_launch<LL, 0>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
    if (variant == 8) {  // 8-point second stage, two CTAs per SM (lengths 32..128)
        switch (L) {
        case 32: return zconv_launch<32, 8>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
        case 64: return zconv_launch<64, 8>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
        case 128: return zconv_launch<128, 8>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, st);
        default: variant = 0;
        }
    }
    switch (L) { DEMAG_CASE(32) DEMAG_CASE(64) DEMAG_CASE(128) DEMAG_CASE(256) DEMAG_CASE(512) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
}

template <typename T>
cudaError_t Passes<T>::sp_zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                int nout, const T *that, int Py, int Kx, const C *tw, const C *phx, const C *phy,
                                const C *phz, cudaStream_t st, int variant)
{
    if (ncols <= 0) return cudaSuccess;
    // zero padding: nz + 1 node rows out of L >= 2 nz
    if (L < 2 || 2 * nrows > L || nout != nrows + 1 || cs != (int64_t)nrows * rs) return cudaErrorInvalidValue;
    if (!pow2_len(L))
        return MixedPasses<T>::sp_zconv(L, S, ncols, width, ss, rs, cs, nrows, nout, that, Py, Kx, tw, phx, phy, phz, st);
    if (variant == 5) {
        cudaError_t e = cudaErrorNotSupported;
        switch (L) {
        case 32: e = sp_zconv_tma<T, 32>(S, ncols, width, ss, rs, cs, nrows, nout, that, Py, Kx, tw, phx, phy, phz, st); break;
        case 64: e = sp_zconv_tma<T, 64>(S, ncols, width, ss, rs, cs, nrows, nout, that, Py, Kx, tw, phx, phy, phz, st); break;
        case 128: e = sp_zconv_tma<T, 128>(S, ncols, width, ss, rs, cs, nrows, nout, that, Py, Kx, tw, phx, phy, phz, st); break;
        case 256: e = sp_zconv_tma<T, 256>(S, ncols, width, ss, rs, cs, nrows, nout, that, Py, Kx, tw, phx, phy, phz, st); break;
        default: break;
        }
        if (e != cudaErrorNotSupported) return e;
    }
    if (L <= 16) {
        const int grid = (ncols + Tile2<T>::NT - 1) / Tile2<T>::NT;
#define DEMAG_CASE(LL)                                                                         \
    case LL:                                                                                   \
        k_sp_z1<T, LL><<<grid, Tile2<T>::NT, 0, st>>>(S, ncols, width, ss, rs, cs, nrows, nout, that, Py, Kx, phx, phy, phz); \
        return cudaGetLastError();
        switch (L) { DEMAG_CASE(2) DEMAG_CASE(4) DEMAG_CASE(8) DEMAG_CASE(16) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
    }
#define DEMAG_CASE(LL)                                                                         \
    case LL: {                                                                                 \
        using Sh = ZShape<T, LL, 0>;                                                           \
        const size_t sm = 3 * swsize(LL * Sh::TC) * sizeof(C) + (LL / 2 + 1) * 3 * Sh::TC * sizeof(T); \
        const int grid = (ncols + Sh::TC - 1) / Sh::TC;                                        \
        cudaError_t e;                                                                         \
        if (2 * nout <= LL) {                                                                  \
            if ((e = allow_smem<k_sp_z2<T, LL, true>>(sm)) != cudaSuccess) return e;           \
            k_sp_z2<T, LL, true><<<grid, Sh::NT, sm, st>>>(S, ncols, width, ss, rs, cs, nrows, nout, that, Py, Kx, tw, phx, phy, phz); \
        } else {                                                                               \
            if ((e = allow_smem<k_sp_z2<T, LL, false>>(sm)) != cudaSuccess) return e;          \
            k_sp_z2<T, LL, false><<<grid, Sh::NT, sm, st>>>(S, ncols, width, ss, rs, cs, nrows, nout, that, Py, Kx, tw, phx, phy, phz); \
        }                                                                                      \
        return cudaGetLastError();                                                             \
    }
    switch (L) { DEMAG_CASE(32) DEMAG_CASE(64) DEMAG_CASE(128) DEMAG_CASE(256) DEMAG_CASE(512) default: return cudaErrorInvalidValue; }
#undef DEMAG_CASE
}

namespace {
// Cell layers per block of the field stencil: enough blocks to fill the GPU
// a few times over, each marching over a contiguous run of layers.
int sp_zchunk(int nx, int ny, int nz)
{
    const int64_t xy = (int64_t)((nx + 31) / 32) * ((ny + 7) / 8);
    const int64_t want = 8 * (int64_t)sm_count();
    int chunk = (int)((xy * nz + want - 1) / want);
    if (chunk < 1) chunk = 1;
    if (chunk > 16) chunk = 16;
    if (chunk > nz) chunk = nz;
    return chunk;
}
}  // namespace

template <typename T>
int Passes<T>::sp_grad_blocks(int nx, int ny, int nz)
{
    const int chunk = sp_zchunk(nx, ny, nz);
    return ((nx + 31) / 32) * ((ny + 7) / 8) * ((nz + chunk - 1) / chunk);
}

template <typename T>
cudaError_t Passes<T>::sp_grad(const T *phi, int nx, int ny, int nz, double dx, double dy, double dz, T *H,
                               const T *Mref, double *partials, cudaStream_t st)
{
    const int chunk = sp_zchunk(nx, ny, nz);
    const dim3 grid((nx + 31) / 32, (ny + 7) / 8, (nz + chunk - 1) / chunk);
    k_sp_grad<T><<<grid, dim3(32, 8), 0, st>>>(phi, nx, ny, nz, chunk, (T)(0.25 / dx), (T)(0.25 / dy),
                                               (T)(0.25 / dz), H, Mref, (T)1, partials);
    return cudaGetLastError();
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
