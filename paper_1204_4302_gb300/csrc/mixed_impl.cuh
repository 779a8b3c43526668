// Launchers of the mixed-radix passes (transform lengths that are not
// powers of two): stage plans and launches of the kernels in mixed.cuh.
#pragma once
#include <string.h>

#include "launch_util.cuh"
#include "mixed.cuh"
#include "plan.h"

namespace demag {

namespace {

// ceil(2^32 / d): n / d == umulhi(n, magic) for n d < 2^32 (d == 1 apart)
unsigned magic_of(int d) { return d <= 1 ? 0u : (unsigned)(((1ull << 32) + (unsigned)d - 1) / (unsigned)d); }

// Elements per tile of the mixed-radix kernels: the column and row passes
// hold two buffers, the z pass six (three components, ping-pong).
template <typename T> constexpr int gen_tile_elems(bool zpass)
{
    return sizeof(T) == 4 ? (zpass ? 2048 : 4096) : (zpass ? 1024 : 2048);
}

// Stage radices of the mixed-radix passes: every length <= 32 with prime
// factors 2, 3, 5, 7 (the in-register DFTs that mixed.cuh instantiates).
bool gen_stage_radix(int r)
{
    if (r < 2 || r > 32) return false;
    for (int f : {2, 3, 5, 7})
        while (r % f == 0) r /= f;
    return r == 1;
}

// Fewest stages (at most `depth`), then the smallest largest radix, radices
// in non-increasing order; false if L has no such split.
bool gen_split(int m, int maxr, int depth, int *cur, int n, int *best, int &bn, int &bmax)
{
    if (m == 1) {
        int mx = 0;
        for (int i = 0; i < n; ++i) mx = cur[i] > mx ? cur[i] : mx;
        if (bn == 0 || n < bn || (n == bn && mx < bmax)) {
            for (int i = 0; i < n; ++i) best[i] = cur[i];
            bn = n;
            bmax = mx;
        }
        return true;
    }
    if (depth == 0) return false;
    bool any = false;
    for (int r = maxr; r >= 2; --r)
        if (m % r == 0 && gen_stage_radix(r)) {
            cur[n] = r;
            any |= gen_split(m / r, r, depth - 1, cur, n + 1, best, bn, bmax);
        }
    return any;
}

// Stage plan of a mixed-radix transform of length L (a product of 2, 3, 5
// and 7, L < 2048) over tiles of about `tile` elements, radices <= maxr;
// comps components per grid column share the tile (z pass: 3).
bool gen_plan(int L, int tile, GenRadix &g, int maxr, int comps = 1)
{
    memset(&g, 0, sizeof g);
    if (L < 2 || L >= 2048) return false;
    g.L = L;
    const int cols = tile / L > 1 ? tile / L : 1;  // grid columns (rows of the x passes) per tile
    g.TC = comps * cols;                             // tile columns: the components side by side
    g.mCols = magic_of(cols);
    int cur[4], r[4], n = 0, mx = 0;
    if (!gen_split(L, maxr, 4, cur, 0, r, n, mx) || n == 0) return false;
    int NS = 1;
    for (int s = 0; s < n; ++s) {
        g.r[s] = r[s];
        g.NS[s] = NS;
        g.mNS[s] = magic_of(NS);
        g.mPer[s] = magic_of(L / r[s] * g.TC);
        g.mNB[s] = magic_of(L / r[s]);
        NS *= r[s];
    }
    g.n = n;
    g.mTC = magic_of(g.TC);
    g.mL = magic_of(L);
    g.mL1 = magic_of(L + 1);
    return true;
}

}  // namespace

template <typename T>
cudaError_t MixedPasses<T>::x_fwd(int L, const XIn<T> &a, int nrows, int nvalid, C *out, int64_t out_rs,
                                  const C *twx, cudaStream_t st)
{
    if (nrows <= 0) return cudaSuccess;
    GenRadix g;
    if (!gen_plan(L, gen_tile_elems<T>(false), g, kGenMaxRadixRows)) return cudaErrorInvalidValue;
    const size_t sm = gen_io_buffers(g.n, false) * swsize(L * g.TC) * sizeof(C);
    cudaError_t e = allow_smem<k_gen_x_fwd<T>>(sm);
    if (e != cudaSuccess) return e;
    k_gen_x_fwd<T><<<(nrows + g.TC - 1) / g.TC, kGenThreads, sm, st>>>(a, nrows, nvalid, out, out_rs, twx, g);
    return cudaGetLastError();
}

template <typename T>
int MixedPasses<T>::x_blocks(int L, int nrows)
{
    GenRadix g;
    if (!gen_plan(L, gen_tile_elems<T>(false), g, kGenMaxRadixRows)) return 1;
    return (nrows + g.TC - 1) / g.TC;
}

template <typename T>
cudaError_t MixedPasses<T>::x_inv(int L, const C *in, int64_t in_rs, int nrows, int nvalid, const XOut<T> &o,
                                  const C *twx, cudaStream_t st)
{
    if (nrows <= 0) return cudaSuccess;
    GenRadix g;
    if (!gen_plan(L, gen_tile_elems<T>(false), g, kGenMaxRadixRows)) return cudaErrorInvalidValue;
    const size_t sm = gen_io_buffers(g.n, true) * swsize(L * g.TC) * sizeof(C);
    cudaError_t e = allow_smem<k_gen_x_inv<T>>(sm);
    if (e != cudaSuccess) return e;
    k_gen_x_inv<T><<<(nrows + g.TC - 1) / g.TC, kGenThreads, sm, st>>>(in, in_rs, nrows, nvalid, o, twx, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t MixedPasses<T>::col(int L, bool inv, const C *in, C *out, int ncols, int width, int64_t iss, int64_t irs,
                                int nin, int64_t oss, int64_t ors, int nout, const C *tw, int twstride, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    GenRadix g;
    if (!gen_plan(L, gen_tile_elems<T>(false), g, kGenMaxRadixRows)) return cudaErrorInvalidValue;
    const size_t sm = gen_io_buffers(g.n, true) * swsize(L * g.TC) * sizeof(C);
    const unsigned mw = magic_of(width);
    const int grid = (ncols + g.TC - 1) / g.TC;
    cudaError_t e;
    if (inv) {
        if ((e = allow_smem<k_gen_col<T, true>>(sm)) != cudaSuccess) return e;
        k_gen_col<T, true><<<grid, kGenThreads, sm, st>>>(in, out, ncols, width, mw, iss, irs, nin, oss, ors, nout, tw,
                                                          twstride, g);
    } else {
        if ((e = allow_smem<k_gen_col<T, false>>(sm)) != cudaSuccess) return e;
        k_gen_col<T, false><<<grid, kGenThreads, sm, st>>>(in, out, ncols, width, mw, iss, irs, nin, oss, ors, nout,
                                                           tw, twstride, g);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t MixedPasses<T>::zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                  const T *nhat, int Py, int Kx, const C *tw, int twstride, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    if (nrows > L) return cudaErrorInvalidValue;
    GenRadix g;
    if (!gen_plan(L, gen_tile_elems<T>(true), g, kGenMaxRadixZ, 3)) return cudaErrorInvalidValue;
    const int cols = g.TC / 3;
    const size_t sm = 2 * swsize(L * g.TC) * sizeof(C);
    cudaError_t e = allow_smem<k_gen_zconv<T>>(sm);
    if (e != cudaSuccess) return e;
    k_gen_zconv<T><<<(ncols + cols - 1) / cols, kGenThreads, sm, st>>>(S, ncols, width, magic_of(width), ss, rs, cs,
                                                                       nrows, nhat, Py, Kx, tw, twstride, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t MixedPasses<T>::sp_zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
                                     int nrows, int nout, const T *that, int Py, int Kx, const C *tw, const C *phx,
                                     const C *phy, const C *phz, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    if (2 * nrows > L || nout != nrows + 1 || cs != (int64_t)nrows * rs) return cudaErrorInvalidValue;
    GenRadix g3, g1;
    if (!gen_plan(L, gen_tile_elems<T>(true), g3, kGenMaxRadixZ, 3)) return cudaErrorInvalidValue;
    if (!gen_plan(L, gen_tile_elems<T>(true), g1, kGenMaxRadixZ, 1)) return cudaErrorInvalidValue;
    const int cols = g1.TC;
    const size_t sm = 2 * swsize(L * g3.TC) * sizeof(C);
    cudaError_t e = allow_smem<k_gen_sp_zconv<T>>(sm);
    if (e != cudaSuccess) return e;
    k_gen_sp_zconv<T><<<(ncols + cols - 1) / cols, kGenThreads, sm, st>>>(S, ncols, width, magic_of(width), ss, rs,
                                                                          cs, nrows, nout, that, Py, Kx, tw, phx, phy,
                                                                          phz, g3, g1);
    return cudaGetLastError();
}

}  // namespace demag
