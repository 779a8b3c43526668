// Kernels of the scalar-potential method (SP, paper Sec. 3.1): the fused z
// pass that forms the potential spectrum from the three magnetization
// spectra, and the finite-difference field of the node potential.
//
// Potential (Eq. "scpot" with Eq. "convolution"): phi = S * M at the grid
// nodes, S the vector kernel of one homogeneously magnetized cell, evaluated
// at node-minus-cell offsets (q - 1/2) d. Its 3-D DFT on the padded grid is
//   S^_j(k) = -i Phi(k) T_j(k),  Phi(k) = exp(-pi i (kx/Px + ky/Py + kz/Pz)),
// with T_j real (S_j is odd along axis j and even along the others, about a
// half-integer centre). T_j is stored for kx < Kx, ky <= Py/2, kz <= Pz/2;
// folding ky -> Py - ky flips the sign of T_x and T_z, folding kz -> Pz - kz
// flips T_x and T_y. The potential spectrum is phi^ = sum_j S^_j M^_j.
//
// Field (Eq. "field"): H = -grad phi, per cell the average of -grad of the
// trilinear interpolant of its 8 corner potentials.
#pragma once
#include "fft2.cuh"

namespace demag {

// Spectral product at one frequency: sum_j sigma_j T_j m_j, times ph.
template <typename T, typename C>
__device__ __forceinline__ C sp_product(T tx, T ty, T tz, C mx, C my, C mz, C ph)
{
    const C a = cmk<C>(tx * mx.x + ty * my.x + tz * mz.x, tx * mx.y + ty * my.y + tz * mz.y);
    return cmul(a, ph);
}

// Fused SP z pass, two stages (32 <= L <= 512). Same tiling as k_z_conv2:
// forward stage 1 (radix R1, rows < nrows, upper half zero) for the three
// components into shared memory; forward stage 2 (radix R2) in registers;
// product with the kernel spectrum and the phase to one component; inverse
// stage 1 (radix R2) in registers to shared memory; inverse stage 2 (radix
// R1) stores the node rows z < nout (nz + 1 rows). The output overwrites
// component 0 in place and continues into the first row of component 1
// (cs == nrows * rs): only this CTA reads or writes its columns.
// POUT: nout <= L/2, so the last stage computes the lower half only.
template <typename T, int L, bool POUT>
__global__ void __launch_bounds__(ZShape<T, L, 0>::NT, 1)
k_sp_z2(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
        int nrows, int nout, const T *__restrict__ that, int Py, int Kx,
        const typename Cplx<T>::type *__restrict__ tw, const typename Cplx<T>::type *__restrict__ phx,
        const typename Cplx<T>::type *__restrict__ phy, const typename Cplx<T>::type *__restrict__ phz)
{
    using C = typename Cplx<T>::type;
    using Sh = ZShape<T, L, 0>;
    constexpr int R1 = Sh::R1, R2 = Sh::R2, NT = Sh::NT, TC = Sh::TC;
    constexpr int TS = swsize(L * TC);
    constexpr int NB1 = TC * R2;
    constexpr int HZ = L / 2 + 1;
    static_assert(NT % TC == 0, "tensor prefetch assumes TC divides the threads");
    static_assert((R1 * TC) % 32 == 0 && (R2 * TC) % 32 == 0, "shared-memory offsets need 32-aligned rows");
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    T *smT = reinterpret_cast<T *>(sm + 3 * TS);  // [kzf][comp][c] kernel block
    const int f0 = blockIdx.x * TC;
    const int hy = Py / 2 + 1;
    const int64_t plane = (int64_t)HZ * hy * Kx;

    tensor_block_prefetch<T, TC, NT, 3, HZ>(smT, that, f0, ncols, width, Py, Kx, plane);

    // forward stage 1, three components: rows j1 + r R2 -> rows j1 R1 + r
#pragma unroll
    for (int q = 0; q < (3 * NB1 + NT - 1) / NT; ++q) {
        const int b = threadIdx.x + q * NT;
        if (b < 3 * NB1) {
            const int comp = b / NB1, bb = b - comp * NB1;
            const int c = bb % TC, j1 = bb / TC, f = f0 + c;
            C u[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
            if (f < ncols) {
                const int i = f / width;
                const C *col = S + (int64_t)ky_pair_order(i, Py) * ss + (f - i * width) + comp * cs + j1 * rs;
#pragma unroll
                for (int r = 0; r < R1 / 2; ++r)
                    if (j1 + r * R2 < nrows) u[r] = col[(int64_t)r * R2 * rs];
            }
            RegDFTHalfIn<R1, false, C>::run(u);
            C *s = sm + comp * TS + sw(j1 * R1 * TC + c);
#pragma unroll
            for (int r = 0; r < R1; ++r) s[r * TC + (r * TC) / 32] = u[r];
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // forward stage 2 (three components) + product + inverse stage 1 (one)
    const bool act2 = threadIdx.x < TC * R1;
    const int c2 = threadIdx.x % TC, j2 = threadIdx.x / TC, f2 = f0 + c2;
    C p[R2];
    if (act2) {
        C v0[R2], v1[R2], v2[R2];
        const C *s = sm + sw(j2 * TC + c2);
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            constexpr int step = R1 * TC + (R1 * TC) / 32;
            v0[r] = s[r * step];
            v1[r] = s[TS + r * step];
            v2[r] = s[2 * TS + r * step];
        }
#pragma unroll
        for (int r = 1; r < R2; ++r) {
            const C w = __ldg(&tw[r * j2]);
            v0[r] = cmul(v0[r], w);
            v1[r] = cmul(v1[r], w);
            v2[r] = cmul(v2[r], w);
        }
        RegDFT<R2, false, C>::run(v0);
        RegDFT<R2, false, C>::run(v1);
        RegDFT<R2, false, C>::run(v2);
        if (f2 < ncols) {
            const int i = f2 / width, kx = f2 - i * width;
            const int ky = ky_pair_order(i, Py);
            const T sy = ky > Py / 2 ? (T)-1 : (T)1;
            // -i phx phy, the column's part of -i Phi
            const C pxy = cmul(__ldg(&phx[kx]), __ldg(&phy[ky]));
            const C cxy = cmk<C>(pxy.y, -pxy.x);
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                const int kz = j2 + r * R1;
                const bool up = kz > L / 2;
                const int kzf = up ? L - kz : kz;
                const T sz = up ? (T)-1 : (T)1;
                const T *t = smT + kzf * 3 * TC + c2;
                const C ph = cmul(cxy, __ldg(&phz[kz]));
                p[r] = sp_product<T, C>(sy * sz * t[0], sz * t[TC], sy * t[2 * TC], v0[r], v1[r], v2[r], ph);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R2; ++r) p[r] = cmk<C>(0, 0);
        }
        RegDFT<R2, true, C>::run(p);
    }
    __syncthreads();  // all stage-2 reads done before buffer 0 is rewritten
    if (act2) {
        C *s = sm + sw(j2 * R2 * TC + c2);
#pragma unroll
        for (int r = 0; r < R2; ++r) s[r * TC + (r * TC) / 32] = p[r];
    }
    __syncthreads();

    // inverse stage 2: radix R1 over rows j1 + r R2 (NS = R2), rows < nout kept
#pragma unroll
    for (int q = 0; q < (NB1 + NT - 1) / NT; ++q) {
        const int b = threadIdx.x + q * NT;
        if (b < NB1) {
            const int c = b % TC, j1 = b / TC, f = f0 + c;
            const C *s = sm + sw(j1 * TC + c);
            C u[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                constexpr int step = R2 * TC + (R2 * TC) / 32;
                u[r] = s[r * step];
            }
#pragma unroll
            for (int r = 1; r < R1; ++r) u[r] = cmulc(u[r], __ldg(&tw[r * j1]));
            if constexpr (POUT) RegDFTHalfOut<R1, true, C>::run(u);
            else RegDFT<R1, true, C>::run(u);
            if (f < ncols) {
                const int i = f / width;
                C *col = S + (int64_t)ky_pair_order(i, Py) * ss + (f - i * width) + j1 * rs;
#pragma unroll
                for (int r = 0; r < (POUT ? R1 / 2 : R1); ++r)
                    if (j1 + r * R2 < nout) col[(int64_t)r * R2 * rs] = u[r];
            }
        }
    }
}

// SP z pass for short columns (L <= 16): one thread per column, whole
// transforms in registers, the kernel spectrum read from global memory.
template <typename T, int L>
__global__ void __launch_bounds__(Tile2<T>::NT)
k_sp_z1(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
        int nrows, int nout, const T *__restrict__ that, int Py, int Kx,
        const typename Cplx<T>::type *__restrict__ phx, const typename Cplx<T>::type *__restrict__ phy,
        const typename Cplx<T>::type *__restrict__ phz)
{
    using C = typename Cplx<T>::type;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= ncols) return;
    const int ky = f / width, kx = f - ky * width;
    C *col = S + (int64_t)ky * ss + kx;
    C v0[L], v1[L], v2[L];
#pragma unroll
    for (int r = 0; r < L; ++r) {
        const bool in = r < nrows;
        v0[r] = in ? col[(int64_t)r * rs] : cmk<C>(0, 0);
        v1[r] = in ? col[cs + (int64_t)r * rs] : cmk<C>(0, 0);
        v2[r] = in ? col[2 * cs + (int64_t)r * rs] : cmk<C>(0, 0);
    }
    RegDFT<L, false, C>::run(v0);
    RegDFT<L, false, C>::run(v1);
    RegDFT<L, false, C>::run(v2);
    const int hy = Py / 2 + 1, HZ = L / 2 + 1;
    const int64_t plane = (int64_t)HZ * hy * Kx;
    const bool yup = ky > Py / 2;
    const int kyf = yup ? Py - ky : ky;
    const T sy = yup ? (T)-1 : (T)1;
    const C pxy = cmul(__ldg(&phx[kx]), __ldg(&phy[ky]));
    const C cxy = cmk<C>(pxy.y, -pxy.x);
#pragma unroll
    for (int kz = 0; kz < L; ++kz) {
        const bool up = kz > L / 2;
        const int kzf = up ? L - kz : kz;
        const T sz = up ? (T)-1 : (T)1;
        const int64_t b = ((int64_t)kzf * hy + kyf) * Kx + kx;
        const T tx = sy * sz * __ldg(&that[b]), ty = sz * __ldg(&that[plane + b]), tz = sy * __ldg(&that[2 * plane + b]);
        v0[kz] = sp_product<T, C>(tx, ty, tz, v0[kz], v1[kz], v2[kz], cmul(cxy, __ldg(&phz[kz])));
    }
    RegDFT<L, true, C>::run(v0);
#pragma unroll
    for (int r = 0; r < L; ++r)
        if (r < nout) col[(int64_t)r * rs] = v0[r];
}

// Field of the node potential phi[nz+1][ny+1][nx+1] (already scaled):
//   H_x = -(1/(4 dx)) sum of the x-differences along the cell's 4 x-edges,
// likewise y and z. Blocks of 32 x 8 cells in x-y march over zchunk cell
// layers; each node plane's differences and sums are computed once and kept
// for the next layer. Optional energy partials: sum over the block of
// mscale * M.H (one per block, in FP64).
template <typename T>
__global__ void __launch_bounds__(256)
k_sp_grad(const T *__restrict__ phi, int nx, int ny, int nz, int zchunk, T cx, T cy, T cz, T *__restrict__ H,
          const T *__restrict__ Mref, T mscale, double *__restrict__ partials)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    const int z0 = blockIdx.z * zchunk, z1 = min(nz, z0 + zchunk);
    const bool on = x < nx && y < ny;
    const int64_t sy = nx + 1, sz = (int64_t)(ny + 1) * (nx + 1);
    const int64_t ncell = (int64_t)nx * ny * nz;
    T gx0 = 0, gy0 = 0, s0 = 0;
    if (on) {
        const T *q = phi + (int64_t)z0 * sz + (int64_t)y * sy + x;
        const T a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + sy), d = __ldg(q + sy + 1);
        gx0 = (b - a) + (d - c);
        gy0 = (c - a) + (d - b);
        s0 = (a + b) + (c + d);
    }
    T acc = 0;
    for (int z = z0; z < z1; ++z) {
        if (!on) continue;
        const T *q = phi + (int64_t)(z + 1) * sz + (int64_t)y * sy + x;
        const T a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + sy), d = __ldg(q + sy + 1);
        const T gx1 = (b - a) + (d - c), gy1 = (c - a) + (d - b), s1 = (a + b) + (c + d);
        const T hx = -cx * (gx0 + gx1), hy = -cy * (gy0 + gy1), hz = -cz * (s1 - s0);
        const int64_t idx = ((int64_t)z * ny + y) * nx + x;
        if (H) {
            H[idx] = hx;
            H[ncell + idx] = hy;
            H[2 * ncell + idx] = hz;
        }
        if (partials) acc += mscale * (Mref[idx] * hx + Mref[ncell + idx] * hy + Mref[2 * ncell + idx] * hz);
        gx0 = gx1; gy0 = gy1; s0 = s1;
    }
    if (partials) {
        // block sum in FP64: warp shuffles, then one value per warp
        double v = (double)acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __shared__ double ws[8];
        const int w = threadIdx.y;  // one warp per threadIdx.y (blockDim.x == 32)
        if (threadIdx.x == 0) ws[w] = v;
        __syncthreads();
        if (w == 0 && threadIdx.x == 0) {
            double t = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) t += ws[k];
            partials[blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z)] = t;
        }
    }
}

}  // namespace demag
