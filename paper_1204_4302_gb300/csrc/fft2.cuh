// Two-stage register FFT kernels for the strided passes (y forward / inverse
// and the fused z pass). A column of length L = R1 * R2 is transformed by
// one radix-R1 stage and one radix-R2 stage, each a register DFT, with a
// single exchange through shared memory in between (Stockham order, the
// output in natural order). Columns with L <= 16 are transformed whole by one
// thread, with no exchange.
//
// The zero padding of the convolution is used twice: the forward input has
// at most L/2 non-zero rows, so the upper half of every first-stage input is
// zero at compile time; the inverse output is needed for at most L/2 rows, so
// the last stage computes only the lower half.
#pragma once
#include "fft_engine.cuh"

namespace demag {

// Radix pair (R1, R2) of a two-stage column transform of length L; variant 1
// swaps the two stages (a tuning choice).
template <int L> struct ColRadix0;
template <> struct ColRadix0<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct ColRadix0<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct ColRadix0<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct ColRadix0<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct ColRadix0<512> { static constexpr int R1 = 32, R2 = 16; };
template <> struct ColRadix0<1024> { static constexpr int R1 = 32, R2 = 32; };
template <int L, int V = 0> struct ColRadix {
    static constexpr int R1 = V == 0 ? ColRadix0<L>::R1 : ColRadix0<L>::R2;
    static constexpr int R2 = V == 0 ? ColRadix0<L>::R2 : ColRadix0<L>::R1;
};

// Radix pair of the fused z pass: the second stage keeps three components in
// registers for the tensor product, so R2 = 16.
template <int L> struct ZRadix { static constexpr int R2 = 16, R1 = L / 16; };

template <typename T> struct Tile2 { static constexpr int NT = 256; };
template <> struct Tile2<double> { static constexpr int NT = 128; };

// CTAs per SM the memory-bound passes are compiled for (register cap); more
// resident CTAs keep more loads in flight.
template <typename T, int L> struct Occ { static constexpr int MIN_CTAS = L <= 256 ? 4 : (L <= 512 ? 3 : 2); };
template <int L> struct Occ<double, L> { static constexpr int MIN_CTAS = 2; };

// Columns per CTA: the stage with fewer butterflies per column gives one
// butterfly to every thread, the other stage loops.
template <typename T, int L, int V = 0> struct ColShape {
    static constexpr int R1 = ColRadix<L, V>::R1, R2 = ColRadix<L, V>::R2;
    static constexpr int NT = Tile2<T>::NT;
    static constexpr int TC = NT / (R1 < R2 ? R1 : R2);
    static_assert((R1 * TC) % 32 == 0 && (TC % 32 == 0 || 32 % TC == 0),
                  "constant swizzled steps need 32-aligned row groups");
};
// z pass: every thread owns one stage-2 butterfly (three components); the
// CTA size NT is a tuning choice (variant 0: Tile2 threads, 1: half).
// Variant 0: TC = Tile2 threads / R1 columns; when R1 = 2 R2 the CTA has
// 3 TC R2 threads so both stage-1 passes give each thread one butterfly.
// Variant 1: half the columns.
// Variant 4: variant 0's thread layout on half the columns, compiled for two
// resident CTAs per SM (one CTA's loads overlap the other's arithmetic).
// Variant 8 (lengths 32..128): an 8-point second stage (three components of
// 8 complex values per thread across the product instead of 16), half-width
// tiles and two CTAs per SM.
template <int L, int V> struct ZRadixV {
    static constexpr int R2 = (V == 8 && L >= 32) ? 8 : ZRadix<L>::R2, R1 = L / R2;
};
template <typename T, int L, int V = 0> struct ZShape {
    static constexpr int R1 = ZRadixV<L, V>::R1, R2 = ZRadixV<L, V>::R2;
    static constexpr int TC = ((V == 1 || V == 4) ? Tile2<T>::NT / 2 : Tile2<T>::NT) / R1;
    static constexpr int NT = ((V == 0 || V == 4) && R1 == 2 * R2) ? 3 * TC * R2 : TC * R1;
    static constexpr int MIN_CTAS = (V == 4 || V == 8) ? 2 : 1;
};

// v[r] *= W_L^(r * k) (or its conjugate), table W_L^m at tw[m * twstride]
template <int R, int L, bool INV, typename C>
__device__ __forceinline__ void twiddle_row(C *v, int k, const C *__restrict__ tw, int twstride)
{
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const C w = __ldg(&tw[((r * k) % L) * twstride]);
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
    }
}

// Global load of a buffer that another CTA of the same launch may have
// written (persistent batch kernel): bypass L1, which is not coherent.
template <bool CG, typename V>
__device__ __forceinline__ V ldp(const V *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// 4-byte asynchronous global -> shared copy (no register staging).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---------------------------------------------------------------- columns
// Strided column transform, column f = slab * width + off, element r at
// slab * ss + r * rs + off. PIN: rows >= L/2 of the input are zero (nin <=
// L/2). POUT: only rows < L/2 are stored (nout <= L/2).
template <typename T, int L, bool INV, bool PIN, bool POUT, bool CG, int V = 0>
__device__ __forceinline__ void k_col2_tile(const typename Cplx<T>::type *__restrict__ in, typename Cplx<T>::type *__restrict__ out, int ncols,
       int width, int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, int nout,
       const typename Cplx<T>::type *__restrict__ tw, int twstride, int tile, unsigned char *smraw)
{
    using C = typename Cplx<T>::type;
    using S = ColShape<T, L, V>;
    constexpr int R1 = S::R1, R2 = S::R2, NT = S::NT, TC = S::TC;
    C *sm = reinterpret_cast<C *>(smraw);
    const int f0 = tile * TC;
    // stage 1: radix R1 over rows j1 + r R2, j1 < R2
#pragma unroll
    for (int q = 0; q < (TC * R2 + NT - 1) / NT; ++q) {
        const int b = threadIdx.x + q * NT;
        if (b < TC * R2) {
            const int c = b % TC, j1 = b / TC, f = f0 + c;
            C u[R1];
            const bool ok = f < ncols;
            int64_t base = 0;
            if (ok) {
                const int slab = f / width;
                base = (int64_t)slab * iss + (f - slab * width);
            }
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int row = j1 + r * R2;
                u[r] = cmk<C>(0, 0);
                if (!(PIN && r >= R1 / 2) && ok && row < nin) u[r] = ldp<CG>(&in[base + (int64_t)row * irs]);
            }
            if constexpr (PIN) RegDFTHalfIn<R1, INV, C>::run(u);
            else RegDFT<R1, INV, C>::run(u);
            // R1 TC is a multiple of 32 and TC a power of two: constant swizzled steps
            C *s = sm + sw(j1 * R1 * TC + c);
#pragma unroll
            for (int r = 0; r < R1; ++r) s[r * TC + (r * TC) / 32] = u[r];
        }
    }
    __syncthreads();
    // stage 2: radix R2 over rows j2 + r R1, j2 < R1; output rows j2 + r R1
#pragma unroll
    for (int q = 0; q < (TC * R1 + NT - 1) / NT; ++q) {
        const int b = threadIdx.x + q * NT;
        if (b < TC * R1) {
            const int c = b % TC, j2 = b / TC, f = f0 + c;
            C v[R2];
            const C *s = sm + sw(j2 * TC + c);
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = s[r * (R1 * TC + (R1 * TC) / 32)];
            twiddle_row<R2, L, INV>(v, j2, tw, twstride);
            if constexpr (POUT) RegDFTHalfOut<R2, INV, C>::run(v);
            else RegDFT<R2, INV, C>::run(v);
            if (f < ncols) {
                const int slab = f / width;
                const int64_t base = (int64_t)slab * oss + (f - slab * width);
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    const int row = j2 + r * R1;
                    if (!(POUT && r >= R2 / 2) && row < nout) out[base + (int64_t)row * ors] = v[r];
                }
            }
        }
    }
}

template <typename T, int L, bool INV, bool PIN, bool POUT, int V = 0>
__global__ void __launch_bounds__(Tile2<T>::NT, Occ<T, L>::MIN_CTAS)
k_col2(const typename Cplx<T>::type *__restrict__ in, typename Cplx<T>::type *__restrict__ out, int ncols,
       int width, int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, int nout,
       const typename Cplx<T>::type *__restrict__ tw, int twstride)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_col2_tile<T, L, INV, PIN, POUT, false, V>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, tw, twstride, blockIdx.x, smraw);
}

// Three-stage column transform for long columns (L = 512, 1024): radices
// 8 x 8 x 8 (or 8 x 8 x 16), so each thread holds at most 16 values and many
// more CTAs fit on an SM; one more shared-memory exchange than k_col2. First
// stage from global memory, middle stage in shared memory, last stage to
// global memory. A tuning variant of k_col2 with the same result.
template <int L> struct Col3Radix;
template <> struct Col3Radix<512> { static constexpr int R1 = 8, R2 = 8, R3 = 8; };
template <> struct Col3Radix<1024> { static constexpr int R1 = 8, R2 = 8, R3 = 16; };

template <typename T, int L> struct Col3Shape {
    static constexpr int R1 = Col3Radix<L>::R1, R2 = Col3Radix<L>::R2, R3 = Col3Radix<L>::R3;
    static constexpr int NT = 2 * Tile2<T>::NT;
    static constexpr int TC = 8;
    static_assert((R1 * TC) % 32 == 0 && ((L / R3) * TC) % 32 == 0 && 32 % TC == 0,
                  "constant swizzled steps need 32-aligned row groups");
};

template <typename T, int L, bool INV, bool PIN, bool POUT>
__global__ void __launch_bounds__(Col3Shape<T, L>::NT)
k_col3(const typename Cplx<T>::type *__restrict__ in, typename Cplx<T>::type *__restrict__ out, int ncols,
       int width, int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, int nout,
       const typename Cplx<T>::type *__restrict__ tw, int twstride)
{
    using C = typename Cplx<T>::type;
    using S = Col3Shape<T, L>;
    constexpr int R1 = S::R1, R2 = S::R2, R3 = S::R3, NT = S::NT, TC = S::TC;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int f0 = blockIdx.x * TC;
    // stage 1: radix R1 over rows j1 + r L/R1 -> rows j1 R1 + r
#pragma unroll
    for (int q = 0; q < (TC * (L / R1) + NT - 1) / NT; ++q) {
        const int b = threadIdx.x + q * NT;
        if (b < TC * (L / R1)) {
            const int c = b % TC, j1 = b / TC, f = f0 + c;
            C u[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
            if (f < ncols) {
                const int slab = f / width;
                const C *col = in + (int64_t)slab * iss + (f - slab * width);
#pragma unroll
                for (int r = 0; r < (PIN ? R1 / 2 : R1); ++r) {
                    const int row = j1 + r * (L / R1);
                    if (row < nin) u[r] = col[(int64_t)row * irs];
                }
            }
            if constexpr (PIN) RegDFTHalfIn<R1, INV, C>::run(u);
            else RegDFT<R1, INV, C>::run(u);
            // R1 TC is a multiple of 32 and TC divides 32: constant swizzled steps
            C *s = sm + sw(j1 * R1 * TC + c);
#pragma unroll
            for (int r = 0; r < R1; ++r) s[r * TC + (r * TC) / 32] = u[r];
        }
    }
    __syncthreads();
    // stage 2 in shared memory (radix R2, NS = R1)
    fft_stage<C, L, R2, R1, INV, NT, TC>(sm, tw, twstride);
    // stage 3: radix R3, NS = R1 R2 = L / R3; outputs rows j + r L/R3
#pragma unroll
    for (int q = 0; q < (TC * (L / R3) + NT - 1) / NT; ++q) {
        const int b = threadIdx.x + q * NT;
        if (b < TC * (L / R3)) {
            const int c = b % TC, j = b / TC, f = f0 + c;
            C v[R3];
            const C *s = sm + sw(j * TC + c);
#pragma unroll
            for (int r = 0; r < R3; ++r) v[r] = s[r * ((L / R3) * TC + (L / R3) * TC / 32)];
            twiddle_row<R3, L, INV>(v, j, tw, twstride);
            if constexpr (POUT) RegDFTHalfOut<R3, INV, C>::run(v);
            else RegDFT<R3, INV, C>::run(v);
            if (f < ncols) {
                const int slab = f / width;
                C *col = out + (int64_t)slab * oss + (f - slab * width);
#pragma unroll
                for (int r = 0; r < (POUT ? R3 / 2 : R3); ++r) {
                    const int row = j + r * (L / R3);
                    if (row < nout) col[(int64_t)row * ors] = v[r];
                }
            }
        }
    }
}

// Short columns (L <= 16): one thread per column, no shared memory.
template <typename T, int L, bool INV, bool CG>
__device__ __forceinline__ void k_col1_tile(const typename Cplx<T>::type *__restrict__ in, typename Cplx<T>::type *__restrict__ out, int ncols,
       int width, int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, int nout, int tile, unsigned char *smraw)
{
    using C = typename Cplx<T>::type;
    const int f = tile * Tile2<T>::NT + threadIdx.x;
    if (f >= ncols) return;
    const int slab = f / width, off = f - slab * width;
    const int64_t bi = (int64_t)slab * iss + off, bo = (int64_t)slab * oss + off;
    C u[L];
#pragma unroll
    for (int r = 0; r < L; ++r) u[r] = r < nin ? ldp<CG>(&in[bi + (int64_t)r * irs]) : cmk<C>(0, 0);
    RegDFT<L, INV, C>::run(u);
#pragma unroll
    for (int r = 0; r < L; ++r)
        if (r < nout) out[bo + (int64_t)r * ors] = u[r];
}

template <typename T, int L, bool INV>
__global__ void __launch_bounds__(Tile2<T>::NT)
k_col1(const typename Cplx<T>::type *__restrict__ in, typename Cplx<T>::type *__restrict__ out, int ncols,
       int width, int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, int nout)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_col1_tile<T, L, INV, false>(in, out, ncols, width, iss, irs, nin, oss, ors, nout, blockIdx.x, smraw);
}

// ---------------------------------------------------------------- z pass
// Tensor product at one frequency: h = -N^ m with the folded, parity-signed
// tensor spectrum (see k_z_conv).
template <typename T, typename C>
__device__ __forceinline__ void tensor_product(const T *__restrict__ nhat, int64_t plane, int64_t b, T sy,
                                               T sz, C &x, C &y, C &z)
{
    const T nxx = __ldg(&nhat[b]), nyy = __ldg(&nhat[plane + b]), nzz = __ldg(&nhat[2 * plane + b]);
    const T nxy = sy * __ldg(&nhat[3 * plane + b]);
    const T nxz = sz * __ldg(&nhat[4 * plane + b]);
    const T nyz = sy * sz * __ldg(&nhat[5 * plane + b]);
    const C mx = x, my = y, mz = z;
    x = cmk<C>(-(nxx * mx.x + nxy * my.x + nxz * mz.x), -(nxx * mx.y + nxy * my.y + nxz * mz.y));
    y = cmk<C>(-(nxy * mx.x + nyy * my.x + nyz * mz.x), -(nxy * mx.y + nyy * my.y + nyz * mz.y));
    z = cmk<C>(-(nxz * mx.x + nyz * my.x + nzz * mz.x), -(nxz * mx.y + nyz * my.y + nzz * mz.y));
}

// m^H N^ m at one frequency for the real symmetric folded tensor (the
// spectral energy density of the Parseval form of E, paper Sec. 2).
template <typename T, typename C>
__device__ __forceinline__ T quad_form(const C &x, const C &y, const C &z, T nxx, T nyy, T nzz, T nxy, T nxz, T nyz)
{
    const T pxx = x.x * x.x + x.y * x.y, pyy = y.x * y.x + y.y * y.y, pzz = z.x * z.x + z.y * z.y;
    const T pxy = x.x * y.x + x.y * y.y, pxz = x.x * z.x + x.y * z.y, pyz = y.x * z.x + y.y * z.y;
    return nxx * pxx + nyy * pyy + nzz * pzz + (T)2 * (nxy * pxy + nxz * pxz + nyz * pyz);
}

// Weight of column kx in the half spectrum's Parseval sum: the columns kx = 0
// and kx = Px/2 (= Kx - 1 for Px >= 2) stand for themselves, every other one
// for itself and its Hermitian partner.
template <typename T>
__device__ __forceinline__ T kx_weight(int kx, int Kx)
{
    return (kx == 0 || kx == Kx - 1) ? (T)1 : (T)2;
}

// Order of the ky rows over the z-pass CTAs: 0, Py/2, 1, Py-1, 2, Py-2, ...
// so that the two rows sharing a folded tensor row run at about the same
// time and the second read of that tensor block hits L2.
__device__ __forceinline__ int ky_pair_order(int i, int Py)
{
    if (i == 0) return 0;
    if (i == 1) return Py / 2;
    const int m = i >> 1;
    return (i & 1) ? Py - m : m;
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem)
{
    if constexpr (sizeof(T) == 4) cp_async4(smem, gmem);
    else cp_async8(smem, gmem);
}

// Copy the CTA's block of a folded spectral table ([NC][HZ][Py/2+1][Kx]) to
// shared memory as [kzf][comp][c] with cp.async. Thread (g, c) handles the
// entries kzf * NC + comp = g, g + G, ... (G = NT / TC); (kzf, comp) and the
// source offset advance incrementally.
template <typename T, int TC, int NT, int NC, int HZ>
__device__ __forceinline__ void tensor_block_prefetch(T *smT, const T *__restrict__ tab, int f0, int ncols, int width,
                                                      int Py, int Kx, int64_t plane)
{
    constexpr int G = NT / TC, GQ = G / NC, GR = G % NC;
    const int c = threadIdx.x % TC, f = f0 + c, g = threadIdx.x / TC;
    if (f >= ncols) return;
    const int i = f / width, kx = f - i * width;
    const int ky = ky_pair_order(i, Py);
    const int kyf = ky > Py / 2 ? Py - ky : ky;
    const int64_t zs = (int64_t)(Py / 2 + 1) * Kx;
    const T *src = tab + (int64_t)kyf * Kx + kx;
    int comp = g % NC;
    int64_t off = comp * plane + (int64_t)(g / NC) * zs;
    const int64_t step = GQ * zs + GR * plane, wrap = zs - NC * plane;
    for (int idx = g; idx < HZ * NC; idx += G) {
        cp_async_elem(&smT[idx * TC + c], src + off);
        comp += GR;
        off += step;
        if (comp >= NC) {
            comp -= NC;
            off += wrap;
        }
    }
}

// Fused z pass, two stages (L >= 32): forward stage 1 (radix R1, rows < nrows
// read, upper half zero) for the three components into shared memory;
// forward stage 2 (radix R2) into registers, which then hold the three
// components at the frequencies kz = j2 + r R1; tensor product in
// registers; inverse stage 1 (radix R2) in registers back to shared memory;
// inverse stage 2 (radix R1) stores the rows z < nrows. Column f = i * width
// + kx with ky = ky_pair_order(i). The CTA's block of the tensor spectrum
// ([6][L/2+1][Py/2+1][Kx], folded in ky and kz) is copied to shared memory
// asynchronously while the first stage runs.
template <typename T, int L, int V, bool CG, bool EONLY = false>
__device__ __forceinline__ void k_z_conv2_tile(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
          int nrows, const T *__restrict__ nhat, int Py, int Kx, const typename Cplx<T>::type *__restrict__ tw,
          int twstride, int tile, unsigned char *smraw, double *partials = nullptr)
{
    using C = typename Cplx<T>::type;
    using Sh = ZShape<T, L, V>;
    constexpr int R1 = Sh::R1, R2 = Sh::R2, NT = Sh::NT, TC = Sh::TC;
    constexpr int TS = swsize(L * TC);
    constexpr int NB1 = TC * R2;  // stage-1 butterflies per component
    constexpr int HZ = L / 2 + 1;
    static_assert(NT % TC == 0, "tensor prefetch assumes TC divides the threads");
    static_assert((R1 * TC) % 32 == 0 && (R2 * TC) % 32 == 0, "shared-memory offsets need 32-aligned rows");
    C *sm = reinterpret_cast<C *>(smraw);
    T *smT = reinterpret_cast<T *>(sm + 3 * TS);  // [kzf][comp][c] tensor block
    const int f0 = tile * TC;
    const int hy = Py / 2 + 1;
    const int64_t plane = (int64_t)HZ * hy * Kx;

    tensor_block_prefetch<T, TC, NT, 6, HZ>(smT, nhat, f0, ncols, width, Py, Kx, plane);

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
                    if (j1 + r * R2 < nrows) u[r] = ldp<CG>(&col[(int64_t)r * R2 * rs]);
            }
            RegDFTHalfIn<R1, false, C>::run(u);
            C *s = sm + comp * TS + sw(j1 * R1 * TC + c);
#pragma unroll
            for (int r = 0; r < R1; ++r) s[r * TC + (r * TC) / 32] = u[r];
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // forward stage 2 + product + inverse stage 1
    const bool act2 = threadIdx.x < TC * R1;
    const int c2 = threadIdx.x % TC, j2 = threadIdx.x / TC, f2 = f0 + c2;
    C v0[R2], v1[R2], v2[R2];
    T e = 0;  // EONLY: this thread's part of sum_k w m^H N^ m
    if (act2) {
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
            const C w = __ldg(&tw[r * j2 * twstride]);
            v0[r] = cmul(v0[r], w);
            v1[r] = cmul(v1[r], w);
            v2[r] = cmul(v2[r], w);
        }
        RegDFT<R2, false, C>::run(v0);
        RegDFT<R2, false, C>::run(v1);
        RegDFT<R2, false, C>::run(v2);
        if (f2 < ncols) {
            const int ky = ky_pair_order(f2 / width, Py);
            const T sy = ky > Py / 2 ? (T)-1 : (T)1;
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                // kz = j2 + r R1: below L/2 for r < R2/2, above for r > R2/2
                int kzf;
                T sz;
                if (r < R2 / 2) { kzf = j2 + r * R1; sz = (T)1; }
                else if (r == R2 / 2) { kzf = L / 2 - j2; sz = j2 == 0 ? (T)1 : (T)-1; }
                else { kzf = (R2 - r) * R1 - j2; sz = (T)-1; }
                const T *t = smT + kzf * 6 * TC + c2;
                const T nxx = t[0], nyy = t[TC], nzz = t[2 * TC];
                const T nxy = sy * t[3 * TC], nxz = sz * t[4 * TC], nyz = sy * sz * t[5 * TC];
                const C mx = v0[r], my = v1[r], mz = v2[r];
                if constexpr (EONLY) {
                    e += quad_form<T>(mx, my, mz, nxx, nyy, nzz, nxy, nxz, nyz);
                } else {
                    v0[r] = cmk<C>(-(nxx * mx.x + nxy * my.x + nxz * mz.x), -(nxx * mx.y + nxy * my.y + nxz * mz.y));
                    v1[r] = cmk<C>(-(nxy * mx.x + nyy * my.x + nyz * mz.x), -(nxy * mx.y + nyy * my.y + nyz * mz.y));
                    v2[r] = cmk<C>(-(nxz * mx.x + nyz * my.x + nzz * mz.x), -(nxz * mx.y + nyz * my.y + nzz * mz.y));
                }
            }
            if constexpr (EONLY) e *= kx_weight<T>(f2 - (f2 / width) * width, Kx);
        }
        if constexpr (!EONLY) {
            RegDFT<R2, true, C>::run(v0);
            RegDFT<R2, true, C>::run(v1);
            RegDFT<R2, true, C>::run(v2);
        }
    }
    if constexpr (EONLY) {
        block_partial<NT>((double)e, partials, tile);
        return;
    }
    __syncthreads();  // all stage-2 reads done before the buffers are rewritten
    if (act2) {
        C *s = sm + sw(j2 * R2 * TC + c2);
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            const int o = r * TC + (r * TC) / 32;
            s[o] = v0[r];
            s[TS + o] = v1[r];
            s[2 * TS + o] = v2[r];
        }
    }
    __syncthreads();

    // inverse stage 2: radix R1 over rows j1 + r R2 (NS = R2), rows < nrows kept
#pragma unroll
    for (int q = 0; q < (3 * NB1 + NT - 1) / NT; ++q) {
        const int b = threadIdx.x + q * NT;
        if (b < 3 * NB1) {
            const int comp = b / NB1, bb = b - comp * NB1;
            const int c = bb % TC, j1 = bb / TC, f = f0 + c;
            const C *s = sm + comp * TS + sw(j1 * TC + c);
            C u[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                constexpr int step = R2 * TC + (R2 * TC) / 32;
                u[r] = s[r * step];
            }
#pragma unroll
            for (int r = 1; r < R1; ++r) u[r] = cmulc(u[r], __ldg(&tw[r * j1 * twstride]));
            RegDFTHalfOut<R1, true, C>::run(u);
            if (f < ncols) {
                const int i = f / width;
                C *col = S + (int64_t)ky_pair_order(i, Py) * ss + (f - i * width) + comp * cs + j1 * rs;
#pragma unroll
                for (int r = 0; r < R1 / 2; ++r)
                    if (j1 + r * R2 < nrows) col[(int64_t)r * R2 * rs] = u[r];
            }
        }
    }
}

template <typename T, int L, int V>
__global__ void __launch_bounds__(ZShape<T, L, V>::NT, ZShape<T, L, V>::MIN_CTAS)
k_z_conv2(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
          int nrows, const T *__restrict__ nhat, int Py, int Kx, const typename Cplx<T>::type *__restrict__ tw,
          int twstride)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_z_conv2_tile<T, L, V, false>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, blockIdx.x, smraw);
}

// Spectral energy of the z columns (EONLY form of k_z_conv2): forward z
// transforms, then per CTA the sum over its columns and all kz of
// w(kx) m^H N^ m into partials[blockIdx.x]; nothing is written back.
template <typename T, int L, int V>
__global__ void __launch_bounds__(ZShape<T, L, V>::NT, ZShape<T, L, V>::MIN_CTAS)
k_z_energy2(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
            int nrows, const T *__restrict__ nhat, int Py, int Kx, const typename Cplx<T>::type *__restrict__ tw,
            int twstride, double *__restrict__ partials)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_z_conv2_tile<T, L, V, false, true>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, tw, twstride, blockIdx.x,
                                         smraw, partials);
}

// Fused z pass, persistent and software pipelined (L >= 32): each CTA loops
// over tiles; while a tile is transformed, the next tile's input rows
// (three components, rows < nrows) and its tensor block are copied into
// shared memory with cp.async, so the copies overlap the arithmetic of the
// current tile. Same arithmetic and result as k_z_conv2.
template <typename T, int L>
__global__ void __launch_bounds__(ZShape<T, L, 0>::NT, 1)
k_z_conv3(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
          int nrows, const T *__restrict__ nhat, int Py, int Kx, const typename Cplx<T>::type *__restrict__ tw,
          int twstride, int ntiles)
{
    using C = typename Cplx<T>::type;
    using Sh = ZShape<T, L, 0>;
    constexpr int R1 = Sh::R1, R2 = Sh::R2, NT = Sh::NT, TC = Sh::TC;
    constexpr int TS = swsize(L * TC);
    constexpr int NB1 = TC * R2;
    constexpr int HZ = L / 2 + 1;
    constexpr int NZ2 = L / 2;  // at most L/2 input rows
    static_assert(NT % TC == 0, "tensor prefetch assumes TC divides the threads");
    static_assert((R1 * TC) % 32 == 0 && (R2 * TC) % 32 == 0, "shared-memory offsets need 32-aligned rows");
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);        // exchange [3][TS]
    C *stg = sm + 3 * TS;                        // staged input [3][NZ2][TC]
    T *smT = reinterpret_cast<T *>(stg + 3 * NZ2 * TC);  // tensor block [HZ][6][TC]
    const int hy = Py / 2 + 1;
    const int64_t plane = (int64_t)HZ * hy * Kx;

    auto issue_input = [&](int tile) {
        // thread -> fixed column c (NT is a multiple of TC); rows strided by NT / TC
        const int c = threadIdx.x % TC, f = tile * TC + c;
        if (f >= ncols) return;
        const int i = f / width;
        const C *base = S + (int64_t)ky_pair_order(i, Py) * ss + (f - i * width);
        for (int row = threadIdx.x / TC; row < nrows; row += NT / TC) {
            const C *src = base + (int64_t)row * rs;
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                C *dst = &stg[(comp * NZ2 + row) * TC + c];
                if constexpr (sizeof(C) == 8) cp_async8(dst, src + comp * cs);
                else {
                    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src + comp * cs) : "memory");
                }
            }
        }
    };
    auto issue_tensor = [&](int tile) {
        const int c = threadIdx.x % TC, f = tile * TC + c;
        if (f < ncols) {
            const int i = f / width, kx = f - i * width;
            const int ky = ky_pair_order(i, Py);
            const int kyf = ky > Py / 2 ? Py - ky : ky;
            const T *src = nhat + (int64_t)kyf * Kx + kx;
            for (int idx = threadIdx.x / TC; idx < HZ * 6; idx += NT / TC) {
                const int kzf = idx / 6, comp = idx - kzf * 6;
                cp_async_elem(&smT[idx * TC + c], src + comp * plane + (int64_t)kzf * hy * Kx);
            }
        }
    };

    int tile = blockIdx.x;
    if (tile < ntiles) {
        issue_input(tile);
        issue_tensor(tile);
    }
    cp_async_wait_all();
    __syncthreads();
    for (; tile < ntiles; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        const int f0 = tile * TC;
        // forward stage 1 from the staged rows
#pragma unroll
        for (int q = 0; q < (3 * NB1 + NT - 1) / NT; ++q) {
            const int b = threadIdx.x + q * NT;
            if (b < 3 * NB1) {
                const int comp = b / NB1, bb = b - comp * NB1;
                const int c = bb % TC, j1 = bb / TC;
                C u[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
                if (f0 + c < ncols) {
                    const C *col = stg + (comp * NZ2 + j1) * TC + c;
#pragma unroll
                    for (int r = 0; r < R1 / 2; ++r)
                        if (j1 + r * R2 < nrows) u[r] = col[r * R2 * TC];
                }
                RegDFTHalfIn<R1, false, C>::run(u);
                C *s = sm + comp * TS + sw(j1 * R1 * TC + c);
#pragma unroll
                for (int r = 0; r < R1; ++r) s[r * TC + (r * TC) / 32] = u[r];
            }
        }
        __syncthreads();
        if (next < ntiles) issue_input(next);  // the staging buffer is free again

        const bool act2 = threadIdx.x < TC * R1;
        const int c2 = threadIdx.x % TC, j2 = threadIdx.x / TC, f2 = f0 + c2;
        C v0[R2], v1[R2], v2[R2];
        if (act2) {
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
                const C w = __ldg(&tw[r * j2 * twstride]);
                v0[r] = cmul(v0[r], w);
                v1[r] = cmul(v1[r], w);
                v2[r] = cmul(v2[r], w);
            }
            RegDFT<R2, false, C>::run(v0);
            RegDFT<R2, false, C>::run(v1);
            RegDFT<R2, false, C>::run(v2);
            if (f2 < ncols) {
                const int ky = ky_pair_order(f2 / width, Py);
                const T sy = ky > Py / 2 ? (T)-1 : (T)1;
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    int kzf;
                    T sz;
                    if (r < R2 / 2) { kzf = j2 + r * R1; sz = (T)1; }
                    else if (r == R2 / 2) { kzf = L / 2 - j2; sz = j2 == 0 ? (T)1 : (T)-1; }
                    else { kzf = (R2 - r) * R1 - j2; sz = (T)-1; }
                    const T *t = smT + kzf * 6 * TC + c2;
                    const T nxx = t[0], nyy = t[TC], nzz = t[2 * TC];
                    const T nxy = sy * t[3 * TC], nxz = sz * t[4 * TC], nyz = sy * sz * t[5 * TC];
                    const C mx = v0[r], my = v1[r], mz = v2[r];
                    v0[r] = cmk<C>(-(nxx * mx.x + nxy * my.x + nxz * mz.x), -(nxx * mx.y + nxy * my.y + nxz * mz.y));
                    v1[r] = cmk<C>(-(nxy * mx.x + nyy * my.x + nyz * mz.x), -(nxy * mx.y + nyy * my.y + nyz * mz.y));
                    v2[r] = cmk<C>(-(nxz * mx.x + nyz * my.x + nzz * mz.x), -(nxz * mx.y + nyz * my.y + nzz * mz.y));
                }
            }
            RegDFT<R2, true, C>::run(v0);
            RegDFT<R2, true, C>::run(v1);
            RegDFT<R2, true, C>::run(v2);
        }
        __syncthreads();  // stage-2 reads of the exchange and the tensor block are done
        if (next < ntiles) issue_tensor(next);
        if (act2) {
            C *s = sm + sw(j2 * R2 * TC + c2);
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                const int o = r * TC + (r * TC) / 32;
                s[o] = v0[r];
                s[TS + o] = v1[r];
                s[2 * TS + o] = v2[r];
            }
        }
        __syncthreads();
        // inverse stage 2, rows < nrows stored
#pragma unroll
        for (int q = 0; q < (3 * NB1 + NT - 1) / NT; ++q) {
            const int b = threadIdx.x + q * NT;
            if (b < 3 * NB1) {
                const int comp = b / NB1, bb = b - comp * NB1;
                const int c = bb % TC, j1 = bb / TC, f = f0 + c;
                const C *s = sm + comp * TS + sw(j1 * TC + c);
                C u[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    constexpr int step = R2 * TC + (R2 * TC) / 32;
                    u[r] = s[r * step];
                }
#pragma unroll
                for (int r = 1; r < R1; ++r) u[r] = cmulc(u[r], __ldg(&tw[r * j1 * twstride]));
                RegDFTHalfOut<R1, true, C>::run(u);
                if (f < ncols) {
                    const int i = f / width;
                    C *col = S + (int64_t)ky_pair_order(i, Py) * ss + (f - i * width) + comp * cs + j1 * rs;
#pragma unroll
                    for (int r = 0; r < R1 / 2; ++r)
                        if (j1 + r * R2 < nrows) col[(int64_t)r * R2 * rs] = u[r];
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();  // next tile's copies have landed; the exchange is free
    }
}

// Fused z pass for L <= 16: one thread per column, all in registers.
template <typename T, int L, bool CG, bool EONLY = false>
__device__ __forceinline__ void k_z_conv1_tile(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
          int nrows, const T *__restrict__ nhat, int Py, int Kx, int tile, unsigned char *smraw, double *partials = nullptr)
{
    using C = typename Cplx<T>::type;
    const int f = tile * Tile2<T>::NT + threadIdx.x;
    if constexpr (EONLY) {
        T e = 0;
        if (f < ncols) {
            const int ky = f / width, kx = f - ky * width;
            const int64_t base = (int64_t)ky * ss + kx;
            C a[L], b[L], c[L];
#pragma unroll
            for (int r = 0; r < L; ++r) {
                const bool ok = r < nrows;
                a[r] = ok ? S[base + (int64_t)r * rs] : cmk<C>(0, 0);
                b[r] = ok ? S[base + (int64_t)r * rs + cs] : cmk<C>(0, 0);
                c[r] = ok ? S[base + (int64_t)r * rs + 2 * cs] : cmk<C>(0, 0);
            }
            RegDFT<L, false, C>::run(a);
            RegDFT<L, false, C>::run(b);
            RegDFT<L, false, C>::run(c);
            const bool fy = ky > Py / 2;
            const int kyf = fy ? Py - ky : ky;
            const T sy = fy ? (T)-1 : (T)1;
            const int hy = Py / 2 + 1;
            const int64_t plane = (int64_t)(L / 2 + 1) * hy * Kx;
#pragma unroll
            for (int r = 0; r < L; ++r) {
                const bool fz = r > L / 2;
                const T sz = fz ? (T)-1 : (T)1;
                const int64_t bb = ((int64_t)(fz ? L - r : r) * hy + kyf) * Kx + kx;
                e += quad_form<T>(a[r], b[r], c[r], __ldg(&nhat[bb]), __ldg(&nhat[plane + bb]),
                                  __ldg(&nhat[2 * plane + bb]), sy * __ldg(&nhat[3 * plane + bb]),
                                  sz * __ldg(&nhat[4 * plane + bb]), sy * sz * __ldg(&nhat[5 * plane + bb]));
            }
            e *= kx_weight<T>(kx, Kx);
        }
        block_partial<Tile2<T>::NT>((double)e, partials, tile);
        return;
    }
    if (f >= ncols) return;
    const int ky = f / width, kx = f - ky * width;
    const int64_t base = (int64_t)ky * ss + kx;
    C a[L], b[L], c[L];
#pragma unroll
    for (int r = 0; r < L; ++r) {
        const bool ok = r < nrows;
        a[r] = ok ? ldp<CG>(&S[base + (int64_t)r * rs]) : cmk<C>(0, 0);
        b[r] = ok ? ldp<CG>(&S[base + (int64_t)r * rs + cs]) : cmk<C>(0, 0);
        c[r] = ok ? ldp<CG>(&S[base + (int64_t)r * rs + 2 * cs]) : cmk<C>(0, 0);
    }
    RegDFT<L, false, C>::run(a);
    RegDFT<L, false, C>::run(b);
    RegDFT<L, false, C>::run(c);
    const bool fy = ky > Py / 2;
    const int kyf = fy ? Py - ky : ky;
    const T sy = fy ? (T)-1 : (T)1;
    const int hy = Py / 2 + 1;
    const int64_t plane = (int64_t)(L / 2 + 1) * hy * Kx;
#pragma unroll
    for (int r = 0; r < L; ++r) {
        const bool fz = r > L / 2;
        const int kzf = fz ? L - r : r;
        tensor_product<T>(nhat, plane, ((int64_t)kzf * hy + kyf) * Kx + kx, sy, fz ? (T)-1 : (T)1, a[r], b[r],
                          c[r]);
    }
    RegDFT<L, true, C>::run(a);
    RegDFT<L, true, C>::run(b);
    RegDFT<L, true, C>::run(c);
#pragma unroll
    for (int r = 0; r < L; ++r)
        if (r < nrows) {
            S[base + (int64_t)r * rs] = a[r];
            S[base + (int64_t)r * rs + cs] = b[r];
            S[base + (int64_t)r * rs + 2 * cs] = c[r];
        }
}

template <typename T, int L>
__global__ void __launch_bounds__(Tile2<T>::NT, (L >= 16 ? 1 : 2))
k_z_conv1(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
          int nrows, const T *__restrict__ nhat, int Py, int Kx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_z_conv1_tile<T, L, false>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, blockIdx.x, smraw);
}

// Spectral energy of the z columns for L <= 16 (EONLY form of k_z_conv1).
template <typename T, int L>
__global__ void __launch_bounds__(Tile2<T>::NT, (L >= 16 ? 1 : 2))
k_z_energy1(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
            int nrows, const T *__restrict__ nhat, int Py, int Kx, double *__restrict__ partials)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_z_conv1_tile<T, L, false, true>(S, ncols, width, ss, rs, cs, nrows, nhat, Py, Kx, blockIdx.x, smraw, partials);
}

}  // namespace demag

namespace demag {

// ---------------------------------------------------------------- x passes
// Rows of 2L reals are packed as L complex values z[n] = x[2n] + i x[2n+1]
// and transformed with two stages, L = R1 * R2 (stage 1 radix R1 by R2
// threads per row, stage 2 radix R2 by R1 threads per row; R1 <= 32 so a
// row's stage-2 threads share a warp). The real-to-complex split needs
// Z[k] and Z[L-k]: Z[j2 + r R1] sits in thread j2, Z[L - j2 - r R1] in thread
// R1 - j2 at r' = R2 - 1 - r (thread 0 holds its own partners), exchanged by
// warp shuffles.
template <int L> struct XRadix;
template <> struct XRadix<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct XRadix<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct XRadix<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct XRadix<512> { static constexpr int R1 = 32, R2 = 16; };

template <typename T, int L> struct XShape {
    static constexpr int R1 = XRadix<L>::R1, R2 = XRadix<L>::R2;
    static_assert(R1 <= 32 && 32 % R1 == 0, "the exchange indexing assumes R1 divides 32");
    static constexpr int NT = Tile2<T>::NT;
    static constexpr int TR = NT / (R1 > R2 ? R1 : R2);  // rows per CTA
    static constexpr int RS = swsize(L);                 // padded row in shared memory
};

// Position in an x row's exchange of element j R1 + c (written by stage-1
// thread j as its output c, read by stage-2 thread c as its input j). For
// R1 = 16 the column is XORed with j: the 16 writers of one column and the 16
// readers of one group then hit 16 different 8-byte bank pairs (two rows per
// warp: two wavefronts, the minimum). Otherwise one padding element per 32
// (j R1 % 32 + c < 32 there).
template <int R1>
__device__ __forceinline__ int xex(int j, int c)
{
    if constexpr (R1 == 16) return j * 16 + (c ^ (j & 15));
    else return sw(j * R1) + c;
}

template <typename C>
__device__ __forceinline__ C shfl_c(C v, int lane)
{
    C r;
    r.x = __shfl_sync(0xffffffffu, v.x, lane);
    r.y = __shfl_sync(0xffffffffu, v.y, lane);
    return r;
}

// Real-to-complex along x (see k_x_fwd for the packing), two stages.
// PIN: the row has at most L reals (the zero-padded field), so the upper half
// of the packed sequence is zero; otherwise all 2L reals are read (setup).
template <typename T, int L, bool PIN, bool CG>
__device__ __forceinline__ void k_x_fwd2_tile(XIn<T> a, int nrows, int nvalid, typename Cplx<T>::type *__restrict__ out, int64_t out_rs,
         const typename Cplx<T>::type *__restrict__ twx, int tile, unsigned char *smraw)
{
    using C = typename Cplx<T>::type;
    using S = XShape<T, L>;
    constexpr int R1 = S::R1, R2 = S::R2, TR = S::TR, RS = S::RS;
    C *sm = reinterpret_cast<C *>(smraw);
    const int row0 = tile * TR;
    // stage 1: thread (row, j1) reads z[j1 + r R2] (r < R1/2 when PIN: the rest is padding)
    if (threadIdx.x < TR * R2) {
        const int rr = threadIdx.x / R2, j1 = threadIdx.x % R2, row = row0 + rr;
        C u[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
        if (row < nrows) {
            const T *p = a.in + (int64_t)row * a.in_rs;
            const T ws = a.wscalar;
            if ((a.in_rs & 1) == 0 && !a.wcell) {
                // even rows: pairs are aligned, one vector load per complex value
#pragma unroll
                for (int r = 0; r < (PIN ? R1 / 2 : R1); ++r) {
                    const int x0 = 2 * (j1 + r * R2);
                    if (x0 + 1 < nvalid) {
                        const C q = *reinterpret_cast<const C *>(p + x0);
                        u[r] = cmk<C>(q.x * ws, q.y * ws);
                    } else if (x0 < nvalid) {
                        u[r].x = p[x0] * ws;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < (PIN ? R1 / 2 : R1); ++r) {
                    const int x0 = 2 * (j1 + r * R2);
                    if (x0 < nvalid) u[r].x = p[x0] * ws * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0);
                    if (x0 + 1 < nvalid)
                        u[r].y = p[x0 + 1] * ws * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0 + 1);
                }
            }
        }
        if constexpr (PIN) RegDFTHalfIn<R1, false, C>::run(u);
        else RegDFT<R1, false, C>::run(u);
        C *s = sm + rr * RS;
#pragma unroll
        for (int r = 0; r < R1; ++r) s[xex<R1>(j1, r)] = u[r];
    }
    __syncthreads();
    // stage 2 + split: thread (row, j2) computes X[k], k = j2 + r R1
    if (threadIdx.x < TR * R1) {
        const int rr = threadIdx.x / R1, j2 = threadIdx.x % R1, row = row0 + rr;
        const C *s = sm + rr * RS;
        C v[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) v[r] = s[xex<R1>(r, j2)];
#pragma unroll
        for (int r = 1; r < R2; ++r) v[r] = cmul(v[r], __ldg(&twx[2 * r * j2]));
        RegDFT<R2, false, C>::run(v);
        const int lane = threadIdx.x & 31;
        const int partner = (lane & ~(R1 - 1)) | ((R1 - j2) & (R1 - 1));
        const T h = (T)0.5;
        C *o = out + (int64_t)row * out_rs;
        const bool live = row < nrows;
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            const C q = shfl_c(v[R2 - 1 - r], partner);
            const C pz = j2 == 0 ? v[(R2 - r) % R2] : q;  // Z[L - k]
            const int k = j2 + r * R1;
            const C E = cmk<C>(h * (v[r].x + pz.x), h * (v[r].y - pz.y));
            const C O = cmk<C>(h * (v[r].y + pz.y), -h * (v[r].x - pz.x));
            if (live) o[k] = cadd(E, cmul(O, __ldg(&twx[k])));
        }
        // X[L] = E(0) - O(0) (W_{2L}^L = -1), from Z[0]
        if (live && j2 == 0) o[L] = cmk<C>(v[0].x - v[0].y, (T)0);
    }
}

template <typename T, int L, bool PIN>
__global__ void __launch_bounds__(Tile2<T>::NT)
k_x_fwd2(XIn<T> a, int nrows, int nvalid, typename Cplx<T>::type *__restrict__ out, int64_t out_rs,
         const typename Cplx<T>::type *__restrict__ twx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_x_fwd2_tile<T, L, PIN, false>(a, nrows, nvalid, out, out_rs, twx, blockIdx.x, smraw);
}

// Complex-to-real along x (see k_x_inv), two stages, XOut epilogue. MP: the
// energy's reference field rows (o.Mref, nvalid a multiple of 4 and rows
// 16-byte aligned) are copied to shared memory with cp.async at the start, so
// their loads overlap the transform instead of following it.
// Epilogue of an inverse x row: the real outputs x, x + 1 (one complex value
// of the half-length transform, scaled), stored and, with the energy, dotted
// with M. Without a cell weight and with even rows, one 8-byte (FP32) or
// 16-byte (FP64) access per pair; otherwise element by element. mref: the
// row of M in shared memory (MP) or nullptr (then M from global memory).
template <typename T>
__device__ __forceinline__ void x_out_pair(const XOut<T> &o, int row, int x, T h0, T h1, T oscale, int nvalid,
                                           const T *mref, T &acc)
{
    using C = typename Cplx<T>::type;
    const int64_t idx = (int64_t)row * o.out_rs + x;
    if (!o.wcell && (o.out_rs & 1) == 0 && x + 1 < nvalid) {
        if (o.out) *reinterpret_cast<C *>(o.out + idx) = cmk<C>(h0 * oscale, h1 * oscale);
        if (o.partials) {
            const C m = mref ? *reinterpret_cast<const C *>(mref + x) : *reinterpret_cast<const C *>(o.Mref + idx);
            acc += o.mscale * (m.x * h0 + m.y * h1);
        }
        return;
    }
    const T hv[2] = {h0, h1};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (x + u >= nvalid) continue;
        const T w = cell_weight(o.wcell, row, o.rows_per_comp, o.out_rs, x + u);
        if (o.out) o.out[idx + u] = hv[u] * oscale * w;
        if (o.partials) acc += o.mscale * w * (mref ? mref[x + u] : o.Mref[idx + u]) * hv[u];
    }
}

template <typename T, int L, bool CG, bool P1 = false, bool MP = false>
__device__ __forceinline__ void k_x_inv2_tile(const typename Cplx<T>::type *__restrict__ in, int64_t in_rs, int nrows, int nvalid, XOut<T> o,
         const typename Cplx<T>::type *__restrict__ twx, int tile, unsigned char *smraw)
{
    using C = typename Cplx<T>::type;
    using S = XShape<T, L>;
    constexpr int R1 = S::R1, R2 = S::R2, NT = S::NT, TR = S::TR, RS = S::RS;
    C *sm = reinterpret_cast<C *>(smraw);
    T *smM = reinterpret_cast<T *>(sm + TR * RS);  // MP: [TR][L] reference rows
    const int row0 = tile * TR;
    if constexpr (MP) {
        const int chunks = nvalid / (16 / (int)sizeof(T));  // 16-byte pieces per row
        for (int i = threadIdx.x; i < TR * chunks; i += NT) {
            const int rr = i / chunks, c = i - rr * chunks, row = row0 + rr;
            if (row < nrows)
                cp_async16(&smM[rr * L + c * (16 / (int)sizeof(T))],
                           o.Mref + (int64_t)row * o.out_rs + c * (16 / (int)sizeof(T)));
        }
    }
    // stage 1: thread (row, j1) builds Z[k], k = j1 + r R2, from X[k] and X[L-k]
    if (threadIdx.x < TR * R2) {
        const int rr = threadIdx.x / R2, j1 = threadIdx.x % R2, row = row0 + rr;
        C u[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
        if (row < nrows) {
            const C *p = in + (int64_t)row * in_rs;
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int k = j1 + r * R2;
                const C a = ldp<CG>(&p[k]);
                const C b = ldp<CG>(&p[L - k]);
                const C E2 = cmk<C>(a.x + b.x, a.y - b.y);
                const C D = cmk<C>(a.x - b.x, a.y + b.y);
                const C O2 = cmulc(D, __ldg(&twx[k]));
                u[r] = cmk<C>(E2.x - O2.y, E2.y + O2.x);
            }
        }
        RegDFT<R1, true, C>::run(u);
        C *s = sm + rr * RS;
#pragma unroll
        for (int r = 0; r < R1; ++r) s[xex<R1>(j1, r)] = u[r];
    }
    if constexpr (MP) cp_async_wait_all();
    __syncthreads();
    T acc = 0;  // per-thread sum of a few dozen terms; blocks reduce in FP64
    if (threadIdx.x < TR * R1) {
        const int rr = threadIdx.x / R1, j2 = threadIdx.x % R1, row = row0 + rr;
        const C *s = sm + rr * RS;
        C v[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) v[r] = s[xex<R1>(r, j2)];
#pragma unroll
        for (int r = 1; r < R2; ++r) v[r] = cmulc(v[r], __ldg(&twx[2 * r * j2]));
        if constexpr (P1) RegDFTHalfOutP1<R2, true, C>::run(v);
        else RegDFTHalfOut<R2, true, C>::run(v);
        if (row < nrows) {
            const T g = o.gdev ? (T)(*o.gdev) : (T)1;
            const T oscale = o.oscale * g;
#pragma unroll
            for (int r = 0; r < (P1 ? R2 / 2 + 1 : R2 / 2); ++r) {  // z[n], n = j2 + r R1 (< L/2 unless P1)
                const int n = j2 + r * R1;
                x_out_pair<T>(o, row, 2 * n, v[r].x * o.scale, v[r].y * o.scale, oscale, nvalid,
                              MP ? smM + rr * L : nullptr, acc);
            }
        }
    }
    if (o.partials) block_partial<NT>((double)acc, o.partials, tile);
}

// P1: one more output pair per row (x = L, L + 1, ...: rows of nx + 1 >= L
// values, the node potential of the scalar-potential method).
template <typename T, int L, bool P1 = false, bool MP = false>
__global__ void __launch_bounds__(Tile2<T>::NT, (L >= 512 ? Occ<T, 2 * L>::MIN_CTAS : Occ<T, L>::MIN_CTAS))
k_x_inv2(const typename Cplx<T>::type *__restrict__ in, int64_t in_rs, int nrows, int nvalid, XOut<T> o,
         const typename Cplx<T>::type *__restrict__ twx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_x_inv2_tile<T, L, false, P1, MP>(in, in_rs, nrows, nvalid, o, twx, blockIdx.x, smraw);
}

}  // namespace demag
