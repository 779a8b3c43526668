// Shared-memory Stockham FFT engine and the five field passes of the
// FFT demagnetization-tensor method (paper Sec. 3.1: H = -N * M evaluated
// with the convolution theorem on the zero-padded grid).
//
// Every pass works on a tile of TC columns x L rows held in shared memory as
// [row][column] (column fastest, one padding element every 32 to spread
// bank accesses). Columns are independent 1-D transforms of length L (a power
// of two <= 1024); each stage of the transform is a radix-R butterfly
// (R <= 16) evaluated in registers, Stockham auto-sorted so the result comes
// out in natural order. Twiddles come from per-axis FP64-accurate tables.
//
// Element types: T = float (complex float2) or double (complex double2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"

namespace demag {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// Threads per CTA and elements per thread of the tile engine.
template <typename T> struct Tile;
template <> struct Tile<float> { static constexpr int NT = 256; static constexpr int EPT = 16; };
template <> struct Tile<double> { static constexpr int NT = 128; static constexpr int EPT = 16; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b)
{
    C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
// a * b
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b)
{
    return cmk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// cos(2 pi m / 32) for m = 0..8 (the quarter wave; the rest by symmetry).
__host__ __device__ constexpr double cos2pi32(int m)
{
    return m == 0 ? 1.0
         : m == 1 ? 0.98078528040323044912618223613424
         : m == 2 ? 0.92387953251128675612818318939679
         : m == 3 ? 0.83146961230254523707878837761791
         : m == 4 ? 0.70710678118654752440084436210485
         : m == 5 ? 0.55557023301960222474283081394853
         : m == 6 ? 0.38268343236508977172845998403040
         : m == 7 ? 0.19509032201612826784828486847702
         : 0.0;
}

// x * W_N^k with W_N = exp(-2 pi i / N) (forward) or its conjugate (inverse),
// N <= 32. k is a compile-time constant after unrolling, so the constants
// fold into the multiplications.
template <int N, bool INV, typename C>
__device__ __forceinline__ C twconst(int k, C x)
{
    using T = decltype(C::x);
    const int m = k * (32 / N);  // angle 2 pi m / 32, 0 <= m < 16
    if (m == 0) return x;
    if (m == 8) return INV ? cmk<C>(-x.y, x.x) : cmk<C>(x.y, -x.x);
    const T c = (T)(m <= 8 ? cos2pi32(m) : -cos2pi32(16 - m));
    const T s = (T)(m <= 8 ? cos2pi32(8 - m) : cos2pi32(m - 8));
    if (INV) return cmk<C>(x.x * c - x.y * s, x.x * s + x.y * c);
    return cmk<C>(x.x * c + x.y * s, x.y * c - x.x * s);
}

// In-register DFT of size N (power of two <= 16), natural order in and out,
// by recursive radix-2 decimation in time.
template <int N, bool INV, typename C> struct RegDFT {
    static __device__ __forceinline__ void run(C *v)
    {
        C e[N / 2], o[N / 2];
#pragma unroll
        for (int k = 0; k < N / 2; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
        RegDFT<N / 2, INV, C>::run(e);
        RegDFT<N / 2, INV, C>::run(o);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const C t = twconst<N, INV>(k, o[k]);
            v[k] = cadd(e[k], t);
            v[k + N / 2] = csub(e[k], t);
        }
    }
};
template <bool INV, typename C> struct RegDFT<1, INV, C> {
    static __device__ __forceinline__ void run(C *) {}
};

// DFT of N points whose inputs v[N/2..N) are zero (the zero padding of the
// convolution): the same decimation in time, with the leaf butterflies of an
// input and a zero reduced to copies. Output v[0..N) in natural order.
template <int N, bool INV, typename C> struct RegDFTHalfIn {
    static __device__ __forceinline__ void run(C *v)
    {
        C e[N / 2], o[N / 2];
#pragma unroll
        for (int k = 0; k < N / 4; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
        RegDFTHalfIn<N / 2, INV, C>::run(e);
        RegDFTHalfIn<N / 2, INV, C>::run(o);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const C t = twconst<N, INV>(k, o[k]);
            v[k] = cadd(e[k], t);
            v[k + N / 2] = csub(e[k], t);
        }
    }
};
template <bool INV, typename C> struct RegDFTHalfIn<2, INV, C> {
    static __device__ __forceinline__ void run(C *v) { v[1] = v[0]; }
};
template <bool INV, typename C> struct RegDFTHalfIn<1, INV, C> {
    static __device__ __forceinline__ void run(C *) {}
};

// DFT of N points of which only the outputs v[0..N/2) are used: the last
// butterfly level computes the sums only.
template <int N, bool INV, typename C> struct RegDFTHalfOut {
    static __device__ __forceinline__ void run(C *v)
    {
        C e[N / 2], o[N / 2];
#pragma unroll
        for (int k = 0; k < N / 2; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
        RegDFT<N / 2, INV, C>::run(e);
        RegDFT<N / 2, INV, C>::run(o);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) v[k] = cadd(e[k], twconst<N, INV>(k, o[k]));
    }
};
template <bool INV, typename C> struct RegDFTHalfOut<1, INV, C> {
    static __device__ __forceinline__ void run(C *) {}
};

// DFT of N points of which the outputs v[0..N/2] are used: one output more
// than RegDFTHalfOut, v[N/2] = E[0] - O[0].
template <int N, bool INV, typename C> struct RegDFTHalfOutP1 {
    static __device__ __forceinline__ void run(C *v)
    {
        C e[N / 2], o[N / 2];
#pragma unroll
        for (int k = 0; k < N / 2; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
        RegDFT<N / 2, INV, C>::run(e);
        RegDFT<N / 2, INV, C>::run(o);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) v[k] = cadd(e[k], twconst<N, INV>(k, o[k]));
        v[N / 2] = csub(e[0], o[0]);
    }
};

__device__ __forceinline__ int sw(int e) { return e + (e >> 5); }

__host__ __device__ constexpr int swsize(int elems) { return elems + (elems >> 5) + 1; }

// One Stockham stage of radix R on a [L][TC] tile, in place (all threads
// read and compute, barrier, then write). NS = product of earlier radices.
// tw: forward twiddle table W_P^m of the axis; twstride = P / L.
template <typename C, int L, int R, int NS, bool INV, int NT, int TC>
__device__ __forceinline__ void fft_stage(C *sm, const C *__restrict__ tw, int twstride)
{
    constexpr int NB = L / R;
    constexpr int BPT = (NB * TC) / NT;
    static_assert((NB * TC) % NT == 0 && BPT >= 1, "tile does not divide the threads");
    C v[BPT][R];
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int b = threadIdx.x + q * NT;
        const int col = b % TC, j = b / TC;
        if constexpr ((NB * TC) % 32 == 0) {
            // sw() is additive across multiples of 32: one swizzled base, constant steps
            const C *s = sm + sw(j * TC + col);
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = s[r * (NB * TC + (NB * TC) / 32)];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = sm[sw((j + r * NB) * TC + col)];
        }
        if (NS > 1) {
            const int k = j % NS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C w = __ldg(&tw[(r * k * (L / (NS * R))) * twstride]);
                v[q][r] = INV ? cmulc(v[q][r], w) : cmul(v[q][r], w);
            }
        }
        RegDFT<R, INV, C>::run(v[q]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int b = threadIdx.x + q * NT;
        const int col = b % TC, j = b / TC;
        const int k = j % NS;
        const int d = (j / NS) * NS * R + k;
        if constexpr ((NS * TC) % 32 == 0) {
            C *s = sm + sw(d * TC + col);
#pragma unroll
            for (int r = 0; r < R; ++r) s[r * (NS * TC + (NS * TC) / 32)] = v[q][r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) sm[sw((d + r * NS) * TC + col)] = v[q][r];
        }
    }
    __syncthreads();
}

// Full length-L transform of every column of the tile (unnormalised).
// Radix schedule: L <= 16 one stage; 32 = 8x4, 64 = 8x8, 128 = 16x8,
// 256 = 16x16, 512 = 8x8x8, 1024 = 16x8x8.
template <typename C, int L, bool INV, int NT, int TC>
__device__ __forceinline__ void tile_fft(C *sm, const C *__restrict__ tw, int twstride)
{
    if constexpr (L == 1) {
    } else if constexpr (L <= 16) {
        fft_stage<C, L, L, 1, INV, NT, TC>(sm, tw, twstride);
    } else if constexpr (L == 32) {
        fft_stage<C, 32, 8, 1, INV, NT, TC>(sm, tw, twstride);
        fft_stage<C, 32, 4, 8, INV, NT, TC>(sm, tw, twstride);
    } else if constexpr (L == 64) {
        fft_stage<C, 64, 8, 1, INV, NT, TC>(sm, tw, twstride);
        fft_stage<C, 64, 8, 8, INV, NT, TC>(sm, tw, twstride);
    } else if constexpr (L == 128) {
        fft_stage<C, 128, 16, 1, INV, NT, TC>(sm, tw, twstride);
        fft_stage<C, 128, 8, 16, INV, NT, TC>(sm, tw, twstride);
    } else if constexpr (L == 256) {
        fft_stage<C, 256, 16, 1, INV, NT, TC>(sm, tw, twstride);
        fft_stage<C, 256, 16, 16, INV, NT, TC>(sm, tw, twstride);
    } else if constexpr (L == 512) {
        fft_stage<C, 512, 8, 1, INV, NT, TC>(sm, tw, twstride);
        fft_stage<C, 512, 8, 8, INV, NT, TC>(sm, tw, twstride);
        fft_stage<C, 512, 8, 64, INV, NT, TC>(sm, tw, twstride);
    } else if constexpr (L == 1024) {
        fft_stage<C, 1024, 16, 1, INV, NT, TC>(sm, tw, twstride);
        fft_stage<C, 1024, 8, 16, INV, NT, TC>(sm, tw, twstride);
        fft_stage<C, 1024, 8, 128, INV, NT, TC>(sm, tw, twstride);
    } else {
        static_assert(L == 1, "unsupported transform length");
    }
}

template <typename T, int L> struct TileShape {
    static constexpr int NT = Tile<T>::NT;
    static constexpr int ELEMS = Tile<T>::NT * Tile<T>::EPT;
    static constexpr int TC = ELEMS / L;
    static_assert(TC >= 1, "length too large for the tile");
};

template <typename T>
__device__ __forceinline__ T cell_weight(const T *wcell, int row, int rows_per_comp, int64_t rs, int x)
{
    return wcell ? __ldg(&wcell[(int64_t)(row % rows_per_comp) * rs + x]) : (T)1;
}

// Block sum of a per-thread double into partials[slot] (slot = the tile).
template <int NT>
__device__ __forceinline__ void block_partial(double v, double *partials, int slot)
{
    __shared__ double red[NT / 32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < NT / 32; ++w) s += red[w];
        partials[slot] = s;
    }
}

// ---------------------------------------------------------------- x forward
// Real-to-complex along x for nrows rows of nvalid real values (zero padded to
// 2L): pack z[n] = x[2n] + i x[2n+1], transform length L, then split into the
// spectrum X[k], k = 0..L, of the length-2L real sequence. twx is the table of
// the x axis (length 2L).
template <typename T, int L, bool CG>
__device__ __forceinline__ void k_x_fwd_tile(XIn<T> a, int nrows, int nvalid, typename Cplx<T>::type *__restrict__ out, int64_t out_rs,
        const typename Cplx<T>::type *__restrict__ twx, int tile, unsigned char *smraw)
{
    using C = typename Cplx<T>::type;
    using S = TileShape<T, L>;
    constexpr int NT = S::NT, TC = S::TC;
    C *sm = reinterpret_cast<C *>(smraw);
    const int row0 = tile * TC;
    for (int e = threadIdx.x; e < L * TC; e += NT) {
        const int n = e % L, rr = e / L, row = row0 + rr;
        C z = cmk<C>(0, 0);
        if (row < nrows) {
            const T *p = a.in + (int64_t)row * a.in_rs;
            const int x0 = 2 * n;
            if (x0 < nvalid) z.x = p[x0] * a.wscalar * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0);
            if (x0 + 1 < nvalid)
                z.y = p[x0 + 1] * a.wscalar * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0 + 1);
        }
        sm[sw(n * TC + rr)] = z;
    }
    __syncthreads();
    tile_fft<C, L, false, NT, TC>(sm, twx, 2);
    const T h = (T)0.5;
    for (int e = threadIdx.x; e < (L + 1) * TC; e += NT) {
        const int k = e % (L + 1), rr = e / (L + 1), row = row0 + rr;
        if (row >= nrows) continue;
        const C p = sm[sw((k == L ? 0 : k) * TC + rr)];
        const C q = sm[sw((k == 0 ? 0 : L - k) * TC + rr)];
        // even part E = (p + conj q)/2, odd part O = (p - conj q)/(2i)
        const C E = cmk<C>(h * (p.x + q.x), h * (p.y - q.y));
        const C O = cmk<C>(h * (p.y + q.y), -h * (p.x - q.x));
        const C w = __ldg(&twx[k]);
        out[(int64_t)row * out_rs + k] = cadd(E, cmul(O, w));
    }
}

template <typename T, int L>
__global__ void __launch_bounds__(Tile<T>::NT)
k_x_fwd(XIn<T> a, int nrows, int nvalid, typename Cplx<T>::type *__restrict__ out, int64_t out_rs,
        const typename Cplx<T>::type *__restrict__ twx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_x_fwd_tile<T, L, false>(a, nrows, nvalid, out, out_rs, twx, blockIdx.x, smraw);
}

// ---------------------------------------------------------------- x inverse
// Complex-to-real along x: from X[k], k = 0..L, rebuild the packed sequence
// Z[k] = (X[k] + conj X[L-k]) + i W^-k (X[k] - conj X[L-k]), inverse transform
// of length L, unpack to 2L reals, keep x < nvalid; epilogue per XOut.
template <typename T, int L, bool CG>
__device__ __forceinline__ void k_x_inv_tile(const typename Cplx<T>::type *__restrict__ in, int64_t in_rs, int nrows, int nvalid, XOut<T> o,
        const typename Cplx<T>::type *__restrict__ twx, int tile, unsigned char *smraw)
{
    using C = typename Cplx<T>::type;
    using S = TileShape<T, L>;
    constexpr int NT = S::NT, TC = S::TC;
    C *sm = reinterpret_cast<C *>(smraw);
    const int row0 = tile * TC;
    for (int e = threadIdx.x; e < L * TC; e += NT) {
        const int k = e % L, rr = e / L, row = row0 + rr;
        C z = cmk<C>(0, 0);
        if (row < nrows) {
            const C *p = in + (int64_t)row * in_rs;
            const C a = CG ? __ldcg(&p[k]) : p[k];
            const C b = CG ? __ldcg(&p[L - k]) : p[L - k];
            const C E2 = cmk<C>(a.x + b.x, a.y - b.y);
            const C D = cmk<C>(a.x - b.x, a.y + b.y);
            const C O2 = cmulc(D, __ldg(&twx[k]));
            z = cmk<C>(E2.x - O2.y, E2.y + O2.x);
        }
        sm[sw(k * TC + rr)] = z;
    }
    __syncthreads();
    tile_fft<C, L, true, NT, TC>(sm, twx, 2);
    const T g = o.gdev ? (T)(*o.gdev) : (T)1;
    const T oscale = o.oscale * g;
    T acc = 0;  // per-thread sum of mscale * w * Mref * h (a few dozen terms)
    for (int e = threadIdx.x; e < L * TC; e += NT) {
        const int n = e % L, rr = e / L, row = row0 + rr;
        if (row >= nrows) continue;
        const C z = sm[sw(n * TC + rr)];
        const T hv[2] = {z.x * o.scale, z.y * o.scale};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int x = 2 * n + u;
            if (x >= nvalid) continue;
            const T w = cell_weight(o.wcell, row, o.rows_per_comp, o.out_rs, x);
            const int64_t idx = (int64_t)row * o.out_rs + x;
            if (o.out) o.out[idx] = hv[u] * oscale * w;
            if (o.partials) acc += o.mscale * w * o.Mref[idx] * hv[u];
        }
    }
    if (o.partials) block_partial<NT>((double)acc, o.partials, tile);
}

template <typename T, int L>
__global__ void __launch_bounds__(Tile<T>::NT)
k_x_inv(const typename Cplx<T>::type *__restrict__ in, int64_t in_rs, int nrows, int nvalid, XOut<T> o,
        const typename Cplx<T>::type *__restrict__ twx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    k_x_inv_tile<T, L, false>(in, in_rs, nrows, nvalid, o, twx, blockIdx.x, smraw);
}


// ---------------------------------------------------------------- z pass
// Forward z transform of the three components, the spectral product
// H^ = -N^ M^ with the real symmetric tensor spectrum (paper Sec. 3.1: the
// element-wise matrix-vector product in Fourier space), inverse z transform,
// rows z < nrows written back in place.
// Columns f = ky * width + kx, ky < Py. The tensor spectrum is stored for
// ky <= Py/2, kz <= Pz/2 only: N^ keeps the parity of each component in k,
// so folding ky -> Py - ky flips the sign of xy and yz, folding kz -> Pz - kz
// flips xz and yz.
template <typename T, int L>
__global__ void __launch_bounds__(Tile<T>::NT)
k_z_conv(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs,
         int64_t cs, int nrows, const T *__restrict__ nhat, int Py, int Kx,
         const typename Cplx<T>::type *__restrict__ tw, int twstride)
{
    using C = typename Cplx<T>::type;
    using Sh = TileShape<T, L>;
    constexpr int NT = Sh::NT, TC = Sh::TC;
    constexpr int TS = swsize(L * TC);
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int f0 = blockIdx.x * TC;
    for (int e = threadIdx.x; e < L * TC; e += NT) {
        const int c = e % TC, r = e / TC, f = f0 + c;
        C v0 = cmk<C>(0, 0), v1 = v0, v2 = v0;
        if (f < ncols && r < nrows) {
            const int slab = f / width, off = f - slab * width;
            const int64_t g = (int64_t)slab * ss + (int64_t)r * rs + off;
            v0 = S[g]; v1 = S[g + cs]; v2 = S[g + 2 * cs];
        }
        sm[sw(e)] = v0; sm[TS + sw(e)] = v1; sm[2 * TS + sw(e)] = v2;
    }
    __syncthreads();
    tile_fft<C, L, false, NT, TC>(sm, tw, twstride);
    tile_fft<C, L, false, NT, TC>(sm + TS, tw, twstride);
    tile_fft<C, L, false, NT, TC>(sm + 2 * TS, tw, twstride);
    const int hy = Py / 2 + 1, hz = L / 2 + 1;
    const int64_t plane = (int64_t)hz * hy * Kx;
    for (int e = threadIdx.x; e < L * TC; e += NT) {
        const int c = e % TC, kz = e / TC, f = f0 + c;
        if (f >= ncols) continue;
        const int ky = f / width, kx = f - ky * width;
        const bool fy = ky > Py / 2, fz = kz > L / 2;
        const int kyf = fy ? Py - ky : ky, kzf = fz ? L - kz : kz;
        const T sy = fy ? (T)-1 : (T)1, sz = fz ? (T)-1 : (T)1;
        const int64_t b = ((int64_t)kzf * hy + kyf) * Kx + kx;
        const T nxx = __ldg(&nhat[b]), nyy = __ldg(&nhat[plane + b]), nzz = __ldg(&nhat[2 * plane + b]);
        const T nxy = sy * __ldg(&nhat[3 * plane + b]);
        const T nxz = sz * __ldg(&nhat[4 * plane + b]);
        const T nyz = sy * sz * __ldg(&nhat[5 * plane + b]);
        const C mx = sm[sw(e)], my = sm[TS + sw(e)], mz = sm[2 * TS + sw(e)];
        sm[sw(e)] = cmk<C>(-(nxx * mx.x + nxy * my.x + nxz * mz.x), -(nxx * mx.y + nxy * my.y + nxz * mz.y));
        sm[TS + sw(e)] = cmk<C>(-(nxy * mx.x + nyy * my.x + nyz * mz.x), -(nxy * mx.y + nyy * my.y + nyz * mz.y));
        sm[2 * TS + sw(e)] = cmk<C>(-(nxz * mx.x + nyz * my.x + nzz * mz.x), -(nxz * mx.y + nyz * my.y + nzz * mz.y));
    }
    __syncthreads();
    tile_fft<C, L, true, NT, TC>(sm, tw, twstride);
    tile_fft<C, L, true, NT, TC>(sm + TS, tw, twstride);
    tile_fft<C, L, true, NT, TC>(sm + 2 * TS, tw, twstride);
    for (int e = threadIdx.x; e < L * TC; e += NT) {
        const int c = e % TC, r = e / TC, f = f0 + c;
        if (f < ncols && r < nrows) {
            const int slab = f / width, off = f - slab * width;
            const int64_t g = (int64_t)slab * ss + (int64_t)r * rs + off;
            S[g] = sm[sw(e)]; S[g + cs] = sm[TS + sw(e)]; S[g + 2 * cs] = sm[2 * TS + sw(e)];
        }
    }
}

}  // namespace demag
