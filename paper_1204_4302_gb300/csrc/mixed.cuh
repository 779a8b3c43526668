// Mixed-radix passes for padded lengths that are not powers of two (products
// of 2, 3, 5 and 7): the zero padding of the convolution only needs P >= 2n - 1,
// and a smooth P just above 2n - 1 can hold far fewer padded cells than the
// next power of two (e.g. n = 80: 160 instead of 256 per axis). These kernels
// trade the compile-time register schedules of the power-of-two passes for
// one generic form: a tile of transforms in shared memory, Stockham stages of
// radix 2, 4, 8, 16, 3, 5, 7 or 9 run from a runtime radix list, ping-ponging
// between two buffers. Same inputs, outputs and epilogues as the power-of-two
// passes.
#pragma once
#include "fft_engine.cuh"

namespace demag {

// Stage plan of one transform of length L (product of the radices), with
// the multipliers that replace the runtime divisions of the index
// arithmetic: q = umulhi(n, m) with m = ceil(2^32 / d) equals n / d for every
// n d < 2^32 (here n < 2^13, d < 2^11), and d == 1 is taken apart.
constexpr int kGenMaxStages = 12;
struct GenRadix {
    int L, n, TC;                  // length, stages, transforms per tile
    int r[kGenMaxStages];          // radices in stage order
    int NS[kGenMaxStages];         // product of the earlier radices
    unsigned mNS[kGenMaxStages];   // division by NS
    unsigned mPer[kGenMaxStages];  // division by (L / r) TC
    unsigned mTC, mL, mL1;         // division by TC, L, L + 1
};

constexpr int kGenThreads = 256;

__device__ __forceinline__ int udiv(int n, int d, unsigned m)
{
    return d == 1 ? n : (int)__umulhi((unsigned)n, m);
}

// cos and sin of 2 pi q / R for the odd radices (q = 1 .. (R - 1) / 2).
template <int R> __device__ __forceinline__ double cos_tab(int q);
template <int R> __device__ __forceinline__ double sin_tab(int q);
template <> __device__ __forceinline__ double cos_tab<3>(int) { return -0.5; }
template <> __device__ __forceinline__ double sin_tab<3>(int) { return 0.866025403784438646764; }
template <> __device__ __forceinline__ double cos_tab<5>(int q)
{
    return q == 1 ? 0.309016994374947424102 : -0.809016994374947424102;
}
template <> __device__ __forceinline__ double sin_tab<5>(int q)
{
    return q == 1 ? 0.951056516295153572116 : 0.587785252292473129169;
}
template <> __device__ __forceinline__ double cos_tab<7>(int q)
{
    return q == 1 ? 0.623489801858733530525 : q == 2 ? -0.222520933956314404289 : -0.900968867902419126236;
}
template <> __device__ __forceinline__ double sin_tab<7>(int q)
{
    return q == 1 ? 0.781831482468029808708 : q == 2 ? 0.974927912181823607018 : 0.433883739117558120476;
}
template <> __device__ __forceinline__ double cos_tab<9>(int q)
{
    return q == 1 ? 0.766044443118978035202
         : q == 2 ? 0.173648177666930348852
         : q == 3 ? -0.5
                  : -0.939692620785908384054;
}
template <> __device__ __forceinline__ double sin_tab<9>(int q)
{
    return q == 1 ? 0.642787609686539326323
         : q == 2 ? 0.984807753012208059367
         : q == 3 ? 0.866025403784438646764
                  : 0.342020143325668733044;
}

// DFT of an odd number R of points, y_m = sum_j x_j w^{jm}, w = exp(-+2 pi i / R):
// with t_k = x_k + x_{R-k} and u_k = x_k - x_{R-k} (k = 1 .. H, H = (R-1)/2),
// a_m = x_0 + sum_k cos(2 pi k m / R) t_k and b_m = sum_k sin(2 pi k m / R) u_k,
// y_m = a_m -+ i b_m and y_{R-m} = a_m +- i b_m.
template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_odd(C *v)
{
    using T = decltype(C::x);
    constexpr int H = (R - 1) / 2;
    C t[H], u[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        t[k] = cadd(v[k + 1], v[R - 1 - k]);
        u[k] = csub(v[k + 1], v[R - 1 - k]);
    }
    const C x0 = v[0];
    C y0 = x0;
#pragma unroll
    for (int k = 0; k < H; ++k) y0 = cadd(y0, t[k]);
    v[0] = y0;
#pragma unroll
    for (int m = 1; m <= H; ++m) {
        C a = x0, b = cmk<C>(0, 0);
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const int q = (k * m) % R;  // angle 2 pi q / R (q = 0 only for R = 9)
            const T cq = (T)(q == 0 ? 1.0 : q <= H ? cos_tab<R>(q) : cos_tab<R>(R - q));
            const T sq = (T)(q == 0 ? 0.0 : q <= H ? sin_tab<R>(q) : -sin_tab<R>(R - q));
            a = cmk<C>(a.x + cq * t[k - 1].x, a.y + cq * t[k - 1].y);
            b = cmk<C>(b.x + sq * u[k - 1].x, b.y + sq * u[k - 1].y);
        }
        const C ib = INV ? cmk<C>(-b.y, b.x) : cmk<C>(b.y, -b.x);
        v[m] = cadd(a, ib);
        v[R - m] = csub(a, ib);
    }
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void small_dft(C *v)
{
    if constexpr (R % 2 == 1) dft_odd<R, INV, C>(v);
    else RegDFT<R, INV, C>::run(v);
}

// One Stockham stage s of radix R from src to dst, ncomp tiles of [L][TC]
// (component stride cstride, swizzled as everywhere). Butterfly b of a
// component: j = b / TC (0 <= j < L / R), column b % TC; it reads rows
// j + r L / R, applies W^{r k} (k = j mod NS, W the root of order NS R) and
// writes rows (j / NS) NS R + k + r NS. tw: W_P^m with P = L twstride.
template <typename C, int R, bool INV>
__device__ __forceinline__ void gen_stage(const C *src, C *dst, int ncomp, int cstride, const GenRadix &g, int s,
                                          const C *__restrict__ tw, int twstride)
{
    const int L = g.L, TC = g.TC, NS = g.NS[s];
    const int NB = L / R, per = NB * TC, total = ncomp * per;
    const int tws = (L / (NS * R)) * twstride;
    const unsigned mPer = g.mPer[s], mNS = g.mNS[s], mTC = g.mTC;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        const int comp = ncomp == 1 ? 0 : udiv(b, per, mPer);
        const int bb = b - comp * per;
        const int j = udiv(bb, TC, mTC), col = bb - j * TC;
        const C *sp = src + comp * cstride;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sp[sw((j + r * NB) * TC + col)];
        const int q = udiv(j, NS, mNS), k = j - q * NS;
        if (k > 0) {
            const int kt = k * tws;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C w = __ldg(&tw[r * kt]);
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        small_dft<R, INV, C>(v);
        C *o = dst + comp * cstride;
        const int d = q * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) o[sw((d + r * NS) * TC + col)] = v[r];
    }
}

// Whole transform of the tiles in a (b is the second buffer); returns the
// buffer that holds the result.
template <typename C, bool INV>
__device__ __forceinline__ C *gen_fft(C *a, C *b, int ncomp, int cstride, const GenRadix &g, const C *__restrict__ tw,
                                      int twstride)
{
    C *src = a, *dst = b;
    for (int s = 0; s < g.n; ++s) {
        switch (g.r[s]) {
        case 2: gen_stage<C, 2, INV>(src, dst, ncomp, cstride, g, s, tw, twstride); break;
        case 3: gen_stage<C, 3, INV>(src, dst, ncomp, cstride, g, s, tw, twstride); break;
        case 4: gen_stage<C, 4, INV>(src, dst, ncomp, cstride, g, s, tw, twstride); break;
        case 5: gen_stage<C, 5, INV>(src, dst, ncomp, cstride, g, s, tw, twstride); break;
        case 7: gen_stage<C, 7, INV>(src, dst, ncomp, cstride, g, s, tw, twstride); break;
        case 8: gen_stage<C, 8, INV>(src, dst, ncomp, cstride, g, s, tw, twstride); break;
        case 9: gen_stage<C, 9, INV>(src, dst, ncomp, cstride, g, s, tw, twstride); break;
        default: gen_stage<C, 16, INV>(src, dst, ncomp, cstride, g, s, tw, twstride); break;
        }
        __syncthreads();
        C *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Column transforms (as k_col2): g.TC columns per CTA, rows < nin read,
// rows < nout written; column f = slab * width + (f mod width), mw the
// multiplier of width.
template <typename T, bool INV>
__global__ void __launch_bounds__(kGenThreads)
k_gen_col(const typename Cplx<T>::type *__restrict__ in, typename Cplx<T>::type *__restrict__ out, int ncols, int width,
          unsigned mw, int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, int nout,
          const typename Cplx<T>::type *__restrict__ tw, int twstride, const __grid_constant__ GenRadix g)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TC = g.TC, TS = swsize(L * TC);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int f0 = blockIdx.x * TC;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int r = udiv(e, TC, g.mTC), f = f0 + e - r * TC;
        C v = cmk<C>(0, 0);
        if (f < ncols && r < nin) {
            const int slab = udiv(f, width, mw);
            v = in[(int64_t)slab * iss + (int64_t)r * irs + (f - slab * width)];
        }
        A[sw(e)] = v;
    }
    __syncthreads();
    const C *res = gen_fft<C, INV>(A, B, 1, 0, g, tw, twstride);
    for (int e = threadIdx.x; e < nout * TC; e += blockDim.x) {
        const int r = udiv(e, TC, g.mTC), f = f0 + e - r * TC;
        if (f < ncols) {
            const int slab = udiv(f, width, mw);
            out[(int64_t)slab * oss + (int64_t)r * ors + (f - slab * width)] = res[sw(e)];
        }
    }
}

// Real-to-complex rows (as k_x_fwd): pack pairs of reals, transform of
// L = Px/2 points, split into X[k], k = 0..L. g.TC rows per CTA.
template <typename T>
__global__ void __launch_bounds__(kGenThreads)
k_gen_x_fwd(XIn<T> a, int nrows, int nvalid, typename Cplx<T>::type *__restrict__ out, int64_t out_rs,
            const typename Cplx<T>::type *__restrict__ twx, const __grid_constant__ GenRadix g)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TR = g.TC, TS = swsize(L * TR);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int row0 = blockIdx.x * TR;
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int rr = udiv(e, L, g.mL), n = e - rr * L, row = row0 + rr;
        C z = cmk<C>(0, 0);
        const int x0 = 2 * n;
        if (row < nrows && x0 < nvalid) {
            const T *p = a.in + (int64_t)row * a.in_rs;
            z.x = p[x0] * a.wscalar * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0);
            if (x0 + 1 < nvalid)
                z.y = p[x0 + 1] * a.wscalar * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0 + 1);
        }
        A[sw(n * TR + rr)] = z;
    }
    __syncthreads();
    const C *Z = gen_fft<C, false>(A, B, 1, 0, g, twx, 2);
    const T h = (T)0.5;
    for (int e = threadIdx.x; e < (L + 1) * TR; e += blockDim.x) {
        const int rr = udiv(e, L + 1, g.mL1), k = e - rr * (L + 1), row = row0 + rr;
        if (row >= nrows) continue;
        const C p = Z[sw((k == L ? 0 : k) * TR + rr)];
        const C q = Z[sw((k == 0 ? 0 : L - k) * TR + rr)];
        const C E = cmk<C>(h * (p.x + q.x), h * (p.y - q.y));
        const C O = cmk<C>(h * (p.y + q.y), -h * (p.x - q.x));
        out[(int64_t)row * out_rs + k] = cadd(E, cmul(O, __ldg(&twx[k])));
    }
}

// Complex-to-real rows (as k_x_inv) with the XOut epilogue; energy partials
// one per CTA.
template <typename T>
__global__ void __launch_bounds__(kGenThreads)
k_gen_x_inv(const typename Cplx<T>::type *__restrict__ in, int64_t in_rs, int nrows, int nvalid, XOut<T> o,
            const typename Cplx<T>::type *__restrict__ twx, const __grid_constant__ GenRadix g)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TR = g.TC, TS = swsize(L * TR);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int row0 = blockIdx.x * TR;
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int rr = udiv(e, L, g.mL), k = e - rr * L, row = row0 + rr;
        C z = cmk<C>(0, 0);
        if (row < nrows) {
            const C *p = in + (int64_t)row * in_rs;
            const C x = p[k], y = p[L - k];
            const C E2 = cmk<C>(x.x + y.x, x.y - y.y);
            const C D = cmk<C>(x.x - y.x, x.y + y.y);
            const C O2 = cmulc(D, __ldg(&twx[k]));
            z = cmk<C>(E2.x - O2.y, E2.y + O2.x);
        }
        A[sw(k * TR + rr)] = z;
    }
    __syncthreads();
    const C *Z = gen_fft<C, true>(A, B, 1, 0, g, twx, 2);
    const T gsc = o.gdev ? (T)(*o.gdev) : (T)1;
    const T oscale = o.oscale * gsc;
    T acc = 0;
    // outputs x < nvalid only: n < (nvalid + 1) / 2 of each row
    const int nh = (nvalid + 1) / 2 < L ? (nvalid + 1) / 2 : L;
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int rr = udiv(e, L, g.mL), n = e - rr * L, row = row0 + rr;
        if (row >= nrows || n >= nh) continue;
        const C z = Z[sw(n * TR + rr)];
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
    if (o.partials) block_partial<kGenThreads>((double)acc, o.partials, blockIdx.x);
}

// Fused z pass (as k_z_conv): three components per column tile, forward
// transforms, the 3x3 product with the folded tensor spectrum, inverse
// transforms, rows < nrows stored. Column f = ky * width + kx.
template <typename T>
__global__ void __launch_bounds__(kGenThreads)
k_gen_zconv(typename Cplx<T>::type *__restrict__ S, int ncols, int width, unsigned mw, int64_t ss, int64_t rs,
            int64_t cs, int nrows, const T *__restrict__ nhat, int Py, int Kx,
            const typename Cplx<T>::type *__restrict__ tw, int twstride, const __grid_constant__ GenRadix g)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TC = g.TC, TS = swsize(L * TC);
    C *A = reinterpret_cast<C *>(smraw), *B = A + 3 * TS;
    const int f0 = blockIdx.x * TC;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int r = udiv(e, TC, g.mTC), f = f0 + e - r * TC;
        C v0 = cmk<C>(0, 0), v1 = v0, v2 = v0;
        if (f < ncols && r < nrows) {
            const int slab = udiv(f, width, mw);
            const int64_t q = (int64_t)slab * ss + (int64_t)r * rs + (f - slab * width);
            v0 = S[q]; v1 = S[q + cs]; v2 = S[q + 2 * cs];
        }
        A[sw(e)] = v0; A[TS + sw(e)] = v1; A[2 * TS + sw(e)] = v2;
    }
    __syncthreads();
    C *F = gen_fft<C, false>(A, B, 3, TS, g, tw, twstride);
    C *G = F == A ? B : A;
    const int hy = Py / 2 + 1, hz = L / 2 + 1;
    const int64_t plane = (int64_t)hz * hy * Kx;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int kz = udiv(e, TC, g.mTC), f = f0 + e - kz * TC;
        if (f >= ncols) continue;
        const int ky = udiv(f, width, mw), kx = f - ky * width;
        const bool fy = ky > Py / 2, fz = kz > L / 2;
        const int kyf = fy ? Py - ky : ky, kzf = fz ? L - kz : kz;
        const T sy = fy ? (T)-1 : (T)1, sz = fz ? (T)-1 : (T)1;
        const int64_t bq = ((int64_t)kzf * hy + kyf) * Kx + kx;
        const T nxx = __ldg(&nhat[bq]), nyy = __ldg(&nhat[plane + bq]), nzz = __ldg(&nhat[2 * plane + bq]);
        const T nxy = sy * __ldg(&nhat[3 * plane + bq]);
        const T nxz = sz * __ldg(&nhat[4 * plane + bq]);
        const T nyz = sy * sz * __ldg(&nhat[5 * plane + bq]);
        const C mx = F[sw(e)], my = F[TS + sw(e)], mz = F[2 * TS + sw(e)];
        F[sw(e)] = cmk<C>(-(nxx * mx.x + nxy * my.x + nxz * mz.x), -(nxx * mx.y + nxy * my.y + nxz * mz.y));
        F[TS + sw(e)] = cmk<C>(-(nxy * mx.x + nyy * my.x + nyz * mz.x), -(nxy * mx.y + nyy * my.y + nyz * mz.y));
        F[2 * TS + sw(e)] = cmk<C>(-(nxz * mx.x + nyz * my.x + nzz * mz.x), -(nxz * mx.y + nyz * my.y + nzz * mz.y));
    }
    __syncthreads();
    const C *res = gen_fft<C, true>(F, G, 3, TS, g, tw, twstride);
    for (int e = threadIdx.x; e < nrows * TC; e += blockDim.x) {
        const int r = udiv(e, TC, g.mTC), f = f0 + e - r * TC;
        if (f < ncols) {
            const int slab = udiv(f, width, mw);
            const int64_t q = (int64_t)slab * ss + (int64_t)r * rs + (f - slab * width);
            S[q] = res[sw(e)]; S[q + cs] = res[TS + sw(e)]; S[q + 2 * cs] = res[2 * TS + sw(e)];
        }
    }
}

}  // namespace demag
