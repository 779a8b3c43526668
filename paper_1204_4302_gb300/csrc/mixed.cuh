// Mixed-radix passes for padded lengths that are not powers of two (products
// of 2, 3, 5 and 7): the zero padding of the convolution only needs P >= 2n - 1,
// and a smooth P just above 2n - 1 can hold far fewer padded cells than the
// next power of two (e.g. n = 80: 160 instead of 256 per axis). These kernels
// trade the compile-time register schedules of the power-of-two passes for
// one generic form: a tile of transforms in shared memory, Stockham stages of
// radix 8, 4, 2, 3, 5 or 7 run with a runtime radix list, ping-ponging between
// two buffers. Same inputs, outputs and epilogues as the power-of-two passes.
#pragma once
#include "fft_engine.cuh"

namespace demag {

// Radices of one transform, in stage order (product L).
struct GenRadix {
    int L;
    int n;
    int r[16];
};

constexpr int kGenThreads = 256;
constexpr int kGenTileElems = 2048;  // transform elements per buffer (L x columns)

// DFT of 3 points: y_k = sum_j x_j w^{jk}, w = exp(-+2 pi i / 3).
template <bool INV, typename C>
__device__ __forceinline__ void dft3(C *v)
{
    using T = decltype(C::x);
    const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
    const C t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    const C y0 = cadd(v[0], t1);
    const C m = cmk<C>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
    // forward: y1 = m - i h t2, y2 = m + i h t2 (inverse: signs swapped)
    const C s = INV ? cmk<C>(-h * t2.y, h * t2.x) : cmk<C>(h * t2.y, -h * t2.x);
    v[0] = y0;
    v[1] = cadd(m, s);
    v[2] = csub(m, s);
}

// DFT of 5 points with the angles 2 pi / 5 and 4 pi / 5.
template <bool INV, typename C>
__device__ __forceinline__ void dft5(C *v)
{
    using T = decltype(C::x);
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
    const C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    const C y0 = cadd(v[0], cadd(t1, t2));
    const C a1 = cmk<C>(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    const C a2 = cmk<C>(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    const C b1 = cmk<C>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
    const C b2 = cmk<C>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
    // forward: y1 = a1 - i b1, y4 = a1 + i b1, y2 = a2 - i b2, y3 = a2 + i b2
    const C ib1 = INV ? cmk<C>(-b1.y, b1.x) : cmk<C>(b1.y, -b1.x);
    const C ib2 = INV ? cmk<C>(-b2.y, b2.x) : cmk<C>(b2.y, -b2.x);
    v[0] = y0;
    v[1] = cadd(a1, ib1);
    v[4] = csub(a1, ib1);
    v[2] = cadd(a2, ib2);
    v[3] = csub(a2, ib2);
}

// DFT of 7 points: pairs x_k +- x_{7-k}, k = 1..3, against cos and sin of
// 2 pi k m / 7 (y_m = a_m - i b_m, y_{7-m} = a_m + i b_m in the forward sense).
template <bool INV, typename C>
__device__ __forceinline__ void dft7(C *v)
{
    using T = decltype(C::x);
    const T c[3] = {(T)0.623489801858733530525, (T)-0.222520933956314404289, (T)-0.900968867902419126236};
    const T s[3] = {(T)0.781831482468029808708, (T)0.974927912181823607018, (T)0.433883739117558120476};
    C t[3], u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        t[k] = cadd(v[k + 1], v[6 - k]);
        u[k] = csub(v[k + 1], v[6 - k]);
    }
    const C x0 = v[0];
    v[0] = cadd(x0, cadd(t[0], cadd(t[1], t[2])));
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        C a = x0, b = cmk<C>(0, 0);
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            const int q = (k * m) % 7;  // angle index of 2 pi k m / 7
            const T cq = q <= 3 ? c[q - 1] : c[7 - q - 1];
            const T sq = q <= 3 ? s[q - 1] : -s[7 - q - 1];
            a = cmk<C>(a.x + cq * t[k - 1].x, a.y + cq * t[k - 1].y);
            b = cmk<C>(b.x + sq * u[k - 1].x, b.y + sq * u[k - 1].y);
        }
        const C ib = INV ? cmk<C>(-b.y, b.x) : cmk<C>(b.y, -b.x);
        v[m] = cadd(a, ib);
        v[7 - m] = csub(a, ib);
    }
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void small_dft(C *v)
{
    if constexpr (R == 3) dft3<INV, C>(v);
    else if constexpr (R == 5) dft5<INV, C>(v);
    else if constexpr (R == 7) dft7<INV, C>(v);
    else RegDFT<R, INV, C>::run(v);
}

// One Stockham stage of radix R from src to dst, ncomp tiles [L][TC] each
// (component stride cstride, swizzled as everywhere). NS = product of the
// earlier radices; tw: table W_P^m of the axis with P = L twstride.
template <typename C, int R, bool INV>
__device__ __forceinline__ void gen_stage(const C *src, C *dst, int ncomp, int cstride, int L, int NS, int TC,
                                          const C *__restrict__ tw, int twstride)
{
    const int NB = L / R, per = NB * TC, total = ncomp * per;
    const int tws = (L / (NS * R)) * twstride;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        const int comp = b / per, bb = b - comp * per;
        const int col = bb % TC, j = bb / TC;
        const C *s = src + comp * cstride;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[sw((j + r * NB) * TC + col)];
        const int k = j % NS;
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C w = __ldg(&tw[r * k * tws]);
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        small_dft<R, INV, C>(v);
        const int d = (j / NS) * NS * R + k;
        C *o = dst + comp * cstride;
#pragma unroll
        for (int r = 0; r < R; ++r) o[sw((d + r * NS) * TC + col)] = v[r];
    }
}

// Whole transform of the tiles in a (b is the second buffer); returns the
// buffer that holds the result.
template <typename C, bool INV>
__device__ C *gen_fft(C *a, C *b, int ncomp, int cstride, const GenRadix &g, int TC, const C *__restrict__ tw,
                      int twstride)
{
    C *src = a, *dst = b;
    int NS = 1;
    for (int s = 0; s < g.n; ++s) {
        const int R = g.r[s];
        switch (R) {
        case 2: gen_stage<C, 2, INV>(src, dst, ncomp, cstride, g.L, NS, TC, tw, twstride); break;
        case 3: gen_stage<C, 3, INV>(src, dst, ncomp, cstride, g.L, NS, TC, tw, twstride); break;
        case 4: gen_stage<C, 4, INV>(src, dst, ncomp, cstride, g.L, NS, TC, tw, twstride); break;
        case 5: gen_stage<C, 5, INV>(src, dst, ncomp, cstride, g.L, NS, TC, tw, twstride); break;
        case 7: gen_stage<C, 7, INV>(src, dst, ncomp, cstride, g.L, NS, TC, tw, twstride); break;
        default: gen_stage<C, 8, INV>(src, dst, ncomp, cstride, g.L, NS, TC, tw, twstride); break;
        }
        __syncthreads();
        NS *= R;
        C *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Column transforms (as k_col2): TC columns per CTA, rows < nin read, rows
// < nout written.
template <typename T, bool INV>
__global__ void __launch_bounds__(kGenThreads)
k_gen_col(const typename Cplx<T>::type *__restrict__ in, typename Cplx<T>::type *__restrict__ out, int ncols, int width,
          int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, int nout,
          const typename Cplx<T>::type *__restrict__ tw, int twstride, GenRadix g, int TC)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TS = swsize(L * TC);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int f0 = blockIdx.x * TC;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int c = e % TC, r = e / TC, f = f0 + c;
        C v = cmk<C>(0, 0);
        if (f < ncols && r < nin) {
            const int slab = f / width;
            v = in[(int64_t)slab * iss + (int64_t)r * irs + (f - slab * width)];
        }
        A[sw(e)] = v;
    }
    __syncthreads();
    const C *res = gen_fft<C, INV>(A, B, 1, 0, g, TC, tw, twstride);
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int c = e % TC, r = e / TC, f = f0 + c;
        if (f < ncols && r < nout) {
            const int slab = f / width;
            out[(int64_t)slab * oss + (int64_t)r * ors + (f - slab * width)] = res[sw(e)];
        }
    }
}

// Real-to-complex rows (as k_x_fwd): pack pairs of reals, transform of
// L = Px/2 points, split into X[k], k = 0..L. TR rows per CTA.
template <typename T>
__global__ void __launch_bounds__(kGenThreads)
k_gen_x_fwd(XIn<T> a, int nrows, int nvalid, typename Cplx<T>::type *__restrict__ out, int64_t out_rs,
            const typename Cplx<T>::type *__restrict__ twx, GenRadix g, int TR)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TS = swsize(L * TR);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int row0 = blockIdx.x * TR;
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int n = e % L, rr = e / L, row = row0 + rr;
        C z = cmk<C>(0, 0);
        if (row < nrows) {
            const T *p = a.in + (int64_t)row * a.in_rs;
            const int x0 = 2 * n;
            if (x0 < nvalid) z.x = p[x0] * a.wscalar * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0);
            if (x0 + 1 < nvalid)
                z.y = p[x0 + 1] * a.wscalar * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0 + 1);
        }
        A[sw(n * TR + rr)] = z;
    }
    __syncthreads();
    const C *Z = gen_fft<C, false>(A, B, 1, 0, g, TR, twx, 2);
    const T h = (T)0.5;
    for (int e = threadIdx.x; e < (L + 1) * TR; e += blockDim.x) {
        const int k = e % (L + 1), rr = e / (L + 1), row = row0 + rr;
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
            const typename Cplx<T>::type *__restrict__ twx, GenRadix g, int TR)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TS = swsize(L * TR);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int row0 = blockIdx.x * TR;
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int k = e % L, rr = e / L, row = row0 + rr;
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
    const C *Z = gen_fft<C, true>(A, B, 1, 0, g, TR, twx, 2);
    const T gsc = o.gdev ? (T)(*o.gdev) : (T)1;
    const T oscale = o.oscale * gsc;
    T acc = 0;
    for (int e = threadIdx.x; e < L * TR; e += blockDim.x) {
        const int n = e % L, rr = e / L, row = row0 + rr;
        if (row >= nrows) continue;
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
k_gen_zconv(typename Cplx<T>::type *__restrict__ S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
            int nrows, const T *__restrict__ nhat, int Py, int Kx, const typename Cplx<T>::type *__restrict__ tw,
            int twstride, GenRadix g, int TC)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TS = swsize(L * TC);
    C *A = reinterpret_cast<C *>(smraw), *B = A + 3 * TS;
    const int f0 = blockIdx.x * TC;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int c = e % TC, r = e / TC, f = f0 + c;
        C v0 = cmk<C>(0, 0), v1 = v0, v2 = v0;
        if (f < ncols && r < nrows) {
            const int slab = f / width;
            const int64_t q = (int64_t)slab * ss + (int64_t)r * rs + (f - slab * width);
            v0 = S[q]; v1 = S[q + cs]; v2 = S[q + 2 * cs];
        }
        A[sw(e)] = v0; A[TS + sw(e)] = v1; A[2 * TS + sw(e)] = v2;
    }
    __syncthreads();
    C *F = gen_fft<C, false>(A, B, 3, TS, g, TC, tw, twstride);
    C *G = F == A ? B : A;
    const int hy = Py / 2 + 1, hz = L / 2 + 1;
    const int64_t plane = (int64_t)hz * hy * Kx;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int c = e % TC, kz = e / TC, f = f0 + c;
        if (f >= ncols) continue;
        const int ky = f / width, kx = f - ky * width;
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
    const C *res = gen_fft<C, true>(F, G, 3, TS, g, TC, tw, twstride);
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int c = e % TC, r = e / TC, f = f0 + c;
        if (f < ncols && r < nrows) {
            const int slab = f / width;
            const int64_t q = (int64_t)slab * ss + (int64_t)r * rs + (f - slab * width);
            S[q] = res[sw(e)]; S[q + cs] = res[TS + sw(e)]; S[q + 2 * cs] = res[2 * TS + sw(e)];
        }
    }
}

}  // namespace demag
