// Mixed-radix passes for padded lengths that are not powers of two (products
// of 2, 3, 5 and 7): the zero padding of the convolution only needs P >= 2n - 1,
// and a smooth P just above 2n - 1 can hold far fewer padded cells than the
// next power of two (e.g. n = 80: 160 instead of 256 per axis). These kernels
// trade the compile-time register schedules of the power-of-two passes for
// one generic form: a tile of transforms in shared memory, Stockham stages
// of any radix R <= 32 with prime factors 2, 3, 5, 7 (in-register DFTs with
// compile-time twiddles) run from a runtime radix list, ping-ponging between
// two buffers; most lengths take two stages, like the power-of-two passes.
// Same inputs, outputs and epilogues as the power-of-two passes.
#pragma once
#include <type_traits>

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
    unsigned mNB[kGenMaxStages];   // division by L / r
    unsigned mTC, mL, mL1;         // division by TC, L, L + 1
    unsigned mCols;                // division by the grid columns of a tile (z pass: TC / 3)
};

constexpr int kGenThreads = 256;

__device__ __forceinline__ int udiv(int n, int d, unsigned m)
{
    return d == 1 ? n : (int)__umulhi((unsigned)n, m);
}

// cos and sin of 2 pi q / R for the odd prime radices (q = 1 .. (R - 1) / 2).
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
            const int q = (k * m) % R;  // angle 2 pi q / R, q != 0 for prime R
            const T cq = (T)(q <= H ? cos_tab<R>(q) : cos_tab<R>(R - q));
            const T sq = (T)(q <= H ? sin_tab<R>(q) : -sin_tab<R>(R - q));
            a = cmk<C>(a.x + cq * t[k - 1].x, a.y + cq * t[k - 1].y);
            b = cmk<C>(b.x + sq * u[k - 1].x, b.y + sq * u[k - 1].y);
        }
        const C ib = INV ? cmk<C>(-b.y, b.x) : cmk<C>(b.y, -b.x);
        v[m] = cadd(a, ib);
        v[R - m] = csub(a, ib);
    }
}

// Compile-time cos and sin of 2 pi e / n (e, n integers, 0 <= e < n) in
// double: reduction to [0, pi/4] by the symmetries of the circle, then the
// Taylor series (12 terms: remainder below 1e-28 on that interval).
__host__ __device__ constexpr double ct_sin_poly(double x)
{
    double term = x, sum = x;
    for (int k = 1; k < 12; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_cos_poly(double x)
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 12; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
constexpr double kCtPi = 3.14159265358979323846264338327950288;
// The angle is kept as an exact fraction num / den of the full turn while the
// symmetries reduce it to at most 1/8 turn; only the final angle is rounded.
__host__ __device__ constexpr double ct_cos2pi(int e, int n)
{
    long long num = e % n, den = n;
    double sg = 1.0;
    if (2 * num > den) num = den - num;  // cos(2 pi - x) = cos x
    if (4 * num > den) {                 // cos x = -cos(pi - x)
        num = den - 2 * num;
        den *= 2;
        sg = -1.0;
    }
    if (8 * num > den) return sg * ct_sin_poly(2.0 * kCtPi * (double)(den - 4 * num) / (4.0 * (double)den));
    return sg * ct_cos_poly(2.0 * kCtPi * (double)num / (double)den);
}
__host__ __device__ constexpr double ct_sin2pi(int e, int n)
{
    long long num = e % n, den = n;
    double sg = 1.0;
    if (2 * num > den) {  // sin(2 pi - x) = -sin x
        num = den - num;
        sg = -1.0;
    }
    if (4 * num > den) {  // sin x = sin(pi - x)
        num = den - 2 * num;
        den *= 2;
    }
    if (8 * num > den) return sg * ct_cos_poly(2.0 * kCtPi * (double)(den - 4 * num) / (4.0 * (double)den));
    return sg * ct_sin_poly(2.0 * kCtPi * (double)num / (double)den);
}

// x W_R^E (forward, W_R = exp(-2 pi i / R)) or x conj(W_R^E) (inverse), the
// constants folded at compile time.
template <int R, int E, bool INV, typename C>
__device__ __forceinline__ C twmul(C x)
{
    using T = decltype(C::x);
    constexpr int e = E % R;
    if constexpr (e == 0) {
        return x;
    } else if constexpr (4 * e == R) {
        return INV ? cmk<C>(-x.y, x.x) : cmk<C>(x.y, -x.x);
    } else if constexpr (2 * e == R) {
        return cmk<C>(-x.x, -x.y);
    } else if constexpr (4 * e == 3 * R) {
        return INV ? cmk<C>(x.y, -x.x) : cmk<C>(-x.y, x.x);
    } else {
        constexpr double c = ct_cos2pi(e, R), s = ct_sin2pi(e, R);
        if (INV) return cmk<C>(x.x * (T)c - x.y * (T)s, x.x * (T)s + x.y * (T)c);
        return cmk<C>(x.x * (T)c + x.y * (T)s, x.y * (T)c - x.x * (T)s);
    }
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1.
template <int B, int E> struct SFor {
    template <typename F> __device__ __forceinline__ static void run(F &&f)
    {
        if constexpr (B < E) {
            f(std::integral_constant<int, B>{});
            SFor<B + 1, E>::run(f);
        }
    }
};

__host__ __device__ constexpr int small_prime_factor(int n) { return n % 2 == 0 ? 2 : n % 3 == 0 ? 3 : n % 5 == 0 ? 5 : n % 7 == 0 ? 7 : n; }
__host__ __device__ constexpr bool pow2_const(int n) { return n > 0 && (n & (n - 1)) == 0; }

// In-register DFT of R points (R a product of 2, 3, 5, 7), natural order in
// and out: powers of two by RegDFT, primes by the pair form, composites by
// decimation in time R = P Q (P the smallest prime factor): Q-point DFTs of
// the P subsequences x[m P + q], twiddles W_R^{q k}, P-point DFTs across q:
// X[k + Q s] = sum_q W_P^{q s} W_R^{q k} Y_q[k].
template <int R, bool INV, typename C> struct MixDFT {
    static __device__ __forceinline__ void run(C *v)
    {
        if constexpr (pow2_const(R)) {
            RegDFT<R, INV, C>::run(v);
        } else if constexpr (small_prime_factor(R) == R) {
            dft_odd<R, INV, C>(v);
        } else {
            constexpr int P = small_prime_factor(R), Q = R / P;
            C sub[P][Q];
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
                for (int m = 0; m < Q; ++m) sub[q][m] = v[m * P + q];
#pragma unroll
            for (int q = 0; q < P; ++q) MixDFT<Q, INV, C>::run(sub[q]);
            SFor<0, Q>::run([&](auto kk) {
                constexpr int k = decltype(kk)::value;
                C t[P];
                SFor<0, P>::run([&](auto qq) {
                    constexpr int q = decltype(qq)::value;
                    t[q] = twmul<R, q * k, INV>(sub[q][k]);
                });
                MixDFT<P, INV, C>::run(t);
#pragma unroll
                for (int s2 = 0; s2 < P; ++s2) v[k + Q * s2] = t[s2];
            });
        }
    }
};

constexpr int kGenMaxRadixRows = 16, kGenMaxRadixZ = 32;

// Stages with caller-supplied ends: the first stage reads its inputs through
// ld(row, col) (global memory, with the pass's prologue) and the last stage
// writes through st(row, col, value) (global memory with the epilogue, or
// shared memory), so a plan of n stages makes n - 1 shared-memory exchanges.
// Tiles in shared memory: XROW = false: [row][col] (columns of the y pass,
// consecutive columns contiguous in global memory); XROW = true: [col][row]
// (rows of the x passes, contiguous along row), and consecutive threads then
// take consecutive butterflies of one transform.
template <typename C, bool XROW> struct GenSmemLd {
    const C *p;
    int TC, L;
    __device__ __forceinline__ C operator()(int row, int col) const
    {
        return p[sw(XROW ? col * L + row : row * TC + col)];
    }
};
template <typename C, bool XROW> struct GenSmemSt {
    C *p;
    int TC, L;
    __device__ __forceinline__ void operator()(int row, int col, C v) const
    {
        p[sw(XROW ? col * L + row : row * TC + col)] = v;
    }
};

template <typename C, int R, bool INV, bool XROW, typename LD, typename ST>
__device__ __forceinline__ void gen_stage_io(const GenRadix &g, int s, const C *__restrict__ tw, int twstride,
                                             const LD &ld, const ST &st)
{
    const int L = g.L, TC = g.TC, NS = g.NS[s];
    const int NB = L / R, total = NB * TC;
    const int tws = (L / (NS * R)) * twstride;
    const unsigned mNS = g.mNS[s];
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        int j, col;
        if constexpr (XROW) {
            col = udiv(b, NB, g.mNB[s]);
            j = b - col * NB;
        } else {
            j = udiv(b, TC, g.mTC);
            col = b - j * TC;
        }
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(j + r * NB, col);
        const int q = udiv(j, NS, mNS), k = j - q * NS;
        if (k > 0) {
            const int kt = k * tws;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C w = __ldg(&tw[r * kt]);
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        MixDFT<R, INV, C>::run(v);
        const int d = q * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) st(d + r * NS, col, v[r]);
    }
}

template <typename C, bool INV, bool XROW, int MAXR, typename LD, typename ST>
__device__ __forceinline__ void gen_stage_any(const GenRadix &g, int s, const C *__restrict__ tw, int twstride,
                                              const LD &ld, const ST &st)
{
    switch (g.r[s]) {
    case 2: gen_stage_io<C, 2, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 3: gen_stage_io<C, 3, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 4: gen_stage_io<C, 4, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 5: gen_stage_io<C, 5, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 6: gen_stage_io<C, 6, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 7: gen_stage_io<C, 7, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 8: gen_stage_io<C, 8, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 9: gen_stage_io<C, 9, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 10: gen_stage_io<C, 10, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 12: gen_stage_io<C, 12, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 14: gen_stage_io<C, 14, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 15: gen_stage_io<C, 15, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 16: gen_stage_io<C, 16, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 18: if constexpr (MAXR >= 18) gen_stage_io<C, 18, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 20: if constexpr (MAXR >= 20) gen_stage_io<C, 20, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 21: if constexpr (MAXR >= 21) gen_stage_io<C, 21, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 24: if constexpr (MAXR >= 24) gen_stage_io<C, 24, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 25: if constexpr (MAXR >= 25) gen_stage_io<C, 25, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 27: if constexpr (MAXR >= 27) gen_stage_io<C, 27, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 28: if constexpr (MAXR >= 28) gen_stage_io<C, 28, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 30: if constexpr (MAXR >= 30) gen_stage_io<C, 30, INV, XROW>(g, s, tw, twstride, ld, st); break;
    case 32: if constexpr (MAXR >= 32) gen_stage_io<C, 32, INV, XROW>(g, s, tw, twstride, ld, st); break;
    default: break;
    }
}

// Whole transform (radices <= MAXR) from ld to st (LASTG) or to a shared
// buffer that is returned (A, or B when the stages end there). Shared
// buffers used: A for the first stage's output, B from the third stage on
// (LASTG) or from the second (otherwise). Every input is read, and a barrier
// passed, before the first output is written (in-place calls are safe).
template <typename C, bool INV, bool XROW, bool LASTG, int MAXR, typename LD, typename ST>
__device__ __forceinline__ C *gen_fft_io(C *A, C *B, const GenRadix &g, const C *__restrict__ tw, int twstride,
                                         const LD &ld0, const ST &stN)
{
    const int n = g.n;
    if constexpr (LASTG) {
        if (n == 1) {
            // one stage: through shared memory, so that an in-place call (the
            // same global buffer read and written) reads every input first
            gen_stage_any<C, INV, XROW, MAXR>(g, 0, tw, twstride, ld0, GenSmemSt<C, XROW>{A, g.TC, g.L});
            __syncthreads();
            for (int e = threadIdx.x; e < g.L * g.TC; e += blockDim.x) {
                int row, col;
                if constexpr (XROW) {
                    col = udiv(e, g.L, g.mL);
                    row = e - col * g.L;
                } else {
                    row = udiv(e, g.TC, g.mTC);
                    col = e - row * g.TC;
                }
                stN(row, col, GenSmemLd<C, XROW>{A, g.TC, g.L}(row, col));
            }
            return nullptr;
        }
    }
    gen_stage_any<C, INV, XROW, MAXR>(g, 0, tw, twstride, ld0, GenSmemSt<C, XROW>{A, g.TC, g.L});
    __syncthreads();
    C *src = A, *dst = B;
    for (int s = 1; s < (LASTG ? n - 1 : n); ++s) {
        gen_stage_any<C, INV, XROW, MAXR>(g, s, tw, twstride, GenSmemLd<C, XROW>{src, g.TC, g.L},
                                    GenSmemSt<C, XROW>{dst, g.TC, g.L});
        __syncthreads();
        C *t = src;
        src = dst;
        dst = t;
    }
    if constexpr (LASTG) {
        gen_stage_any<C, INV, XROW, MAXR>(g, n - 1, tw, twstride, GenSmemLd<C, XROW>{src, g.TC, g.L}, stN);
        return nullptr;
    } else {
        return src;
    }
}

// Shared buffers a kernel of the I/O form needs for a plan of n stages.
inline int gen_io_buffers(int n, bool last_global) { return last_global ? (n >= 3 ? 2 : 1) : (n >= 2 ? 2 : 1); }

// Column transforms (as k_col2): g.TC columns per CTA, rows < nin read,
// rows < nout written; column f = slab * width + (f mod width), mw the
// multiplier of width. The first stage reads global memory, the last writes it.
template <typename T, bool INV>
__global__ void __launch_bounds__(kGenThreads, sizeof(T) == 4 ? 3 : 1)
k_gen_col(const typename Cplx<T>::type *__restrict__ in, typename Cplx<T>::type *__restrict__ out, int ncols, int width,
          unsigned mw, int64_t iss, int64_t irs, int nin, int64_t oss, int64_t ors, int nout,
          const typename Cplx<T>::type *__restrict__ tw, int twstride, const __grid_constant__ GenRadix g)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int TS = swsize(g.L * g.TC);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int f0 = blockIdx.x * g.TC;
    auto ld = [&](int row, int col) {
        const int f = f0 + col;
        C v = cmk<C>(0, 0);
        if (f < ncols && row < nin) {
            const int slab = udiv(f, width, mw);
            v = in[(int64_t)slab * iss + (int64_t)row * irs + (f - slab * width)];
        }
        return v;
    };
    auto st = [&](int row, int col, C v) {
        const int f = f0 + col;
        if (f < ncols && row < nout) {
            const int slab = udiv(f, width, mw);
            out[(int64_t)slab * oss + (int64_t)row * ors + (f - slab * width)] = v;
        }
    };
    gen_fft_io<C, INV, false, true, kGenMaxRadixRows>(A, B, g, tw, twstride, ld, st);
}

// Real-to-complex rows (as k_x_fwd): pack pairs of reals, transform of
// L = Px/2 points (first stage from global memory), split into X[k],
// k = 0..L. g.TC rows per CTA.
template <typename T>
__global__ void __launch_bounds__(kGenThreads, sizeof(T) == 4 ? 3 : 1)
k_gen_x_fwd(XIn<T> a, int nrows, int nvalid, typename Cplx<T>::type *__restrict__ out, int64_t out_rs,
            const typename Cplx<T>::type *__restrict__ twx, const __grid_constant__ GenRadix g)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TR = g.TC, TS = swsize(L * TR);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int row0 = blockIdx.x * TR;
    const bool pairs = (a.in_rs & 1) == 0;  // rows start on a pair boundary: one vector load per pair
    auto ld = [&](int n, int rr) {
        const int row = row0 + rr, x0 = 2 * n;
        C z = cmk<C>(0, 0);
        if (row < nrows && x0 < nvalid) {
            const T *p = a.in + (int64_t)row * a.in_rs;
            if (pairs && x0 + 1 < nvalid) {
                z = *reinterpret_cast<const C *>(p + x0);
            } else {
                z.x = p[x0];
                if (x0 + 1 < nvalid) z.y = p[x0 + 1];
            }
            z.x *= a.wscalar * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0);
            if (x0 + 1 < nvalid) z.y *= a.wscalar * cell_weight(a.wcell, row, a.rows_per_comp, a.in_rs, x0 + 1);
        }
        return z;
    };
    const GenSmemSt<C, true> none{nullptr, TR, L};
    const C *Z = gen_fft_io<C, false, true, false, kGenMaxRadixRows>(A, B, g, twx, 2, ld, none);
    const T h = (T)0.5;
    for (int e = threadIdx.x; e < (L + 1) * TR; e += blockDim.x) {
        const int rr = udiv(e, L + 1, g.mL1), k = e - rr * (L + 1), row = row0 + rr;
        if (row >= nrows) continue;
        const C p = Z[sw(rr * L + (k == L ? 0 : k))];
        const C q = Z[sw(rr * L + (k == 0 ? 0 : L - k))];
        const C E = cmk<C>(h * (p.x + q.x), h * (p.y - q.y));
        const C O = cmk<C>(h * (p.y + q.y), -h * (p.x - q.x));
        out[(int64_t)row * out_rs + k] = cadd(E, cmul(O, __ldg(&twx[k])));
    }
}

// Complex-to-real rows (as k_x_inv): the first stage forms the packed
// spectrum from X[k] and X[L-k] in global memory, the last applies the XOut
// epilogue (energy partials one per CTA).
template <typename T>
__global__ void __launch_bounds__(kGenThreads, sizeof(T) == 4 ? 3 : 1)
k_gen_x_inv(const typename Cplx<T>::type *__restrict__ in, int64_t in_rs, int nrows, int nvalid, XOut<T> o,
            const typename Cplx<T>::type *__restrict__ twx, const __grid_constant__ GenRadix g)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TR = g.TC, TS = swsize(L * TR);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int row0 = blockIdx.x * TR;
    auto ld = [&](int k, int rr) {
        const int row = row0 + rr;
        C z = cmk<C>(0, 0);
        if (row < nrows) {
            const C *p = in + (int64_t)row * in_rs;
            const C x = p[k], y = p[L - k];
            const C E2 = cmk<C>(x.x + y.x, x.y - y.y);
            const C D = cmk<C>(x.x - y.x, x.y + y.y);
            const C O2 = cmulc(D, __ldg(&twx[k]));
            z = cmk<C>(E2.x - O2.y, E2.y + O2.x);
        }
        return z;
    };
    const T gsc = o.gdev ? (T)(*o.gdev) : (T)1;
    const T oscale = o.oscale * gsc;
    T acc = 0;
    const bool pairs = (o.out_rs & 1) == 0;  // rows start on a pair boundary: vector stores and loads
    auto st = [&](int n, int rr, C z) {
        const int row = row0 + rr, x0 = 2 * n;
        if (row >= nrows || x0 >= nvalid) return;
        const T hv[2] = {z.x * o.scale, z.y * o.scale};
        const int64_t idx0 = (int64_t)row * o.out_rs + x0;
        if (pairs && x0 + 1 < nvalid) {
            const T w0 = cell_weight(o.wcell, row, o.rows_per_comp, o.out_rs, x0);
            const T w1 = cell_weight(o.wcell, row, o.rows_per_comp, o.out_rs, x0 + 1);
            if (o.out) *reinterpret_cast<C *>(o.out + idx0) = cmk<C>(hv[0] * oscale * w0, hv[1] * oscale * w1);
            if (o.partials) {
                const C m = *reinterpret_cast<const C *>(o.Mref + idx0);
                acc += o.mscale * (w0 * m.x * hv[0] + w1 * m.y * hv[1]);
            }
            return;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int x = x0 + u;
            if (x >= nvalid) continue;
            const T w = cell_weight(o.wcell, row, o.rows_per_comp, o.out_rs, x);
            const int64_t idx = idx0 + u;
            if (o.out) o.out[idx] = hv[u] * oscale * w;
            if (o.partials) acc += o.mscale * w * o.Mref[idx] * hv[u];
        }
    };
    gen_fft_io<C, true, true, true, kGenMaxRadixRows>(A, B, g, twx, 2, ld, st);
    if (o.partials) block_partial<kGenThreads>((double)acc, o.partials, blockIdx.x);
}

// Fused z pass (as k_z_conv): the three components of TC = g.TC / 3 columns
// form one [row][3 TC] tile (component-major columns). Forward transform
// with the first stage reading global memory (rows < nrows), the 3x3
// product with the folded tensor spectrum in shared memory, inverse
// transform whose last stage stores rows < nrows. Column f = ky * width + kx.
template <typename T>
__global__ void __launch_bounds__(kGenThreads)
k_gen_zconv(typename Cplx<T>::type *__restrict__ S, int ncols, int width, unsigned mw, int64_t ss, int64_t rs,
            int64_t cs, int nrows, const T *__restrict__ nhat, int Py, int Kx,
            const typename Cplx<T>::type *__restrict__ tw, int twstride, const __grid_constant__ GenRadix g)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g.L, TCC = g.TC, TC = TCC / 3, TS = swsize(L * TCC);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int f0 = blockIdx.x * TC;
    // column cc of the tile: component cc / TC, grid column f0 + cc % TC
    auto gaddr = [&](int row, int cc, bool &ok) {
        const int comp = cc >= 2 * TC ? 2 : (cc >= TC ? 1 : 0), f = f0 + cc - comp * TC;
        ok = f < ncols && row < nrows;
        const int slab = udiv(f, width, mw);
        return (int64_t)slab * ss + (int64_t)row * rs + (f - slab * width) + comp * cs;
    };
    auto ld = [&](int row, int cc) {
        bool ok;
        const int64_t q = gaddr(row, cc, ok);
        return ok ? S[q] : cmk<C>(0, 0);
    };
    const GenSmemSt<C, false> none{nullptr, TCC, L};
    C *F = gen_fft_io<C, false, false, false, kGenMaxRadixZ>(A, B, g, tw, twstride, ld, none);
    C *G = F == A ? B : A;
    const int hy = Py / 2 + 1, hz = L / 2 + 1;
    const int64_t plane = (int64_t)hz * hy * Kx;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int kz = udiv(e, TC, g.mCols), c = e - kz * TC, f = f0 + c;
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
        // row kz: the components at columns c, TC + c, 2 TC + c
        const int i0 = sw(kz * TCC + c), i1 = sw(kz * TCC + TC + c), i2 = sw(kz * TCC + 2 * TC + c);
        const C mx = F[i0], my = F[i1], mz = F[i2];
        F[i0] = cmk<C>(-(nxx * mx.x + nxy * my.x + nxz * mz.x), -(nxx * mx.y + nxy * my.y + nxz * mz.y));
        F[i1] = cmk<C>(-(nxy * mx.x + nyy * my.x + nyz * mz.x), -(nxy * mx.y + nyy * my.y + nyz * mz.y));
        F[i2] = cmk<C>(-(nxz * mx.x + nyz * my.x + nzz * mz.x), -(nxz * mx.y + nyz * my.y + nzz * mz.y));
    }
    __syncthreads();
    auto st = [&](int row, int cc, C v) {
        bool ok;
        const int64_t q = gaddr(row, cc, ok);
        if (ok) S[q] = v;
    };
    gen_fft_io<C, true, false, true, kGenMaxRadixZ>(G, F, g, tw, twstride, GenSmemLd<C, false>{F, TCC, L}, st);
}

// Fused SP z pass (as k_sp_z2) for lengths that are not powers of two: the
// forward transforms of the three components run as in k_gen_zconv; the
// product with the kernel tables and the half-cell phase (-i Phi, from the
// per-axis tables phx, phy, phz) leaves one component in the first TC tile
// columns; its inverse transform (plan g1, TC columns) stores the nout = nrows
// + 1 node rows over component 0 (running on into the first row of component
// 1, cs == nrows * rs: only this CTA reads or writes its columns, and every
// input was read before the first output is written).
template <typename T>
__global__ void __launch_bounds__(kGenThreads)
k_gen_sp_zconv(typename Cplx<T>::type *__restrict__ S, int ncols, int width, unsigned mw, int64_t ss, int64_t rs,
               int64_t cs, int nrows, int nout, const T *__restrict__ that, int Py, int Kx,
               const typename Cplx<T>::type *__restrict__ tw, const typename Cplx<T>::type *__restrict__ phx,
               const typename Cplx<T>::type *__restrict__ phy, const typename Cplx<T>::type *__restrict__ phz,
               const __grid_constant__ GenRadix g3, const __grid_constant__ GenRadix g1)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = g3.L, TCC = g3.TC, TC = g1.TC, TS = swsize(L * TCC);
    C *A = reinterpret_cast<C *>(smraw), *B = A + TS;
    const int f0 = blockIdx.x * TC;
    auto ld = [&](int row, int cc) {
        const int comp = cc >= 2 * TC ? 2 : (cc >= TC ? 1 : 0), f = f0 + cc - comp * TC;
        C v = cmk<C>(0, 0);
        if (f < ncols && row < nrows) {
            const int slab = udiv(f, width, mw);
            v = S[(int64_t)slab * ss + (int64_t)row * rs + (f - slab * width) + comp * cs];
        }
        return v;
    };
    const GenSmemSt<C, false> none{nullptr, TCC, L};
    C *F = gen_fft_io<C, false, false, false, kGenMaxRadixZ>(A, B, g3, tw, 1, ld, none);
    C *G = F == A ? B : A;
    const int hy = Py / 2 + 1, hz = L / 2 + 1;
    const int64_t plane = (int64_t)hz * hy * Kx;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int kz = udiv(e, TC, g3.mCols), c = e - kz * TC, f = f0 + c;
        C p = cmk<C>(0, 0);
        const C mx = F[sw(kz * TCC + c)], my = F[sw(kz * TCC + TC + c)], mz = F[sw(kz * TCC + 2 * TC + c)];
        if (f < ncols) {
            const int ky = udiv(f, width, mw), kx = f - ky * width;
            const bool fy = ky > Py / 2, fz = kz > L / 2;
            const int kyf = fy ? Py - ky : ky, kzf = fz ? L - kz : kz;
            const T sy = fy ? (T)-1 : (T)1, sz = fz ? (T)-1 : (T)1;
            const int64_t bq = ((int64_t)kzf * hy + kyf) * Kx + kx;
            // folds: ky flips T_x and T_z, kz flips T_x and T_y
            const T tx = sy * sz * __ldg(&that[bq]), ty = sz * __ldg(&that[plane + bq]),
                    tz = sy * __ldg(&that[2 * plane + bq]);
            const C pxy = cmul(__ldg(&phx[kx]), __ldg(&phy[ky]));
            const C ph = cmul(cmk<C>(pxy.y, -pxy.x), __ldg(&phz[kz]));  // -i Phi
            const C a = cmk<C>(tx * mx.x + ty * my.x + tz * mz.x, tx * mx.y + ty * my.y + tz * mz.y);
            p = cmul(a, ph);
        }
        F[sw(kz * TCC + c)] = p;  // only this thread reads or writes element (kz, c)
    }
    __syncthreads();
    auto ldf = [&](int row, int c) { return F[sw(row * TCC + c)]; };
    auto st = [&](int row, int c, C v) {
        const int f = f0 + c;
        if (f < ncols && row < nout) {
            const int slab = udiv(f, width, mw);
            S[(int64_t)slab * ss + (int64_t)row * rs + (f - slab * width)] = v;
        }
    };
    gen_fft_io<C, true, false, true, kGenMaxRadixZ>(G, F, g1, tw, 1, ldf, st);
}

}  // namespace demag
