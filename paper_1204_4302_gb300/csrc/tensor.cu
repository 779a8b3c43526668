// FP64 setup of the demagnetization tensor (paper Sec. 3.1, the tensor N of
// Eq. "demag"; Sec. 4: computed once per geometry; Sec. 5.1: homogeneously
// magnetized cells with the field averaged over each cell).
//
// N_ij(R) = (1/V) Int_cell(R) Int_cell(0) G_ij(r - r') dr' dr,
// G_ij(r) = -(1/4pi) d_i d_j (1/|r|),  positive definite at R = 0 (trace 1).
//
// Offsets R = (i dx, j dy, k dz), 0 <= i < nx etc. (the other octants follow
// by parity): far offsets one thread each, near and separated ones one warp
// each (k_tensor_octant_warp). Three regimes, all in FP64 with lengths scaled
// by the largest cell edge (N is scale invariant):
//   near  (cells touch: |i|,|j|,|k| <= 1): Newell's closed form, the
//         27-point second-difference stencil of f and g (Newell, Williams
//         and Dunlop 1993). Exact, but its cancellation grows like (R/d)^6.
//   mid   (separated, |R| < 20 max d): tensor-product Gauss-Legendre
//         quadrature of G over the tent density of the difference of two
//         uniform points in the two cells (n nodes on each half axis, n from
//         the Bernstein-ellipse bound of the analytic integrand).
//   far   (|R| >= 20 max d): multipole expansion of the same cell average,
//         N_ij = -(V/4pi) sum_a prod_axis mu_{a}(d)/a! d^a d_i d_j (1/|R|)
//         over even multi-indices a of total order <= 10; the tent moments
//         are mu_{2k}(d) = 2 d^{2k} / ((2k+1)(2k+2)). Taylor coefficients of
//         1/|R| come from their three-term recurrence. Truncation ~1e-15.
#include <math.h>

#include <algorithm>
#include <cmath>

#include <vector>

#include "plan.h"

namespace demag {

namespace {

constexpr int kMaxGL = 32;                 // largest half-axis node count
constexpr int kGLTable = kMaxGL * (kMaxGL + 1) / 2;
constexpr int kOrder = 10;                 // multipole truncation (even)
constexpr int kTaylor = kOrder + 2;        // highest derivative order of 1/R
constexpr int kNumTaylor = (kTaylor + 1) * (kTaylor + 2) * (kTaylor + 3) / 6;
constexpr double kFar = 20.0;              // far regime: |R| >= kFar * max d

__constant__ double c_glx[kGLTable];  // rule n at offset n(n-1)/2, nodes on [-1,1]
__constant__ double c_glw[kGLTable];

// Gauss-Legendre nodes and weights by Newton iteration on P_n, started from
// the asymptotic root estimate of Tricomi; host side, FP64.
void legendre_rule(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 1; i <= n; ++i) {
        const double th = pi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
        double t = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(th);
        double d = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, p = t;  // P_{k-1}, P_k
            for (int k = 1; k < n; ++k) {
                const double pn = ((2.0 * k + 1.0) * t * p - k * pm) / (k + 1.0);
                pm = p; p = pn;
            }
            d = (n == 1) ? 1.0 : n * (pm - t * p) / (1.0 - t * t);
            const double step = p / d;
            t -= step;
            if (fabs(step) < 1e-16) {
                // refresh the derivative at the final point
                pm = 1.0; p = t;
                for (int k = 1; k < n; ++k) {
                    const double pn = ((2.0 * k + 1.0) * t * p - k * pm) / (k + 1.0);
                    pm = p; p = pn;
                }
                d = (n == 1) ? 1.0 : n * (pm - t * p) / (1.0 - t * t);
                break;
            }
        }
        x[i - 1] = t;  // descending from +1
        w[i - 1] = 2.0 / ((1.0 - t * t) * d * d);
    }
}

bool upload_rules()
{
    static int done_for = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (done_for == dev) return true;
    std::vector<double> X(kGLTable), W(kGLTable);
    for (int n = 1; n <= kMaxGL; ++n) legendre_rule(n, &X[n * (n - 1) / 2], &W[n * (n - 1) / 2]);
    if (cudaMemcpyToSymbol(c_glx, X.data(), sizeof(double) * kGLTable) != cudaSuccess) return false;
    if (cudaMemcpyToSymbol(c_glw, W.data(), sizeof(double) * kGLTable) != cudaSuccess) return false;
    done_for = dev;
    return true;
}

// Newell's f (even in all arguments) and g (odd in x and y, even in z).
__device__ double newell_f(double x, double y, double z)
{
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z;
    const double r = sqrt(xx + yy + zz);
    if (r == 0.0) return 0.0;
    double v = (2.0 * xx - yy - zz) * r * (1.0 / 6.0);
    const double rxz = sqrt(xx + zz), rxy = sqrt(xx + yy);
    if (y > 0.0 && rxz > 0.0) v += 0.5 * y * (zz - xx) * asinh(y / rxz);
    if (z > 0.0 && rxy > 0.0) v += 0.5 * z * (yy - xx) * asinh(z / rxy);
    if (x > 0.0 && y > 0.0 && z > 0.0) v -= x * y * z * atan(y * z / (x * r));
    return v;
}

__device__ double newell_g(double x, double y, double z)
{
    const double sgn = copysign(1.0, x) * copysign(1.0, y);
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z;
    const double r = sqrt(xx + yy + zz);
    if (r == 0.0) return 0.0;
    const double rxy = sqrt(xx + yy), ryz = sqrt(yy + zz), rxz = sqrt(xx + zz);
    double v = -x * y * r * (1.0 / 3.0);
    if (z > 0.0 && rxy > 0.0) v += x * y * z * asinh(z / rxy);
    if (x > 0.0 && ryz > 0.0) v += y * (3.0 * zz - yy) * (1.0 / 6.0) * asinh(x / ryz);
    if (y > 0.0 && rxz > 0.0) v += x * (3.0 * zz - xx) * (1.0 / 6.0) * asinh(y / rxz);
    if (z > 0.0) v -= zz * z * (1.0 / 6.0) * atan(x * y / (z * r));
    if (y > 0.0) v -= z * yy * 0.5 * atan(x * z / (y * r));
    if (x > 0.0) v -= z * xx * 0.5 * atan(y * z / (x * r));
    return sgn * v;
}

__device__ int half_axis_nodes(double gap, double d)
{
    const double b = gap / d;
    const int n = (int)ceil(17.0 / log(b + sqrt(1.0 + b * b)));
    return n < 2 ? 2 : (n > kMaxGL ? kMaxGL : n);
}

// Tent-weighted 1-D node (i < 2n): mirror pairs of GL nodes on [0, d].
__device__ __forceinline__ void tent_node(int n, int i, double d, double &u, double &w)
{
    const int base = n * (n - 1) / 2;
    const int g = i >> 1;
    const double t = 0.5 * d * (1.0 + c_glx[base + g]);
    w = 0.5 * c_glw[base + g] * (1.0 - t / d);
    u = (i & 1) ? -t : t;
}

// Index of the multi-index (b1, b2, n - b1 - b2) among all of order <= n.
__device__ __forceinline__ int tidx(int b1, int b2, int b3)
{
    const int n = b1 + b2 + b3;
    return n * (n + 1) * (n + 2) / 6 + b1 * (n + 1) - b1 * (b1 - 1) / 2 + b2;
}

// Taylor coefficients t_beta = (1/beta!) d^beta_y 1/|R - y| at y = 0 for all
// multi-indices of order <= kTaylor (index tidx), by the three-term
// recurrence n R^2 t_beta = (2n-1) sum_a R_a t_{beta-e_a} - (n-1) sum_a t_{beta-2e_a}.
__device__ void taylor_inv_r(double X, double Y, double Z, double *t)
{
    const double R2 = X * X + Y * Y + Z * Z;
    const double Rv[3] = {X, Y, Z};
    t[0] = rsqrt(R2);
    for (int n = 1; n <= kTaylor; ++n) {
        const double inv = 1.0 / (n * R2);
        for (int b1 = n; b1 >= 0; --b1)
            for (int b2 = n - b1; b2 >= 0; --b2) {
                const int b3 = n - b1 - b2;
                const int bb[3] = {b1, b2, b3};
                double s = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    if (bb[ax] >= 1) {
                        int m[3] = {b1, b2, b3};
                        m[ax] -= 1;
                        s += (2.0 * n - 1.0) * Rv[ax] * t[tidx(m[0], m[1], m[2])];
                    }
                    if (bb[ax] >= 2) {
                        int m[3] = {b1, b2, b3};
                        m[ax] -= 2;
                        s -= (n - 1.0) * t[tidx(m[0], m[1], m[2])];
                    }
                }
                t[tidx(b1, b2, b3)] = s * inv;
            }
    }
}

__device__ void far_multipole(double X, double Y, double Z, double a, double b, double c, double *out)
{
    // t_beta equal (1/beta!) d^beta (1/|R|) for even |beta| (the only ones used).
    double t[kNumTaylor];
    taylor_inv_r(X, Y, Z, t);
    // per-axis moment factors m_k(d) = mu_{2k}(d) / (2k)! = 2 d^{2k} / (2k+2)!
    double fact[kTaylor + 1];
    fact[0] = 1.0;
    for (int i = 1; i <= kTaylor; ++i) fact[i] = fact[i - 1] * i;
    double mx[kOrder / 2 + 1], my[kOrder / 2 + 1], mz[kOrder / 2 + 1];
    for (int k = 0; k <= kOrder / 2; ++k) {
        mx[k] = 2.0 * pow(a, 2 * k) / fact[2 * k + 2];
        my[k] = 2.0 * pow(b, 2 * k) / fact[2 * k + 2];
        mz[k] = 2.0 * pow(c, 2 * k) / fact[2 * k + 2];
    }
    const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) {
        double s = 0.0;
        // highest orders first: small terms before large ones
        for (int k1 = kOrder / 2; k1 >= 0; --k1)
            for (int k2 = kOrder / 2 - k1; k2 >= 0; --k2)
                for (int k3 = kOrder / 2 - k1 - k2; k3 >= 0; --k3) {
                    int be[3] = {2 * k1, 2 * k2, 2 * k3};
                    be[ci[q]] += 1;
                    be[cj[q]] += 1;
                    s += mx[k1] * my[k2] * mz[k3] * fact[be[0]] * fact[be[1]] * fact[be[2]] *
                         t[tidx(be[0], be[1], be[2])];
                }
        out[q] = -a * b * c / (4.0 * 3.14159265358979323846) * s;
    }
}

// Regime of an offset: touching cells (closed form), separated within
// kFar cells (tent quadrature), far (multipole).
__device__ __forceinline__ int tensor_regime(int i, int j, int k, double X, double Y, double Z, double dmax)
{
    if (i <= 1 && j <= 1 && k <= 1) return 0;
    return X * X + Y * Y + Z * Z >= (kFar * dmax) * (kFar * dmax) ? 2 : 1;
}

// Far offsets, one thread each (the near and mid offsets are left to
// k_tensor_octant_warp).
__global__ void k_tensor_octant(double *__restrict__ out, int nx, int ny, int nz, double a, double b,
                                double c)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((int64_t)nx * ny));
        const double X = i * a, Y = j * b, Z = k * c;
        const double dmax = fmax(a, fmax(b, c));
        if (tensor_regime(i, j, k, X, Y, Z, dmax) != 2) continue;
        double v[6];
        far_multipole(X, Y, Z, a, b, c, v);
        for (int q = 0; q < 6; ++q) out[q * n + idx] = v[q];
    }
}

// Near and mid offsets, one warp each: the 27 stencil points of the closed
// form, or the (z, y) node pairs of the tent quadrature, are spread over the
// lanes and the six sums reduced across the warp. The offsets of the box
// [0, bx) x [0, by) x [0, bz) (which holds every near and mid offset of the
// table) that are far are skipped (warp-uniform).
__global__ void __launch_bounds__(256) k_tensor_octant_warp(double *__restrict__ out, int nx, int ny, int nz,
                                                            double a, double b, double c, int bx, int by, int bz)
{
    const int64_t n = (int64_t)nx * ny * nz;
    const int lane = threadIdx.x & 31;
    const int64_t nbox = (int64_t)bx * by * bz;
    const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nbox; w += wstep) {
        const int i = (int)(w % bx), j = (int)((w / bx) % by), k = (int)(w / ((int64_t)bx * by));
        const double X = i * a, Y = j * b, Z = k * c;
        const double dmax = fmax(a, fmax(b, c));
        const int reg = tensor_regime(i, j, k, X, Y, Z, dmax);
        if (reg == 2) continue;
        double s[6] = {0, 0, 0, 0, 0, 0};
        double scale;
        if (reg == 0) {
            if (lane < 27) {
                const int p = lane % 3 - 1, q = (lane / 3) % 3 - 1, t = lane / 9 - 1;
                const double wt = (p == 0 ? 2.0 : -1.0) * (q == 0 ? 2.0 : -1.0) * (t == 0 ? 2.0 : -1.0);
                const double x = X + p * a, y = Y + q * b, z = Z + t * c;
                s[0] = wt * newell_f(x, y, z);
                s[1] = wt * newell_f(y, x, z);
                s[2] = wt * newell_f(z, y, x);
                s[3] = wt * newell_g(x, y, z);
                s[4] = wt * newell_g(x, z, y);
                s[5] = wt * newell_g(y, z, x);
            }
            scale = 1.0 / (4.0 * 3.14159265358979323846 * a * b * c);
        } else {
            const double gx = fmax(0.0, fabs(X) - a), gy = fmax(0.0, fabs(Y) - b), gz = fmax(0.0, fabs(Z) - c);
            const double gap = sqrt(gx * gx + gy * gy + gz * gz);
            const int nxn = half_axis_nodes(gap, a), nyn = half_axis_nodes(gap, b), nzn = half_axis_nodes(gap, c);
            const int pairs = 4 * nzn * nyn;
            for (int pr = lane; pr < pairs; pr += 32) {
                const int kk = pr / (2 * nyn), jj = pr - kk * (2 * nyn);
                double uz, wz, uy, wy;
                tent_node(nzn, kk, c, uz, wz);
                tent_node(nyn, jj, b, uy, wy);
                const double rz = Z + uz, ry = Y + uy;
                double pp[6] = {0, 0, 0, 0, 0, 0};
                for (int ii = 0; ii < 2 * nxn; ++ii) {
                    double ux, wx;
                    tent_node(nxn, ii, a, ux, wx);
                    const double rx = X + ux;
                    const double r2 = rx * rx + ry * ry + rz * rz;
                    const double ir = rsqrt(r2);
                    const double ir2 = ir * ir;
                    const double f = wx * ir2 * ir2 * ir;  // w / r^5
                    pp[0] += f * (3.0 * rx * rx - r2);
                    pp[1] += f * (3.0 * ry * ry - r2);
                    pp[2] += f * (3.0 * rz * rz - r2);
                    pp[3] += f * 3.0 * rx * ry;
                    pp[4] += f * 3.0 * rx * rz;
                    pp[5] += f * 3.0 * ry * rz;
                }
                const double wyz = wy * wz;
                for (int q = 0; q < 6; ++q) s[q] += wyz * pp[q];
            }
            scale = -a * b * c / (4.0 * 3.14159265358979323846);
        }
        for (int q = 0; q < 6; ++q)
            for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
        if (lane == 0) {
            const int64_t idx = ((int64_t)k * ny + j) * nx + i;
            for (int q = 0; q < 6; ++q) out[q * n + idx] = scale * s[q];
        }
    }
}

__global__ void k_wrap(const double *__restrict__ oct, int comp, int nx, int ny, int nz, int Px, int Py,
                       int Pz, double *__restrict__ out)
{
    const int64_t total = (int64_t)Px * Py * Pz;
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int px = (int)(idx % Px), py = (int)((idx / Px) % Py), pz = (int)(idx / ((int64_t)Px * Py));
        // wrapped index -> signed offset, or none if no pair of cells has it
        const int i = px < nx ? px : (px > Px - nx ? px - Px : INT_MIN);
        const int j = py < ny ? py : (py > Py - ny ? py - Py : INT_MIN);
        const int k = pz < nz ? pz : (pz > Pz - nz ? pz - Pz : INT_MIN);
        double v = 0.0;
        if (i != INT_MIN && j != INT_MIN && k != INT_MIN) {
            const int64_t t = ((int64_t)abs(k) * ny + abs(j)) * nx + abs(i);
            v = oct[comp * n + t];
            const double si = i < 0 ? -1.0 : 1.0, sj = j < 0 ? -1.0 : 1.0, sk = k < 0 ? -1.0 : 1.0;
            if (comp == 3) v *= si * sj;
            else if (comp == 4) v *= si * sk;
            else if (comp == 5) v *= sj * sk;
        }
        out[idx] = v;
    }
}

// Largest |imaginary residue| of a block (256 threads) into *imag_max with
// one atomic per block (non-negative doubles order like their bit patterns).
__device__ __forceinline__ void block_max_to(double local, unsigned long long *imag_max)
{
    __shared__ double red[8];
    for (int off = 16; off > 0; off >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        atomicMax(imag_max, (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void k_extract(const double2 *__restrict__ S, int comp, int Kx, int Py, int Pz, int Kxp,
                          double *__restrict__ nhat64, float *__restrict__ nhat32,
                          unsigned long long *__restrict__ imag_max)
{
    const int hy = Py / 2 + 1, hz = Pz / 2 + 1;
    const int64_t plane = (int64_t)hz * hy * Kx;
    double local = 0.0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < plane;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(idx % Kx), ky = (int)((idx / Kx) % hy), kz = (int)(idx / ((int64_t)Kx * hy));
        const double2 v = S[((int64_t)kz * Py + ky) * Kxp + kx];
        nhat64[comp * plane + idx] = v.x;
        if (nhat32) nhat32[comp * plane + idx] = (float)v.x;
        local = fmax(local, fabs(v.y));
    }
    block_max_to(local, imag_max);
}

constexpr int kFinalizeThreads = 256;

// Compensated pair sum (s, c) + (s2, c2) -> (s, c): Neumaier's two-sum of the
// leading parts, the error and both compensations in c.
__device__ __forceinline__ void two_sum_add(double &s, double &c, double s2, double c2)
{
    const double t = s + s2;
    const double e = fabs(s) >= fabs(s2) ? (s - t) + s2 : (s2 - t) + s;
    c += c2 + e;
    s = t;
}

// Warp-wide compensated sum by shuffles (five levels, fixed pairing).
__device__ __forceinline__ void warp_two_sum(double &s, double &c)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        two_sum_add(s, c, s2, c2);
    }
}

// Sum of n FP64 partials times `factor` into *E. The CUDA cores' FP64 rate
// per SM is low on this GPU, so the sum is spread over up to kFinalizeBlocks
// CTAs and kept shallow: CTA b sums the contiguous chunk b (Neumaier-
// compensated per thread, then warp shuffles and one shared-memory step over
// the warps) into scratch[2b], scratch[2b + 1]; the CTA that finishes last (a
// counter after the scratch) combines the CTA results the same way in its
// first two warps, writes *E and resets the counter. The pairing is fixed, so
// the result does not depend on which CTA finishes last.
__global__ void __launch_bounds__(kFinalizeThreads) k_energy_finalize(const double *__restrict__ partials, int n,
                                                                      double factor, double *__restrict__ E,
                                                                      double *__restrict__ scratch)
{
    constexpr int NW = kFinalizeThreads / 32;
    __shared__ double ss[NW], sc[NW];
    __shared__ bool s_last;
    const int nb = gridDim.x, chunk = (n + nb - 1) / nb;
    const int lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0, c = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) two_sum_add(s, c, partials[i], 0.0);
    warp_two_sum(s, c);
    if (lane == 0) {
        ss[warp] = s;
        sc[warp] = c;
    }
    __syncthreads();
    unsigned int *count = reinterpret_cast<unsigned int *>(scratch + 2 * kFinalizeBlocks);
    if (warp == 0) {
        s = lane < NW ? ss[lane] : 0.0;
        c = lane < NW ? sc[lane] : 0.0;
        warp_two_sum(s, c);
        if (lane == 0) {
            scratch[2 * blockIdx.x] = s;
            scratch[2 * blockIdx.x + 1] = c;
            __threadfence();
            s_last = atomicAdd(count, 1u) == (unsigned)(nb - 1);
        }
    }
    __syncthreads();
    if (s_last && warp == 0) {
        __threadfence();
        const volatile double *vs = scratch;
        double S = 0.0, C = 0.0;
        for (int b = lane; b < nb; b += 32) two_sum_add(S, C, vs[2 * b], vs[2 * b + 1]);
        warp_two_sum(S, C);
        if (lane == 0) {
            *E = factor * (S + C);
            *count = 0u;
        }
    }
}

// ------------------------------------------------------------------ SP kernel
// Vector kernel of the scalar-potential method (paper Sec. 3.1, Eq. "scpot"):
// the potential at R of a cell of edges (a, b, c) centred at 0 with unit
// magnetization along j,
//   S_j(R) = (1/4pi) Int_cell d/du_j (1/|R - u|) du
//          = (1/4pi) (Int over the face u_j = +d_j/2 - over u_j = -d_j/2) dA / |R - u|.
// Offsets are node-minus-cell-centre, (i + 1/2, j + 1/2, k + 1/2) edges in
// the stored octant. Lengths scaled by the longest edge (S scales like a
// length). Three regimes:
//   near (|X| <= 2.5a, |Y| <= 2.5b, |Z| <= 2.5c): closed form of each face
//        integral, a signed corner sum of F(p, v, w) = v ln(w + r) +
//        w ln(v + r) - p atan(v w / (p r)), r = |(p, v, w)| (d^2F/dv dw = 1/r);
//   mid: Gauss-Legendre quadrature of (R - u)_j / |R - u|^3 over the cell,
//        nodes per axis from the Bernstein ellipse through the nearest
//        singularity of the integrand (R_a + i rho, rho >= the distance of R
//        from the cell in the other two axes);
//   far (|R| >= 20 max d): multipole expansion of the cell's Newtonian
//        potential, S_j = (1/4pi) sum_beta mu_beta (beta_j + 1) t_{beta + e_j}
//        over even beta of order <= 10, mu_beta = V prod_a h_a^beta_a /
//        (beta_a + 1), h = d/2.

// ln(w + r), r = sqrt(q2 + w^2): the form without cancellation for w < 0.
__device__ __forceinline__ double sp_lnwr(double w, double r, double q2)
{
    return w >= 0.0 ? log(w + r) : log(q2 / (r - w));
}

__device__ double sp_F(double p, double v, double w)
{
    const double pp = p * p, vv = v * v, ww = w * w;
    const double r = sqrt(pp + vv + ww);
    if (r == 0.0) return 0.0;
    double s = 0.0;
    if (v != 0.0) s += v * sp_lnwr(w, r, pp + vv);
    if (w != 0.0) s += w * sp_lnwr(v, r, pp + ww);
    if (p != 0.0) s -= p * atan(v * w / (p * r));
    return s;
}

// Integral of 1/|(p, V - v, W - w)| over v in [-hv, hv], w in [-hw, hw].
__device__ double sp_face(double p, double V, double W, double hv, double hw)
{
    return (sp_F(p, V + hv, W + hw) - sp_F(p, V - hv, W + hw)) - (sp_F(p, V + hv, W - hw) - sp_F(p, V - hv, W - hw));
}

__device__ void sp_near(double X, double Y, double Z, double a, double b, double c, double *out)
{
    const double k = 1.0 / (4.0 * 3.14159265358979323846);
    out[0] = k * (sp_face(X - 0.5 * a, Y, Z, 0.5 * b, 0.5 * c) - sp_face(X + 0.5 * a, Y, Z, 0.5 * b, 0.5 * c));
    out[1] = k * (sp_face(Y - 0.5 * b, Z, X, 0.5 * c, 0.5 * a) - sp_face(Y + 0.5 * b, Z, X, 0.5 * c, 0.5 * a));
    out[2] = k * (sp_face(Z - 0.5 * c, X, Y, 0.5 * a, 0.5 * b) - sp_face(Z + 0.5 * c, X, Y, 0.5 * a, 0.5 * b));
}

// GL node count on [-h, h] for a singularity at Ra + i rho: the ellipse with
// foci -+h through it has semi-major axis s h, s = (|z - 1| + |z + 1|) / 2,
// z = (Ra + i rho)/h, and parameter s + sqrt(s^2 - 1).
__device__ int sp_axis_nodes(double Ra, double rho, double h)
{
    const double x = Ra / h, y = rho / h;
    const double s = 0.5 * (sqrt((x - 1.0) * (x - 1.0) + y * y) + sqrt((x + 1.0) * (x + 1.0) + y * y));
    const double e = s + sqrt(fmax(s * s - 1.0, 0.0));
    const int n = e > 1.0 ? (int)ceil(17.0 / log(e)) : kMaxGL;
    return n < 2 ? 2 : (n > kMaxGL ? kMaxGL : n);
}

__device__ void sp_mid(double X, double Y, double Z, double a, double b, double c, double *out)
{
    const double R[3] = {X, Y, Z}, h[3] = {0.5 * a, 0.5 * b, 0.5 * c};
    double g[3];
    for (int q = 0; q < 3; ++q) g[q] = fmax(0.0, fabs(R[q]) - h[q]);
    int n[3];
    for (int q = 0; q < 3; ++q) {
        const double g1 = g[(q + 1) % 3], g2 = g[(q + 2) % 3];
        n[q] = sp_axis_nodes(fabs(R[q]), sqrt(g1 * g1 + g2 * g2), h[q]);
    }
    const int bx = n[0] * (n[0] - 1) / 2, by = n[1] * (n[1] - 1) / 2, bz = n[2] * (n[2] - 1) / 2;
    double s[3] = {0, 0, 0};
    for (int k = 0; k < n[2]; ++k) {
        const double rz = Z - h[2] * c_glx[bz + k], wz = h[2] * c_glw[bz + k];
        for (int j = 0; j < n[1]; ++j) {
            const double ry = Y - h[1] * c_glx[by + j], wy = h[1] * c_glw[by + j];
            double p[3] = {0, 0, 0};
            for (int i = 0; i < n[0]; ++i) {
                const double rx = X - h[0] * c_glx[bx + i];
                const double r2 = rx * rx + ry * ry + rz * rz;
                const double ir = rsqrt(r2);
                const double f = h[0] * c_glw[bx + i] * ir * ir * ir;
                p[0] += f * rx;
                p[1] += f * ry;
                p[2] += f * rz;
            }
            const double w = wy * wz;
            for (int q = 0; q < 3; ++q) s[q] += w * p[q];
        }
    }
    for (int q = 0; q < 3; ++q) out[q] = s[q] * (1.0 / (4.0 * 3.14159265358979323846));
}

__device__ void sp_far(double X, double Y, double Z, double a, double b, double c, double *out)
{
    double t[kNumTaylor];
    taylor_inv_r(X, Y, Z, t);
    // per-axis moments h^{2k} / (2k + 1), h = d/2
    double mx[kOrder / 2 + 1], my[kOrder / 2 + 1], mz[kOrder / 2 + 1];
    for (int k = 0; k <= kOrder / 2; ++k) {
        mx[k] = pow(0.5 * a, 2 * k) / (2 * k + 1);
        my[k] = pow(0.5 * b, 2 * k) / (2 * k + 1);
        mz[k] = pow(0.5 * c, 2 * k) / (2 * k + 1);
    }
    for (int q = 0; q < 3; ++q) {
        double s = 0.0;
        for (int k1 = kOrder / 2; k1 >= 0; --k1)
            for (int k2 = kOrder / 2 - k1; k2 >= 0; --k2)
                for (int k3 = kOrder / 2 - k1 - k2; k3 >= 0; --k3) {
                    int be[3] = {2 * k1, 2 * k2, 2 * k3};
                    const double fac = be[q] + 1.0;
                    be[q] += 1;
                    s += mx[k1] * my[k2] * mz[k3] * fac * t[tidx(be[0], be[1], be[2])];
                }
        out[q] = a * b * c / (4.0 * 3.14159265358979323846) * s;
    }
}

// Octant of S at half-integer offsets: out[3][nz][ny][nx], entry (k, j, i)
// = S((i + 1/2) a, (j + 1/2) b, (k + 1/2) c), edges scaled by the longest (L);
// the stored value is L * S (S scales like a length).
__global__ void k_sp_octant(double *__restrict__ out, int nx, int ny, int nz, double a, double b, double c,
                            double L)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((int64_t)nx * ny));
        const double X = (i + 0.5) * a, Y = (j + 0.5) * b, Z = (k + 0.5) * c;
        const double dmax = fmax(a, fmax(b, c));
        double v[3];
        if (X <= 2.5 * a && Y <= 2.5 * b && Z <= 2.5 * c) sp_near(X, Y, Z, a, b, c, v);
        else if (X * X + Y * Y + Z * Z >= (kFar * dmax) * (kFar * dmax)) sp_far(X, Y, Z, a, b, c, v);
        else sp_mid(X, Y, Z, a, b, c, v);
        for (int q = 0; q < 3; ++q) out[q * n + idx] = L * v[q];
    }
}

// Wrapped node kernel of component comp on the padded grid: index p of an
// axis with n cells holds node-minus-cell offset q = p (p <= n) or p - P
// (p >= P - n + 1), at distance (q - 1/2) d, i.e. octant index q - 1 (q >= 1)
// or -q (q <= 0, where component comp takes the sign of its own axis).
__global__ void k_sp_wrap(const double *__restrict__ oct, int comp, int nx, int ny, int nz, int Px, int Py,
                          int Pz, double *__restrict__ out)
{
    const int64_t total = (int64_t)Px * Py * Pz;
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int px = (int)(idx % Px), py = (int)((idx / Px) % Py), pz = (int)(idx / ((int64_t)Px * Py));
        const int qx = px <= nx ? px : (px >= Px - nx + 1 ? px - Px : INT_MIN);
        const int qy = py <= ny ? py : (py >= Py - ny + 1 ? py - Py : INT_MIN);
        const int qz = pz <= nz ? pz : (pz >= Pz - nz + 1 ? pz - Pz : INT_MIN);
        double v = 0.0;
        if (qx != INT_MIN && qy != INT_MIN && qz != INT_MIN) {
            const int tx = qx >= 1 ? qx - 1 : -qx, ty = qy >= 1 ? qy - 1 : -qy, tz = qz >= 1 ? qz - 1 : -qz;
            v = oct[comp * n + ((int64_t)tz * ny + ty) * nx + tx];
            const int q = comp == 0 ? qx : (comp == 1 ? qy : qz);
            if (q <= 0) v = -v;
        }
        out[idx] = v;
    }
}

// T_comp(k) = Re(i conj(Phi(k)) S^(k)), Phi(k) = exp(-pi i (kx/Px + ky/Py + kz/Pz)),
// for kx < Kx, ky <= Py/2, kz <= Pz/2; the largest |Im| goes to imag_max.
__global__ void k_sp_extract(const double2 *__restrict__ S, int comp, int Px, int Kx, int Py, int Pz, int Kxp,
                             double *__restrict__ t64, float *__restrict__ t32,
                             unsigned long long *__restrict__ imag_max)
{
    const int hy = Py / 2 + 1, hz = Pz / 2 + 1;
    const int64_t plane = (int64_t)hz * hy * Kx;
    double local = 0.0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < plane;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(idx % Kx), ky = (int)((idx / Kx) % hy), kz = (int)(idx / ((int64_t)Kx * hy));
        const double2 v = S[((int64_t)kz * Py + ky) * Kxp + kx];
        // theta / pi = kx/Px + ky/Py + kz/Pz (exact for power-of-two P, to rounding otherwise)
        const double th = (double)kx / Px + (double)ky / Py + (double)kz / Pz;
        double sn, cs;
        sincospi(th, &sn, &cs);
        // i conj(Phi) = -sin + i cos
        const double re = -sn * v.x - cs * v.y;
        const double im = cs * v.x - sn * v.y;
        t64[comp * plane + idx] = re;
        if (t32) t32[comp * plane + idx] = (float)re;
        local = fmax(local, fabs(im));
    }
    block_max_to(local, imag_max);
}

int grid_for(int64_t n, int block)
{
    const int64_t g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 65535 * 4 ? 65535 * 4 : g));
}

}  // namespace

cudaError_t tensor_octant(double *out, int nx, int ny, int nz, double dx, double dy, double dz,
                          cudaStream_t st)
{
    if (!upload_rules()) return cudaErrorUnknown;
    const double h = fmax(dx, fmax(dy, dz));
    const int64_t n = (int64_t)nx * ny * nz;
    const double a = dx / h, b = dy / h, c = dz / h;
    k_tensor_octant<<<grid_for(n, 64), 64, 0, st>>>(out, nx, ny, nz, a, b, c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the box that holds every offset closer than kFar cells (and the 2x2x2
    // touching ones): |i a| < kFar (max edge = 1 after scaling)
    const int bx = (int)std::min<double>(nx, std::max(2.0, std::floor(kFar / a) + 1));
    const int by = (int)std::min<double>(ny, std::max(2.0, std::floor(kFar / b) + 1));
    const int bz = (int)std::min<double>(nz, std::max(2.0, std::floor(kFar / c) + 1));
    const int64_t warps = (int64_t)bx * by * bz;
    k_tensor_octant_warp<<<grid_for(warps * 32, 256), 256, 0, st>>>(out, nx, ny, nz, a, b, c, bx, by, bz);
    return cudaGetLastError();
}

cudaError_t tensor_wrap(const double *oct, int comp, int nx, int ny, int nz, int Px, int Py, int Pz,
                        double *out, cudaStream_t st)
{
    const int64_t total = (int64_t)Px * Py * Pz;
    k_wrap<<<grid_for(total, 256), 256, 0, st>>>(oct, comp, nx, ny, nz, Px, Py, Pz, out);
    return cudaGetLastError();
}

cudaError_t tensor_extract(const double2 *S, int comp, int Px, int Py, int Pz, int Kxp,
                           double *nhat64, float *nhat32, unsigned long long *imag_max,
                           cudaStream_t st)
{
    const int Kx = Px / 2 + 1;
    const int64_t plane = (int64_t)(Pz / 2 + 1) * (Py / 2 + 1) * Kx;
    k_extract<<<grid_for(plane, 256), 256, 0, st>>>(S, comp, Kx, Py, Pz, Kxp, nhat64, nhat32, imag_max);
    return cudaGetLastError();
}

cudaError_t sp_octant(double *out, int nx, int ny, int nz, double dx, double dy, double dz, cudaStream_t st)
{
    if (!upload_rules()) return cudaErrorUnknown;
    const double h = fmax(dx, fmax(dy, dz));
    const int64_t n = (int64_t)nx * ny * nz;
    k_sp_octant<<<grid_for(n, 64), 64, 0, st>>>(out, nx, ny, nz, dx / h, dy / h, dz / h, h);
    return cudaGetLastError();
}

cudaError_t sp_wrap(const double *oct, int comp, int nx, int ny, int nz, int Px, int Py, int Pz, double *out,
                    cudaStream_t st)
{
    const int64_t total = (int64_t)Px * Py * Pz;
    k_sp_wrap<<<grid_for(total, 256), 256, 0, st>>>(oct, comp, nx, ny, nz, Px, Py, Pz, out);
    return cudaGetLastError();
}

cudaError_t sp_extract(const double2 *S, int comp, int Px, int Py, int Pz, int Kxp, double *t64, float *t32,
                       unsigned long long *imag_max, cudaStream_t st)
{
    const int Kx = Px / 2 + 1;
    const int64_t plane = (int64_t)(Pz / 2 + 1) * (Py / 2 + 1) * Kx;
    k_sp_extract<<<grid_for(plane, 256), 256, 0, st>>>(S, comp, Px, Kx, Py, Pz, Kxp, t64, t32, imag_max);
    return cudaGetLastError();
}

cudaError_t energy_finalize(const double *partials, int n, double factor, double *E, double *scratch, cudaStream_t st)
{
    const int nb = std::max(1, std::min(kFinalizeBlocks, (n + 127) / 128));
    k_energy_finalize<<<nb, kFinalizeThreads, 0, st>>>(partials, n, factor, E, scratch);
    return cudaGetLastError();
}

}  // namespace demag
