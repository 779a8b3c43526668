// FP64 setup of the demagnetization tensor (paper Sec. 3.1, the tensor N of
// Eq. "demag"; Sec. 4: computed once per geometry; Sec. 5.1: homogeneously
// magnetized cells with the field averaged over each cell).
//
// N_ij(R) = (1/V) Int_cell(R) Int_cell(0) G_ij(r - r') dr' dr,
// G_ij(r) = -(1/4pi) d_i d_j (1/|r|),  positive definite at R = 0 (trace 1).
//
// One thread per offset R = (i dx, j dy, k dz), 0 <= i < nx etc. (the other
// octants follow by parity). Three regimes, all in FP64 with lengths scaled
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

__device__ void near_closed(double X, double Y, double Z, double a, double b, double c, double *out)
{
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int p = -1; p <= 1; ++p) {
        const double wp = p == 0 ? 2.0 : -1.0, x = X + p * a;
        for (int q = -1; q <= 1; ++q) {
            const double wq = q == 0 ? 2.0 : -1.0, y = Y + q * b;
            for (int t = -1; t <= 1; ++t) {
                const double wt = wp * wq * (t == 0 ? 2.0 : -1.0), z = Z + t * c;
                s[0] += wt * newell_f(x, y, z);
                s[1] += wt * newell_f(y, x, z);
                s[2] += wt * newell_f(z, y, x);
                s[3] += wt * newell_g(x, y, z);
                s[4] += wt * newell_g(x, z, y);
                s[5] += wt * newell_g(y, z, x);
            }
        }
    }
    const double k = 1.0 / (4.0 * 3.14159265358979323846 * a * b * c);
    for (int i = 0; i < 6; ++i) out[i] = s[i] * k;
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

__device__ void mid_quadrature(double X, double Y, double Z, double a, double b, double c, double *out)
{
    const double gx = fmax(0.0, fabs(X) - a), gy = fmax(0.0, fabs(Y) - b), gz = fmax(0.0, fabs(Z) - c);
    const double gap = sqrt(gx * gx + gy * gy + gz * gz);
    const int nx = half_axis_nodes(gap, a), ny = half_axis_nodes(gap, b), nz = half_axis_nodes(gap, c);
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 2 * nz; ++k) {
        double uz, wz;
        tent_node(nz, k, c, uz, wz);
        const double rz = Z + uz;
        for (int j = 0; j < 2 * ny; ++j) {
            double uy, wy;
            tent_node(ny, j, b, uy, wy);
            const double ry = Y + uy;
            double p[6] = {0, 0, 0, 0, 0, 0};
            for (int i = 0; i < 2 * nx; ++i) {
                double ux, wx;
                tent_node(nx, i, a, ux, wx);
                const double rx = X + ux;
                const double r2 = rx * rx + ry * ry + rz * rz;
                const double ir = rsqrt(r2);
                const double ir2 = ir * ir;
                const double f = wx * ir2 * ir2 * ir;  // w / r^5
                p[0] += f * (3.0 * rx * rx - r2);
                p[1] += f * (3.0 * ry * ry - r2);
                p[2] += f * (3.0 * rz * rz - r2);
                p[3] += f * 3.0 * rx * ry;
                p[4] += f * 3.0 * rx * rz;
                p[5] += f * 3.0 * ry * rz;
            }
            const double w = wy * wz;
            for (int q = 0; q < 6; ++q) s[q] += w * p[q];
        }
    }
    const double k = -a * b * c / (4.0 * 3.14159265358979323846);
    for (int q = 0; q < 6; ++q) out[q] = k * s[q];
}

// Index of the multi-index (b1, b2, n - b1 - b2) among all of order <= n.
__device__ __forceinline__ int tidx(int b1, int b2, int b3)
{
    const int n = b1 + b2 + b3;
    return n * (n + 1) * (n + 2) / 6 + b1 * (n + 1) - b1 * (b1 - 1) / 2 + b2;
}

__device__ void far_multipole(double X, double Y, double Z, double a, double b, double c, double *out)
{
    // Taylor coefficients t_beta = (1/beta!) d^beta_y 1/|R - y| at y = 0, which
    // equal (1/beta!) d^beta (1/|R|) for even |beta| (the only ones used).
    double t[kNumTaylor];
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

__global__ void k_tensor_octant(double *__restrict__ out, int nx, int ny, int nz, double a, double b,
                                double c)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((int64_t)nx * ny));
        const double X = i * a, Y = j * b, Z = k * c;
        const double dmax = fmax(a, fmax(b, c));
        double v[6];
        if (i <= 1 && j <= 1 && k <= 1) near_closed(X, Y, Z, a, b, c, v);
        else if (X * X + Y * Y + Z * Z >= (kFar * dmax) * (kFar * dmax)) far_multipole(X, Y, Z, a, b, c, v);
        else mid_quadrature(X, Y, Z, a, b, c, v);
        for (int q = 0; q < 6; ++q) out[q * n + idx] = v[q];
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
    // non-negative doubles order like their bit patterns
    atomicMax(imag_max, (unsigned long long)__double_as_longlong(local));
}

__global__ void k_energy_finalize(const double *__restrict__ partials, int n, double factor,
                                  double *__restrict__ E)
{
    // one block; Neumaier-compensated sums per thread, then a tree of pairs
    __shared__ double ss[256], sc[256];
    double s = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = partials[i];
        const double t = s + v;
        c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const double a = ss[threadIdx.x], b = ss[threadIdx.x + w];
            const double t = a + b;
            const double e = fabs(a) >= fabs(b) ? (a - t) + b : (b - t) + a;
            ss[threadIdx.x] = t;
            sc[threadIdx.x] += sc[threadIdx.x + w] + e;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = factor * (ss[0] + sc[0]);
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
    k_tensor_octant<<<grid_for(n, 64), 64, 0, st>>>(out, nx, ny, nz, dx / h, dy / h, dz / h);
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

cudaError_t energy_finalize(const double *partials, int n, double factor, double *E, cudaStream_t st)
{
    k_energy_finalize<<<1, 256, 0, st>>>(partials, n, factor, E);
    return cudaGetLastError();
}

}  // namespace demag
