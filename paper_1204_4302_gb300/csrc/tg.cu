// Tensor-grid method (TG, paper Sec. 3.2) for magnetization in CP format
// (App. A): the potential at the cell centres as the block-CP sum of
// Eq. "sumpot", evaluated densely, and the field by second-order finite
// differences.
//
//   1/|r|^3 = (2/sqrt(pi)) Int tau^2 exp(-tau^2 |r|^2) dtau      (Eq. "transform")
//           ~= sum_l W_l exp(-s_l^2 |r|^2),  tau = e^t, s_l = e^{t_l},
//              W_l = (4 h / sqrt(pi)) e^{3 t_l}  (sinc / trapezoidal rule in t)
//   Phi = (1/4pi) sum_l W_l sum_p M^(p) x_1 D_1^(l,p) x_2 D_2^(l,p) x_3 D_3^(l,p)
//
// with the Gaussian matrices of Eqs. "Dmat", "gs": on the axis q, for a target
// cell centre x_i and a source cell j, the integral over the source cell of
// exp(-s^2 (x_i - x')^2) (q != p) or (x_i - x') exp(-s^2 (x_i - x')^2) (q = p).
// On a uniform axis both depend on i - j only (Toeplitz): the plan keeps the
// 2n - 1 values per (node, axis, kind), computed in FP64 in closed form (erf,
// exp). A CP magnetization M^(p) = sum_m lam_m u_m o v_m o w_m passes the mode
// products factor by factor, (u o v o w) x_1 A x_2 B x_3 C = (A u) o (B v) o (C w),
// so per call the library
//   1. transforms every factor vector by its Toeplitz matrix (k_tg_apply),
//   2. sums the K = 3 R r rank-one terms densely: Phi[k][j][i] =
//      sum_K Z[K][k] Y[K][j] X[K][i] (k_tg_dense, a tiled contraction whose
//      first operand is formed on the fly as the products Z Y),
//   3. differences Phi (k_tg_field) and forms the energy with M rebuilt from
//      its factors.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "demag.h"
#include "plan.h"

namespace demag {
namespace {

// Toeplitz tables: tab[((l * 3 + q) * 2 + kind) * tstride + (delta + n_q - 1)],
// delta = i - j in [-(n_q - 1), n_q - 1].
__device__ double tg_plain(double s, double d, int delta)
{
    // Int_{(delta - 1/2) d}^{(delta + 1/2) d} exp(-s^2 u^2) du, without the
    // cancellation of erf(a) - erf(b) when a and b have the same sign
    const double a = s * (delta + 0.5) * d, b = s * (delta - 0.5) * d;
    double diff;
    if (b >= 0.0) diff = erfc(b) - erfc(a);
    else if (a <= 0.0) diff = erfc(-a) - erfc(-b);
    else diff = erf(a) - erf(b);
    return 0.88622692545275801365 / s * diff;  // sqrt(pi)/2 / s
}

__device__ double tg_odd(double s, double d, int delta)
{
    // Int_{(delta - 1/2) d}^{(delta + 1/2) d} u exp(-s^2 u^2) du
    const double lo = (delta - 0.5) * d, hi = (delta + 0.5) * d;
    return (exp(-s * s * lo * lo) - exp(-s * s * hi * hi)) / (2.0 * s * s);
}

template <typename T>
__global__ void k_tg_tables(const double *__restrict__ snode, int R, int nx, int ny, int nz, double dx, double dy,
                            double dz, int tstride, T *__restrict__ tab)
{
    const int n[3] = {nx, ny, nz};
    const double d[3] = {dx, dy, dz};
    const int64_t total = (int64_t)R * 3 * 2 * tstride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e % tstride);
        const int64_t rest = e / tstride;
        const int kind = (int)(rest % 2), q = (int)((rest / 2) % 3), l = (int)(rest / 6);
        const int delta = t - (n[q] - 1);
        double v = 0.0;
        if (delta <= n[q] - 1) v = kind ? tg_odd(snode[l], d[q], delta) : tg_plain(snode[l], d[q], delta);
        tab[e] = (T)v;
    }
}

// Factor transform on axis q: out[v][i] = sum_j D[i - j] u[v][j] for the
// vectors v = (l, p, m) (K = 3 R r of them), D the plain table (p != q) or
// the odd one (p = q) of node l. On axis x the weight W_l lam_m^(p) / (4 pi)
// is folded in. One block per vector; the factor and the table sit in
// shared memory.
template <typename T>
__global__ void __launch_bounds__(512)
k_tg_apply(const T *__restrict__ tab, int tstride, const T *__restrict__ U, const T *__restrict__ lam,
           const double *__restrict__ wnode, int R, int r, int q, int n, T *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T *su = reinterpret_cast<T *>(smraw);   // [n]
    T *st = su + n;                          // [2n - 1]
    const int v = blockIdx.x;                // (l * 3 + p) * r + m
    const int m = v % r, p = (v / r) % 3, l = v / (3 * r);
    const T *u = U + ((int64_t)p * r + m) * n;
    const T *tb = tab + ((int64_t)(l * 3 + q) * 2 + (p == q ? 1 : 0)) * tstride;
    for (int j = threadIdx.x; j < n; j += blockDim.x) su[j] = u[j];
    for (int t = threadIdx.x; t < 2 * n - 1; t += blockDim.x) st[t] = tb[t];
    __syncthreads();
    T scale = (T)1;
    if (q == 0) scale = (T)(wnode[l] * (double)lam[p * r + m] * (1.0 / (4.0 * 3.14159265358979323846)));
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T acc = 0;
        for (int j = 0; j < n; ++j) acc += st[i - j + n - 1] * su[j];
        out[(int64_t)v * n + i] = acc * scale;
    }
}

// Dense block-CP contraction Phi[k][j][i] = sum_K Z[K][k] Y[K][j] X[K][i].
// CTA tile: 8 k x 16 j rows (128) by 128 i; K in chunks of 16; each of the
// 256 threads accumulates 8 rows x 8 columns (columns strided by 16).
constexpr int kTgBK = 16, kTgRows = 128, kTgCols = 128;

template <typename T>
__global__ void __launch_bounds__(256)
k_tg_dense(const T *__restrict__ X, const T *__restrict__ Y, const T *__restrict__ Z, int K, int nx, int ny, int nz,
           T *__restrict__ phi)
{
    __shared__ T sP[kTgBK][kTgRows];   // Z[K][k] Y[K][j] for the tile's rows
    __shared__ T sQ[kTgBK][kTgCols];   // X[K][i]
    const int i0 = blockIdx.x * kTgCols;
    const int jt = (ny + 15) / 16;
    const int j0 = (blockIdx.y % jt) * 16, k0 = (blockIdx.y / jt) * 8;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // rows ty*8 .. +8, columns tx + 16 c
    T acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0;
    for (int kb = 0; kb < K; kb += kTgBK) {
        // rows: row = kk * 16 + jj
        for (int e = threadIdx.x; e < kTgBK * kTgRows; e += 256) {
            const int kk = e / kTgRows, row = e % kTgRows;
            const int Kk = kb + kk, k = k0 + row / 16, j = j0 + row % 16;
            T v = 0;
            if (Kk < K && k < nz && j < ny) v = Z[(int64_t)Kk * nz + k] * Y[(int64_t)Kk * ny + j];
            sP[kk][row] = v;
        }
        for (int e = threadIdx.x; e < kTgBK * kTgCols; e += 256) {
            const int kk = e / kTgCols, c = e % kTgCols;
            const int Kk = kb + kk, i = i0 + c;
            sQ[kk][c] = (Kk < K && i < nx) ? X[(int64_t)Kk * nx + i] : (T)0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kTgBK; ++kk) {
            T a[8], b[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) a[t] = sP[kk][ty * 8 + t];
#pragma unroll
            for (int t = 0; t < 8; ++t) b[t] = sQ[kk][tx + 16 * t];
#pragma unroll
            for (int s = 0; s < 8; ++s)
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[s][t] += a[s] * b[t];
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int row = ty * 8 + s, k = k0 + row / 16, j = j0 + row % 16;
        if (k >= nz || j >= ny) continue;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int i = i0 + tx + 16 * t;
            if (i < nx) phi[((int64_t)k * ny + j) * nx + i] = acc[s][t];
        }
    }
}

// Second-order differences of the cell-centre potential (central inside,
// one-sided at the ends; n >= 3 per axis), H = -grad Phi, and optionally the
// energy partials sum over the block of M . H with M rebuilt from its factors.
template <typename T>
__global__ void __launch_bounds__(256)
k_tg_field(const T *__restrict__ phi, int nx, int ny, int nz, T hx, T hy, T hz, T *__restrict__ H,
           const T *__restrict__ lam, const T *__restrict__ Ux, const T *__restrict__ Uy, const T *__restrict__ Uz, int r,
           double *__restrict__ partials)
{
    const int64_t ncell = (int64_t)nx * ny * nz;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (c < ncell) {
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((int64_t)nx * ny));
        const int64_t sy = nx, sz = (int64_t)nx * ny;
        auto deriv = [&](int idx, int n, int64_t st, T h) -> T {
            const T *f = phi + c;
            if (idx == 0) return ((T)-3 * f[0] + (T)4 * f[st] - f[2 * st]) / ((T)2 * h);
            if (idx == n - 1) return ((T)3 * f[0] - (T)4 * f[-st] + f[-2 * st]) / ((T)2 * h);
            return (f[st] - f[-st]) / ((T)2 * h);
        };
        const T h0 = -deriv(i, nx, 1, hx), h1 = -deriv(j, ny, sy, hy), h2 = -deriv(k, nz, sz, hz);
        if (H) {
            H[c] = h0;
            H[ncell + c] = h1;
            H[2 * ncell + c] = h2;
        }
        if (partials) {
            const T hv[3] = {h0, h1, h2};
            for (int p = 0; p < 3; ++p) {
                T mp = 0;
                for (int m = 0; m < r; ++m)
                    mp += lam[p * r + m] * Ux[((int64_t)p * r + m) * nx + i] * Uy[((int64_t)p * r + m) * ny + j] *
                          Uz[((int64_t)p * r + m) * nz + k];
                acc += (double)(mp * hv[p]);
            }
        }
    }
    if (partials) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __shared__ double ws[8];
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int w = 0; w < 8; ++w) t += ws[w];
            partials[blockIdx.x] = t;
        }
    }
}

}  // namespace
}  // namespace demag

// ---------------------------------------------------------------- the plan
struct demag_tg_plan {
    int nx, ny, nz, rank, R;
    double dx, dy, dz;
    demag_prec prec;
    int device;
    int tstride;            // 2 max(n) - 1
    double *snode, *wnode;  // sinc nodes / weights (device)
    void *tab;              // Toeplitz tables [R][3][2][tstride]
    void *X, *Y, *Z;        // transformed factors [K][n_q]
    void *phi;              // cell-centre potential [nz][ny][nx]
    double *partials;
    int npartials;
    size_t device_bytes;
    long launches;
};

namespace {

demag_status tg_fail(demag_status s, const std::string &m)
{
    demag::set_last_error(m);
    return s;
}

template <typename T>
demag_status tg_run(demag_tg_plan *p, const void *lam, const void *Ux, const void *Uy, const void *Uz, void *H,
                    double *E_dev, bool want_field, void *phi_out, cudaStream_t st)
{
    using namespace demag;
    const int K = 3 * p->R * p->rank;
    const int n[3] = {p->nx, p->ny, p->nz};
    const void *U[3] = {Ux, Uy, Uz};
    void *out[3] = {p->X, p->Y, p->Z};
    for (int q = 0; q < 3; ++q) {
        const size_t sm = (size_t)(3 * n[q]) * sizeof(T);
        k_tg_apply<T><<<K, n[q] >= 512 ? 512 : ((n[q] + 31) / 32) * 32, sm, st>>>(
            static_cast<const T *>(p->tab), p->tstride, static_cast<const T *>(U[q]), static_cast<const T *>(lam),
            p->wnode, p->R, p->rank, q, n[q], static_cast<T *>(out[q]));
        p->launches++;
    }
    T *phi = phi_out ? static_cast<T *>(phi_out) : static_cast<T *>(p->phi);
    const dim3 grid((p->nx + kTgCols - 1) / kTgCols, ((p->ny + 15) / 16) * ((p->nz + 7) / 8));
    k_tg_dense<T><<<grid, 256, 0, st>>>(static_cast<const T *>(p->X), static_cast<const T *>(p->Y),
                                        static_cast<const T *>(p->Z), K, p->nx, p->ny, p->nz, phi);
    p->launches++;
    if (want_field || E_dev) {
        const int64_t ncell = (int64_t)p->nx * p->ny * p->nz;
        const int blocks = (int)((ncell + 255) / 256);
        k_tg_field<T><<<blocks, 256, 0, st>>>(phi, p->nx, p->ny, p->nz, (T)p->dx, (T)p->dy, (T)p->dz,
                                              static_cast<T *>(H), static_cast<const T *>(lam),
                                              static_cast<const T *>(Ux), static_cast<const T *>(Uy),
                                              static_cast<const T *>(Uz), p->rank, E_dev ? p->partials : nullptr);
        p->launches++;
        if (E_dev) {
            const double V = p->dx * p->dy * p->dz;
            cudaError_t e = energy_finalize(p->partials, blocks, -0.5 * 4e-7 * 3.14159265358979323846 * V, E_dev, st);
            if (e != cudaSuccess) return tg_fail(DEMAG_ERR_CUDA, std::string("TG energy: ") + cudaGetErrorString(e));
            p->launches++;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tg_fail(DEMAG_ERR_CUDA, std::string("TG pass: ") + cudaGetErrorString(e));
    return DEMAG_OK;
}

demag_status tg_check_ptr(const demag_tg_plan *p, const void *ptr, const char *name)
{
    if (!ptr) return tg_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is NULL");
    if (((uintptr_t)ptr & 15u) != 0) return tg_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return tg_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return tg_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not device memory");
    if (a.type == cudaMemoryTypeDevice && a.device != p->device)
        return tg_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " lives on another device");
    return DEMAG_OK;
}

struct TgGuard {
    int prev = -1;
    bool ok = true;
    explicit TgGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~TgGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

demag_status tg_job(demag_tg_plan *p, const void *lam, const void *Ux, const void *Uy, const void *Uz, void *H,
                    double *E_dev, void *phi, void *stream)
{
    if (!p) return tg_fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    TgGuard g(p->device);
    if (!g.ok) return tg_fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    demag_status s;
    if ((s = tg_check_ptr(p, lam, "lam")) != DEMAG_OK || (s = tg_check_ptr(p, Ux, "Ux")) != DEMAG_OK ||
        (s = tg_check_ptr(p, Uy, "Uy")) != DEMAG_OK || (s = tg_check_ptr(p, Uz, "Uz")) != DEMAG_OK)
        return s;
    if (H && (s = tg_check_ptr(p, H, "H")) != DEMAG_OK) return s;
    if (phi && (s = tg_check_ptr(p, phi, "phi")) != DEMAG_OK) return s;
    {
        // outputs must not overlap the factors (the kernels read them throughout)
        const size_t es = p->prec == DEMAG_F32 ? 4 : 8, r = (size_t)p->rank;
        const size_t ncell = (size_t)p->nx * p->ny * p->nz;
        const void *in[4] = {lam, Ux, Uy, Uz};
        const size_t inb[4] = {3 * r * es, 3 * r * p->nx * es, 3 * r * p->ny * es, 3 * r * p->nz * es};
        auto hits = [&](const void *o, size_t ob) {
            for (int q = 0; q < 4; ++q) {
                const uintptr_t a = (uintptr_t)o, b = (uintptr_t)in[q];
                if (a < b + inb[q] && b < a + ob) return true;
            }
            return false;
        };
        if (H && hits(H, 3 * ncell * es)) return tg_fail(DEMAG_ERR_INVALID_ARG, "H overlaps a factor");
        if (phi && hits(phi, ncell * es)) return tg_fail(DEMAG_ERR_INVALID_ARG, "phi overlaps a factor");
    }
    if (E_dev) {
        if (((uintptr_t)E_dev & 7u) != 0) return tg_fail(DEMAG_ERR_INVALID_ARG, "E_dev is not 8-byte aligned");
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, E_dev) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return tg_fail(DEMAG_ERR_INVALID_ARG, "E_dev is not device memory");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prec == DEMAG_F32) return tg_run<float>(p, lam, Ux, Uy, Uz, H, E_dev, H != nullptr, phi, st);
    return tg_run<double>(p, lam, Ux, Uy, Uz, H, E_dev, H != nullptr, phi, st);
}

}  // namespace

extern "C" {

void demag_tg_plan_destroy(demag_tg_plan_t p)
{
    if (!p) return;
    TgGuard g(p->device);
    cudaFree(p->snode);
    cudaFree(p->wnode);
    cudaFree(p->tab);
    cudaFree(p->X);
    cudaFree(p->Y);
    cudaFree(p->Z);
    cudaFree(p->phi);
    cudaFree(p->partials);
    delete p;
}

demag_status demag_tg_plan_create(int nx, int ny, int nz, double dx, double dy, double dz, int rank, demag_prec prec,
                                  demag_tg_plan_t *out)
{
    if (!out) return tg_fail(DEMAG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 3 || ny < 3 || nz < 3)
        return tg_fail(DEMAG_ERR_INVALID_ARG, "the second-order differences need at least 3 cells per axis");
    if (nx > 512 || ny > 512 || nz > 512) return tg_fail(DEMAG_ERR_UNSUPPORTED, "TG grids are built up to 512 per axis");
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz))
        return tg_fail(DEMAG_ERR_INVALID_ARG, "cell edges must be positive and finite");
    if (rank < 1 || rank > 64) return tg_fail(DEMAG_ERR_INVALID_ARG, "CP rank must be in 1..64");
    if (prec != DEMAG_F32 && prec != DEMAG_F64) return tg_fail(DEMAG_ERR_INVALID_ARG, "unknown precision");
    demag_tg_plan *p = new demag_tg_plan;
    memset(p, 0, sizeof(*p));
    p->nx = nx; p->ny = ny; p->nz = nz;
    p->dx = dx; p->dy = dy; p->dz = dz;
    p->rank = rank;
    p->prec = prec;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return tg_fail(DEMAG_ERR_CUDA, "no CUDA device");
    }
    // sinc rule in t (tau = e^t) covering |r| from half the shortest edge to
    // twice the body diagonal; step and tail by precision (rule error ~1e-15
    // for FP64 plans, ~2e-9 for FP32 plans)
    const double a_min = 0.5 * fmin(dx, fmin(dy, dz));
    const double a_max = 2.0 * sqrt((nx * dx) * (nx * dx) + (ny * dy) * (ny * dy) + (nz * dz) * (nz * dz));
    const double h = prec == DEMAG_F64 ? 0.1 : 0.2, tail = prec == DEMAG_F64 ? 14.0 : 10.0;
    const double t0 = -log(a_max) - tail, t1 = log(6.0 / a_min) + 1.0;
    const int R = (int)ceil((t1 - t0) / h) + 1;
    std::vector<double> s(R), w(R);
    for (int l = 0; l < R; ++l) {
        const double t = t0 + h * l;
        s[l] = exp(t);
        w[l] = 4.0 * h / sqrt(3.14159265358979323846) * exp(3.0 * t);
    }
    p->R = R;
    const int nmax = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
    p->tstride = 2 * nmax - 1;
    const size_t es = prec == DEMAG_F32 ? 4 : 8;
    const int K = 3 * R * rank;
    const int64_t ncell = (int64_t)nx * ny * nz;
    p->npartials = (int)((ncell + 255) / 256);
    auto cleanup = [&](cudaError_t e, const char *what) {
        demag_tg_plan_destroy(p);
        return tg_fail(e == cudaErrorMemoryAllocation ? DEMAG_ERR_OOM : DEMAG_ERR_CUDA,
                       std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    const size_t tab_bytes = (size_t)R * 6 * p->tstride * es;
    if ((e = cudaMalloc(&p->snode, sizeof(double) * R)) != cudaSuccess) return cleanup(e, "cudaMalloc sinc nodes");
    if ((e = cudaMalloc(&p->wnode, sizeof(double) * R)) != cudaSuccess) return cleanup(e, "cudaMalloc sinc weights");
    if ((e = cudaMalloc(&p->tab, tab_bytes)) != cudaSuccess) return cleanup(e, "cudaMalloc tables");
    if ((e = cudaMalloc(&p->X, (size_t)K * nx * es)) != cudaSuccess) return cleanup(e, "cudaMalloc factors");
    if ((e = cudaMalloc(&p->Y, (size_t)K * ny * es)) != cudaSuccess) return cleanup(e, "cudaMalloc factors");
    if ((e = cudaMalloc(&p->Z, (size_t)K * nz * es)) != cudaSuccess) return cleanup(e, "cudaMalloc factors");
    if ((e = cudaMalloc(&p->phi, (size_t)ncell * es)) != cudaSuccess) return cleanup(e, "cudaMalloc potential");
    if ((e = cudaMalloc(&p->partials, sizeof(double) * p->npartials)) != cudaSuccess) return cleanup(e, "cudaMalloc partials");
    if ((e = cudaMemcpy(p->snode, s.data(), sizeof(double) * R, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(e, "upload sinc nodes");
    if ((e = cudaMemcpy(p->wnode, w.data(), sizeof(double) * R, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(e, "upload sinc weights");
    const int64_t total = (int64_t)R * 6 * p->tstride;
    const int blocks = (int)((total + 255) / 256 < 65535 * 4 ? (total + 255) / 256 : 65535 * 4);
    if (prec == DEMAG_F32)
        demag::k_tg_tables<float><<<blocks, 256>>>(p->snode, R, nx, ny, nz, dx, dy, dz, p->tstride,
                                                   static_cast<float *>(p->tab));
    else
        demag::k_tg_tables<double><<<blocks, 256>>>(p->snode, R, nx, ny, nz, dx, dy, dz, p->tstride,
                                                    static_cast<double *>(p->tab));
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(e, "TG tables");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup(e, "TG tables");
    p->launches = 1;
    p->device_bytes = 2 * sizeof(double) * R + tab_bytes + (size_t)K * (nx + ny + nz) * es + (size_t)ncell * es +
                      sizeof(double) * p->npartials;
    *out = p;
    demag::set_last_error("");
    return DEMAG_OK;
}

demag_status demag_tg_field_cp(demag_tg_plan_t p, const void *lam, const void *Ux, const void *Uy, const void *Uz,
                               void *H, double *E_dev, void *stream)
{
    if (!H && !E_dev) return tg_fail(DEMAG_ERR_INVALID_ARG, "nothing to compute (no field, no energy)");
    return tg_job(p, lam, Ux, Uy, Uz, H, E_dev, nullptr, stream);
}

demag_status demag_tg_potential_cp(demag_tg_plan_t p, const void *lam, const void *Ux, const void *Uy, const void *Uz,
                                   void *phi, void *stream)
{
    if (!phi) return tg_fail(DEMAG_ERR_INVALID_ARG, "phi is NULL");
    return tg_job(p, lam, Ux, Uy, Uz, nullptr, nullptr, phi, stream);
}

demag_status demag_tg_plan_info(demag_tg_plan_t p, int *sinc_terms, size_t *device_bytes, long *launches)
{
    if (!p) return tg_fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (sinc_terms) *sinc_terms = p->R;
    if (device_bytes) *device_bytes = p->device_bytes;
    if (launches) *launches = p->launches;
    return DEMAG_OK;
}

}  // extern "C"
