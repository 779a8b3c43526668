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
//      sum_K Z[K][k] Y[K][j] X[K][i], a GEMM whose first operand is formed on
//      the fly as the products Z Y: on the tensor cores for FP32 plans
//      (k_tg_mma in tg_mma.cuh, three TF32 products per term), as a tiled
//      FP32 / FP64 CUDA-core contraction otherwise (k_tg_dense),
//   3. differences Phi (k_tg_field) and forms the energy with M rebuilt from
//      its factors.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include <algorithm>
#include <type_traits>

#include "demag.h"
#include "launch_util.cuh"
#include "plan.h"
#include "tg_mma.cuh"

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
// is folded in. One block per (l, p): its r vectors share the table, so a
// thread (output i) takes each table entry once for VC vectors at a time
// (VC = 8, 4, 2 or 1 by the rank), whose factors sit in shared memory as
// [j][VC] (read two at a time).
template <typename T, int VC>
__global__ void __launch_bounds__(512)
k_tg_apply(const T *__restrict__ tab, int tstride, const T *__restrict__ U, const T *__restrict__ lam,
           const double *__restrict__ wnode, int R, int r, int q, int n, T *__restrict__ out)
{
    using V2 = typename CplxOf<T>::type;  // two values (float2 / double2)
    extern __shared__ __align__(16) unsigned char smraw[];
    T *su = reinterpret_cast<T *>(smraw);   // [n][VC]
    T *st = su + (size_t)n * VC;             // [2n - 1]
    const int lp = blockIdx.x;               // l * 3 + p
    const int p = lp % 3, l = lp / 3;
    const T *tb = tab + ((int64_t)(l * 3 + q) * 2 + (p == q ? 1 : 0)) * tstride;
    for (int t = threadIdx.x; t < 2 * n - 1; t += blockDim.x) st[t] = tb[t];
    for (int m0 = 0; m0 < r; m0 += VC) {
        const int mc = min(VC, r - m0);
        __syncthreads();  // the previous chunk's factors are read
        for (int e = threadIdx.x; e < n * VC; e += blockDim.x) {
            const int j = e / VC, mm = e % VC;
            su[e] = mm < mc ? U[((int64_t)p * r + m0 + mm) * n + j] : (T)0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            T acc[VC];
#pragma unroll
            for (int mm = 0; mm < VC; ++mm) acc[mm] = 0;
            for (int j = 0; j < n; ++j) {
                const T d = st[i - j + n - 1];
                if constexpr (VC == 1) {
                    acc[0] += d * su[j];
                } else {
                    const V2 *f = reinterpret_cast<const V2 *>(su + (size_t)j * VC);
#pragma unroll
                    for (int h = 0; h < VC / 2; ++h) {
                        const V2 w = f[h];
                        acc[2 * h] += d * w.x;
                        acc[2 * h + 1] += d * w.y;
                    }
                }
            }
            for (int mm = 0; mm < mc; ++mm) {
                const int m = m0 + mm, v = lp * r + m;
                T scale = (T)1;
                if (q == 0) scale = (T)(wnode[l] * (double)lam[p * r + m] * (1.0 / (4.0 * 3.14159265358979323846)));
                out[(int64_t)v * n + i] = acc[mm] * scale;
            }
        }
    }
}

template <typename T>
void tg_apply(const T *tab, int tstride, const T *U, const T *lam, const double *wnode, int R, int r, int q, int n,
              T *out, cudaStream_t st)
{
    const int threads = n >= 512 ? 512 : ((n + 31) / 32) * 32;
    const int vc = r >= 8 ? 8 : (r >= 4 ? 4 : (r >= 2 ? 2 : 1));
    const size_t sm = (size_t)(vc * n + 2 * n) * sizeof(T);
    switch (vc) {
    case 8: k_tg_apply<T, 8><<<3 * R, threads, sm, st>>>(tab, tstride, U, lam, wnode, R, r, q, n, out); break;
    case 4: k_tg_apply<T, 4><<<3 * R, threads, sm, st>>>(tab, tstride, U, lam, wnode, R, r, q, n, out); break;
    case 2: k_tg_apply<T, 2><<<3 * R, threads, sm, st>>>(tab, tstride, U, lam, wnode, R, r, q, n, out); break;
    default: k_tg_apply<T, 1><<<3 * R, threads, sm, st>>>(tab, tstride, U, lam, wnode, R, r, q, n, out); break;
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
constexpr int kTgFieldThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kTgFieldThreads)
k_tg_field(const T *__restrict__ phi, int nx, int ny, int nz, T hx, T hy, T hz, T *__restrict__ H,
           const T *__restrict__ lam, const T *__restrict__ Ux, const T *__restrict__ Uy, const T *__restrict__ Uz, int r,
           double *__restrict__ partials, const T *__restrict__ G = nullptr, int r2 = 0, int r3 = 0)
{
    // One block per x row (j, k) at a time (grid-stride over rows), threads
    // over i. The energy's M^(p)[k][j][i] = sum_m w[p r + m] Ux[p r + m][i]
    // takes the row-constant part from shared memory (CP: w = lam Uy[j]
    // Uz[k]; Tucker, G given: w[p r + a] = sum_{b,c} G B[b][j] C[c][k] with
    // r = r1), so a cell costs 3 r coalesced factor loads and no index
    // divisions; the energy leaves one FP64 partial per block.
    __shared__ T w[3 * 64];
    __shared__ double ws[kTgFieldThreads / 32];
    const int64_t sy = nx, sz = (int64_t)nx * ny, ncell = sz * nz;
    const T ix = (T)0.5 / hx, iy = (T)0.5 / hy, iz = (T)0.5 / hz;
    const int nrows = ny * nz;
    T acc = 0;
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int j = row % ny, k = row / ny;
        if (partials) {
            __syncthreads();  // the previous row's w is read
            if (G) {
                // Tucker: w[p r + a] = sum_{b,c} G^(p)[c][b][a] B^(p)[b][j] C^(p)[c][k]
                for (int v = threadIdx.x; v < 3 * r; v += blockDim.x) {
                    const int p = v / r, a = v % r;
                    const T *Gp = G + (int64_t)p * r3 * r2 * r;
                    T acc = 0;
                    for (int c = 0; c < r3; ++c) {
                        T t = 0;
                        for (int b = 0; b < r2; ++b) t += Gp[(c * r2 + b) * r + a] * Uy[(p * r2 + b) * ny + j];
                        acc += t * Uz[(p * r3 + c) * nz + k];
                    }
                    w[v] = acc;
                }
            } else {
                for (int v = threadIdx.x; v < 3 * r; v += blockDim.x) w[v] = lam[v] * Uy[v * ny + j] * Uz[v * nz + k];
            }
            __syncthreads();
        }
        const T *prow = phi + (int64_t)row * nx;
        // y and z differences: central inside, one-sided at the ends
        const int64_t jm = j == 0 ? 0 : (j == ny - 1 ? -2 * sy : -sy), jp = j == 0 ? 2 * sy : (j == ny - 1 ? 0 : sy);
        const int64_t km = k == 0 ? 0 : (k == nz - 1 ? -2 * sz : -sz), kp = k == 0 ? 2 * sz : (k == nz - 1 ? 0 : sz);
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const T *f = prow + i;
            T d0, d1, d2;
            if (i == 0) d0 = ((T)-3 * f[0] + (T)4 * f[1] - f[2]) * ix;
            else if (i == nx - 1) d0 = ((T)3 * f[0] - (T)4 * f[-1] + f[-2]) * ix;
            else d0 = (f[1] - f[-1]) * ix;
            if (j == 0) d1 = ((T)-3 * f[0] + (T)4 * f[sy] - f[jp]) * iy;
            else if (j == ny - 1) d1 = ((T)3 * f[0] - (T)4 * f[-sy] + f[jm]) * iy;
            else d1 = (f[jp] - f[jm]) * iy;
            if (k == 0) d2 = ((T)-3 * f[0] + (T)4 * f[sz] - f[kp]) * iz;
            else if (k == nz - 1) d2 = ((T)3 * f[0] - (T)4 * f[-sz] + f[km]) * iz;
            else d2 = (f[kp] - f[km]) * iz;
            const int64_t c = (int64_t)row * nx + i;
            if (H) {
                H[c] = -d0;
                H[ncell + c] = -d1;
                H[2 * ncell + c] = -d2;
            }
            if (partials) {
                const T hv[3] = {-d0, -d1, -d2};
                for (int p = 0; p < 3; ++p) {
                    T mp = 0;
                    for (int m = 0; m < r; ++m) mp += w[p * r + m] * Ux[(p * r + m) * nx + i];
                    acc += mp * hv[p];
                }
            }
        }
    }
    if (partials) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = (double)acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int q = 0; q < kTgFieldThreads / 32; ++q) t += ws[q];
            partials[blockIdx.x] = t;
        }
    }
}

// Tucker input: the contraction's first operand Q[g][K], g = k ny + j,
// K = (l 3 + p) r1 + a, of the potential's block sum
//   Phi[k][j][i] = sum_{l,p,a} Q[g][(l,p,a)] X[(l,p,a)][i],
//   Q = sum_{b,c} G^(p)[c][b][a] Y[(l,p,b)][j] Z[(l,p,c)][k]
// (the core times the transformed y and z factors). One block per ((l,p), k):
// U[a][b] = sum_c G[c][b][a] Z[(l,p,c)][k] in shared memory, then
// Q = sum_b U[a][b] Y[(l,p,b)][j] over the block's threads. KMAJOR: Q stored
// [g][Kp] (rows of the tensor-core operand), else [K][g] (the CUDA-core form).
template <typename T, bool KMAJOR>
__global__ void __launch_bounds__(256)
k_tg_tucker_q(const T *__restrict__ G, const T *__restrict__ Y, const T *__restrict__ Z, int r1, int r2, int r3,
              int ny, int nz, int Kp, int64_t M, T *__restrict__ Q)
{
    __shared__ T U[16 * 16];
    const int lp = blockIdx.x, k = blockIdx.y;  // lp = l 3 + p
    const int p = lp % 3;
    const T *Gp = G + (int64_t)p * r3 * r2 * r1;
    for (int e = threadIdx.x; e < r1 * r2; e += blockDim.x) {
        const int a = e / r2, b = e % r2;
        T acc = 0;
        for (int c = 0; c < r3; ++c) acc += Gp[(c * r2 + b) * r1 + a] * Z[((int64_t)lp * r3 + c) * nz + k];
        U[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ny * r1; e += blockDim.x) {
        const int j = KMAJOR ? e / r1 : e % ny, a = KMAJOR ? e % r1 : e / ny;
        T acc = 0;
        for (int b = 0; b < r2; ++b) acc += U[a * r2 + b] * Y[((int64_t)lp * r2 + b) * ny + j];
        const int64_t g = (int64_t)k * ny + j, K = (int64_t)lp * r1 + a;
        if (KMAJOR) Q[g * Kp + K] = acc;
        else Q[K * M + g] = acc;
    }
    if (KMAJOR && lp == (int)gridDim.x - 1) {
        // the padding terms K .. Kp - 1 of this k's rows are zero (the K-major
        // and term-major forms share the buffer)
        const int K = (int)gridDim.x * r1, pad = Kp - K;
        for (int e = threadIdx.x; e < ny * pad; e += blockDim.x)
            Q[((int64_t)k * ny + e / pad) * Kp + K + e % pad] = (T)0;
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
    // tensor-core contraction (FP32 plans): transposed factors, the B operand
    // in stage order, its tiling, the timeout word
    int contraction;        // 0 CUDA cores, 1 tensor cores
    // Tucker input (ranks r1, r2, r3; rank == r1): the first operand of the
    // contraction, Q, and a row of ones (the unit z operand / CP weights)
    bool tucker;
    int r1, r2, r3;
    void *Q, *ones;
    int Kp, BN, ntn, nkc;
    float *Yt, *Zt, *Bsw;
    int *err;
    // per-stage event timing (factor transforms, operand preparation,
    // contraction, differences and energy)
    bool timing;
    cudaEvent_t ev[5];
    double stage_ms[4];
    long timed_calls;
};

namespace {

demag_status tg_fail(demag_status s, const std::string &m)
{
    demag::set_last_error(m);
    return s;
}

// The FP32 contraction on the tensor cores: operand preparation (B in stage
// order with its TF32 split, Y and Z transposed to K-contiguous rows), then
// the persistent tcgen05 kernel.
// Tucker plans pass their operand Q [nz ny][Kp] as the y factor of ny_eff =
// nz ny rows and a row of ones as the z factor (nz_eff = 1): A = Q * 1.
cudaError_t tg_contract_mma(demag_tg_plan *p, float *phi, cudaStream_t st, cudaEvent_t between)
{
    using namespace demag;
    const int K = 3 * p->R * p->r1;
    const int64_t nb = (int64_t)p->ntn * p->nkc * p->BN * tgm::kBK;
    const int bb = (int)std::min<int64_t>((nb + 255) / 256, 4096);
    tgm::k_tg_prep_b<<<bb, 256, 0, st>>>(static_cast<const float *>(p->X), K, p->nx, p->BN, p->ntn, p->nkc, p->Bsw);
    p->launches++;
    const float *Yt = p->Yt, *Zt = p->Zt;
    int ny = p->ny, nz = p->nz;
    if (p->tucker) {
        Yt = static_cast<const float *>(p->Q);
        Zt = static_cast<const float *>(p->ones);
        ny = p->ny * p->nz;
        nz = 1;
    } else {
        const int by = (int)std::min<int64_t>(((int64_t)p->ny * p->Kp + 255) / 256, 4096);
        tgm::k_tg_transpose<<<by, 256, 0, st>>>(static_cast<const float *>(p->Y), K, p->ny, p->Kp, p->Yt);
        const int bz = (int)std::min<int64_t>(((int64_t)p->nz * p->Kp + 255) / 256, 4096);
        tgm::k_tg_transpose<<<bz, 256, 0, st>>>(static_cast<const float *>(p->Z), K, p->nz, p->Kp, p->Zt);
        p->launches += 2;
    }
    if (between) cudaEventRecord(between, st);
    const size_t sm = tgm::smem_bytes(p->BN);
    cudaError_t e = allow_smem<tgm::k_tg_mma>(sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tgm::k_tg_mma, tgm::kThreads, sm)) != cudaSuccess)
        return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int64_t M = (int64_t)p->nz * p->ny;
    const int ntiles = (int)((M + tgm::kBM - 1) / tgm::kBM) * p->ntn;
    const int cap = sm_count() * occ;
    const int grid = ntiles < cap ? ntiles : cap;
    tgm::k_tg_mma<<<grid, tgm::kThreads, sm, st>>>(Yt, Zt, p->Bsw, p->Kp, p->nx, ny, nz, p->BN, p->ntn, ntiles, phi,
                                                   p->err);
    p->launches++;
    return cudaGetLastError();
}

// One TG call. CP plans: lam [3][r], factors [3][r][n]. Tucker plans: G
// [3][r3][r2][r1] in place of lam, factors [3][r_q][n_q].
template <typename T>
demag_status tg_run(demag_tg_plan *p, const void *lam, const void *Ux, const void *Uy, const void *Uz, void *H,
                    double *E_dev, bool want_field, void *phi_out, cudaStream_t st)
{
    using namespace demag;
    const int K = 3 * p->R * p->r1;
    const int n[3] = {p->nx, p->ny, p->nz}, rq[3] = {p->r1, p->r2, p->r3};
    const void *U[3] = {Ux, Uy, Uz};
    void *out[3] = {p->X, p->Y, p->Z};
    const T *G = p->tucker ? static_cast<const T *>(lam) : nullptr;
    const T *weights = p->tucker ? static_cast<const T *>(p->ones) : static_cast<const T *>(lam);
    if (p->timing) cudaEventRecord(p->ev[0], st);
    for (int q = 0; q < 3; ++q) {
        tg_apply<T>(static_cast<const T *>(p->tab), p->tstride, static_cast<const T *>(U[q]), weights, p->wnode, p->R,
                    rq[q], q, n[q], static_cast<T *>(out[q]), st);
        p->launches++;
    }
    const bool mma = std::is_same<T, float>::value && p->contraction == 1;
    if (p->tucker) {
        const dim3 grid(3 * p->R, p->nz);
        const int64_t M = (int64_t)p->ny * p->nz;
        if (mma)
            k_tg_tucker_q<T, true><<<grid, 256, 0, st>>>(G, static_cast<const T *>(p->Y), static_cast<const T *>(p->Z),
                                                        p->r1, p->r2, p->r3, p->ny, p->nz, p->Kp, M,
                                                        static_cast<T *>(p->Q));
        else
            k_tg_tucker_q<T, false><<<grid, 256, 0, st>>>(G, static_cast<const T *>(p->Y), static_cast<const T *>(p->Z),
                                                         p->r1, p->r2, p->r3, p->ny, p->nz, p->Kp, M,
                                                         static_cast<T *>(p->Q));
        p->launches++;
    }
    if (p->timing) cudaEventRecord(p->ev[1], st);
    T *phi = phi_out ? static_cast<T *>(phi_out) : static_cast<T *>(p->phi);
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (p->contraction == 1) {
            cudaError_t e = tg_contract_mma(p, phi, st, p->timing ? p->ev[2] : nullptr);
            if (e != cudaSuccess) return tg_fail(DEMAG_ERR_CUDA, std::string("TG tensor-core contraction: ") +
                                                                     cudaGetErrorString(e));
            done = true;
        }
    }
    if (!done) {
        if (p->timing) cudaEventRecord(p->ev[2], st);
        // Tucker: y operand Q [K][nz ny] over ny_eff = nz ny rows, z operand a
        // row of ones (nz_eff = 1)
        const int ny = p->tucker ? p->ny * p->nz : p->ny, nz = p->tucker ? 1 : p->nz;
        const T *Yop = static_cast<const T *>(p->tucker ? p->Q : p->Y);
        const T *Zop = static_cast<const T *>(p->tucker ? p->ones : p->Z);
        const dim3 grid((p->nx + kTgCols - 1) / kTgCols, ((ny + 15) / 16) * ((nz + 7) / 8));
        k_tg_dense<T><<<grid, 256, 0, st>>>(static_cast<const T *>(p->X), Yop, Zop, K, p->nx, ny, nz, phi);
        p->launches++;
    }
    if (p->timing) cudaEventRecord(p->ev[3], st);
    if (want_field || E_dev) {
        // a grid-stride kernel: no more blocks than are resident at once
        const int64_t nrows = (int64_t)p->ny * p->nz;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tg_field<T>, kTgFieldThreads, 0) != cudaSuccess ||
            occ < 1)
            occ = 1;
        const int blocks =
            (int)std::min<int64_t>(std::min<int64_t>(nrows, (int64_t)sm_count() * occ), p->npartials);
        k_tg_field<T><<<blocks, kTgFieldThreads, 0, st>>>(phi, p->nx, p->ny, p->nz, (T)p->dx, (T)p->dy, (T)p->dz,
                                              static_cast<T *>(H), static_cast<const T *>(lam),
                                              static_cast<const T *>(Ux), static_cast<const T *>(Uy),
                                              static_cast<const T *>(Uz), p->r1, E_dev ? p->partials : nullptr, G,
                                              p->r2, p->r3);
        p->launches++;
        if (E_dev) {
            const double V = p->dx * p->dy * p->dz;
            cudaError_t e = energy_finalize(p->partials, blocks, -0.5 * 4e-7 * 3.14159265358979323846 * V, E_dev,
                                            p->partials + p->npartials, st);
            if (e != cudaSuccess) return tg_fail(DEMAG_ERR_CUDA, std::string("TG energy: ") + cudaGetErrorString(e));
            p->launches++;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tg_fail(DEMAG_ERR_CUDA, std::string("TG pass: ") + cudaGetErrorString(e));
    if (p->timing) {
        cudaEventRecord(p->ev[4], st);
        if ((e = cudaEventSynchronize(p->ev[4])) != cudaSuccess)
            return tg_fail(DEMAG_ERR_CUDA, std::string("TG timing: ") + cudaGetErrorString(e));
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->ev[k], p->ev[k + 1]);
            p->stage_ms[k] += ms;
        }
        p->timed_calls++;
    }
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
    const char *n0 = p->tucker ? "G" : "lam", *n1 = p->tucker ? "A" : "Ux", *n2 = p->tucker ? "B" : "Uy",
               *n3 = p->tucker ? "C" : "Uz";
    if ((s = tg_check_ptr(p, lam, n0)) != DEMAG_OK || (s = tg_check_ptr(p, Ux, n1)) != DEMAG_OK ||
        (s = tg_check_ptr(p, Uy, n2)) != DEMAG_OK || (s = tg_check_ptr(p, Uz, n3)) != DEMAG_OK)
        return s;
    if (H && (s = tg_check_ptr(p, H, "H")) != DEMAG_OK) return s;
    if (phi && (s = tg_check_ptr(p, phi, "phi")) != DEMAG_OK) return s;
    {
        // outputs must not overlap the factors (the kernels read them throughout)
        const size_t es = p->prec == DEMAG_F32 ? 4 : 8, r1 = p->r1, r2 = p->r2, r3 = p->r3;
        const size_t ncell = (size_t)p->nx * p->ny * p->nz;
        const void *in[4] = {lam, Ux, Uy, Uz};
        const size_t inb[4] = {(p->tucker ? 3 * r1 * r2 * r3 : 3 * r1) * es, 3 * r1 * p->nx * es, 3 * r2 * p->ny * es,
                               3 * r3 * p->nz * es};
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
    cudaFree(p->Yt);
    cudaFree(p->Zt);
    cudaFree(p->Bsw);
    cudaFree(p->err);
    cudaFree(p->Q);
    cudaFree(p->ones);
    for (int k = 0; k < 5; ++k)
        if (p->ev[k]) cudaEventDestroy(p->ev[k]);
    delete p;
}

}  // extern "C"

namespace {

demag_status tg_create(int nx, int ny, int nz, double dx, double dy, double dz, int rank, int r2, int r3, bool tucker,
                       demag_prec prec, demag_tg_plan_t *out)
{
    if (!out) return tg_fail(DEMAG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 3 || ny < 3 || nz < 3)
        return tg_fail(DEMAG_ERR_INVALID_ARG, "the second-order differences need at least 3 cells per axis");
    if (nx > 512 || ny > 512 || nz > 512) return tg_fail(DEMAG_ERR_UNSUPPORTED, "TG grids are built up to 512 per axis");
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz))
        return tg_fail(DEMAG_ERR_INVALID_ARG, "cell edges must be positive and finite");
    if (!tucker && (rank < 1 || rank > 64)) return tg_fail(DEMAG_ERR_INVALID_ARG, "CP rank must be in 1..64");
    if (tucker && (rank < 1 || r2 < 1 || r3 < 1 || rank > 16 || r2 > 16 || r3 > 16))
        return tg_fail(DEMAG_ERR_INVALID_ARG, "Tucker ranks must be in 1..16");
    if (prec != DEMAG_F32 && prec != DEMAG_F64) return tg_fail(DEMAG_ERR_INVALID_ARG, "unknown precision");
    demag_tg_plan *p = new demag_tg_plan;
    memset(p, 0, sizeof(*p));
    p->nx = nx; p->ny = ny; p->nz = nz;
    p->dx = dx; p->dy = dy; p->dz = dz;
    p->rank = rank;
    p->tucker = tucker;
    p->r1 = rank;
    p->r2 = tucker ? r2 : rank;
    p->r3 = tucker ? r3 : rank;
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
    const int K = 3 * R * rank, K2 = 3 * R * p->r2, K3 = 3 * R * p->r3;
    const int64_t ncell = (int64_t)nx * ny * nz;
    p->npartials = (int)std::min<int64_t>((int64_t)ny * nz, 4096);  // one per block of the field kernel
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
    if ((e = cudaMalloc(&p->Y, (size_t)K2 * ny * es)) != cudaSuccess) return cleanup(e, "cudaMalloc factors");
    if ((e = cudaMalloc(&p->Z, (size_t)K3 * nz * es)) != cudaSuccess) return cleanup(e, "cudaMalloc factors");
    if ((e = cudaMalloc(&p->phi, (size_t)ncell * es)) != cudaSuccess) return cleanup(e, "cudaMalloc potential");
    if ((e = cudaMalloc(&p->partials, sizeof(double) * (p->npartials + demag::kFinalizeScratch))) != cudaSuccess)
        return cleanup(e, "cudaMalloc partials");
    if ((e = cudaMemset(p->partials, 0, sizeof(double) * (p->npartials + demag::kFinalizeScratch))) != cudaSuccess)
        return cleanup(e, "clear partials");
    size_t mma_bytes = 0;
    p->Kp = (K + demag::tgm::kBK - 1) / demag::tgm::kBK * demag::tgm::kBK;
    if (tucker) {
        // Q: [nz ny][Kp] (tensor cores) or [K][nz ny] (CUDA cores); ones: the
        // unit z operand of Kp terms and the unit CP weights of the x factors
        const size_t qb = (size_t)ncell / nx * p->Kp * es;
        if ((e = cudaMalloc(&p->Q, qb)) != cudaSuccess) return cleanup(e, "cudaMalloc Tucker operand");
        if ((e = cudaMemset(p->Q, 0, qb)) != cudaSuccess) return cleanup(e, "clear Tucker operand");
        const size_t no = std::max<size_t>((size_t)p->Kp, (size_t)3 * rank);
        if ((e = cudaMalloc(&p->ones, no * es)) != cudaSuccess) return cleanup(e, "cudaMalloc ones");
        if (prec == DEMAG_F32) {
            std::vector<float> one(no, 1.0f);
            e = cudaMemcpy(p->ones, one.data(), no * es, cudaMemcpyHostToDevice);
        } else {
            std::vector<double> one(no, 1.0);
            e = cudaMemcpy(p->ones, one.data(), no * es, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return cleanup(e, "upload ones");
        mma_bytes += qb + no * es;
    }
    if (prec == DEMAG_F32) {
        // tensor-core contraction: K padded to the 16-term stage, the columns
        // split into ceil(nx / 256) tiles of BN (a multiple of 32) columns
        p->contraction = 1;
        p->nkc = p->Kp / demag::tgm::kBK;
        p->ntn = (nx + 255) / 256;
        p->BN = ((nx + p->ntn - 1) / p->ntn + 31) / 32 * 32;
        const size_t yb = tucker ? 0 : (size_t)ny * p->Kp * 4, zb = tucker ? 0 : (size_t)nz * p->Kp * 4;
        const size_t bb = (size_t)p->ntn * p->nkc * p->BN * 2 * demag::tgm::kBK * 4;
        if (!tucker && (e = cudaMalloc(&p->Yt, yb)) != cudaSuccess) return cleanup(e, "cudaMalloc transposed factors");
        if (!tucker && (e = cudaMalloc(&p->Zt, zb)) != cudaSuccess) return cleanup(e, "cudaMalloc transposed factors");
        if ((e = cudaMalloc(&p->Bsw, bb)) != cudaSuccess) return cleanup(e, "cudaMalloc tensor-core operand");
        if ((e = cudaMalloc(&p->err, sizeof(int))) != cudaSuccess) return cleanup(e, "cudaMalloc status word");
        if ((e = cudaMemset(p->err, 0, sizeof(int))) != cudaSuccess) return cleanup(e, "clear status word");
        mma_bytes += yb + zb + bb + sizeof(int);
    }
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
    p->device_bytes = 2 * sizeof(double) * R + tab_bytes + ((size_t)K * nx + (size_t)K2 * ny + (size_t)K3 * nz) * es +
                      (size_t)ncell * es + sizeof(double) * (p->npartials + demag::kFinalizeScratch) + mma_bytes;
    *out = p;
    demag::set_last_error("");
    return DEMAG_OK;
}

}  // namespace

extern "C" {

demag_status demag_tg_plan_create(int nx, int ny, int nz, double dx, double dy, double dz, int rank, demag_prec prec,
                                  demag_tg_plan_t *out)
{
    return tg_create(nx, ny, nz, dx, dy, dz, rank, rank, rank, false, prec, out);
}

demag_status demag_tg_plan_create_tucker(int nx, int ny, int nz, double dx, double dy, double dz, int r1, int r2,
                                         int r3, demag_prec prec, demag_tg_plan_t *out)
{
    return tg_create(nx, ny, nz, dx, dy, dz, r1, r2, r3, true, prec, out);
}

demag_status demag_tg_field_tucker(demag_tg_plan_t p, const void *G, const void *A, const void *B, const void *C,
                                   void *H, double *E_dev, void *stream)
{
    if (p && !p->tucker) return tg_fail(DEMAG_ERR_INVALID_ARG, "a CP plan takes demag_tg_field_cp");
    if (!H && !E_dev) return tg_fail(DEMAG_ERR_INVALID_ARG, "nothing to compute (no field, no energy)");
    return tg_job(p, G, A, B, C, H, E_dev, nullptr, stream);
}

demag_status demag_tg_potential_tucker(demag_tg_plan_t p, const void *G, const void *A, const void *B, const void *C,
                                       void *phi, void *stream)
{
    if (p && !p->tucker) return tg_fail(DEMAG_ERR_INVALID_ARG, "a CP plan takes demag_tg_potential_cp");
    if (!phi) return tg_fail(DEMAG_ERR_INVALID_ARG, "phi is NULL");
    return tg_job(p, G, A, B, C, nullptr, nullptr, phi, stream);
}

demag_status demag_tg_field_cp(demag_tg_plan_t p, const void *lam, const void *Ux, const void *Uy, const void *Uz,
                               void *H, double *E_dev, void *stream)
{
    if (p && p->tucker) return tg_fail(DEMAG_ERR_INVALID_ARG, "a Tucker plan takes demag_tg_field_tucker");
    if (!H && !E_dev) return tg_fail(DEMAG_ERR_INVALID_ARG, "nothing to compute (no field, no energy)");
    return tg_job(p, lam, Ux, Uy, Uz, H, E_dev, nullptr, stream);
}

demag_status demag_tg_potential_cp(demag_tg_plan_t p, const void *lam, const void *Ux, const void *Uy, const void *Uz,
                                   void *phi, void *stream)
{
    if (p && p->tucker) return tg_fail(DEMAG_ERR_INVALID_ARG, "a Tucker plan takes demag_tg_potential_tucker");
    if (!phi) return tg_fail(DEMAG_ERR_INVALID_ARG, "phi is NULL");
    return tg_job(p, lam, Ux, Uy, Uz, nullptr, nullptr, phi, stream);
}

demag_status demag_tg_set_contraction(demag_tg_plan_t p, int contraction)
{
    if (!p) return tg_fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (contraction != 0 && contraction != 1) return tg_fail(DEMAG_ERR_INVALID_ARG, "contraction must be 0 or 1");
    if (contraction == 1 && p->prec != DEMAG_F32)
        return tg_fail(DEMAG_ERR_UNSUPPORTED, "the tensor-core contraction is built for FP32 plans");
    p->contraction = contraction;
    return DEMAG_OK;
}

demag_status demag_tg_get_contraction(demag_tg_plan_t p, int *contraction)
{
    if (!p || !contraction) return tg_fail(DEMAG_ERR_INVALID_ARG, "plan or output is NULL");
    *contraction = p->contraction;
    return DEMAG_OK;
}

demag_status demag_tg_set_timing(demag_tg_plan_t p, int enable)
{
    if (!p) return tg_fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    TgGuard g(p->device);
    if (!g.ok) return tg_fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    if (enable && !p->ev[0])
        for (int k = 0; k < 5; ++k)
            if (cudaEventCreate(&p->ev[k]) != cudaSuccess) {
                cudaGetLastError();
                for (int q = 0; q < k; ++q) cudaEventDestroy(p->ev[q]);
                for (int q = 0; q < 5; ++q) p->ev[q] = nullptr;
                return tg_fail(DEMAG_ERR_CUDA, "creating timing events");
            }
    p->timing = enable != 0;
    for (int k = 0; k < 4; ++k) p->stage_ms[k] = 0.0;
    p->timed_calls = 0;
    return DEMAG_OK;
}

demag_status demag_tg_get_timing(demag_tg_plan_t p, double *ms, long *calls)
{
    if (!p || !ms) return tg_fail(DEMAG_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < 4; ++k) ms[k] = p->stage_ms[k];
    if (calls) *calls = p->timed_calls;
    return DEMAG_OK;
}

demag_status demag_tg_status(demag_tg_plan_t p, void *stream)
{
    if (!p) return tg_fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (!p->err) return DEMAG_OK;
    TgGuard g(p->device);
    if (!g.ok) return tg_fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    int flag = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&flag, p->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return tg_fail(DEMAG_ERR_CUDA, "reading the TG status");
    if (flag) {
        cudaMemsetAsync(p->err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        return tg_fail(DEMAG_ERR_TIMEOUT, "a bounded wait of the tensor-core contraction ran out of time");
    }
    return DEMAG_OK;
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
