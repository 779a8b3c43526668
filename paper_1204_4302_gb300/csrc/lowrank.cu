// Low-rank magnetization for the tensor-grid method (paper Sec. 3.2,
// "Low-Rank Magnetization"): each component M^(p) approximated in CP format
// or in Tucker format by alternating least squares (the ALS algorithms of
// Kolda and Bader's tensor survey, which the paper uses for both formats),
// and the relative error of Eq. "relr". FP64 throughout.
//
// Layouts: M [3][nz][ny][nx] (x fastest); factors [3][r][n] (row m of a
// component's factor is the m-th column vector over the axis' cells, the
// layout the TG entry points take); Tucker cores [3][r3][r2][r1].
//
// CP-ALS sweep (x, then y, then z):
//   A <- X_(x) (C kr B) V^+, V = (C^T C) * (B^T B); lambda <- column norms,
//   A <- A / lambda; likewise B and C.
// The MTTKRP X_(x) (C kr B) = sum_{k,j} X[k][j][i] B[j][m] C[k][m] is taken
// as a mode product over j (k_ttm_mid) and a diagonal contraction over k
// (k_diag_outer); y and z the same way with the roles permuted. V^+ is the
// pseudo-inverse of the symmetric V through its eigen-decomposition (cyclic
// Jacobi in one CTA), eigenvalues at or below 1e-12 of the largest dropped.
//
// Tucker-ALS (higher-order orthogonal iteration) sweep:
//   A <- r1 leading left singular vectors of (X x_y B^T x_z C^T)_(x), then B,
//   then C likewise, and after the last sweep G = X x_x A^T x_y B^T x_z C^T.
// The leading singular vectors come from the Jacobi eigen-decomposition of
// the smaller Gram matrix of the unfolding Y (n x q): Y Y^T when n <= q, else
// Y^T Y and u = Y v / |Y v| (zero for a null direction).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "demag.h"
#include "launch_util.cuh"
#include "plan.h"

namespace demag {
namespace {

constexpr int kLrThreads = 128;
constexpr int kLrChunk = 8;          // factor rows per CTA in the mode products
constexpr double kPinvRcond = 1e-12;

__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += red[q];
    return t;
}

// out[o][m][i] = sum_t X[(o n1 + t) n0 + i] F[m n1 + t]  (contract the middle
// axis of a [n2][n1][n0] tensor with the rows of F [r][n1]).
__global__ void __launch_bounds__(kLrThreads)
k_ttm_mid(const double *__restrict__ X, int n1, int n0, const double *__restrict__ F, int r, double *__restrict__ out)
{
    extern __shared__ double sF[];  // [kLrChunk][n1]
    const int o = blockIdx.x, i = blockIdx.y * kLrThreads + threadIdx.x, m0 = blockIdx.z * kLrChunk;
    const int mc = min(kLrChunk, r - m0);
    for (int e = threadIdx.x; e < mc * n1; e += blockDim.x) sF[e] = F[(int64_t)(m0 + e / n1) * n1 + e % n1];
    __syncthreads();
    if (i >= n0) return;
    double acc[kLrChunk];
#pragma unroll
    for (int q = 0; q < kLrChunk; ++q) acc[q] = 0.0;
    const double *x = X + (int64_t)o * n1 * n0 + i;
    for (int t = 0; t < n1; ++t) {
        const double v = x[(int64_t)t * n0];
#pragma unroll
        for (int q = 0; q < kLrChunk; ++q)
            if (q < mc) acc[q] += v * sF[q * n1 + t];
    }
    for (int q = 0; q < mc; ++q) out[((int64_t)o * r + m0 + q) * n0 + i] = acc[q];
}

// out[m][t][i] = sum_o F[m n2 + o] X[(o n1 + t) n0 + i]  (contract the outer axis).
__global__ void __launch_bounds__(kLrThreads)
k_ttm_outer(const double *__restrict__ X, int n2, int n1, int n0, const double *__restrict__ F, int r,
            double *__restrict__ out)
{
    extern __shared__ double sF[];  // [kLrChunk][n2]
    const int t = blockIdx.x, i = blockIdx.y * kLrThreads + threadIdx.x, m0 = blockIdx.z * kLrChunk;
    const int mc = min(kLrChunk, r - m0);
    for (int e = threadIdx.x; e < mc * n2; e += blockDim.x) sF[e] = F[(int64_t)(m0 + e / n2) * n2 + e % n2];
    __syncthreads();
    if (i >= n0) return;
    double acc[kLrChunk];
#pragma unroll
    for (int q = 0; q < kLrChunk; ++q) acc[q] = 0.0;
    const double *x = X + (int64_t)t * n0 + i;
    for (int o = 0; o < n2; ++o) {
        const double v = x[(int64_t)o * n1 * n0];
#pragma unroll
        for (int q = 0; q < kLrChunk; ++q)
            if (q < mc) acc[q] += v * sF[q * n2 + o];
    }
    for (int q = 0; q < mc; ++q) out[((int64_t)(m0 + q) * n1 + t) * n0 + i] = acc[q];
}

// out[row][m] = sum_i X[row n0 + i] F[m n0 + i]  (contract the inner axis; one
// CTA per row and factor-row chunk).
__global__ void __launch_bounds__(kLrThreads)
k_ttm_inner(const double *__restrict__ X, int n0, const double *__restrict__ F, int r, double *__restrict__ out)
{
    __shared__ double red[kLrThreads / 32];
    const int64_t row = blockIdx.x;
    const int m0 = blockIdx.y * kLrChunk, mc = min(kLrChunk, r - m0);
    double acc[kLrChunk];
#pragma unroll
    for (int q = 0; q < kLrChunk; ++q) acc[q] = 0.0;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const double v = X[row * n0 + i];
#pragma unroll
        for (int q = 0; q < kLrChunk; ++q)
            if (q < mc) acc[q] += v * F[(int64_t)(m0 + q) * n0 + i];
    }
    for (int q = 0; q < mc; ++q) {
        const double s = block_sum(acc[q], red);
        if (threadIdx.x == 0) out[row * r + m0 + q] = s;
    }
}

// out[m][i] = sum_o F[m no + o] T[o sto + m stm + i]  (diagonal contraction
// over the outer axis; the Khatri-Rao step of the x-mode MTTKRP).
__global__ void __launch_bounds__(kLrThreads)
k_diag_outer(const double *__restrict__ T, int no, int64_t sto, int64_t stm, int n0, const double *__restrict__ F,
             double *__restrict__ out)
{
    const int m = blockIdx.y, i = blockIdx.x * kLrThreads + threadIdx.x;
    if (i >= n0) return;
    double acc = 0.0;
    for (int o = 0; o < no; ++o) acc += F[(int64_t)m * no + o] * T[o * sto + m * stm + i];
    out[(int64_t)m * n0 + i] = acc;
}

// out[m][o] = sum_i F[m n0 + i] T[o sto + m stm + i]  (diagonal contraction
// over the inner axis; one CTA per (o, m)).
__global__ void __launch_bounds__(kLrThreads)
k_diag_inner(const double *__restrict__ T, int no, int64_t sto, int64_t stm, int n0, const double *__restrict__ F,
             double *__restrict__ out)
{
    __shared__ double red[kLrThreads / 32];
    const int o = blockIdx.x, m = blockIdx.y;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) acc += F[(int64_t)m * n0 + i] * T[o * sto + m * stm + i];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) out[(int64_t)m * no + o] = s;
}

// G[a][b] = sum_i F[a n + i] F[b n + i] (one CTA per entry).
__global__ void __launch_bounds__(kLrThreads) k_gram(const double *__restrict__ F, int n, int r, double *__restrict__ G)
{
    __shared__ double red[kLrThreads / 32];
    const int a = blockIdx.x / r, b = blockIdx.x % r;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += F[(int64_t)a * n + i] * F[(int64_t)b * n + i];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) G[a * r + b] = s;
}

// Cyclic Jacobi eigen-decomposition of the symmetric m x m matrix A (row
// major, overwritten: its diagonal ends as the eigenvalues) with Q the
// eigenvectors in columns, by one CTA. Each round applies m'/2 disjoint
// rotations (round-robin pairing, m' = m rounded up to even, the extra index
// idle) as A <- J^T A J in two passes (columns, then rows) and Q <- Q J;
// sweeps of m' - 1 rounds until the off-diagonal norm is below 1e-15 of the
// matrix norm or 60 sweeps.
__device__ void jacobi_eig(double *A, double *Q, int m, double *cs, double *red)
{
    const int me = m + (m & 1), np = me / 2;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Q[e] = (e / m == e % m) ? 1.0 : 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const double v = A[e] * A[e];
            tot += v;
            if (e / m != e % m) off += v;
        }
        off = block_sum(off, red);
        tot = block_sum(tot, red);
        if (off <= 1e-30 * tot || tot == 0.0) break;
        for (int round = 0; round < me - 1; ++round) {
            // pairing: position 0 fixed, the others rotated by `round`
            for (int k = threadIdx.x; k < np; k += blockDim.x) {
                const int pa = k, pb = me - 1 - k;
                int p = pa == 0 ? 0 : 1 + (pa - 1 + round) % (me - 1);
                int q = 1 + (pb - 1 + round) % (me - 1);
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0;
                if (q < m) {
                    const double apq = A[p * m + q];
                    if (apq != 0.0) {
                        const double th = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                }
                cs[4 * k] = p;
                cs[4 * k + 1] = q;
                cs[4 * k + 2] = c;
                cs[4 * k + 3] = s;
            }
            __syncthreads();
            // columns p, q of A and Q
            for (int e = threadIdx.x; e < np * m; e += blockDim.x) {
                const int k = e / m, row = e % m;
                const int p = (int)cs[4 * k], q = (int)cs[4 * k + 1];
                if (q >= m) continue;
                const double c = cs[4 * k + 2], s = cs[4 * k + 3];
                const double ap = A[row * m + p], aq = A[row * m + q];
                A[row * m + p] = c * ap - s * aq;
                A[row * m + q] = s * ap + c * aq;
                const double qp = Q[row * m + p], qq = Q[row * m + q];
                Q[row * m + p] = c * qp - s * qq;
                Q[row * m + q] = s * qp + c * qq;
            }
            __syncthreads();
            // rows p, q of A
            for (int e = threadIdx.x; e < np * m; e += blockDim.x) {
                const int k = e / m, col = e % m;
                const int p = (int)cs[4 * k], q = (int)cs[4 * k + 1];
                if (q >= m) continue;
                const double c = cs[4 * k + 2], s = cs[4 * k + 3];
                const double ap = A[p * m + col], aq = A[q * m + col];
                A[p * m + col] = c * ap - s * aq;
                A[q * m + col] = s * ap + c * aq;
            }
            __syncthreads();
        }
    }
}

constexpr int kEigThreads = 256;

// P = (G1 * G2)^+ (Hadamard product, then the pseudo-inverse of the
// symmetric result), r <= 64, one CTA; the matrices live in shared memory.
__global__ void __launch_bounds__(kEigThreads)
k_pinv_hadamard(const double *__restrict__ G1, const double *__restrict__ G2, int r, double *__restrict__ P)
{
    extern __shared__ double sm[];  // [r][r] matrix, [r][r] eigenvectors
    double *sA = sm, *sQ = sm + r * r;
    __shared__ double cs[4 * 32], red[kEigThreads / 32];
    __shared__ double s_cut;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) sA[e] = G1[e] * G2[e];
    __syncthreads();
    jacobi_eig(sA, sQ, r, cs, red);
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int a = 0; a < r; ++a) mx = fmax(mx, sA[a * r + a]);
        s_cut = kPinvRcond * mx;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int a = e / r, b = e % r;
        double v = 0.0;
        for (int t = 0; t < r; ++t) {
            const double w = sA[t * r + t];
            if (w > s_cut) v += sQ[a * r + t] * sQ[b * r + t] / w;
        }
        P[e] = v;
    }
}

// out[m][i] = sum_a Mt[a][i] P[a][m] (n x r times r x r).
__global__ void __launch_bounds__(kLrThreads)
k_apply_pinv(const double *__restrict__ Mt, int n, int r, const double *__restrict__ P, double *__restrict__ out)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * r) return;
    const int m = (int)(e / n), i = (int)(e % n);
    double v = 0.0;
    for (int a = 0; a < r; ++a) v += Mt[(int64_t)a * n + i] * P[a * r + m];
    out[e] = v;
}

// lam[m] = |F[m][:]|_2 and F[m][:] /= lam[m] (when non-zero); one CTA per row.
__global__ void __launch_bounds__(kLrThreads) k_normalize(double *__restrict__ F, int n, double *__restrict__ lam)
{
    __shared__ double red[kLrThreads / 32];
    const int m = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += F[(int64_t)m * n + i] * F[(int64_t)m * n + i];
    const double nrm = sqrt(block_sum(acc, red));
    if (threadIdx.x == 0) lam[m] = nrm;
    if (nrm > 0.0)
        for (int i = threadIdx.x; i < n; i += blockDim.x) F[(int64_t)m * n + i] /= nrm;
}

// Generic unfolding of a 3-way array: Y(row, hi, lo) = Y[row srow + hi shi +
// lo slo], columns col = hi qlo + lo (q = qhi qlo).
struct Unfold {
    const double *Y;
    int n, qhi, qlo;
    int64_t srow, shi, slo;
    __device__ double at(int row, int col) const
    {
        return Y[row * srow + (int64_t)(col / qlo) * shi + (int64_t)(col % qlo) * slo];
    }
};

// W = Y Y^T (rows, n x n) when by_rows, else Y^T Y (q x q); one CTA per entry.
__global__ void __launch_bounds__(kLrThreads) k_unfold_gram(Unfold u, bool by_rows, double *__restrict__ W)
{
    __shared__ double red[kLrThreads / 32];
    const int q = u.qhi * u.qlo, m = by_rows ? u.n : q;
    const int a = blockIdx.x / m, b = blockIdx.x % m;
    double acc = 0.0;
    if (by_rows)
        for (int c = threadIdx.x; c < q; c += blockDim.x) acc += u.at(a, c) * u.at(b, c);
    else
        for (int row = threadIdx.x; row < u.n; row += blockDim.x) acc += u.at(row, a) * u.at(row, b);
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) W[a * m + b] = s;
}

// Eigen-decomposition of W (m x m, global memory) by one CTA, then the r
// leading eigenvectors (eigenvalues descending) as the rows of `sel`
// [r][m] and the eigenvalues in `val` [r].
__global__ void __launch_bounds__(kEigThreads)
k_eig_leading(double *__restrict__ W, double *__restrict__ Q, int m, int r, double *__restrict__ sel,
              double *__restrict__ val)
{
    __shared__ double cs[4 * 128], red[kEigThreads / 32];
    __shared__ int order[256];
    jacobi_eig(W, Q, m, cs, red);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < m; ++a) order[a] = a;
        for (int a = 0; a < r; ++a) {  // partial selection sort, largest first (ties: lower index)
            int best = a;
            for (int b = a + 1; b < m; ++b)
                if (W[order[b] * m + order[b]] > W[order[best] * m + order[best]]) best = b;
            const int t = order[a]; order[a] = order[best]; order[best] = t;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r * m; e += blockDim.x) {
        const int a = e / m, row = e % m;
        sel[e] = Q[row * m + order[a]];
    }
    if (threadIdx.x < r) val[threadIdx.x] = W[order[threadIdx.x] * m + order[threadIdx.x]];
}

// Left singular vectors from right ones, by one CTA: u_a = Y v_a for a = 0 ..
// r - 1 (eigenvalues descending), each orthogonalised against u_0 .. u_{a-1}
// (two Gram-Schmidt passes: Y v_a loses orthogonality as sigma_a / sigma_0
// falls, the Gram matrix squaring the condition) and normalised into
// F[a][.]. A direction whose eigenvalue is at or below 1e-20 of the largest
// (sigma below 1e-10 of sigma_0: rounding noise of the Gram matrix), or
// whose norm after orthogonalisation falls below 1e-8 of its norm before,
// is a direction the tensor does not hold: zero.
__global__ void __launch_bounds__(kLrThreads)
k_left_from_right(Unfold u, const double *__restrict__ V, const double *__restrict__ val, int r, double *__restrict__ F)
{
    __shared__ double red[kLrThreads / 32];
    const int q = u.qhi * u.qlo, n = u.n;
    const double top = val[0] > 0.0 ? val[0] : 0.0;
    for (int a = 0; a < r; ++a) {
        double *fa = F + (int64_t)a * n;
        double acc = 0.0;
        for (int row = threadIdx.x; row < n; row += blockDim.x) {
            double v = 0.0;
            for (int c = 0; c < q; ++c) v += u.at(row, c) * V[(int64_t)a * q + c];
            fa[row] = v;
            acc += v * v;
        }
        const double n0 = sqrt(block_sum(acc, red));
        for (int pass = 0; pass < 2; ++pass)
            for (int b = 0; b < a; ++b) {
                const double *fb = F + (int64_t)b * n;
                double d = 0.0;
                for (int row = threadIdx.x; row < n; row += blockDim.x) d += fb[row] * fa[row];
                d = block_sum(d, red);
                for (int row = threadIdx.x; row < n; row += blockDim.x) fa[row] -= d * fb[row];
            }
        acc = 0.0;
        for (int row = threadIdx.x; row < n; row += blockDim.x) acc += fa[row] * fa[row];
        const double n1 = sqrt(block_sum(acc, red));
        const bool null_dir = !(val[a] > 1e-20 * top) || !(n0 > 0.0) || !(n1 > 1e-8 * n0);
        for (int row = threadIdx.x; row < n; row += blockDim.x) fa[row] = null_dir ? 0.0 : fa[row] / n1;
        __syncthreads();
    }
}

// Relative error of Eq. "relr" for all three components: one CTA per x row
// (grid-stride), the row-constant part of the reconstruction in shared
// memory: CP w[m] = lam_m B[m][j] C[m][k]; Tucker w[a] = sum_{b,c}
// G[c][b][a] B[b][j] C[c][k]; L[k][j][i] = sum_a w[a] A[a][i]. Partials
// (sum (M - L)^2, sum M^2) per CTA.
__global__ void __launch_bounds__(kLrThreads)
k_relerr_partials(const double *__restrict__ M, int nx, int ny, int nz, const double *__restrict__ lam,
                  const double *__restrict__ G, const double *__restrict__ A, const double *__restrict__ B,
                  const double *__restrict__ C, int r1, int r2, int r3, double *__restrict__ part)
{
    __shared__ double w[64], red[kLrThreads / 32];
    const int nrows = ny * nz;
    const int64_t ncell = (int64_t)nrows * nx;
    double e2 = 0.0, m2 = 0.0;
    for (int p = 0; p < 3; ++p) {
        const double *Ap = A + (int64_t)p * r1 * nx, *Bp = B + (int64_t)p * r2 * ny, *Cp = C + (int64_t)p * r3 * nz;
        for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
            const int j = row % ny, k = row / ny;
            __syncthreads();
            for (int a = threadIdx.x; a < r1; a += blockDim.x) {
                double v = 0.0;
                if (G) {
                    const double *Gp = G + (int64_t)p * r3 * r2 * r1;
                    for (int c = 0; c < r3; ++c)
                        for (int b = 0; b < r2; ++b)
                            v += Gp[((int64_t)c * r2 + b) * r1 + a] * Bp[(int64_t)b * ny + j] * Cp[(int64_t)c * nz + k];
                } else {
                    v = lam[p * r1 + a] * Bp[(int64_t)a * ny + j] * Cp[(int64_t)a * nz + k];
                }
                w[a] = v;
            }
            __syncthreads();
            const double *mrow = M + p * ncell + (int64_t)row * nx;
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                double l = 0.0;
                for (int a = 0; a < r1; ++a) l += w[a] * Ap[(int64_t)a * nx + i];
                const double mv = mrow[i];
                e2 += (mv - l) * (mv - l);
                m2 += mv * mv;
            }
        }
    }
    const double se = block_sum(e2, red), sm = block_sum(m2, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = se;
        part[2 * blockIdx.x + 1] = sm;
    }
}

__global__ void __launch_bounds__(kLrThreads) k_relerr_final(const double *__restrict__ part, int n, double *__restrict__ out)
{
    __shared__ double red[kLrThreads / 32];
    double e = 0.0, m = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        e += part[2 * q];
        m += part[2 * q + 1];
    }
    e = block_sum(e, red);
    m = block_sum(m, red);
    if (threadIdx.x == 0) *out = m > 0.0 ? sqrt(e / m) : sqrt(e);
}

// ---------------------------------------------------------------- host side
demag_status lr_fail(demag_status s, const std::string &m)
{
    set_last_error(m);
    return s;
}

demag_status lr_check(const void *ptr, const char *name, bool may_be_null = false)
{
    if (!ptr) return may_be_null ? DEMAG_OK : lr_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is NULL");
    if (((uintptr_t)ptr & 7u) != 0) return lr_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not 8-byte aligned");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return lr_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return lr_fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not device memory");
    return DEMAG_OK;
}

struct Workspace {
    std::vector<void *> bufs;
    cudaError_t err = cudaSuccess;
    double *get(size_t count)
    {
        void *p = nullptr;
        if (err == cudaSuccess) err = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(double));
        if (err != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return static_cast<double *>(p);
    }
    ~Workspace()
    {
        for (void *p : bufs) cudaFree(p);
    }
};

inline dim3 grid3(int a, int b, int c) { return dim3((unsigned)a, (unsigned)b, (unsigned)c); }
inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// out [n2][r][n0] = X [n2][n1][n0] x_mid F [r][n1]
void ttm_mid(const double *X, int n2, int n1, int n0, const double *F, int r, double *out, cudaStream_t st)
{
    k_ttm_mid<<<grid3(n2, cdiv(n0, kLrThreads), cdiv(r, kLrChunk)), kLrThreads, kLrChunk * n1 * sizeof(double), st>>>(
        X, n1, n0, F, r, out);
}

// out [r][n1][n0] = X [n2][n1][n0] x_outer F [r][n2]
void ttm_outer(const double *X, int n2, int n1, int n0, const double *F, int r, double *out, cudaStream_t st)
{
    k_ttm_outer<<<grid3(n1, cdiv(n0, kLrThreads), cdiv(r, kLrChunk)), kLrThreads, kLrChunk * n2 * sizeof(double),
                  st>>>(X, n2, n1, n0, F, r, out);
}

// out [rows][r] = X [rows][n0] x_inner F [r][n0]
void ttm_inner(const double *X, int rows, int n0, const double *F, int r, double *out, cudaStream_t st)
{
    k_ttm_inner<<<grid3(rows, cdiv(r, kLrChunk), 1), kLrThreads, 0, st>>>(X, n0, F, r, out);
}

// One CP-ALS mode update: F <- MT V^+ (MT [r][n] the MTTKRP), lam <- norms.
void cp_update(double *F, int n, int r, const double *MT, const double *G1, const double *G2, double *P, double *lam,
               cudaStream_t st)
{
    k_pinv_hadamard<<<1, kEigThreads, 2 * r * r * sizeof(double), st>>>(G1, G2, r, P);
    k_apply_pinv<<<cdiv(n * r, kLrThreads), kLrThreads, 0, st>>>(MT, n, r, P, F);
    k_normalize<<<r, kLrThreads, 0, st>>>(F, n, lam);
}

void gram(const double *F, int n, int r, double *G, cudaStream_t st)
{
    k_gram<<<r * r, kLrThreads, 0, st>>>(F, n, r, G);
}

// r leading left singular vectors of the unfolding into F [r][n].
void leading_vectors(const Unfold &u, int r, double *F, double *W, double *Q, double *sel, double *val,
                     cudaStream_t st)
{
    const int q = u.qhi * u.qlo;
    const bool by_rows = u.n <= q;
    const int m = by_rows ? u.n : q;
    k_unfold_gram<<<m * m, kLrThreads, 0, st>>>(u, by_rows, W);
    k_eig_leading<<<1, kEigThreads, 0, st>>>(W, Q, m, r, by_rows ? F : sel, val);
    if (!by_rows) k_left_from_right<<<1, kLrThreads, 0, st>>>(u, sel, val, r, F);
}

demag_status relerr_run(const double *M, int nx, int ny, int nz, const double *lam, const double *G, const double *A,
                        const double *B, const double *C, int r1, int r2, int r3, double *out, Workspace &ws,
                        cudaStream_t st)
{
    const int blocks = std::min(ny * nz, 1024);
    double *part = ws.get(2 * (size_t)blocks);
    if (!part) return lr_fail(DEMAG_ERR_OOM, "workspace for the relative error");
    k_relerr_partials<<<blocks, kLrThreads, 0, st>>>(M, nx, ny, nz, lam, G, A, B, C, r1, r2, r3, part);
    k_relerr_final<<<1, kLrThreads, 0, st>>>(part, blocks, out);
    return DEMAG_OK;
}

demag_status lr_finish(cudaStream_t st, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return lr_fail(DEMAG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    set_last_error("");
    return DEMAG_OK;
}

}  // namespace
}  // namespace demag

extern "C" {

demag_status demag_cp_als(int nx, int ny, int nz, const double *M, int rank, int iters, double *lam, double *Ux,
                          double *Uy, double *Uz, double *relerr, void *stream)
{
    using namespace demag;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 512 || ny > 512 || nz > 512)
        return lr_fail(DEMAG_ERR_INVALID_ARG, "grid sizes must be 1..512 per axis");
    if (rank < 1 || rank > 64) return lr_fail(DEMAG_ERR_INVALID_ARG, "CP rank must be in 1..64");
    if (iters < 0) return lr_fail(DEMAG_ERR_INVALID_ARG, "iters must be >= 0");
    demag_status s;
    if ((s = lr_check(M, "M")) != DEMAG_OK || (s = lr_check(lam, "lam")) != DEMAG_OK ||
        (s = lr_check(Ux, "Ux")) != DEMAG_OK || (s = lr_check(Uy, "Uy")) != DEMAG_OK ||
        (s = lr_check(Uz, "Uz")) != DEMAG_OK || (s = lr_check(relerr, "relerr", true)) != DEMAG_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int r = rank;
    if (allow_smem<k_pinv_hadamard>(2 * (size_t)r * r * sizeof(double)) != cudaSuccess)
        return lr_fail(DEMAG_ERR_CUDA, "shared memory for the rank-r eigen-decomposition");
    const int64_t ncell = (int64_t)nx * ny * nz;
    Workspace ws;
    const int nmax = std::max(nx, std::max(ny, nz));
    double *T = ws.get((size_t)r * nx * std::max(ny, nz));  // [nz][r][nx] or [r][ny][nx]
    double *MT = ws.get((size_t)r * nmax);
    double *GA = ws.get((size_t)r * r), *GB = ws.get((size_t)r * r), *GC = ws.get((size_t)r * r);
    double *P = ws.get((size_t)r * r);
    if (ws.err != cudaSuccess) return lr_fail(DEMAG_ERR_OOM, "ALS workspace");
    for (int p = 0; p < 3; ++p) {
        const double *X = M + p * ncell;
        double *A = Ux + (int64_t)p * r * nx, *B = Uy + (int64_t)p * r * ny, *C = Uz + (int64_t)p * r * nz;
        double *lp = lam + p * r;
        gram(B, ny, r, GB, st);
        gram(C, nz, r, GC, st);
        for (int it = 0; it < iters; ++it) {
            // x: T[k][m][i] = sum_j X B, MT[m][i] = sum_k C[m][k] T[k][m][i]
            ttm_mid(X, nz, ny, nx, B, r, T, st);
            k_diag_outer<<<grid3(cdiv(nx, kLrThreads), r, 1), kLrThreads, 0, st>>>(T, nz, (int64_t)r * nx, nx, nx, C,
                                                                                     MT);
            cp_update(A, nx, r, MT, GC, GB, P, lp, st);
            gram(A, nx, r, GA, st);
            // y: S[m][j][i] = sum_k C[m][k] X, MT[m][j] = sum_i A[m][i] S[m][j][i]
            ttm_outer(X, nz, ny, nx, C, r, T, st);
            k_diag_inner<<<grid3(ny, r, 1), kLrThreads, 0, st>>>(T, ny, nx, (int64_t)ny * nx, nx, A, MT);
            cp_update(B, ny, r, MT, GC, GA, P, lp, st);
            gram(B, ny, r, GB, st);
            // z: T[k][m][i] = sum_j X B, MT[m][k] = sum_i A[m][i] T[k][m][i]
            ttm_mid(X, nz, ny, nx, B, r, T, st);
            k_diag_inner<<<grid3(nz, r, 1), kLrThreads, 0, st>>>(T, nz, (int64_t)r * nx, nx, nx, A, MT);
            cp_update(C, nz, r, MT, GB, GA, P, lp, st);
            gram(C, nz, r, GC, st);
        }
    }
    if (relerr) {
        if ((s = relerr_run(M, nx, ny, nz, lam, nullptr, Ux, Uy, Uz, r, r, r, relerr, ws, st)) != DEMAG_OK) return s;
    }
    return lr_finish(st, "CP-ALS");
}

demag_status demag_tucker_als(int nx, int ny, int nz, const double *M, int r1, int r2, int r3, int iters, double *G,
                              double *A, double *B, double *C, double *relerr, void *stream)
{
    using namespace demag;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 512 || ny > 512 || nz > 512)
        return lr_fail(DEMAG_ERR_INVALID_ARG, "grid sizes must be 1..512 per axis");
    if (r1 < 1 || r2 < 1 || r3 < 1 || r1 > 16 || r2 > 16 || r3 > 16 || r1 > nx || r2 > ny || r3 > nz)
        return lr_fail(DEMAG_ERR_INVALID_ARG, "Tucker ranks must be in 1..16 and at most the axis length");
    if (iters < 1) return lr_fail(DEMAG_ERR_INVALID_ARG, "iters must be >= 1");
    demag_status s;
    if ((s = lr_check(M, "M")) != DEMAG_OK || (s = lr_check(G, "G")) != DEMAG_OK || (s = lr_check(A, "A")) != DEMAG_OK ||
        (s = lr_check(B, "B")) != DEMAG_OK || (s = lr_check(C, "C")) != DEMAG_OK ||
        (s = lr_check(relerr, "relerr", true)) != DEMAG_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ncell = (int64_t)nx * ny * nz;
    Workspace ws;
    // T1 [nz][r2][nx] or [nz][ny][r1]; Y [r3][r2][nx], [r3][ny][r1] or [nz][r2][r1]
    const size_t t1 = (size_t)nz * std::max((size_t)r2 * nx, (size_t)ny * r1);
    const size_t ysz = std::max((size_t)r3 * r2 * nx, std::max((size_t)r3 * ny * r1, (size_t)nz * r2 * r1));
    const int mmax = 256;
    double *T1 = ws.get(t1), *Y = ws.get(ysz);
    double *W = ws.get((size_t)mmax * mmax), *Q = ws.get((size_t)mmax * mmax);
    double *sel = ws.get((size_t)16 * mmax), *val = ws.get(16);
    if (ws.err != cudaSuccess) return lr_fail(DEMAG_ERR_OOM, "ALS workspace");
    for (int p = 0; p < 3; ++p) {
        const double *X = M + p * ncell;
        double *Ap = A + (int64_t)p * r1 * nx, *Bp = B + (int64_t)p * r2 * ny, *Cp = C + (int64_t)p * r3 * nz;
        for (int it = 0; it < iters; ++it) {
            // x: Y[c][b][i] = sum_k C[c][k] sum_j X[k][j][i] B[b][j]; unfold rows i, columns (c, b)
            ttm_mid(X, nz, ny, nx, Bp, r2, T1, st);
            ttm_outer(T1, nz, r2, nx, Cp, r3, Y, st);
            leading_vectors(Unfold{Y, nx, r3, r2, 1, (int64_t)r2 * nx, nx}, r1, Ap, W, Q, sel, val, st);
            // y: Y[c][j][a] = sum_k C[c][k] sum_i X[k][j][i] A[a][i]; unfold rows j, columns (c, a)
            ttm_inner(X, nz * ny, nx, Ap, r1, T1, st);
            ttm_outer(T1, nz, ny, r1, Cp, r3, Y, st);
            leading_vectors(Unfold{Y, ny, r3, r1, r1, (int64_t)ny * r1, 1}, r2, Bp, W, Q, sel, val, st);
            // z: Y[k][b][a] = sum_j B[b][j] sum_i X[k][j][i] A[a][i]; unfold rows k, columns (b, a)
            ttm_inner(X, nz * ny, nx, Ap, r1, T1, st);
            ttm_mid(T1, nz, ny, r1, Bp, r2, Y, st);
            leading_vectors(Unfold{Y, nz, r2, r1, (int64_t)r2 * r1, r1, 1}, r3, Cp, W, Q, sel, val, st);
        }
        // G[c][b][a] = sum_k C[c][k] Y[k][b][a] (Y of the last z update, with the final A and B)
        ttm_inner(X, nz * ny, nx, Ap, r1, T1, st);
        ttm_mid(T1, nz, ny, r1, Bp, r2, Y, st);
        ttm_outer(Y, nz, r2, r1, Cp, r3, G + (int64_t)p * r3 * r2 * r1, st);
    }
    if (relerr) {
        if ((s = relerr_run(M, nx, ny, nz, nullptr, G, A, B, C, r1, r2, r3, relerr, ws, st)) != DEMAG_OK) return s;
    }
    return lr_finish(st, "Tucker-ALS");
}

}  // extern "C"
