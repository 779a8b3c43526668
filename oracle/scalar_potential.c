/*
 * FP64 CPU oracle of the scalar-potential method (SP) of paper Sec. 3.1.
 *
 * TEST INFRASTRUCTURE. Only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark load this file's library. It shares no code
 * with the CUDA library it checks and stays plain: no blocking, no fusion.
 *
 * What it computes. The potential of a magnetization M is the integral of
 * Eq. "scpot": phi(r) = (1/4pi) Int M(r') . grad' (1/|r - r'|) dr'. For cells
 * of constant M this is a sum over cells of M_b . S(r - r_b) with the vector
 * kernel of one cell centred at the origin,
 *
 *   S_j(R) = (1/4pi) Int_cell d/du_j (1/|R - u|) du
 *          = (1/4pi) [ Int_{face u_j = +d_j/2} - Int_{face u_j = -d_j/2} ] dA / |R - u|
 *          = (1/4pi) Int_cell (R - u)_j / |R - u|^3 du ,
 *
 * and the field is H = -grad phi (Eq. "field") by finite differences.
 *
 * Readings (the paper states the method by these equations and defers the
 * discretisation to its reference implementation):
 *   - the potential is evaluated at the grid nodes (cell corners);
 *   - the field of a cell is the average over the cell of -grad of the
 *     trilinear interpolant of its 8 corner potentials, i.e.
 *     H_x = -(1/(4 dx)) sum over the cell's 4 edges along x of
 *     (phi(upper node) - phi(lower node)), and likewise for y and z.
 * With these readings the SP energies of the paper's cube and thin-film
 * tables are reproduced to every printed digit (see the tests).
 *
 * Two independent evaluations of S are provided:
 *   - closed form: each face integral of 1/|R - u| over a rectangle is a
 *     signed sum over the rectangle's corners of the antiderivative
 *     F(a, v, w) = v ln(w + r) + w ln(v + r) - a atan(v w / (a r)),
 *     r = sqrt(a^2 + v^2 + w^2), for which d^2 F / dv dw = 1 / r;
 *   - Gauss-Legendre quadrature of the volume form (R - u)_j / |R - u|^3
 *     over the cell, for points away from the cell, with the node count per
 *     axis taken from the Bernstein ellipse of the nearest singularity.
 * The closed form cancels digits at large |R| (a difference of two face
 * integrals, each a corner sum), so the oracle uses it only near the cell.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

int oracle_gl_rule(int n, double *x, double *w); /* newell.c */

/* ln(w + r) with r = sqrt(q2 + w^2), q2 >= 0; for w < 0 the equivalent
 * ln(q2 / (r - w)) avoids the cancellation of w + r. */
static double log_w_plus_r(double w, double r, double q2)
{
    if (w >= 0.0) return log(w + r);
    return log(q2 / (r - w));
}

/* Antiderivative F of 1/r over a rectangle in a plane at distance a. Terms
 * whose factor vanishes are dropped: that is their limit value. */
static double rect_F(double a, double v, double w)
{
    const double a2 = a * a, v2 = v * v, w2 = w * w;
    const double r = sqrt(a2 + v2 + w2);
    if (r == 0.0) return 0.0;
    double s = 0.0;
    if (v != 0.0) s += v * log_w_plus_r(w, r, a2 + v2);
    if (w != 0.0) s += w * log_w_plus_r(v, r, a2 + w2);
    if (a != 0.0) s -= a * atan(v * w / (a * r));
    return s;
}

/* Int_{-hv}^{hv} Int_{-hw}^{hw} dv' dw' / sqrt(a^2 + (V - v')^2 + (W - w')^2). */
double oracle_sp_rect(double a, double V, double W, double hv, double hw)
{
    return rect_F(a, V + hv, W + hw) - rect_F(a, V - hv, W + hw) - rect_F(a, V + hv, W - hw) +
           rect_F(a, V - hv, W - hw);
}

/* S(R) by the face integrals (closed form). out = (S_x, S_y, S_z). S scales
 * like a length (S(sR; s d) = s S(R; d)); lengths are taken in units of the
 * longest edge so the logarithms of the corner sum stay of order one. */
void oracle_sp_kernel_closed(double X, double Y, double Z, double dx, double dy, double dz,
                             double out[3])
{
    const double L = fmax(dx, fmax(dy, dz));
    X /= L; Y /= L; Z /= L;
    dx /= L; dy /= L; dz /= L;
    const double k = L / (4.0 * M_PI);
    out[0] = k * (oracle_sp_rect(X - 0.5 * dx, Y, Z, 0.5 * dy, 0.5 * dz) -
                  oracle_sp_rect(X + 0.5 * dx, Y, Z, 0.5 * dy, 0.5 * dz));
    out[1] = k * (oracle_sp_rect(Y - 0.5 * dy, Z, X, 0.5 * dz, 0.5 * dx) -
                  oracle_sp_rect(Y + 0.5 * dy, Z, X, 0.5 * dz, 0.5 * dx));
    out[2] = k * (oracle_sp_rect(Z - 0.5 * dz, X, Y, 0.5 * dx, 0.5 * dy) -
                  oracle_sp_rect(Z + 0.5 * dz, X, Y, 0.5 * dx, 0.5 * dy));
}

#define SP_MAX_NODES 96

/* GL nodes for axis a: the integrand, as a function of u_a on [-h, h], is
 * analytic except at u_a = R_a +- i rho with rho >= rho_min, the distance of
 * R from the cell in the other two axes. The Bernstein ellipse through the
 * nearest such point has parameter |z + sqrt(z^2 - 1)|, z = (R_a + i rho_min)
 * / h, and the GL error decays like its -2n-th power: n = ceil(20 / ln) nodes
 * give ~e^-40. */
static int sp_axis_nodes(double Ra, double rho_min, double h)
{
    const double complex z = (Ra + I * rho_min) / h;
    double complex s = csqrt(z * z - 1.0);
    double rb = cabs(z + s);
    const double rb2 = cabs(z - s);
    if (rb2 > rb) rb = rb2;
    if (!(rb > 1.0)) return -1;
    int n = (int)ceil(20.0 / log(rb));
    if (n < 4) n = 4;
    return n;
}

/* S(R) by tensor-product GL quadrature of the volume form. Returns -1 when
 * R lies in or on the closed cell (the integrand is singular), -2 when a
 * rule would need more than SP_MAX_NODES nodes. n_ = 0 picks the counts. */
int oracle_sp_kernel_quad(double X, double Y, double Z, double dx, double dy, double dz, int nx_,
                          int ny_, int nz_, double out[3])
{
    const double R[3] = {X, Y, Z}, h[3] = {0.5 * dx, 0.5 * dy, 0.5 * dz};
    double g[3];
    for (int a = 0; a < 3; ++a) g[a] = fmax(0.0, fabs(R[a]) - h[a]);
    if (!(g[0] > 0.0 || g[1] > 0.0 || g[2] > 0.0)) return -1;
    int n[3] = {nx_, ny_, nz_};
    for (int a = 0; a < 3; ++a) {
        if (n[a] > 0) continue;
        const double rho = sqrt(g[(a + 1) % 3] * g[(a + 1) % 3] + g[(a + 2) % 3] * g[(a + 2) % 3]);
        n[a] = sp_axis_nodes(R[a], rho, h[a]);
        if (n[a] < 0) return -1;
    }
    if (n[0] > SP_MAX_NODES || n[1] > SP_MAX_NODES || n[2] > SP_MAX_NODES) return -2;
    double x[3][SP_MAX_NODES], w[3][SP_MAX_NODES];
    for (int a = 0; a < 3; ++a) {
        oracle_gl_rule(n[a], x[a], w[a]);
        for (int i = 0; i < n[a]; ++i) {
            x[a][i] *= h[a];
            w[a][i] *= h[a];
        }
    }
    double s[3] = {0, 0, 0};
    for (int k = 0; k < n[2]; ++k) {
        const double rz = Z - x[2][k];
        for (int j = 0; j < n[1]; ++j) {
            const double ry = Y - x[1][j];
            double p[3] = {0, 0, 0};
            for (int i = 0; i < n[0]; ++i) {
                const double rx = X - x[0][i];
                const double r2 = rx * rx + ry * ry + rz * rz;
                const double f = w[0][i] / (r2 * sqrt(r2));
                p[0] += f * rx;
                p[1] += f * ry;
                p[2] += f * rz;
            }
            const double wyz = w[1][j] * w[2][k];
            for (int q = 0; q < 3; ++q) s[q] += wyz * p[q];
        }
    }
    for (int q = 0; q < 3; ++q) out[q] = s[q] / (4.0 * M_PI);
    return 0;
}

/* The oracle's kernel: closed form within 2.5 cell edges on every axis,
 * quadrature beyond. */
void oracle_sp_kernel(double X, double Y, double Z, double dx, double dy, double dz, double out[3])
{
    if (fabs(X) <= 2.5 * dx && fabs(Y) <= 2.5 * dy && fabs(Z) <= 2.5 * dz) {
        oracle_sp_kernel_closed(X, Y, Z, dx, dy, dz, out);
        return;
    }
    if (oracle_sp_kernel_quad(X, Y, Z, dx, dy, dz, 0, 0, 0, out) != 0)
        oracle_sp_kernel_closed(X, Y, Z, dx, dy, dz, out);
}

/* ------------------------------------------------------------ node tables */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double *out;     /* [3][nz][ny][nx] */
    int64_t next;
    pthread_mutex_t lock;
} sp_job;

static void *sp_worker(void *arg)
{
    sp_job *J = (sp_job *)arg;
    const int64_t rows = (int64_t)J->nz * J->ny;
    const int64_t plane = rows * J->nx;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        const int64_t r = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (r >= rows) break;
        const int k = (int)(r / J->ny), j = (int)(r % J->ny);
        for (int i = 0; i < J->nx; ++i) {
            double s[3];
            oracle_sp_kernel((i + 0.5) * J->dx, (j + 0.5) * J->dy, (k + 0.5) * J->dz, J->dx, J->dy,
                             J->dz, s);
            const int64_t idx = ((int64_t)k * J->ny + j) * J->nx + i;
            for (int q = 0; q < 3; ++q) J->out[q * plane + idx] = s[q];
        }
    }
    return NULL;
}

/* Kernel at the positive half-integer offsets: out[3][nz][ny][nx], entry
 * (k, j, i) = S((i + 1/2) dx, (j + 1/2) dy, (k + 1/2) dz). The offsets from a
 * cell centre to the grid nodes are half-integer multiples of the edges; the
 * other octants follow from the parities (S_x odd in X and even in Y, Z;
 * S_y odd in Y; S_z odd in Z). */
int oracle_sp_kernel_nodes(int nx, int ny, int nz, double dx, double dy, double dz, int nthreads,
                           double *out)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0) || !out) return -1;
    sp_job J;
    memset(&J, 0, sizeof J);
    J.nx = nx; J.ny = ny; J.nz = nz;
    J.dx = dx; J.dy = dy; J.dz = dz;
    J.out = out;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    pthread_mutex_init(&J.lock, NULL);
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, sp_worker, &J) == 0) ++started;
    sp_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.lock);
    return 0;
}

/* Potential at every node by the direct sum over cells (Eq. "scpot" on the
 * grid), each pair's kernel evaluated on its own. M[3][nz][ny][nx];
 * phi[nz+1][ny+1][nx+1], node (i, j, k) at (i dx, j dy, k dz), cell (a, b, c)
 * centred at ((a + 1/2) dx, ...). O(nodes x cells): tiny grids only. */
int oracle_sp_potential_bruteforce(int nx, int ny, int nz, double dx, double dy, double dz,
                                   const double *M, double *phi)
{
    if (nx < 1 || ny < 1 || nz < 1 || !M || !phi) return -1;
    const int64_t nc = (int64_t)nx * ny * nz;
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                double acc = 0.0;
                for (int c = 0; c < nz; ++c)
                    for (int b = 0; b < ny; ++b)
                        for (int a = 0; a < nx; ++a) {
                            double s[3];
                            oracle_sp_kernel((i - a - 0.5) * dx, (j - b - 0.5) * dy, (k - c - 0.5) * dz,
                                             dx, dy, dz, s);
                            const int64_t idx = ((int64_t)c * ny + b) * nx + a;
                            acc += s[0] * M[idx] + s[1] * M[nc + idx] + s[2] * M[2 * nc + idx];
                        }
                phi[((int64_t)k * (ny + 1) + j) * (nx + 1) + i] = acc;
            }
    return 0;
}
