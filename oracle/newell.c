/*
 * FP64 CPU oracle: the cell-averaged demagnetization tensor and the direct
 * O(N^2) stray-field sum of the FFT demagnetization-tensor method (DM).
 *
 * TEST INFRASTRUCTURE. Only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark load this file's library. It shares no code
 * with the CUDA library it checks and must stay plain: no blocking, no
 * fusion, no tricks beyond the definitions written below.
 *
 * What it computes (paper Sec. 3.1, Eq. "demag" and the remark of Sec. 5.1
 * that the tensor is built for homogeneously magnetized cells with the field
 * averaged over each cell):
 *
 *   H(r_a) = -sum_b N(r_a - r_b) M_b,
 *   N_ij(R) = (1 / V_t) Int_{target} Int_{source} G_ij(r - r') dr' dr,
 *   G_ij(r) = -(1/4pi) d_i d_j (1/|r|) = -(1/4pi) (3 r_i r_j - d_ij |r|^2) / |r|^5 .
 *
 * The paper does not print the cell-averaged formulas (it cites OOMMF and
 * MicroMagnum for them); the closed form used here is the published one of
 * Newell, Williams and Dunlop (J. Geophys. Res. 98, 9551, 1993): the tensor
 * of two boxes is a signed sum of an auxiliary function over the 8 x 8 pairs
 * of box corners. N(0) is positive definite with trace 1 (sign reading: the
 * paper writes H = N * M with the opposite sign convention for N).
 *
 * Two independent evaluations of the same integral are provided:
 *   - closed form (64 corner pairs of f or g), used when the two cells touch
 *     or overlap, where the integrand is singular;
 *   - Gauss-Legendre quadrature of the point kernel G averaged over the
 *     difference of two uniform points in the two cells (a tent density per
 *     axis), used when the cells are separated by a gap. The closed form
 *     loses digits to cancellation roughly like (R/d)^6 at large R; the
 *     quadrature does not.
 * The node count is chosen from the Bernstein-ellipse bound of the analytic
 * integrand so the quadrature error stays near 1e-17 relative.
 *
 * Component order everywhere: xx, yy, zz, xy, xz, yz.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- closed form
 * Newell f(x,y,z), evaluated at |x|,|y|,|z| (even in every argument). Each
 * term whose factor vanishes is dropped, which is its limit value. */
static double newell_f(double x, double y, double z)
{
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    const double xz2 = x2 + z2, xy2 = x2 + y2;
    double s = (2.0 * x2 - y2 - z2) * R / 6.0;
    if (y > 0.0 && xz2 > 0.0) s += 0.5 * y * (z2 - x2) * asinh(y / sqrt(xz2));
    if (z > 0.0 && xy2 > 0.0) s += 0.5 * z * (y2 - x2) * asinh(z / sqrt(xy2));
    if (x > 0.0 && y > 0.0 && z > 0.0) s -= x * y * z * atan(y * z / (x * R));
    return s;
}

/* Newell g(x,y,z): odd in x and in y, even in z. */
static double newell_g(double x, double y, double z)
{
    const double sgn = (x < 0.0 ? -1.0 : 1.0) * (y < 0.0 ? -1.0 : 1.0);
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    const double xy2 = x2 + y2, yz2 = y2 + z2, xz2 = x2 + z2;
    double s = -x * y * R / 3.0;
    if (z > 0.0 && xy2 > 0.0) s += x * y * z * asinh(z / sqrt(xy2));
    if (x > 0.0 && yz2 > 0.0) s += y / 6.0 * (3.0 * z2 - y2) * asinh(x / sqrt(yz2));
    if (y > 0.0 && xz2 > 0.0) s += x / 6.0 * (3.0 * z2 - x2) * asinh(y / sqrt(xz2));
    if (z > 0.0) s -= z2 * z / 6.0 * atan(x * y / (z * R));
    if (y > 0.0) s -= z * y2 / 2.0 * atan(x * z / (y * R));
    if (x > 0.0) s -= z * x2 / 2.0 * atan(y * z / (x * R));
    return sgn * s;
}

/* Mutual tensor of a target box (centre tc, edges td) and a source box
 * (centre sc, edges sd): the field averaged over the target produced by unit
 * magnetization filling the source is -N m. Sum over the 8 x 8 corner pairs
 * with sign (-1)^(number of upper corners), divided by 4 pi V_target. */
void oracle_box_tensor(const double tc[3], const double td[3],
                       const double sc[3], const double sd[3], double out[6])
{
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int e = 0; e < 64; ++e) {
        const int et = e & 7, es = e >> 3;
        double D[3];
        int upper = 0;
        for (int a = 0; a < 3; ++a) {
            const int bt = (et >> a) & 1, bs = (es >> a) & 1;
            const double t = tc[a] + (bt ? 0.5 : -0.5) * td[a];
            const double s = sc[a] + (bs ? 0.5 : -0.5) * sd[a];
            D[a] = t - s;
            upper += bt + bs;
        }
        const double sign = (upper & 1) ? -1.0 : 1.0;
        acc[0] += sign * newell_f(D[0], D[1], D[2]);
        acc[1] += sign * newell_f(D[1], D[0], D[2]);
        acc[2] += sign * newell_f(D[2], D[1], D[0]);
        acc[3] += sign * newell_g(D[0], D[1], D[2]);
        acc[4] += sign * newell_g(D[0], D[2], D[1]);
        acc[5] += sign * newell_g(D[1], D[2], D[0]);
    }
    const double scale = 1.0 / (4.0 * M_PI * td[0] * td[1] * td[2]);
    for (int c = 0; c < 6; ++c) out[c] = acc[c] * scale;
}

/* Closed-form tensor between two equal cells at offset (X,Y,Z). */
void oracle_cell_tensor_closed(double X, double Y, double Z,
                               double dx, double dy, double dz, double out[6])
{
    const double tc[3] = {X, Y, Z}, sc[3] = {0.0, 0.0, 0.0};
    const double d[3] = {dx, dy, dz};
    oracle_box_tensor(tc, d, sc, d, out);
}

/* ------------------------------------------------------------ quadrature
 * Gauss-Legendre nodes and weights on [-1, 1]: roots of P_n by Newton's
 * method from the usual cosine first guesses, weights 2 / ((1-x^2) P_n'(x)^2). */
int oracle_gl_rule(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = (n == 1) ? 1.0 : n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) <= 1e-17) break;
        }
        /* derivative at the converged root for the weight */
        {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = (n == 1) ? 1.0 : n * (t * p1 - p0) / (t * t - 1.0);
        }
        const double wi = 2.0 / ((1.0 - t * t) * dp * dp);
        x[i] = -t; w[i] = wi;
        x[n - 1 - i] = t; w[n - 1 - i] = wi;
    }
    if (n & 1) x[n / 2] = 0.0;
    return 0;
}

#define ORACLE_MAX_HALF_NODES 64

/* 1-D rule for E[phi(u)] with u the difference of two uniform points in
 * cells of edge d: density (1 - |u|/d)/d on [-d, d]. n GL nodes on each half,
 * where the density is linear. Returns 2n nodes. */
static void tent_rule(int n, double d, double *u, double *wt)
{
    double x[ORACLE_MAX_HALF_NODES], w[ORACLE_MAX_HALF_NODES];
    oracle_gl_rule(n, x, w);
    for (int i = 0; i < n; ++i) {
        const double ui = 0.5 * d * (1.0 + x[i]);
        const double wi = 0.5 * w[i] * (1.0 - ui / d);
        u[2 * i] = ui;      wt[2 * i] = wi;
        u[2 * i + 1] = -ui; wt[2 * i + 1] = wi;
    }
}

/* Gap between two equal cells at offset R: the smallest |r - r'|. */
static double cell_gap(double X, double Y, double Z, double dx, double dy, double dz)
{
    const double gx = fmax(0.0, fabs(X) - dx);
    const double gy = fmax(0.0, fabs(Y) - dy);
    const double gz = fmax(0.0, fabs(Z) - dz);
    return sqrt(gx * gx + gy * gy + gz * gz);
}

/* Nodes per half interval on one axis. The integrand is analytic in each
 * variable within distance gap of the real box; shrinking that margin by half
 * bounds the integrand on the Bernstein ellipse of semi-minor axis
 * b = gap / d (half-interval half-length d/2), rho = b + sqrt(1 + b^2), and
 * the error decays like rho^(-2n): n = ceil(20 / ln rho) gives ~e^-40. */
static int half_nodes(double gap, double d)
{
    const double b = gap / d;
    const double rho = b + sqrt(1.0 + b * b);
    int n = (int)ceil(20.0 / log(rho));
    if (n < 3) n = 3;
    if (n > ORACLE_MAX_HALF_NODES) n = ORACLE_MAX_HALF_NODES;
    return n;
}

static inline void neumaier_add(double *s, double *c, double v)
{
    const double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else *c += (v - t) + *s;
    *s = t;
}

/* Tensor between two separated equal cells by tensor-product quadrature of
 * the point kernel. nx_, ny_, nz_ nodes per half interval (0 = automatic).
 * Returns -1 when the cells touch (gap 0), where the integrand is singular. */
int oracle_cell_tensor_quad(double X, double Y, double Z,
                            double dx, double dy, double dz,
                            int nx_, int ny_, int nz_, double out[6])
{
    const double gap = cell_gap(X, Y, Z, dx, dy, dz);
    if (!(gap > 0.0)) return -1;
    const int nx = nx_ > 0 ? nx_ : half_nodes(gap, dx);
    const int ny = ny_ > 0 ? ny_ : half_nodes(gap, dy);
    const int nz = nz_ > 0 ? nz_ : half_nodes(gap, dz);
    if (nx > ORACLE_MAX_HALF_NODES || ny > ORACLE_MAX_HALF_NODES || nz > ORACLE_MAX_HALF_NODES)
        return -2;
    double ux[2 * ORACLE_MAX_HALF_NODES], wx[2 * ORACLE_MAX_HALF_NODES];
    double uy[2 * ORACLE_MAX_HALF_NODES], wy[2 * ORACLE_MAX_HALF_NODES];
    double uz[2 * ORACLE_MAX_HALF_NODES], wz[2 * ORACLE_MAX_HALF_NODES];
    tent_rule(nx, dx, ux, wx);
    tent_rule(ny, dy, uy, wy);
    tent_rule(nz, dz, uz, wz);
    double s[6] = {0}, c[6] = {0};
    for (int k = 0; k < 2 * nz; ++k) {
        const double rz = Z + uz[k];
        for (int j = 0; j < 2 * ny; ++j) {
            const double ry = Y + uy[j];
            double p[6] = {0};
            for (int i = 0; i < 2 * nx; ++i) {
                const double rx = X + ux[i];
                const double r2 = rx * rx + ry * ry + rz * rz;
                const double r = sqrt(r2);
                const double w = wx[i] / (r2 * r2 * r);
                p[0] += w * (3.0 * rx * rx - r2);
                p[1] += w * (3.0 * ry * ry - r2);
                p[2] += w * (3.0 * rz * rz - r2);
                p[3] += w * (3.0 * rx * ry);
                p[4] += w * (3.0 * rx * rz);
                p[5] += w * (3.0 * ry * rz);
            }
            const double wyz = wy[j] * wz[k];
            for (int q = 0; q < 6; ++q) neumaier_add(&s[q], &c[q], wyz * p[q]);
        }
    }
    const double scale = -dx * dy * dz / (4.0 * M_PI);
    for (int q = 0; q < 6; ++q) out[q] = scale * (s[q] + c[q]);
    return 0;
}

/* The oracle's tensor entry: closed form for touching cells, quadrature for
 * separated ones. */
void oracle_cell_tensor(double X, double Y, double Z,
                        double dx, double dy, double dz, double out[6])
{
    if (oracle_cell_tensor_quad(X, Y, Z, dx, dy, dz, 0, 0, 0, out) != 0)
        oracle_cell_tensor_closed(X, Y, Z, dx, dy, dz, out);
}

/* ------------------------------------------------------------ tables */
typedef struct {
    int nx, ny, nz;       /* table extents per axis */
    int ox, oy, oz;       /* offset index of the first entry (0 or -(n-1)) */
    double dx, dy, dz;
    double *out;          /* [6][nz][ny][nx] */
    int64_t next;         /* shared work counter over z-y rows */
    pthread_mutex_t lock;
} table_job;

static void *table_worker(void *arg)
{
    table_job *J = (table_job *)arg;
    const int64_t rows = (int64_t)J->nz * J->ny;
    const int64_t plane = (int64_t)J->nz * J->ny * J->nx;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        const int64_t r = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (r >= rows) break;
        const int k = (int)(r / J->ny), j = (int)(r % J->ny);
        for (int i = 0; i < J->nx; ++i) {
            double t[6];
            oracle_cell_tensor((i + J->ox) * J->dx, (j + J->oy) * J->dy, (k + J->oz) * J->dz,
                               J->dx, J->dy, J->dz, t);
            const int64_t idx = ((int64_t)k * J->ny + j) * J->nx + i;
            for (int q = 0; q < 6; ++q) J->out[q * plane + idx] = t[q];
        }
    }
    return NULL;
}

static int run_table(table_job *J, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    J->next = 0;
    pthread_mutex_init(&J->lock, NULL);
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, table_worker, J) == 0) ++started;
    table_worker(J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J->lock);
    return 0;
}

/* Octant table: out[6][nz][ny][nx], entry (k,j,i) = N(i dx, j dy, k dz),
 * 0 <= i < nx etc. The other octants follow from the parities of the
 * components (xx, yy, zz even in every axis; xy odd in x and y; xz odd in
 * x and z; yz odd in y and z). */
int oracle_tensor_octant(int nx, int ny, int nz, double dx, double dy, double dz,
                         int nthreads, double *out)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0) || !out) return -1;
    table_job J;
    memset(&J, 0, sizeof J);
    J.nx = nx; J.ny = ny; J.nz = nz;
    J.dx = dx; J.dy = dy; J.dz = dz;
    J.out = out;
    return run_table(&J, nthreads);
}

/* Signed-offset table: out[6][2nz-1][2ny-1][2nx-1], entry (k,j,i) holds
 * N((i-nx+1) dx, (j-ny+1) dy, (k-nz+1) dz), every offset evaluated directly. */
int oracle_tensor_signed(int nx, int ny, int nz, double dx, double dy, double dz,
                         int nthreads, double *out)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0) || !out) return -1;
    table_job J;
    memset(&J, 0, sizeof J);
    J.nx = 2 * nx - 1; J.ny = 2 * ny - 1; J.nz = 2 * nz - 1;
    J.ox = -(nx - 1); J.oy = -(ny - 1); J.oz = -(nz - 1);
    J.dx = dx; J.dy = dy; J.dz = dz;
    J.out = out;
    return run_table(&J, nthreads);
}

/* Direct pair sum H_a = -sum_b N(r_a - r_b) M_b over all cell pairs.
 * M, H: [3][nz][ny][nx]; tab: the signed-offset table above. O(N^2). */
int oracle_field_bruteforce(int nx, int ny, int nz, const double *tab,
                            const double *M, double *H)
{
    if (nx < 1 || ny < 1 || nz < 1 || !tab || !M || !H) return -1;
    const int64_t n = (int64_t)nx * ny * nz;
    const int sx = 2 * nx - 1, sy = 2 * ny - 1, sz = 2 * nz - 1;
    const int64_t tplane = (int64_t)sx * sy * sz;
    for (int64_t a = 0; a < n; ++a) {
        const int az = (int)(a / ((int64_t)nx * ny)), ay = (int)((a / nx) % ny), ax = (int)(a % nx);
        double h[3] = {0, 0, 0};
        for (int64_t b = 0; b < n; ++b) {
            const int bz = (int)(b / ((int64_t)nx * ny)), by = (int)((b / nx) % ny), bx = (int)(b % nx);
            const int64_t t = ((int64_t)(az - bz + nz - 1) * sy + (ay - by + ny - 1)) * sx + (ax - bx + nx - 1);
            const double xx = tab[0 * tplane + t], yy = tab[1 * tplane + t], zz = tab[2 * tplane + t];
            const double xy = tab[3 * tplane + t], xz = tab[4 * tplane + t], yz = tab[5 * tplane + t];
            const double mx = M[b], my = M[n + b], mz = M[2 * n + b];
            h[0] += xx * mx + xy * my + xz * mz;
            h[1] += xy * mx + yy * my + yz * mz;
            h[2] += xz * mx + yz * my + zz * mz;
        }
        H[a] = -h[0]; H[n + a] = -h[1]; H[2 * n + a] = -h[2];
    }
    return 0;
}

/* The same direct sum at a list of target cells only, with the tensor taken
 * from an octant table and the other octants by parity. cells: ncell triples
 * (x, y, z). Hout: [ncell][3]. Used to check single outputs of large grids. */
int oracle_field_at(int nx, int ny, int nz, const double *oct, const double *M,
                    int ncell, const int *cells, double *Hout)
{
    if (nx < 1 || ny < 1 || nz < 1 || !oct || !M || !cells || !Hout) return -1;
    const int64_t n = (int64_t)nx * ny * nz;
    for (int q = 0; q < ncell; ++q) {
        const int ax = cells[3 * q], ay = cells[3 * q + 1], az = cells[3 * q + 2];
        if (ax < 0 || ax >= nx || ay < 0 || ay >= ny || az < 0 || az >= nz) return -2;
        double h[3] = {0, 0, 0};
        for (int bz = 0; bz < nz; ++bz)
            for (int by = 0; by < ny; ++by)
                for (int bx = 0; bx < nx; ++bx) {
                    const int di = ax - bx, dj = ay - by, dk = az - bz;
                    const double si = di < 0 ? -1.0 : 1.0, sj = dj < 0 ? -1.0 : 1.0, sk = dk < 0 ? -1.0 : 1.0;
                    const int64_t t = ((int64_t)abs(dk) * ny + abs(dj)) * nx + abs(di);
                    const double xx = oct[0 * n + t], yy = oct[1 * n + t], zz = oct[2 * n + t];
                    const double xy = si * sj * oct[3 * n + t];
                    const double xz = si * sk * oct[4 * n + t];
                    const double yz = sj * sk * oct[5 * n + t];
                    const int64_t b = ((int64_t)bz * ny + by) * nx + bx;
                    const double mx = M[b], my = M[n + b], mz = M[2 * n + b];
                    h[0] += xx * mx + xy * my + xz * mz;
                    h[1] += xy * mx + yy * my + yz * mz;
                    h[2] += xz * mx + yz * my + zz * mz;
                }
        Hout[3 * q] = -h[0]; Hout[3 * q + 1] = -h[1]; Hout[3 * q + 2] = -h[2];
    }
    return 0;
}
