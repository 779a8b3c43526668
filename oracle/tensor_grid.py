"""FP64 CPU oracle of the tensor-grid method (TG, paper Sec. 3.2).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke
check and the CPU legs of the benchmark import it; the CUDA library shares no
code with it.

What the method computes. The potential of Eq. "scpot" at the cell centres,
with the kernel 1/|r|^3 written as a Gaussian integral (Eq. "transform"),
1/|r|^3 = (2/sqrt(pi)) Int tau^2 exp(-tau^2 |r|^2) dtau, so that the integral
over the body separates into 1-D integrals along the axes (Eq. "gausspot").
The tau integral is done by a sinc (trapezoidal) quadrature after the
substitution tau = e^t, which converges exponentially:

    1/a^3 ~= sum_l W_l exp(-s_l^2 a^2),  s_l = e^{t_l},  W_l = (4 h / sqrt(pi)) e^{3 t_l},

and on a tensor-product grid the potential becomes the block sum of mode
products of Eq. "sumpot":

    Phi = (1/4pi) sum_l W_l sum_p M^(p) x_1 D_1^(l,p) x_2 D_2^(l,p) x_3 D_3^(l,p),

with the Gaussian matrices of Eqs. "Dmat" and "gs" (target cell centre x_i,
source cell j on the axis):

    q != p:  d_ij = Int_{cell j} exp(-s^2 (x_i - x')^2) dx'
    q == p:  d_ij = Int_{cell j} (x_i - x') exp(-s^2 (x_i - x')^2) dx'

evaluated here in closed form (erf and exp). The field is H = -grad Phi by
second-order finite differences at the cell centres: central differences
inside, the one-sided second-order formula at the first and last cell of each
axis (a reading: the paper names the order only; with it the TG energies of
the paper's cube and thin-film tables are reproduced to the printed digits).

Low-rank magnetization (App. A): a CP tensor sum_m lambda_m u_m o v_m o w_m
goes through the mode products factor by factor, (u o v o w) x_1 A x_2 B x_3 C
= (A u) o (B v) o (C w), so the potential is a block-CP tensor whose dense
values are sums over (l, p, m) of products of three vectors.

Layout: M is (3, nz, ny, nx); potentials (nz, ny, nx); CP factors per
component p: lam[p] (r,), U[p] = (Ux (nx, r), Uy (ny, r), Uz (nz, r)).
Uniform cells only (the method allows any tensor grid; the library builds
the uniform one).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def sinc_rule(a_min: float, a_max: float, h: float = 0.08, tail: float = 12.0):
    """Nodes s_l and weights W_l with 1/a^3 ~= sum_l W_l exp(-s_l^2 a^2) on
    [a_min, a_max]: trapezoidal rule in t (tau = e^t) with step h on
    [-ln(a_max) - tail, ln(6 / a_min) + 1]."""
    t0 = -math.log(a_max) - tail
    t1 = math.log(6.0 / a_min) + 1.0
    n = int(math.ceil((t1 - t0) / h)) + 1
    t = t0 + h * np.arange(n)
    return np.exp(t), (4.0 * h / math.sqrt(math.pi)) * np.exp(3.0 * t)


def gauss_matrix(n: int, d: float, s: float, odd: bool) -> np.ndarray:
    """D[i, j] for centres x_i = (i + 1/2) d and cells [j d, (j + 1) d]."""
    x = (np.arange(n) + 0.5) * d
    lo = np.arange(n) * d
    hi = lo + d
    X = x[:, None]
    if odd:
        return (np.exp(-(s * (X - hi[None, :])) ** 2) - np.exp(-(s * (X - lo[None, :])) ** 2)) / (2.0 * s * s)
    return (math.sqrt(math.pi) / (2.0 * s)) * (erf(s * (X - lo[None, :])) - erf(s * (X - hi[None, :])))


def _rule_for(n, d, h):
    dmin, L = min(d), math.sqrt(sum((a * b) ** 2 for a, b in zip(n, d)))
    return sinc_rule(0.5 * dmin, 2.0 * L, h)


def tg_potential_dense(M: np.ndarray, d, h: float = 0.08) -> np.ndarray:
    """Phi at the cell centres from a dense M (Eq. "sumpot"), shape (nz, ny, nx)."""
    M = np.asarray(M, dtype=np.float64)
    _, nz, ny, nx = M.shape
    n = (nx, ny, nz)
    s, W = _rule_for(n, d, h)
    phi = np.zeros((nz, ny, nx))
    for sl, wl in zip(s, W):
        G = [gauss_matrix(n[q], d[q], sl, False) for q in range(3)]
        O = [gauss_matrix(n[q], d[q], sl, True) for q in range(3)]
        for p in range(3):
            Dx = O[0] if p == 0 else G[0]
            Dy = O[1] if p == 1 else G[1]
            Dz = O[2] if p == 2 else G[2]
            T = np.einsum("kja,ia->kji", M[p], Dx)
            T = np.einsum("kbi,jb->kji", T, Dy)
            T = np.einsum("cji,kc->kji", T, Dz)
            phi += wl * T
    return phi / (4.0 * math.pi)


def cp_to_dense(lam, Ux, Uy, Uz) -> np.ndarray:
    """Dense (nz, ny, nx) tensor of a CP tensor (App. A, Eq. "CP")."""
    return np.einsum("m,im,jm,km->kji", np.asarray(lam, float), Ux, Uy, Uz)


def tg_potential_cp(cp, d, n, h: float = 0.08) -> np.ndarray:
    """Phi from CP factors per component: cp[p] = (lam, Ux, Uy, Uz). The mode
    products act on the factors (A u_m, B v_m, C w_m); the block-CP result is
    then summed densely."""
    nx, ny, nz = n
    s, W = _rule_for(n, d, h)
    phi = np.zeros((nz, ny, nx))
    for sl, wl in zip(s, W):
        G = [gauss_matrix(n[q], d[q], sl, False) for q in range(3)]
        O = [gauss_matrix(n[q], d[q], sl, True) for q in range(3)]
        for p in range(3):
            lam, Ux, Uy, Uz = cp[p]
            A = (O[0] if p == 0 else G[0]) @ Ux
            B = (O[1] if p == 1 else G[1]) @ Uy
            C = (O[2] if p == 2 else G[2]) @ Uz
            phi += wl * cp_to_dense(lam, A, B, C)
    return phi / (4.0 * math.pi)


def cell_potential_direct(M: np.ndarray, d, kernel) -> np.ndarray:
    """Exact Phi at the cell centres by the direct sum over cells of M . S,
    S the potential of one homogeneously magnetized cell (``kernel(R, d)``,
    e.g. ``oracle.sp_kernel``) at integer-cell offsets. Tiny grids only."""
    M = np.asarray(M, dtype=np.float64)
    _, nz, ny, nx = M.shape
    phi = np.zeros((nz, ny, nx))
    cache = {}
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                acc = 0.0
                for c in range(nz):
                    for b in range(ny):
                        for a in range(nx):
                            key = (i - a, j - b, k - c)
                            if key not in cache:
                                cache[key] = kernel((key[0] * d[0], key[1] * d[1], key[2] * d[2]), d)
                            acc += float(np.dot(cache[key], M[:, c, b, a]))
                phi[k, j, i] = acc
    return phi


def tg_field_from_potential(phi: np.ndarray, d) -> np.ndarray:
    """H = -grad Phi at the cell centres, second order: central differences
    inside, (-3 f0 + 4 f1 - f2) / (2h) and its mirror at the ends. Needs at
    least 3 cells per axis."""
    phi = np.asarray(phi, dtype=np.float64)
    if min(phi.shape) < 3:
        raise ValueError("second-order one-sided differences need 3 cells per axis")
    H = np.zeros((3,) + phi.shape)
    for c, (axis, h) in enumerate(((2, d[0]), (1, d[1]), (0, d[2]))):
        f = np.moveaxis(phi, axis, -1)
        g = np.empty_like(f)
        g[..., 1:-1] = (f[..., 2:] - f[..., :-2]) / (2 * h)
        g[..., 0] = (-3 * f[..., 0] + 4 * f[..., 1] - f[..., 2]) / (2 * h)
        g[..., -1] = (3 * f[..., -1] - 4 * f[..., -2] + f[..., -3]) / (2 * h)
        H[c] = -np.moveaxis(g, -1, axis)
    return H


def cell_kernel_octant(n, d, kernel) -> np.ndarray:
    """(3, nz, ny, nx): S(i dx, j dy, k dz) for 0 <= i < nx etc. (S_x odd in
    x and even in y, z; likewise for S_y, S_z)."""
    nx, ny, nz = (int(v) for v in n)
    out = np.zeros((3, nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                out[:, k, j, i] = kernel((i * d[0], j * d[1], k * d[2]), d)
    return out


def cell_potential_fft(M: np.ndarray, d, kernel, octant=None) -> np.ndarray:
    """Exact Phi at the cell centres as a zero-padded float64 FFT convolution
    of M with S at integer-cell offsets (period >= 2n - 1 per axis)."""
    M = np.asarray(M, dtype=np.float64)
    _, nz, ny, nx = M.shape
    n = (nx, ny, nz)
    P = []
    for v in n:
        p = 1
        while p < 2 * v - 1:
            p *= 2
        P.append(p)
    if octant is None:
        octant = cell_kernel_octant(n, d, kernel)
    W = np.zeros((3, P[2], P[1], P[0]))
    for sz in (1, -1):
        for sy in (1, -1):
            for sx in (1, -1):
                ix = np.arange(nx) if sx > 0 else np.arange(1, nx)
                iy = np.arange(ny) if sy > 0 else np.arange(1, ny)
                iz = np.arange(nz) if sz > 0 else np.arange(1, nz)
                if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
                    continue
                px = ix if sx > 0 else P[0] - ix
                py = iy if sy > 0 else P[1] - iy
                pz = iz if sz > 0 else P[2] - iz
                signs = (sx, sy, sz)
                for c in range(3):
                    W[c][np.ix_(pz, py, px)] = signs[c] * octant[c][np.ix_(iz, iy, ix)]
    Sh = np.fft.rfftn(W, axes=(1, 2, 3))
    Mh = np.fft.rfftn(M, s=(P[2], P[1], P[0]), axes=(1, 2, 3))
    phi = np.fft.irfftn(Sh[0] * Mh[0] + Sh[1] * Mh[1] + Sh[2] * Mh[2], s=(P[2], P[1], P[0]), axes=(0, 1, 2))
    return np.ascontiguousarray(phi[:nz, :ny, :nx])
