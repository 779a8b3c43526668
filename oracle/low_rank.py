"""FP64 CPU oracle of the low-rank magnetization approximations of the
tensor-grid method (paper Sec. 3.2, "Low-Rank Magnetization"): each
component M^(p) (a 3-way tensor) in CP or in Tucker format, found by
alternating least squares (the paper uses the ALS algorithms of Kolda and
Bader's tensor survey for both formats), with the relative error of
Eq. "relr" (Frobenius norms over the three components).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke
check and the CPU legs of the benchmark import it; the CUDA library shares no
code with it.

Layout: a component X is (nz, ny, nx) (x fastest, as M[p]); factor matrices
are A (nx, r), B (ny, r), C (nz, r) with rows indexed by the cell along the
axis; the initial guesses are inputs (the paper starts from random ones).

CP-ALS (one sweep = the three mode updates in the order x, y, z):
    A <- X_(x) (C kr B) V^+,   V = (C^T C) * (B^T B)   (* = Hadamard product,
                                                      kr = Khatri-Rao product)
    lambda <- column 2-norms of A, A <- A / lambda
    the same for B (V = (C^T C) * (A^T A)) and C (V = (B^T B) * (A^T A)),
lambda ending as the column norms of the last update. X_(x) (C kr B) is the
MTTKRP sum_{k,j} X[k,j,i] B[j,m] C[k,m]; V is symmetric positive definite
when the factors have full column rank, and V^+ is then V^-1 (here the
pseudo-inverse through the eigen-decomposition of V, which stays defined
when the rank asked for exceeds what the tensor holds).

Tucker-ALS (higher-order orthogonal iteration), one sweep:
    A <- r1 leading left singular vectors of (X x_y B^T x_z C^T)_(x)
    B <- r2 leading ones of (X x_x A^T x_z C^T)_(y)
    C <- r3 leading ones of (X x_x A^T x_y B^T)_(z)
and the core G = X x_x A^T x_y B^T x_z C^T after the last sweep. The
approximation A, B, C, G is unique up to rotations within the factor
subspaces (the projectors A A^T are unique when the singular values at each
cut are separated); its reconstruction is unique.
"""
from __future__ import annotations

import numpy as np


def cp_reconstruct(lam, A, B, C) -> np.ndarray:
    """X[k, j, i] = sum_m lam[m] A[i, m] B[j, m] C[k, m]."""
    return np.einsum("m,im,jm,km->kji", np.asarray(lam, float), A, B, C)


def mttkrp(X: np.ndarray, F1, F2, mode: str) -> np.ndarray:
    """The matricized tensor times the Khatri-Rao product of the two other
    factors: mode 'x': sum_{k,j} X[k,j,i] F1[j,m] F2[k,m] (F1 = B, F2 = C);
    'y': sum_{k,i} X[k,j,i] F1[i,m] F2[k,m] (A, C); 'z': sum_{j,i} X[k,j,i]
    F1[i,m] F2[j,m] (A, B)."""
    spec = {"x": "kji,jm,km->im", "y": "kji,im,km->jm", "z": "kji,im,jm->km"}[mode]
    return np.einsum(spec, X, F1, F2)


def _normalize(F):
    lam = np.linalg.norm(F, axis=0)
    safe = np.where(lam > 0, lam, 1.0)
    return F / safe, lam


PINV_RCOND = 1e-12


def pinv_sym(V: np.ndarray, rcond: float = PINV_RCOND) -> np.ndarray:
    """Pseudo-inverse of the symmetric positive semi-definite V through its
    eigen-decomposition, eigenvalues at or below rcond * the largest taken as
    zero (V is singular when the rank exceeds what the tensor holds)."""
    w, Q = np.linalg.eigh(V)
    cut = rcond * (w.max() if w.size else 0.0)
    inv = np.where(w > cut, 1.0 / np.where(w > cut, w, 1.0), 0.0)
    return (Q * inv) @ Q.T


def cp_als(X: np.ndarray, init, iters: int):
    """CP-ALS of one component from the initial factors init = (A, B, C);
    returns (lam, A, B, C) after `iters` sweeps."""
    X = np.asarray(X, dtype=np.float64)
    A, B, C = (np.array(f, dtype=np.float64) for f in init)
    lam = np.ones(A.shape[1])
    for _ in range(iters):
        A = mttkrp(X, B, C, "x") @ pinv_sym((C.T @ C) * (B.T @ B))
        A, lam = _normalize(A)
        B = mttkrp(X, A, C, "y") @ pinv_sym((C.T @ C) * (A.T @ A))
        B, lam = _normalize(B)
        C = mttkrp(X, A, B, "z") @ pinv_sym((B.T @ B) * (A.T @ A))
        C, lam = _normalize(C)
    return lam, A, B, C


def ttm(X: np.ndarray, F: np.ndarray, mode: str) -> np.ndarray:
    """Mode product with the transposed factor, X x_mode F^T: the axis of
    `mode` (length n) becomes r (F is (n, r)); layout (z, y, x) kept."""
    spec = {"x": "kji,ia->kja", "y": "kji,jb->kbi", "z": "kji,kc->cji"}[mode]
    return np.einsum(spec, X, F)


def leading_left_singular_vectors(Y: np.ndarray, mode: str, r: int) -> np.ndarray:
    """The r leading left singular vectors of the mode unfolding of Y."""
    axis = {"x": 2, "y": 1, "z": 0}[mode]
    unf = np.moveaxis(Y, axis, 0).reshape(Y.shape[axis], -1)
    U, _, _ = np.linalg.svd(unf, full_matrices=False)
    return U[:, :r]


def tucker_core(X, A, B, C) -> np.ndarray:
    """G[c, b, a] = sum X[k, j, i] A[i, a] B[j, b] C[k, c] (layout (r3, r2, r1))."""
    return ttm(ttm(ttm(X, A, "x"), B, "y"), C, "z")


def tucker_reconstruct(G, A, B, C) -> np.ndarray:
    """X[k, j, i] = sum G[c, b, a] A[i, a] B[j, b] C[k, c]."""
    return np.einsum("cba,ia,jb,kc->kji", G, A, B, C)


def tucker_als(X: np.ndarray, init, iters: int):
    """Tucker-ALS (HOOI) of one component from init = (A, B, C); the initial
    A is not read (the first mode update uses B and C only) and no factor
    needs orthonormal columns. Returns (G, A, B, C) after `iters` sweeps."""
    X = np.asarray(X, dtype=np.float64)
    A, B, C = (np.array(f, dtype=np.float64) for f in init)
    r1, r2, r3 = A.shape[1], B.shape[1], C.shape[1]
    for _ in range(iters):
        A = leading_left_singular_vectors(ttm(ttm(X, B, "y"), C, "z"), "x", r1)
        B = leading_left_singular_vectors(ttm(ttm(X, A, "x"), C, "z"), "y", r2)
        C = leading_left_singular_vectors(ttm(ttm(X, A, "x"), B, "y"), "z", r3)
    return tucker_core(X, A, B, C), A, B, C


def relerr(M: np.ndarray, L: np.ndarray) -> float:
    """Eq. "relr": sqrt(sum_p ||M^(p) - L^(p)||_F^2) / sqrt(sum_p ||M^(p)||_F^2)."""
    M = np.asarray(M, dtype=np.float64)
    return float(np.sqrt(np.sum((M - L) ** 2)) / np.sqrt(np.sum(M ** 2)))
