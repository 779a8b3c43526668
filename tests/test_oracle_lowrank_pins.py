"""Pins for the low-rank oracle (CP-ALS and Tucker-ALS of paper Sec. 3.2,
"Low-Rank Magnetization"; relative error of Eq. "relr"): the contractions
against loops, exact recovery of tensors of exactly the asked rank, a rank-one
tensor after one sweep, the monotone decrease of the ALS error, the
orthogonal-projection identity of Tucker, the symmetric pseudo-inverse
against numpy's, Eq. relr against the pinned rel-RMS, and the paper's TG
energies of the flower (CP rank 6) and vortex (Tucker rank 10) cubes
recovered from ALS-compressed states."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import low_rank as lr
from oracle import tensor_grid as tg
from paper_1204_4302_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_mttkrp_and_ttm_against_loops():
    nz, ny, nx, r = 3, 4, 5, 2
    X = _rand((nz, ny, nx), 1)
    A, B, C = _rand((nx, r), 2), _rand((ny, r), 3), _rand((nz, r), 4)
    ex = np.zeros((nx, r)); ey = np.zeros((ny, r)); ez = np.zeros((nz, r))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for m in range(r):
                    ex[i, m] += X[k, j, i] * B[j, m] * C[k, m]
                    ey[j, m] += X[k, j, i] * A[i, m] * C[k, m]
                    ez[k, m] += X[k, j, i] * A[i, m] * B[j, m]
    assert np.allclose(lr.mttkrp(X, B, C, "x"), ex, rtol=1e-14, atol=1e-14)
    assert np.allclose(lr.mttkrp(X, A, C, "y"), ey, rtol=1e-14, atol=1e-14)
    assert np.allclose(lr.mttkrp(X, A, B, "z"), ez, rtol=1e-14, atol=1e-14)
    tx = np.zeros((nz, ny, r))
    for k in range(nz):
        for j in range(ny):
            for a in range(r):
                tx[k, j, a] = sum(X[k, j, i] * A[i, a] for i in range(nx))
    assert np.allclose(lr.ttm(X, A, "x"), tx, rtol=1e-14, atol=1e-14)
    ty = np.zeros((nz, r, nx))
    for k in range(nz):
        for b in range(r):
            for i in range(nx):
                ty[k, b, i] = sum(X[k, j, i] * B[j, b] for j in range(ny))
    assert np.allclose(lr.ttm(X, B, "y"), ty, rtol=1e-14, atol=1e-14)
    tz = np.zeros((r, ny, nx))
    for c in range(r):
        for j in range(ny):
            for i in range(nx):
                tz[c, j, i] = sum(X[k, j, i] * C[k, c] for k in range(nz))
    assert np.allclose(lr.ttm(X, C, "z"), tz, rtol=1e-14, atol=1e-14)
    # CP and Tucker reconstructions against loops
    lam = np.array([2.0, -0.5])
    G = _rand((r, r, r), 5)
    cp = np.zeros((nz, ny, nx)); tk = np.zeros((nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                cp[k, j, i] = sum(lam[m] * A[i, m] * B[j, m] * C[k, m] for m in range(r))
                tk[k, j, i] = sum(G[c, b, a] * A[i, a] * B[j, b] * C[k, c]
                                  for a in range(r) for b in range(r) for c in range(r))
    assert np.allclose(lr.cp_reconstruct(lam, A, B, C), cp, rtol=1e-14, atol=1e-14)
    assert np.allclose(lr.tucker_reconstruct(G, A, B, C), tk, rtol=1e-14, atol=1e-14)


def test_pinv_sym_against_numpy():
    Q = np.linalg.qr(_rand((6, 6), 7))[0]
    w = np.array([3.0, 2.0, 1.0, 0.5, 1e-20, 0.0])
    V = (Q * w) @ Q.T
    assert np.allclose(lr.pinv_sym(V), np.linalg.pinv(V, rcond=1e-12, hermitian=True), atol=1e-12)
    S = _rand((5, 5), 8)
    S = S @ S.T + 5 * np.eye(5)
    assert np.allclose(lr.pinv_sym(S), np.linalg.inv(S), rtol=1e-12, atol=1e-13)


def test_cp_als_recovers_an_exact_rank_r_tensor():
    n, r = (9, 7, 6), 3
    A0, B0, C0 = (_rand((v, r), 10 + q) for q, v in enumerate(n))
    lam0 = np.array([3.0, 2.0, 1.0])
    X = lr.cp_reconstruct(lam0, A0, B0, C0)
    init = [F + 0.1 * _rand(F.shape, 20 + q) for q, F in enumerate((A0, B0, C0))]
    lam, A, B, C = lr.cp_als(X, init, 200)
    assert lr.relerr(X[None], lr.cp_reconstruct(lam, A, B, C)[None]) < 1e-10
    assert np.allclose(np.linalg.norm(A, axis=0), 1.0)


def test_cp_als_rank_one_after_one_sweep():
    n = (8, 5, 4)
    u, v, w = (_rand(k, 30 + q) for q, k in enumerate(n))
    X = np.einsum("i,j,k->kji", u, v, w)
    init = [_rand((k, 1), 40 + q) for q, k in enumerate(n)]
    lam, A, B, C = lr.cp_als(X, init, 1)
    assert lr.relerr(X[None], lr.cp_reconstruct(lam, A, B, C)[None]) < 1e-13
    assert abs(lam[0] - np.linalg.norm(u) * np.linalg.norm(v) * np.linalg.norm(w)) < 1e-12 * lam[0]


def test_cp_als_error_does_not_increase():
    X = _rand((6, 7, 8), 50)
    f = [_rand((k, 4), 60 + q) for q, k in enumerate((8, 7, 6))]
    errs = []
    for _ in range(12):
        lam, A, B, C = lr.cp_als(X, f, 1)
        f = [A, B, C]
        errs.append(lr.relerr(X[None], lr.cp_reconstruct(lam, A, B, C)[None]))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:])), errs


def test_tucker_full_rank_and_exact_multilinear_rank():
    X = _rand((5, 6, 7), 70)
    init = [_rand((k, k), 71 + q) for q, k in enumerate((7, 6, 5))]
    G, A, B, C = lr.tucker_als(X, init, 1)
    assert lr.relerr(X[None], lr.tucker_reconstruct(G, A, B, C)[None]) < 1e-13
    # multilinear rank (2, 3, 2)
    G0 = _rand((2, 3, 2), 72)
    A0, B0, C0 = _rand((9, 2), 73), _rand((8, 3), 74), _rand((7, 2), 75)
    Y = lr.tucker_reconstruct(G0, A0, B0, C0)
    init = [_rand((9, 2), 76), _rand((8, 3), 77), _rand((7, 2), 78)]
    G, A, B, C = lr.tucker_als(Y, init, 2)
    assert lr.relerr(Y[None], lr.tucker_reconstruct(G, A, B, C)[None]) < 1e-13
    assert np.allclose(A.T @ A, np.eye(2), atol=1e-13)


def test_tucker_orthogonal_projection_identity():
    """||X||^2 = ||G||^2 + ||X - X^||^2 for orthonormal factors, and the error
    does not increase from sweep to sweep."""
    X = _rand((8, 9, 10), 80)
    f = [_rand((k, 3), 81 + q) for q, k in enumerate((10, 9, 8))]
    errs = []
    for _ in range(6):
        G, A, B, C = lr.tucker_als(X, f, 1)
        f = [A, B, C]
        L = lr.tucker_reconstruct(G, A, B, C)
        assert abs(np.sum(X ** 2) - np.sum(G ** 2) - np.sum((X - L) ** 2)) < 1e-12 * np.sum(X ** 2)
        errs.append(lr.relerr(X[None], L[None]))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:])), errs


def test_relr_is_the_pinned_rel_rms():
    M = _rand((3, 4, 5, 6), 90)
    L = M + 0.01 * _rand(M.shape, 91)
    assert abs(lr.relerr(M, L) - oracle.rel_errors(L, M)["rel_rms"]) < 1e-15


@pytest.mark.parametrize("name,fmt,rank", [("cube_flower", "cp", 6), ("cube_vortex", "tucker", 10)])
def test_paper_tg_energies_from_als_compressed_states(name, fmt, rank):
    """The paper's TG rows use low-rank states (flower: CP rank 6; vortex:
    Tucker rank 10, Tables cube_flower and cube_vortex); the TG energy of the
    ALS approximation (random initial guesses, seed 5) reproduces the printed
    values to their four digits."""
    with open(os.path.join(GOLDEN, "paper_tg_energies.json")) as fh:
        case = {c["name"]: c for c in json.load(fh)["cases"]}[name]
    n = tuple(case["grid"])
    d = tuple(e / k for e, k in zip(case["extent"], n))
    M = inputs.flower(n, tuple(case["extent"])) if case["state"] == "flower" else \
        inputs.vortex(n, tuple(case["extent"]), rc=0.14)
    rng = np.random.default_rng(5)
    L = np.zeros_like(M)
    for p in range(3):
        init = [rng.standard_normal((v, rank)) for v in n]
        if fmt == "cp":
            lam, A, B, C = lr.cp_als(M[p], init, 60)
            L[p] = lr.cp_reconstruct(lam, A, B, C)
        else:
            G, A, B, C = lr.tucker_als(M[p], init, 10)
            L[p] = lr.tucker_reconstruct(G, A, B, C)
    assert lr.relerr(M, L) < 1e-4
    phi = tg.cell_potential_fft(L, d, oracle.sp_kernel)
    e = oracle.energy_reduced(L, tg.tg_field_from_potential(phi, d), d)
    mag = 10 ** (math.floor(math.log10(abs(case["e"]))) - case["digits"] + 1)
    assert abs(e - case["e"]) <= 0.5 * mag, e
