"""Pins for the tensor-grid (TG) oracle: the sinc rule against 1/a^3, the
Gaussian matrices against quadrature, the TG potential against the exact
cell-centre potential of the separately pinned SP kernel (direct sum and
FFT), CP factor paths against dense ones, the finite differences on exact
polynomials, and the TG energies the paper prints."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import tensor_grid as tg
from paper_1204_4302_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("h", [0.08, 0.12])
def test_sinc_rule_reproduces_inverse_cube(h):
    """sum_l W_l exp(-s_l^2 a^2) = 1/a^3 (the Gaussian integral of Eq.
    "transform" with tau = e^t) over four decades of a."""
    s, W = tg.sinc_rule(0.25, 2000.0, h)
    a = np.geomspace(0.25, 2000.0, 400)
    approx = (W[None, :] * np.exp(-(s[None, :] * a[:, None]) ** 2)).sum(1)
    assert np.max(np.abs(approx * a ** 3 - 1.0)) < 1e-13


@pytest.mark.parametrize("s", [0.05, 0.7, 3.0, 20.0])
@pytest.mark.parametrize("odd", [False, True])
def test_gauss_matrix_closed_form_vs_quadrature(s, odd):
    """The erf / exp closed forms of the 1-D cell integrals of Eq. "gs" against
    Gauss-Legendre quadrature of the integrand over each cell (the diagonal
    cells of the odd kind vanish by symmetry)."""
    n, d = 7, 0.8
    D = tg.gauss_matrix(n, d, s, odd)
    x, w = oracle.gl_rule(60)
    ref = np.zeros((n, n))
    for i in range(n):
        xi = (i + 0.5) * d
        for j in range(n):
            xp = (j + 0.5) * d + 0.5 * d * x
            f = np.exp(-(s * (xi - xp)) ** 2)
            if odd:
                f = f * (xi - xp)
            ref[i, j] = 0.5 * d * np.sum(w * f)
    assert np.max(np.abs(D - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    if odd:
        np.testing.assert_allclose(np.diag(D), 0.0, atol=1e-15)


@pytest.mark.parametrize("n,d", [((5, 4, 3), (1.0, 0.8, 1.3)), ((3, 6, 4), (2e-9, 1e-9, 1.5e-9))])
def test_tg_potential_equals_exact_cell_potential(n, d):
    """The TG potential (sinc quadrature + mode products) equals the exact
    potential at the cell centres, the direct sum of M . S with the SP
    oracle's cell kernel S (pinned on its own), to rounding: the method's
    only approximation, the sinc rule, is at machine precision."""
    rng = np.random.default_rng(sum(n))
    M = rng.standard_normal((3, n[2], n[1], n[0]))
    exact = tg.cell_potential_direct(M, d, oracle.sp_kernel)
    phi = tg.tg_potential_dense(M, d)
    assert np.max(np.abs(phi - exact)) <= 1e-12 * np.max(np.abs(exact))
    fft = tg.cell_potential_fft(M, d, oracle.sp_kernel)
    assert np.max(np.abs(fft - exact)) <= 1e-12 * np.max(np.abs(exact))


def test_cp_factor_path_equals_dense_path():
    """Mode products applied to CP factors (App. A) give the dense result of
    the expanded CP tensor."""
    rng = np.random.default_rng(4)
    n, d, r = (6, 5, 4), (1.0, 1.1, 0.9), 3
    cp = []
    M = np.zeros((3, n[2], n[1], n[0]))
    for p in range(3):
        lam = rng.standard_normal(r)
        U = (rng.standard_normal((n[0], r)), rng.standard_normal((n[1], r)), rng.standard_normal((n[2], r)))
        cp.append((lam,) + U)
        M[p] = tg.cp_to_dense(lam, *U)
    a = tg.tg_potential_cp(cp, d, n)
    b = tg.tg_potential_dense(M, d)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


def test_second_order_differences_exact_for_quadratics():
    """Central and one-sided second-order differences are exact for quadratic
    potentials at the cell centres."""
    rng = np.random.default_rng(5)
    n, d = (6, 5, 4), (0.7, 1.3, 0.9)
    c = rng.standard_normal(10)
    k, j, i = np.meshgrid(*(np.arange(v) + 0.5 for v in (n[2], n[1], n[0])), indexing="ij")
    x, y, z = i * d[0], j * d[1], k * d[2]
    phi = (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
           + c[7] * x * y + c[8] * x * z + c[9] * y * z)
    H = tg.tg_field_from_potential(phi, d)
    gx = c[1] + 2 * c[4] * x + c[7] * y + c[8] * z
    gy = c[2] + 2 * c[5] * y + c[7] * x + c[9] * z
    gz = c[3] + 2 * c[6] * z + c[8] * x + c[9] * y
    np.testing.assert_allclose(H, -np.stack([gx, gy, gz]), rtol=0, atol=1e-11)


def _state(case, n):
    ext = tuple(case["extent"])
    if case["state"] == "uniform_z":
        return inputs.uniform(n, (0, 0, 1))
    if case["state"] == "flower":
        return inputs.flower(n, ext)
    return inputs.vortex(n, ext, rc=0.14)


def test_paper_tg_energies():
    """The TG energies the paper prints (tests/golden/paper_tg_energies.json):
    cell-centre potential and second-order differences, to the printed digits."""
    with open(os.path.join(GOLDEN, "paper_tg_energies.json")) as fh:
        cases = json.load(fh)["cases"]
    octs = {}
    for case in cases:
        n = tuple(case["grid"])
        d = tuple(e / k for e, k in zip(case["extent"], n))
        key = (n, d)
        if key not in octs:
            octs[key] = tg.cell_kernel_octant(n, d, oracle.sp_kernel)
        m = _state(case, n)
        phi = tg.cell_potential_fft(m, d, oracle.sp_kernel, octant=octs[key])
        e = oracle.energy_reduced(m, tg.tg_field_from_potential(phi, d), d)
        if "relerr_vs_exact" in case:
            val, ref = abs(e - case["exact"]) / case["exact"], case["relerr_vs_exact"]
        else:
            val, ref = e, case["e"]
        mag = 10 ** (math.floor(math.log10(abs(ref))) - case["digits"] + 1)
        assert abs(val - ref) <= 0.5 * mag, (case["name"], val)
