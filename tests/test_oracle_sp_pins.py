"""Pins for the scalar-potential (SP) oracle: its cell kernel S, the FFT
potential and the finite-difference field, each checked against something
other than the oracle's own formulas: textbook integrals, an independent
quadrature, the dipole limit, the demagnetization tensor of the DM oracle
(pinned on its own), direct sums, exact polynomial cases and the SP energies
the paper prints.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1204_4302_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LN1P2 = math.log(1.0 + math.sqrt(2.0))


# ------------------------------------------------------------ rectangle integral
def test_rect_integral_textbook_values():
    """Int over a square of side s of 1/r, seen from a corner in its plane, is
    2 s ln(1 + sqrt 2); from the centre, 4 such squares of side s/2. Catches a
    wrong corner sign or a dropped log term of the antiderivative."""
    for s in (1.0, 0.3, 7.0):
        h = s / 2
        assert oracle.sp_rect(0.0, h, h, h, h) == pytest.approx(2 * s * LN1P2, rel=1e-14)
        assert oracle.sp_rect(0.0, 0.0, 0.0, h, h) == pytest.approx(4 * s * LN1P2, rel=1e-14)


@pytest.mark.parametrize("a,V,W,hv,hw", [(0.7, 0.1, -0.2, 0.5, 0.4), (2.0, 3.0, 1.0, 0.5, 0.5),
                                          (-1.5, 0.0, 0.0, 1.0, 0.25), (0.3, 2.0, -2.5, 0.6, 0.9)])
def test_rect_integral_vs_quadrature(a, V, W, hv, hw):
    """Off the plane the integrand is smooth: a 2-D Gauss-Legendre rule agrees
    with the closed form. Catches a wrong atan term (it is what carries the
    dependence on the distance a)."""
    x, w = oracle.gl_rule(60)
    v = hv * x
    u = hw * x
    VV, UU = np.meshgrid(v, u, indexing="ij")
    f = 1.0 / np.sqrt(a * a + (V - VV) ** 2 + (W - UU) ** 2)
    q = hv * hw * np.einsum("i,j,ij->", w, w, f)
    assert oracle.sp_rect(a, V, W, hv, hw) == pytest.approx(q, rel=1e-13)


# ------------------------------------------------------------ the cell kernel S
D_CASES = [(1.0, 1.0, 1.0), (1.0, 1.3, 0.7), (2e-9, 2e-9, 5e-10)]


@pytest.mark.parametrize("d", D_CASES)
@pytest.mark.parametrize("R", [(3.5, 0.5, 0.5), (2.5, -1.5, 0.5), (4.5, 2.5, -3.5), (0.5, 3.5, -0.5),
                               (-2.5, 2.5, 2.5), (1.0, 0.2, 4.0)])
def test_kernel_closed_form_vs_volume_quadrature(R, d):
    """Two independent forms of S (face integrals in closed form; GL of the
    volume integrand (R - u)/|R - u|^3) agree away from the cell. Catches a
    swapped face sign or a permuted axis in either."""
    Rv = tuple(r * e for r, e in zip(R, d))
    a = oracle.sp_kernel_closed(Rv, d)
    b = oracle.sp_kernel_quad(Rv, d)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_kernel_parity_and_centre():
    """S_x is odd in X and even in Y and Z (likewise for y, z); at the cell
    centre S = 0 by symmetry."""
    d = (1.0, 1.3, 0.7)
    R = np.array([1.5, 0.5, 2.5]) * d
    s = oracle.sp_kernel(R, d)
    for ax in range(3):
        f = np.ones(3)
        f[ax] = -1
        t = oracle.sp_kernel(R * f, d)
        exp = s.copy()
        exp[ax] = -exp[ax]
        np.testing.assert_allclose(t, exp, rtol=1e-13, atol=1e-18)
    np.testing.assert_allclose(oracle.sp_kernel((0, 0, 0), d), 0.0, atol=1e-15)


def test_kernel_dipole_limit():
    """Far away a magnetized cell is a point dipole: S(R) -> V R / (4 pi |R|^3),
    with a relative correction of order (d/R)^2."""
    d = (1.0, 1.3, 0.7)
    V = d[0] * d[1] * d[2]
    for R in [(1000.0, 300.0, -200.0), (0.0, 0.0, 2000.0)]:
        R = np.array(R)
        r = np.linalg.norm(R)
        dip = V * R / (4 * math.pi * r ** 3)
        s = oracle.sp_kernel(R, d)
        assert np.max(np.abs(s - dip)) <= 1e-5 * np.max(np.abs(dip))


@pytest.mark.parametrize("d", [(1.0, 1.0, 1.0), (1.0, 1.3, 0.7)])
@pytest.mark.parametrize("R", [(3, 0, 0), (3, 1, 2), (-2, 3, 1), (0, 0, 4), (2, -2, -3)])
def test_face_average_of_kernel_is_the_demag_tensor(R, d):
    """H = -grad phi with phi = S . M, so the point tensor is d_k S_j, and its
    average over a target cell is (1/V) times the difference of the integrals
    of S_j over the target's two faces normal to k. At separated cells this
    must reproduce the DM oracle's cell-averaged tensor, which the DM pins
    fix on their own (Newell closed form, Aharoni prism factors). Catches a
    sign, an axis permutation or a wrong normalisation of S."""
    R = np.array(R, dtype=float) * np.array(d)
    V = d[0] * d[1] * d[2]
    x, w = oracle.gl_rule(14)
    Nsp = np.zeros((3, 3))
    for k in range(3):
        a, b = [ax for ax in range(3) if ax != k]
        ua, ub = 0.5 * d[a] * x, 0.5 * d[b] * x
        wab = np.outer(w, w) * (0.25 * d[a] * d[b])
        for side in (+1, -1):
            acc = np.zeros(3)
            for i in range(len(x)):
                for j in range(len(x)):
                    t = np.zeros(3)
                    t[k] = side * 0.5 * d[k]
                    t[a] = ua[i]
                    t[b] = ub[j]
                    acc += wab[i, j] * oracle.sp_kernel(R + t, d)
            Nsp[k] += side * acc / V
    t6 = oracle.cell_tensor(R, d)
    Ndm = np.array([[t6[0], t6[3], t6[4]], [t6[3], t6[1], t6[5]], [t6[4], t6[5], t6[2]]])
    assert np.max(np.abs(Nsp - Ndm)) <= 1e-10 * np.max(np.abs(Ndm))


# ------------------------------------------------------------ potential and field
@pytest.mark.parametrize("n", [(1, 1, 1), (3, 2, 4), (2, 1, 3), (5, 3, 2), (4, 4, 1)])
def test_fft_potential_matches_direct_sum(n):
    """Zero-padded FFT convolution with the wrapped half-integer kernel equals
    the direct sum over cells at every node, ragged sizes and single layers
    included. Catches a wrap-around index or parity-sign mistake."""
    rng = np.random.default_rng(sum(n))
    d = (1.0, 0.8, 1.3)
    M = rng.standard_normal((3, n[2], n[1], n[0]))
    a = oracle.sp_potential_bruteforce(M, d)
    b = oracle.sp_potential_fft(M, d)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
    # any larger power-of-two period gives the same potential
    P = tuple(2 * oracle.sp_padded_size(v) for v in n)
    c = oracle.sp_potential_fft(M, d, P=P)
    assert np.max(np.abs(c - a)) <= 1e-13 * np.max(np.abs(a))


def test_uniform_body_potential_is_the_body_potential():
    """Superposition: for uniform M the node potential is that of the whole
    box, (1/4pi) M_j times the difference of the integrals of 1/|r - r'| over
    the box's two faces normal to j, evaluated once for the whole body."""
    n, d = (6, 5, 3), (1.0, 0.8, 1.3)
    mv = np.array([0.3, -0.5, 0.8])
    M = np.empty((3, n[2], n[1], n[0]))
    for c in range(3):
        M[c] = mv[c]
    phi = oracle.sp_potential_fft(M, d)
    L = np.array(n) * np.array(d)
    for (i, j, k) in [(0, 0, 0), (6, 5, 3), (3, 2, 1), (6, 0, 2), (1, 4, 3)]:
        r = np.array([i, j, k]) * np.array(d) - L / 2
        s = 0.0
        for ax in range(3):
            a, b = [q for q in range(3) if q != ax]
            plus = oracle.sp_rect(r[ax] - L[ax] / 2, r[a], r[b], L[a] / 2, L[b] / 2)
            minus = oracle.sp_rect(r[ax] + L[ax] / 2, r[a], r[b], L[a] / 2, L[b] / 2)
            s += mv[ax] * (plus - minus) / (4 * math.pi)
        assert phi[k, j, i] == pytest.approx(s, rel=1e-12, abs=1e-14)


def test_fd_field_is_exact_for_quadratic_potentials():
    """The cell average of -grad of the trilinear interpolant is exact when phi
    is a quadratic polynomial: -grad phi at the cell centre. Catches a wrong
    edge set, a missing 1/4 or a wrong spacing per axis."""
    rng = np.random.default_rng(3)
    n, d = (5, 4, 3), (0.7, 1.1, 1.9)
    c = rng.standard_normal(10)
    k, j, i = np.meshgrid(*(np.arange(v + 1) for v in (n[2], n[1], n[0])), indexing="ij")
    x, y, z = i * d[0], j * d[1], k * d[2]

    def phi_of(x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
                + c[7] * x * y + c[8] * x * z + c[9] * y * z)

    H = oracle.sp_field_from_potential(phi_of(x, y, z), d)
    kc, jc, ic = np.meshgrid(*(np.arange(v) + 0.5 for v in (n[2], n[1], n[0])), indexing="ij")
    xc, yc, zc = ic * d[0], jc * d[1], kc * d[2]
    gx = c[1] + 2 * c[4] * xc + c[7] * yc + c[8] * zc
    gy = c[2] + 2 * c[5] * yc + c[7] * xc + c[9] * zc
    gz = c[3] + 2 * c[6] * zc + c[8] * xc + c[9] * yc
    np.testing.assert_allclose(H, -np.stack([gx, gy, gz]), rtol=0, atol=1e-12)


def test_sp_field_of_uniform_film_interior():
    """A single-layer film (nz = 1) magnetized out of plane: far from the edges
    the potential drops by M dz across the layer, so H_z = -M there (the thin
    film limit), to within the edge influence at the film's centre."""
    n, d = (64, 64, 1), (1.0, 1.0, 0.05)
    M = np.zeros((3, 1, 64, 64))
    M[2] = 1.0
    H = oracle.sp_field(M, d)
    assert H[2, 0, 32, 32] == pytest.approx(-1.0, abs=2e-3)
    assert abs(H[0, 0, 32, 32]) < 1e-12 and abs(H[1, 0, 32, 32]) < 1e-12


# ------------------------------------------------------------ paper values
def _state(case, n):
    ext = tuple(case["extent"])
    if case["state"] == "uniform_z":
        return inputs.uniform(n, (0, 0, 1))
    if case["state"] == "flower":
        return inputs.flower(n, ext)
    if case["state"] == "vortex":
        return inputs.vortex(n, ext, rc=0.14)
    raise KeyError(case["state"])


def test_paper_sp_energies():
    """The SP energies of the paper's cube and thin-film tables
    (tests/golden/paper_sp_energies.json), to the printed digits. These fix the
    readings of the discretisation (node potential, cell-averaged difference
    field): a potential at the cell centres with central or one-sided
    differences misses several of them."""
    with open(os.path.join(GOLDEN, "paper_sp_energies.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        n = tuple(case["grid"])
        d = tuple(e / k for e, k in zip(case["extent"], n))
        m = _state(case, n)
        e = oracle.energy_reduced(m, oracle.sp_field(m, d), d)
        digits = case["digits"]
        if "relerr_vs_exact" in case:
            val, ref = abs(e - case["exact"]) / case["exact"], case["relerr_vs_exact"]
        else:
            val, ref = e, case["e"]
        mag = 10 ** (math.floor(math.log10(abs(ref))) - digits + 1)
        assert abs(val - ref) <= 0.5 * mag, (case["name"], val)
