"""Pins for the FP64 oracle: checks against what the paper and the mathematics
fix, never against the oracle's own formulas retyped.

Each test states what it pins and which plausible mistake it would catch.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1204_4302_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ Gauss-Legendre
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 24, 40, 64])
def test_gl_rule_integrates_polynomials_exactly(n):
    """An n-point Gauss-Legendre rule is exact for degree <= 2n-1: int x^k = 2/(k+1)
    for even k, 0 for odd k (closed form)."""
    x, w = oracle.gl_rule(n)
    assert np.all(np.diff(x) > 0)
    for k in range(0, 2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 2e-14 * max(1.0, n / 8)


# ------------------------------------------------------------ self tensor
def test_self_tensor_cube_is_one_third():
    """Cube: by symmetry Nxx = Nyy = Nzz and the trace is 1, so each is exactly 1/3,
    off-diagonals 0. Catches a sign error or a wrong normalisation of the stencil."""
    t = oracle.cell_tensor((0, 0, 0), (1.0, 1.0, 1.0))
    np.testing.assert_allclose(t[:3], [1 / 3] * 3, rtol=0, atol=1e-15)
    np.testing.assert_allclose(t[3:], 0.0, atol=1e-17)
    t2 = oracle.cell_tensor((0, 0, 0), (2e-9, 2e-9, 2e-9))  # scale invariance (dimensionless)
    np.testing.assert_allclose(t2, t, atol=1e-15)


def _aharoni_dz(a, b, c):
    """Aharoni (J. Appl. Phys. 83, 3432, 1998): demagnetizing factor along the
    c edge of a rectangular prism 2a x 2b x 2c. An independent published closed
    form, not derived from Newell's f."""
    r = math.sqrt(a * a + b * b + c * c)
    ab = math.sqrt(a * a + b * b)
    bc = math.sqrt(b * b + c * c)
    ac = math.sqrt(a * a + c * c)
    s = (b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
    s += (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
    s += b / (2 * c) * math.log((ab + a) / (ab - a))
    s += a / (2 * c) * math.log((ab + b) / (ab - b))
    s += c / (2 * a) * math.log((bc - b) / (bc + b))
    s += c / (2 * b) * math.log((ac - a) / (ac + a))
    s += 2 * math.atan(a * b / (c * r))
    s += (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
    s += (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
    s += c / (a * b) * (ac + bc)
    s -= (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c)
    return s / math.pi


@pytest.mark.parametrize("edges", [(1, 1, 1), (1, 2, 3), (1, 1, 0.1), (5, 0.3, 2), (0.7, 0.7, 4.0)])
def test_self_tensor_matches_aharoni_prism(edges):
    """Diagonal self terms = demagnetizing factors of the prism (Aharoni). Pins f
    (and through the trace all three diagonal permutations)."""
    ex, ey, ez = edges
    t = oracle.cell_tensor((0, 0, 0), edges)
    a, b, c = ex / 2, ey / 2, ez / 2
    want = [_aharoni_dz(b, c, a), _aharoni_dz(c, a, b), _aharoni_dz(a, b, c)]
    np.testing.assert_allclose(t[:3], want, rtol=0, atol=5e-14)
    assert abs(sum(want) - 1.0) < 1e-13
    np.testing.assert_allclose(t[3:], 0.0, atol=1e-15)


def test_thin_film_body_factor():
    """Homogeneous 1 x 1 x 0.1 film: e = (1/2) Nzz V = 4.025e-2 (paper Sec. 5.3,
    Table thin_homo, DM row), so Nzz(film) = 0.8050 to the printed digits."""
    t = oracle.cell_tensor((0, 0, 0), (1.0, 1.0, 0.1))
    e = 0.5 * t[2] * 0.1
    assert round(e, 5) == pytest.approx(4.025e-2, abs=5e-6)


# ------------------------------------------------------------ off-origin
OFFSETS = [(1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 0, 0), (2, 1, 0), (3, 1.0, 0.5),
           (2, 2, 2), (5, 3, 1), (7, -2, 3), (-12, 5, -9), (40, 0, 0), (30, 20, 10)]


@pytest.mark.parametrize("R", OFFSETS)
def test_trace_vanishes_off_origin(R):
    """Away from the self term the kernel is a Hessian of the harmonic 1/r, so the
    trace of N vanishes (Laplace). Catches a dropped term in f or a wrong
    diagonal permutation."""
    for d in [(1, 1, 1), (1.0, 0.5, 2.0)]:
        Rphys = tuple(r * dd for r, dd in zip(R, d))
        t = oracle.cell_tensor(Rphys, d)
        scale = max(1e-300, np.max(np.abs(t)))
        assert abs(t[0] + t[1] + t[2]) < 1e-12 * scale + 1e-14


@pytest.mark.parametrize("R", [(2, 0, 0), (2, 1, 0), (2, 1, 1), (3, 1.0, 0.5), (2, 2, 2), (3, -2, 1), (0, 3, -2)])
@pytest.mark.parametrize("d", [(1, 1, 1), (1.0, 0.5, 2.0), (2.0, 2.0, 0.25)])
def test_closed_form_equals_quadrature(R, d):
    """Two independent evaluations of the same cell-averaged integral: the corner
    formula of f and g, and quadrature of the point-dipole kernel. At 2-3 cells
    the closed form still holds ~13 digits. Pins g, its signs, and the
    quadrature's tent weights."""
    Rp = tuple(r * dd for r, dd in zip(R, d))
    c = oracle.cell_tensor_closed(Rp, d)
    q = oracle.cell_tensor_quad(Rp, d)
    scale = np.max(np.abs(q))
    # the closed form's own rounding grows with R / min(d); flat cells lose more
    tol = 5e-12 if max(d) / min(d) <= 2 else 1e-10
    np.testing.assert_allclose(c, q, rtol=0, atol=tol * scale)


@pytest.mark.parametrize("R", [(2, 0, 0), (3, 1, 0), (9, 4, 2), (60, 20, -10)])
def test_quadrature_converged(R):
    """Raising the node count changes nothing (the automatic rule is converged)."""
    a = oracle.cell_tensor_quad(R, (1, 1, 1))
    b = oracle.cell_tensor_quad(R, (1, 1, 1), nodes=(60, 60, 60))
    scale = np.max(np.abs(b))
    np.testing.assert_allclose(a, b, rtol=0, atol=2e-14 * scale)


def test_dipole_limit():
    """Far away N -> -(V/4pi)(3 R R^T/R^5 - I/R^3): the point-dipole field. For
    cubic cells the (d/R)^2 correction vanishes (harmonicity), so the relative
    deviation falls like (d/R)^4."""
    def dev(R):
        R = np.asarray(R, dtype=float)
        t = oracle.cell_tensor(R, (1, 1, 1))
        r = np.linalg.norm(R)
        full = -(3 * np.outer(R, R) / r ** 5 - np.eye(3) / r ** 3) / (4 * math.pi)
        want = np.array([full[0, 0], full[1, 1], full[2, 2], full[0, 1], full[0, 2], full[1, 2]])
        return np.max(np.abs(t - want)) / np.max(np.abs(want))
    d1 = dev((20.0, 12.0, 6.0))
    d2 = dev((40.0, 24.0, 12.0))
    assert d1 < 1e-4
    assert 10.0 < d1 / d2 < 22.0   # ~ 2^4


def test_parity_of_components():
    """xx, yy, zz even in every axis; xy odd in x and y; xz odd in x and z; yz odd
    in y and z (from the symmetry of the integrand under reflections)."""
    R = (3.0, 2.0, 1.5)
    d = (1.0, 0.8, 1.3)
    base = oracle.cell_tensor(R, d)
    odd = {3: (0, 1), 4: (0, 2), 5: (1, 2)}
    for flip in [(-1, 1, 1), (1, -1, 1), (1, 1, -1), (-1, -1, 1), (-1, -1, -1)]:
        t = oracle.cell_tensor(tuple(f * r for f, r in zip(flip, R)), d)
        for c in range(6):
            s = 1.0
            for ax in odd.get(c, ()):
                s *= flip[ax]
            assert abs(t[c] - s * base[c]) < 1e-15 * np.max(np.abs(base))


def test_additivity_box_of_cells():
    """The field of a block of cells is the sum of the cells' fields: the mutual
    tensor of a cell and a 2 x 3 x 2 block (64-corner formula with unequal boxes)
    equals the sum of the cell-cell tensors (closed form or quadrature)."""
    d = np.array([1.0, 0.7, 1.2])
    for tgt in [(3, 1, 0), (0, 0, 0), (1, 2, 1), (-2, 0, 3)]:
        tc = np.array(tgt, dtype=float) * d
        acc = np.zeros(6)
        for k in range(2):
            for j in range(3):
                for i in range(2):
                    sc = np.array([i, j, k]) * d
                    acc += oracle.cell_tensor(tc - sc, d)
        block_centre = np.array([0.5, 1.0, 0.5]) * d
        block_edges = np.array([2, 3, 2]) * d
        got = oracle.box_tensor(tc, d, block_centre, block_edges)
        np.testing.assert_allclose(got, acc, rtol=0, atol=1e-12 * np.max(np.abs(acc)))


# ------------------------------------------------------------ convolution
TINY = [(1, 1, 1), (2, 1, 1), (1, 3, 1), (1, 1, 4), (3, 2, 2), (5, 4, 3), (8, 6, 5), (7, 1, 6)]


@pytest.mark.parametrize("n", TINY)
def test_bruteforce_equals_fft(n):
    """The direct pair sum over directly evaluated signed offsets equals the FFT
    convolution built from the octant table mirrored by parity. Catches a wrong
    parity sign, a wrapping off-by-one, a transposed operand."""
    d = (1.0, 0.9, 1.3)
    M = inputs.random_unit(n, seed=11)
    Hb = oracle.field_bruteforce(M, d)
    Hf = oracle.field_fft(M, d)
    np.testing.assert_allclose(Hf, Hb, rtol=0, atol=1e-13 * np.max(np.abs(Hb)))


@pytest.mark.parametrize("n", [(5, 4, 3), (7, 1, 6)])
def test_threaded_fft_path_equals_bruteforce(n):
    """The threaded transforms (workers > 1, used for the full-size grids)
    give the direct pair sum too."""
    pytest.importorskip("scipy")
    d = (1.0, 0.9, 1.3)
    M = inputs.random_unit(n, seed=12)
    Hb = oracle.field_bruteforce(M, d)
    Hf = oracle.field_fft(M, d, workers=4)
    np.testing.assert_allclose(Hf, Hb, rtol=0, atol=1e-13 * np.max(np.abs(Hb)))


def test_padding_invariance():
    """Any period P >= 2N - 1 gives the same field on the physical cells."""
    n = (6, 5, 3)
    d = (1.0, 1.0, 1.0)
    M = inputs.random_unit(n, seed=3)
    oct_ = oracle.tensor_octant(n, d)
    ref = oracle.field_fft(M, d, P=(11, 9, 5), octant=oct_)
    for P in [(12, 10, 6), (16, 16, 8), (13, 27, 7)]:
        H = oracle.field_fft(M, d, P=P, octant=oct_)
        np.testing.assert_allclose(H, ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))


def test_operator_is_symmetric():
    """<K a, b> = <a, K b> for K: M -> H (N symmetric and even). Catches a sign
    error in the odd components' mirroring."""
    n = (9, 7, 4)
    d = (1.0, 1.3, 0.8)
    a = inputs.random_unit(n, seed=5)
    b = inputs.random_unit(n, seed=6)
    oct_ = oracle.tensor_octant(n, d)
    Ka = oracle.field_fft(a, d, octant=oct_)
    Kb = oracle.field_fft(b, d, octant=oct_)
    lhs, rhs = float(np.sum(Ka * b)), float(np.sum(a * Kb))
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1)


def test_uniform_field_equals_body_tensor():
    """Uniform M: the cell-averaged field is exact for any grid (paper Sec. 5.1),
    H_cell = -N(cell, body) M with the mutual tensor of the cell and the whole
    body (one 64-corner evaluation per cell)."""
    n = (5, 4, 3)
    d = np.array([1.0, 0.6, 1.5])
    m = inputs.uniform(n, (0.3, -0.5, 0.8))
    H = oracle.field_fft(m, d)
    body_c = np.array(n) * d / 2
    body_e = np.array(n) * d
    mv = m[:, 0, 0, 0]
    for (i, j, k) in [(0, 0, 0), (4, 3, 2), (2, 1, 1), (1, 3, 0)]:
        tc = (np.array([i, j, k]) + 0.5) * d
        t = oracle.box_tensor(tc, d, body_c, body_e)
        N = np.array([[t[0], t[3], t[4]], [t[3], t[1], t[5]], [t[4], t[5], t[2]]])
        np.testing.assert_allclose(H[:, k, j, i], -N @ mv, rtol=0, atol=1e-14)


@pytest.mark.parametrize("n,ext", [((16, 16, 16), (1, 1, 1)), ((12, 9, 5), (1.2, 0.9, 0.5))])
def test_uniform_energy_equals_demag_factor(n, ext):
    """E = (1/2) mu0 Ms^2 V_body N_body for uniform M, exact up to rounding (paper
    Sec. 5.1: for the unit cube e = 1/6 mu0 Ms^2). N_body from Aharoni."""
    d = tuple(e / k for e, k in zip(ext, n))
    m = inputs.uniform(n, (0, 0, 1))
    h = oracle.field_fft(m, d)
    e = oracle.energy_reduced(m, h, d)
    V = ext[0] * ext[1] * ext[2]
    want = 0.5 * V * _aharoni_dz(ext[0] / 2, ext[1] / 2, ext[2] / 2)
    assert abs(e - want) < 1e-13 * want
    Ms = 8e5
    E = oracle.energy(Ms * m, Ms * h, d)
    assert abs(E - oracle.MU0 * Ms ** 2 * want) < 1e-12 * abs(E)


def _state(case, n):
    ext = tuple(case["extent"])
    if case["state"] == "uniform_z":
        return inputs.uniform(n, (0, 0, 1))
    if case["state"] == "flower":
        return inputs.flower(n, ext)
    if case["state"] == "vortex":
        return inputs.vortex(n, ext, rc=0.14)
    raise KeyError(case["state"])


def test_paper_dm_energies():
    """The DM energies the paper prints (tests/golden/paper_energies.json, each
    with its table), to the printed digits; the cube to better than the paper's
    own 2.9e-9 relative error."""
    with open(os.path.join(GOLDEN, "paper_energies.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        n = tuple(case["grid"])
        d = tuple(e / k for e, k in zip(case["extent"], n))
        m = _state(case, n)
        e = oracle.energy_reduced(m, oracle.field_fft(m, d), d)
        if case.get("exact"):
            assert abs(e - case["e"]) / case["e"] < case["paper_relerr"], case["name"]
        else:
            digits = case["digits"]
            mag = 10 ** (math.floor(math.log10(abs(case["e"]))) - digits + 1)
            assert abs(e - case["e"]) <= 0.5 * mag, (case["name"], e)


def test_sphere_energy_tends_to_continuum():
    """Staircase sphere (paper Sec. 5.4): as the grid refines the energy tends to
    the continuum value (1/2)(1/3) V_sphere = pi/36 [mu0 Ms^2] for radius 1/2.
    The paper prints no number, so this is a soft pin: the error shrinks."""
    errs = []
    for k in (8, 16, 24):
        n = (k, k, k)
        d = (1.0 / k,) * 3
        mask = inputs.sphere_mask(n, k / 2)
        m = inputs.uniform(n, (0, 0, 1)) * mask[None]
        e = oracle.energy_reduced(m, oracle.field_fft(m, d), d)
        errs.append(abs(e - math.pi / 36) / (math.pi / 36))
    assert errs[-1] < 0.05
    assert errs[-1] < errs[0]


def test_field_at_matches_full_field():
    """Sampled direct sums with the octant table reproduce the full field."""
    n = (7, 5, 4)
    d = (1.0, 1.0, 1.0)
    M = inputs.random_unit(n, seed=8)
    oct_ = oracle.tensor_octant(n, d)
    H = oracle.field_fft(M, d, octant=oct_)
    cells = [(0, 0, 0), (6, 4, 3), (3, 2, 1)]
    got = oracle.field_at(M, oct_, cells)
    for q, (i, j, k) in enumerate(cells):
        np.testing.assert_allclose(got[q], H[:, k, j, i], rtol=0, atol=1e-14)


def test_mpmath_closed_form_rounding():
    """The FP64 closed form near the origin agrees with the same integral at
    50 digits (mpmath, quadrature of the point kernel for a separated pair and
    the prism factor of Aharoni for the self term)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    a, b, c = (mpmath.mpf(1) / 2, mpmath.mpf(1), mpmath.mpf(3) / 2)
    r = mpmath.sqrt(a * a + b * b + c * c)
    ab, bc, ac = mpmath.sqrt(a * a + b * b), mpmath.sqrt(b * b + c * c), mpmath.sqrt(a * a + c * c)
    s = (b * b - c * c) / (2 * b * c) * mpmath.log((r - a) / (r + a))
    s += (a * a - c * c) / (2 * a * c) * mpmath.log((r - b) / (r + b))
    s += b / (2 * c) * mpmath.log((ab + a) / (ab - a))
    s += a / (2 * c) * mpmath.log((ab + b) / (ab - b))
    s += c / (2 * a) * mpmath.log((bc - b) / (bc + b))
    s += c / (2 * b) * mpmath.log((ac - a) / (ac + a))
    s += 2 * mpmath.atan(a * b / (c * r))
    s += (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
    s += (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
    s += c / (a * b) * (ac + bc)
    s -= (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c)
    dz = s / mpmath.pi
    t = oracle.cell_tensor((0, 0, 0), (1.0, 2.0, 3.0))
    assert abs(t[2] - float(dz)) < 1e-15


def test_rel_errors_two_cell_case_by_hand():
    """The error measures on a two-cell field worked out by hand: H_ref has
    3 and -4 in two entries (max |H_ref| = 4, ||H_ref||_2 = 5); H differs by
    0.5 and -1.2 in two others (max 1.2, ||diff||_2 = 1.3). rel-max = 0.3,
    rel-RMS = 0.26 (the Frobenius form of Sec. 3.2, Eq. "relr"), and the
    field error of Sec. 5.1, Eq. "relerr", sqrt(sum |diff|^2 / N) with N = 2
    cells: sqrt(1.69 / 2)."""
    Href = np.zeros((3, 1, 1, 2))
    Href[0, 0, 0, 0] = 3.0
    Href[1, 0, 0, 1] = -4.0
    H = Href.copy()
    H[2, 0, 0, 0] += 0.5
    H[0, 0, 0, 1] -= 1.2
    e = oracle.rel_errors(H, Href)
    assert e["rel_max"] == pytest.approx(0.3, rel=1e-15)
    assert e["rel_rms"] == pytest.approx(0.26, rel=1e-15)
    assert e["paper_relerr"] == pytest.approx(math.sqrt(0.845), rel=1e-15)
    # swapped operands change the normaliser: ||H||_2 = sqrt(26.69)
    f = oracle.rel_errors(Href, H)
    assert f["rel_rms"] == pytest.approx(1.3 / math.sqrt(26.69), rel=1e-15)
