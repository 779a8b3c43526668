"""Tensor-grid (TG) method on the GPU against the TG oracle: the cell-centre
potential of CP magnetizations (FP64 to 1e-12; FP32 to a bound derived
below), the second-order field and the energy, uniform bodies at full size
against the closed-form body potential, and the TG energies of the paper's
homogeneous states.

FP32 bound. The potential is a sum of K = 3 R r rank-one terms accumulated in
FP32 (relative error ~ eps32 sqrt(K) of the largest partial sums) and the
field divides potential differences by one cell edge, amplifying by
A = max|phi| / (max|H| min(d)) as for the SP method; the tests allow
eps32 sqrt(K) (16 + 8 A) against max|H|.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import tensor_grid as tg  # noqa: E402

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _random_cp(n, r, seed, scale=8e5):
    rng = np.random.default_rng(seed)
    lam = scale * rng.standard_normal((3, r))
    U = [rng.standard_normal((3, r, v)) for v in n]
    return lam, U[0], U[1], U[2]


def _dense(lam, Ux, Uy, Uz):
    return np.stack([tg.cp_to_dense(lam[p], Ux[p].T, Uy[p].T, Uz[p].T) for p in range(3)])


def _torch(a, dt):
    return torch.tensor(a, dtype=dt, device="cuda")


@pytest.mark.parametrize("n,d,r", [((5, 4, 3), (2e-9, 1.5e-9, 2.5e-9), 2), ((17, 9, 6), (1e-9, 1e-9, 1e-9), 3),
                                   ((33, 20, 12), (1e-9, 2e-9, 1e-9), 1), ((130, 7, 5), (1e-9, 1e-9, 3e-9), 4)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tg_cp_matches_oracle(n, d, r, prec):
    from paper_1204_4302_gb300.tg import TGPlan
    lam, Ux, Uy, Uz = _random_cp(n, r, seed=sum(n) + r)
    M = _dense(lam, Ux, Uy, Uz)
    phi_ref = tg.cell_potential_fft(M, d, oracle.sp_kernel)
    H_ref = tg.tg_field_from_potential(phi_ref, d)
    E_ref = oracle.energy(M, H_ref, d)
    dt = torch.float32 if prec == "f32" else torch.float64
    p = TGPlan(n, d, r, prec=prec)
    args = [_torch(a, dt) for a in (lam, Ux, Uy, Uz)]
    phi = p.potential(*args).double().cpu().numpy()
    H, E = p.field(*args, energy=True)
    H = H.double().cpu().numpy()
    if prec == "f64":
        assert _relmax(phi, phi_ref) <= 1e-12
        assert _relmax(H, H_ref) <= 1e-12
        assert abs(E.item() - E_ref) <= 1e-12 * abs(E_ref) + 1e-12 * oracle.MU0 * np.sum(np.abs(M * H_ref))
    else:
        K = 3 * p.info()["sinc_terms"] * r
        A = float(np.max(np.abs(phi_ref)) / (np.max(np.abs(H_ref)) * min(d)))
        tol = EPS32 * math.sqrt(K) * (16 + 8 * A)
        assert _relmax(phi, phi_ref) <= EPS32 * math.sqrt(K) * 16, _relmax(phi, phi_ref)
        assert _relmax(H, H_ref) <= tol, (_relmax(H, H_ref), tol)
        assert abs(E.item() - E_ref) <= tol * np.sum(np.abs(M * H_ref)) * 0.5 * oracle.MU0 * np.prod(d)
    p.close()


def _uniform_cp(n, mv):
    r = 1
    lam = np.array(mv, dtype=float).reshape(3, 1)
    U = [np.ones((3, r, v)) for v in n]
    return lam, U[0], U[1], U[2]


@pytest.mark.parametrize("prec", ["f64"])
def test_tg_paper_homogeneous_energies(prec):
    """Rank-one CP magnetizations of the paper's homogeneous cube (relative
    energy error 3.8e-4, Table cube_homo, TG row) and thin film (4.025e-2,
    Table thin_homo, TG row), by the CUDA path."""
    from paper_1204_4302_gb300.tg import TGPlan
    for n, ext, ref, rel in (((40, 40, 40), (1.0, 1.0, 1.0), 3.8e-4, True), ((80, 80, 8), (1.0, 1.0, 0.1), 4.025e-2, False)):
        d = tuple(e / k for e, k in zip(ext, n))
        lam, Ux, Uy, Uz = _uniform_cp(n, (0.0, 0.0, 1.0))
        p = TGPlan(n, d, 1, prec=prec)
        H = p.field(*[_torch(a, torch.float64) for a in (lam, Ux, Uy, Uz)]).cpu().numpy()
        p.close()
        m = np.zeros((3,) + tuple(reversed(n)))
        m[2] = 1.0
        e = oracle.energy_reduced(m, H, d)
        if rel:
            val = abs(e - 1 / 6) * 6
            assert abs(val - ref) <= 0.05e-4, val
        else:
            assert abs(e - ref) <= 0.5e-5, e


@pytest.mark.parametrize("n", [(256, 256, 256), (512, 512, 128)])
def test_tg_full_size_uniform_body(n):
    """Full size, uniform M: the potential at sampled cell centres equals the
    potential of the whole box (its face integrals in closed form), FP64 to
    1e-12 and FP32 to the bound above; the field of FP32 within the bound of
    FP64."""
    from paper_1204_4302_gb300.tg import TGPlan
    d = (1e-9, 1e-9, 1e-9)
    mv = np.array([0.3, -0.5, 0.8]) * 8e5
    L = np.array(n) * np.array(d)
    rng = np.random.default_rng(7)
    cells = [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (n[0] // 2, n[1] // 3, n[2] - 1)]
    cells += [tuple(int(rng.integers(0, v)) for v in n) for _ in range(12)]
    ref = []
    for (i, j, k) in cells:
        rr = (np.array([i, j, k]) + 0.5) * np.array(d) - L / 2
        s = 0.0
        for ax in range(3):
            a, b = [q for q in range(3) if q != ax]
            plus = oracle.sp_rect(rr[ax] - L[ax] / 2, rr[a], rr[b], L[a] / 2, L[b] / 2)
            minus = oracle.sp_rect(rr[ax] + L[ax] / 2, rr[a], rr[b], L[a] / 2, L[b] / 2)
            s += mv[ax] * (plus - minus) / (4 * math.pi)
        ref.append(s)
    ref = np.array(ref)
    lam, Ux, Uy, Uz = _uniform_cp(n, mv)
    Hs = {}
    for prec in ("f64", "f32"):
        dt = torch.float32 if prec == "f32" else torch.float64
        p = TGPlan(n, d, 1, prec=prec)
        args = [_torch(a, dt) for a in (lam, Ux, Uy, Uz)]
        phi = p.potential(*args)
        got = np.array([float(phi[k, j, i]) for (i, j, k) in cells])
        K = 3 * p.info()["sinc_terms"]
        tol = 1e-12 if prec == "f64" else EPS32 * math.sqrt(K) * 16
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), prec
        Hs[prec] = p.field(*args)
        p.close()
        del phi
    H64 = Hs["f64"]
    diff = float((Hs["f32"].double() - H64).abs().max() / H64.abs().max())
    assert diff <= 1e-3, diff


@pytest.mark.parametrize("n,d,r", [((64, 40, 7), (1e-9, 1e-9, 1e-9), 2),     # M = 280: a ragged last row tile
                                   ((300, 33, 9), (1e-9, 2e-9, 1e-9), 1),    # nx > 256: two column tiles of 160
                                   ((37, 11, 5), (2e-9, 1e-9, 1e-9), 3),     # nx not a multiple of 4 (scalar stores)
                                   ((5, 4, 3), (1e-9, 1e-9, 1e-9), 1)])      # one partial tile
def test_tg_tensor_core_contraction(n, d, r):
    """FP32 plans contract on the tensor cores by default (three TF32
    products per term, FP32 accumulators in tensor memory): the potential
    against the oracle within the FP32 bound, against the CUDA-core
    contraction of the same plan, the per-stage timing and the status word."""
    from paper_1204_4302_gb300.tg import TGPlan
    lam, Ux, Uy, Uz = _random_cp(n, r, seed=7 * sum(n) + r)
    M = _dense(lam, Ux, Uy, Uz)
    phi_ref = tg.cell_potential_fft(M, d, oracle.sp_kernel)
    p = TGPlan(n, d, r, prec="f32")
    assert p.contraction() == TGPlan.TENSOR_CORES
    args = [_torch(a, torch.float32) for a in (lam, Ux, Uy, Uz)]
    K = 3 * p.info()["sinc_terms"] * r
    bound = EPS32 * math.sqrt(K) * 16
    p.set_timing(True)
    phi_tc = p.potential(*args).double().cpu().numpy()
    ms, calls = p.get_timing()
    assert calls == 1 and len(ms) == 4 and all(v >= 0 for v in ms) and ms[2] > 0
    p.set_timing(False)
    p.status()
    p.set_contraction(TGPlan.CUDA_CORES)
    phi_cc = p.potential(*args).double().cpu().numpy()
    assert _relmax(phi_tc, phi_ref) <= bound, (_relmax(phi_tc, phi_ref), bound)
    assert _relmax(phi_cc, phi_ref) <= bound
    assert _relmax(phi_tc, phi_cc) <= bound
    p.close()


def test_tg_contraction_choice():
    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.tg import TGPlan
    p = TGPlan((8, 8, 8), (1e-9, 1e-9, 1e-9), 1, prec="f64")
    assert p.contraction() == TGPlan.CUDA_CORES
    with pytest.raises(B.DemagError):
        p.set_contraction(TGPlan.TENSOR_CORES)
    with pytest.raises(B.DemagError):
        p.set_contraction(2)
    p.close()


def test_tg_tensor_core_full_size_rank8():
    """256^3 cells, CP rank 8 (K = 3 R 8 terms, the benchmark's TG case):
    the tensor-core FP32 potential against the FP64 plan's within the FP32
    bound, on every cell."""
    from paper_1204_4302_gb300.tg import TGPlan
    n, d, r = (256, 256, 256), (2e-9, 2e-9, 2e-9), 8
    rng = np.random.default_rng(11)
    lam = 8e5 * rng.standard_normal((3, r)) / r
    U = [rng.standard_normal((3, r, v)) for v in n]
    p32 = TGPlan(n, d, r, prec="f32")
    phi32 = p32.potential(*[_torch(a, torch.float32) for a in [lam] + U])
    p32.status()
    K = 3 * p32.info()["sinc_terms"] * r
    p32.close()
    p64 = TGPlan(n, d, r, prec="f64")
    phi64 = p64.potential(*[_torch(a, torch.float64) for a in [lam] + U])
    p64.close()
    rel = float((phi32.double() - phi64).abs().max() / phi64.abs().max())
    assert rel <= EPS32 * math.sqrt(K) * 16, (rel, K)
