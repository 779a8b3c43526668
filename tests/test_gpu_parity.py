"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle,
element by element, on seeded inputs.

Tolerances (rel-max = max|H - H_ref| / max|H_ref|):
  FP64 plans <= 1e-12, FP32 plans <= 1e-5 (the targets of the method's FP32
  form: FFTs and spectral product in FP32, tensor set up in FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1204_4302_gb300 import inputs  # noqa: E402

TOL = {"f32": 1e-5, "f64": 1e-12}
DT = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def _plan(n, d, prec, pad=None):
    from paper_1204_4302_gb300.plan import Plan
    return Plan(n, d, prec=prec, pad=pad)


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _gpu_field(n, d, M, prec, pad=None):
    plan = _plan(n, d, prec, pad)
    H = plan.field(torch.tensor(M, dtype=DT[prec], device="cuda"))
    torch.cuda.synchronize()
    out = H.double().cpu().numpy()
    plan.close()
    return out


SHAPES = [
    ((16, 16, 16), (1e-9, 1e-9, 1e-9)),      # the 16^3 cube of the paper-style check
    ((20, 12, 7), (1e-9, 1.5e-9, 0.7e-9)),   # ragged, non-cubic cells
    ((33, 17, 5), (2e-9, 2e-9, 2e-9)),       # odd sizes, several tiles
    ((1, 1, 1), (1e-9, 2e-9, 3e-9)),         # single cell: H = -N(0) M
    ((1, 1, 8), (1e-9, 1e-9, 1e-9)),         # degenerate axes
    ((9, 1, 1), (1e-9, 1e-9, 1e-9)),
    ((1, 7, 1), (1e-9, 1e-9, 1e-9)),
    ((2, 2, 2), (1e-9, 1e-9, 1e-9)),
    ((64, 16, 1), (2e-9, 2e-9, 2e-9)),       # 2-D film, Pz = 1
    ((48, 40, 3), (3e-9, 3e-9, 3e-9)),
    ((3, 130, 9), (1e-9, 1e-9, 1e-9)),       # long y axis, short x
    ((70, 5, 3), (1e-9, 1e-9, 1e-9)),        # x transform of 128 complex points
    ((140, 6, 3), (1e-9, 1e-9, 1e-9)),       # 256
    ((300, 3, 2), (1e-9, 1e-9, 1e-9)),       # 512 (padded 1024)
    ((9, 5, 40), (1e-9, 1e-9, 1e-9)),        # z pass of length 128
    ((5, 4, 70), (1e-9, 1e-9, 1e-9)),        # z pass of length 256
    ((4, 3, 130), (1e-9, 1e-9, 1e-9)),       # z pass of length 512
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,d", SHAPES)
def test_field_matches_oracle(n, d, prec):
    M = 8e5 * inputs.random_unit(n, seed=sum(n))
    Href = oracle.field_fft(M, d)
    H = _gpu_field(n, d, M, prec)
    assert _relmax(H, Href) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_explicit_padding_gives_same_field(prec):
    n, d = (10, 6, 5), (1e-9, 1e-9, 1e-9)
    M = inputs.random_unit(n, seed=2)
    Href = oracle.field_fft(M, d)
    for pad in [(32, 16, 16), (64, 32, 16), (32, 128, 64)]:
        H = _gpu_field(n, d, M, prec, pad=pad)
        assert _relmax(H, Href) <= TOL[prec], pad


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_paper_flower_energy(prec):
    """Flower state in the unit cube at 40^3 (paper Sec. 5.2, Table cube_flower,
    DM row: e = 1.528e-1 mu0 Ms^2)."""
    n = (40, 40, 40)
    d = (1.0 / 40,) * 3
    m = inputs.flower(n)
    plan = _plan(n, d, prec)
    E, _ = plan.energy_grad(torch.tensor(m, dtype=DT[prec], device="cuda"), 1.0, want_grad=False)
    mu0 = oracle.MU0
    e = E.item() / mu0  # energy in units of mu0 Ms^2 (Ms = 1)
    eref = oracle.energy_reduced(m, oracle.field_fft(m, d), d)
    assert abs(e - eref) <= 10 * TOL[prec] * abs(eref)
    assert round(e, 4) == pytest.approx(0.1528, abs=1e-12)
    plan.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_uniform_cube_energy(prec):
    """Uniform M in a cube: E = mu0 Ms^2 V / 6 (paper Sec. 5.1), exact up to rounding."""
    n = (16, 16, 16)
    d = (1e-9,) * 3
    Ms = 8e5
    plan = _plan(n, d, prec)
    M = torch.tensor(Ms * inputs.uniform(n, (1, 0, 0)), dtype=DT[prec], device="cuda")
    E = plan.energy(M)
    V = (16e-9) ** 3
    Eexact = oracle.MU0 * Ms ** 2 * V / 6
    assert abs(E - Eexact) <= 10 * TOL[prec] * Eexact
    plan.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_energy_and_gradient_with_mask(prec):
    """Sphere mask (paper Sec. 5.4 staircase): M = Ms w m; E and dE/dm against the
    oracle's field of the masked magnetization."""
    n = (24, 24, 24)
    d = (2e-9,) * 3
    Ms = 8e5
    w = inputs.sphere_mask(n, 12)
    m = inputs.random_unit(n, seed=9)
    M = Ms * w[None] * m
    Href = oracle.field_fft(M, d)
    Eref = oracle.energy(M, Href, d)
    Gref = -oracle.MU0 * d[0] * d[1] * d[2] * Ms * w[None] * Href
    plan = _plan(n, d, prec)
    mt = torch.tensor(m, dtype=DT[prec], device="cuda")
    wt = torch.tensor(w, dtype=DT[prec], device="cuda")
    E, G = plan.energy_grad(mt, Ms, wt)
    torch.cuda.synchronize()
    assert abs(E.item() - Eref) <= 10 * TOL[prec] * abs(Eref)
    assert _relmax(G.double().cpu().numpy(), Gref) <= TOL[prec]
    plan.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_field_energy_matches(prec):
    n, d = (18, 14, 6), (1e-9, 1e-9, 2e-9)
    M = 8e5 * inputs.random_unit(n, seed=4)
    Href = oracle.field_fft(M, d)
    plan = _plan(n, d, prec)
    H, E = plan.field_energy(torch.tensor(M, dtype=DT[prec], device="cuda"))
    torch.cuda.synchronize()
    assert _relmax(H.double().cpu().numpy(), Href) <= TOL[prec]
    Eref = oracle.energy(M, Href, d)
    assert abs(E.item() - Eref) <= 10 * TOL[prec] * abs(Eref)
    plan.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_identity(prec):
    """<K a, b> = <a, K^T b> with K^T the adjoint entry point."""
    n, d = (21, 11, 6), (1e-9, 1.2e-9, 0.9e-9)
    a = inputs.random_unit(n, seed=12)
    b = inputs.random_unit(n, seed=13)
    plan = _plan(n, d, prec)
    at = torch.tensor(a, dtype=DT[prec], device="cuda")
    bt = torch.tensor(b, dtype=DT[prec], device="cuda")
    Ka = plan.field(at).double()
    KTb = plan.field_adjoint(bt).double()
    lhs = float((Ka * bt.double()).sum())
    rhs = float((at.double() * KTb).sum())
    scale = float(Ka.abs().sum())
    assert abs(lhs - rhs) <= 10 * TOL[prec] * scale
    plan.close()


def test_tensor_spectrum_is_real():
    """The wrapped tensor is even or odd in every axis, so its spectrum is real:
    the imaginary parts left by the FP64 setup are rounding only."""
    for n in [(16, 16, 16), (33, 7, 5), (1, 9, 4)]:
        plan = _plan(n, (1e-9, 1e-9, 1e-9), "f64")
        assert plan.info()["tensor_imag_max"] < 1e-13
        plan.close()


def test_tensor_values_through_unit_impulse():
    """A unit moment in one cell: H at every cell is -N(offset) e_j, so the field
    of an impulse reads out the device tensor column by column; compare with
    the oracle's tensor table (mid and far regimes, and their switch)."""
    n = (48, 30, 26)
    d = (1e-9, 1.3e-9, 0.8e-9)
    plan = _plan(n, d, "f64")
    tab = oracle.tensor_octant(n, d)
    for j in range(3):
        M = np.zeros((3,) + n[::-1])
        M[j, 0, 0, 0] = 1.0
        H = plan.field(torch.tensor(M, device="cuda")).cpu().numpy()
        # column j of N: (xx,xy,xz), (xy,yy,yz), (xz,yz,zz)
        comps = [(0, 3, 4), (3, 1, 5), (4, 5, 2)][j]
        for i in range(3):
            want = tab[comps[i]]
            got = -H[i]
            scale = np.max(np.abs(tab[:3]))
            assert np.max(np.abs(got - want)) <= 1e-13 * scale, (i, j)
    plan.close()


def test_host_entry_point_matches_device():
    n, d = (20, 18, 9), (1e-9, 1e-9, 1e-9)
    M = 8e5 * inputs.random_unit(n, seed=21)
    plan = _plan(n, d, "f32")
    Md = torch.tensor(M, dtype=torch.float32, device="cuda")
    Hd = plan.field(Md).cpu()
    Mh = torch.tensor(M, dtype=torch.float32).pin_memory()
    Hh = plan.field_host(Mh)
    assert torch.equal(Hd, Hh)
    Hh2 = plan.field_host(torch.tensor(M, dtype=torch.float32))  # pageable
    assert torch.equal(Hd, Hh2)
    # streamed: seven states through the three rotating device slots
    Ms = [torch.tensor(inputs.random_unit(n, seed=50 + i) * 8e5, dtype=torch.float32).pin_memory() for i in range(7)]
    Hs = [torch.empty_like(m).pin_memory() for m in Ms]
    for m, h in zip(Ms, Hs):
        plan.field_host_async(m, h)
    plan.host_wait()
    for m, h in zip(Ms, Hs):
        assert torch.equal(plan.field(m.cuda()).cpu(), h)
    # streamed with the energy: H and E of every state, as on the device
    Es = [torch.zeros(1, dtype=torch.float64).pin_memory() for _ in Ms]
    for m, h, e in zip(Ms, Hs, Es):
        plan.field_energy_host_async(m, h, e)
    plan.host_wait()
    for m, h, e in zip(Ms, Hs, Es):
        Hd, Ed = plan.field_energy(m.cuda())
        torch.cuda.synchronize()
        assert torch.equal(Hd.cpu(), h) and Ed.item() == e.item()
    plan.close()
