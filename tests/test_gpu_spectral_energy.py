"""Energy without a field by the spectral (Parseval) sum (demag_energy and
demag_energy_grad with no gradient output): E = (mu0/2) (V / (Px Py Pz))
sum_k w(kx) M^H N^ M over the half spectrum, formed in the z pass after the
forward transforms (paper Sec. 2 energy; Sec. 3.1 tensor product). Checked
through the C ABI against the FP64 oracle's E = -(mu0/2) V sum M.H (FP32
rel 1e-5, FP64 rel 1e-12) and against the same plan's field-pipeline energy,
on z lengths 1..512 (one-thread, two-stage and persistent TMA z kernels),
Px = 1 (a single column in x), Py = 1, ragged tiles, a cell-weight mask,
and plans without a spectral form (smooth padding) that keep the field
pipeline. Field calls with the energy on FP32 plans with the persistent z
pass take the same spectral sum in that pass (demag_info.energy_in_z): their
E against the oracle and against the last pass's sum of M.H, their H against
the field of the other route."""
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


SHAPES = [
    (16, 16, 16),    # Pz = 32: two-stage kernel
    (20, 12, 7),     # Pz = 16: one thread per column
    (1, 1, 8),       # Px = Py = 1
    (9, 1, 1),       # Pz = 1
    (33, 17, 5),     # ragged
    (9, 17, 129),    # Pz = 512: persistent TMA kernel (FP32) / two-stage (FP64)
    (40, 6, 200),
    (40, 6, 100),    # Pz = 256: persistent TMA kernel at L = 256 (FP32)
]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", SHAPES)
def test_spectral_energy_matches_oracle_and_field_pipeline(n, prec):
    from paper_1204_4302_gb300.plan import Plan
    d = (2e-9, 1.5e-9, 1e-9)
    M = 8e5 * inputs.random_unit(n, seed=61)
    Href = oracle.field_fft(M, d)
    Eref = oracle.energy(M, Href, d)
    p = Plan(n, d, prec=prec)
    Mt = torch.tensor(M, dtype=DT[prec], device="cuda")
    zvs = (0, 6, 7) if prec == "f32" else (0,)
    for zv in zvs:
        p.set_variants(zv, 0, 1)
        p.set_spectral_energy(True)
        Es = p.energy(Mt)
        p.set_spectral_energy(False)
        Ef = p.energy(Mt)
        assert abs(Es - Eref) <= TOL[prec] * abs(Eref), (zv, Es, Eref)
        assert abs(Es - Ef) <= TOL[prec] * abs(Eref), (zv, Es, Ef)
    p.check_pipeline()
    p.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_spectral_energy_with_cell_weight(prec):
    """Sphere mask (M = Ms w m): energy_grad with no gradient output."""
    from paper_1204_4302_gb300.plan import Plan
    n, d, Ms = (24, 24, 24), (2e-9, 2e-9, 2e-9), 8e5
    w = inputs.sphere_mask(n, 12)
    m = inputs.random_unit(n, seed=62)
    M = Ms * w[None] * m
    Eref = oracle.energy(M, oracle.field_fft(M, d), d)
    p = Plan(n, d, prec=prec)
    mt = torch.tensor(m, dtype=DT[prec], device="cuda")
    wt = torch.tensor(w, dtype=DT[prec], device="cuda")
    E, G = p.energy_grad(mt, Ms, w=wt, want_grad=False)
    assert G is None
    assert abs(E.item() - Eref) <= TOL[prec] * abs(Eref)
    p.close()


def test_smooth_padding_keeps_the_field_pipeline():
    """Lengths that are not powers of two have no spectral form: the energy
    still comes out right (from the field pipeline)."""
    from paper_1204_4302_gb300.plan import Plan
    n, d = (30, 14, 11), (1e-9, 1e-9, 1e-9)
    M = 8e5 * inputs.random_unit(n, seed=63)
    Eref = oracle.energy(M, oracle.field_fft(M, d), d)
    p = Plan(n, d, prec="f64", pad="smooth")
    E = p.energy(torch.tensor(M, dtype=torch.float64, device="cuda"))
    assert abs(E - Eref) <= 1e-12 * abs(Eref)
    p.close()


def test_spectral_energy_full_size_headline_grid():
    """256^3 (padded 512^3): the spectral energy against the field-pipeline
    energy of the same plan, and the time of each (the spectral route skips
    the two inverse passes)."""
    from paper_1204_4302_gb300.plan import Plan
    n, d = (256, 256, 256), (2e-9, 2e-9, 2e-9)
    g = torch.Generator(device="cuda").manual_seed(9)
    M = torch.randn(3, 256, 256, 256, device="cuda", generator=g)
    M = 8e5 * M / M.norm(dim=0, keepdim=True)
    p = Plan(n, d, prec="f32")
    for zv in (6, 0):
        p.set_variants(zv, 2, 1)
        p.set_spectral_energy(True)
        Es = p.energy(M)
        p.set_spectral_energy(False)
        Ef = p.energy(M)
        assert abs(Es - Ef) <= 2e-6 * abs(Ef), (zv, Es, Ef)
    p.close()


FE_SHAPES = [
    (9, 17, 129),    # Pz = 512, ragged x tiles
    (40, 6, 100),    # Pz = 256
    (24, 20, 200),
]


@pytest.mark.parametrize("n", FE_SHAPES)
@pytest.mark.parametrize("zv", [6, 7])
def test_field_energy_in_the_z_pass(n, zv):
    from paper_1204_4302_gb300.plan import Plan
    d = (2e-9, 1.5e-9, 1e-9)
    M = 8e5 * inputs.random_unit(n, seed=64)
    Href = oracle.field_fft(M, d)
    Eref = oracle.energy(M, Href, d)
    p = Plan(n, d, prec="f32")
    Mt = torch.tensor(M, dtype=torch.float32, device="cuda")
    p.set_variants(zv, 0, 1)
    p.set_spectral_energy(True)
    assert p.info()["energy_in_z"] == 1
    Hz, Ez = p.field_energy(Mt)
    p.set_spectral_energy(False)
    assert p.info()["energy_in_z"] == 0
    Hx, Ex = p.field_energy(Mt)
    torch.cuda.synchronize()
    Ez, Ex = Ez.item(), Ex.item()
    assert abs(Ez - Eref) <= 1e-5 * abs(Eref), (Ez, Eref)
    assert abs(Ez - Ex) <= 1e-5 * abs(Eref), (Ez, Ex)
    hmax = np.abs(Href).max()
    assert np.abs(Hz.cpu().numpy() - Href).max() <= 1e-5 * hmax
    assert (Hz - Hx).abs().max().item() <= 1e-6 * hmax
    p.check_pipeline()
    p.close()


def test_energy_grad_in_the_z_pass_with_cell_weight():
    """M = Ms w m with a sphere mask: E taken in the z pass and the gradient
    -mu0 V Ms w H from the last pass, against the oracle."""
    from paper_1204_4302_gb300.plan import Plan
    n, d, Ms = (40, 36, 72), (2e-9, 2e-9, 2e-9), 8e5
    w = inputs.sphere_mask(n, 18)
    m = inputs.random_unit(n, seed=65)
    M = Ms * w[None] * m
    Href = oracle.field_fft(M, d)
    Eref = oracle.energy(M, Href, d)
    p = Plan(n, d, prec="f32")
    p.set_variants(6, 0, 1)
    assert p.info()["energy_in_z"] == 1
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    wt = torch.tensor(w, dtype=torch.float32, device="cuda")
    E, G = p.energy_grad(mt, Ms, w=wt)
    torch.cuda.synchronize()
    assert abs(E.item() - Eref) <= 1e-5 * abs(Eref)
    Gref = -oracle.MU0 * np.prod(d) * Ms * w[None] * Href
    assert np.abs(G.cpu().numpy() - Gref).max() <= 1e-5 * np.abs(Gref).max()
    p.close()


def test_energy_route_flag_off_the_persistent_pass():
    """FP64 plans, other z forms and smooth padding keep the last pass's sum."""
    from paper_1204_4302_gb300.plan import Plan
    d = (1e-9, 1e-9, 1e-9)
    p = Plan((16, 16, 100), d, prec="f64")
    assert p.info()["energy_in_z"] == 0
    p.close()
    p = Plan((16, 16, 100), d, prec="f32")
    p.set_variants(0, 0, 1)
    assert p.info()["energy_in_z"] == 0
    p.set_variants(6, 0, 1)
    assert p.info()["energy_in_z"] == 1
    p.close()
    p = Plan((16, 16, 30), d, prec="f32", pad="smooth")
    assert p.info()["energy_in_z"] == 0
    p.close()
