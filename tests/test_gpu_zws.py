"""The persistent TMA z pass (z variants 6 and 7: 8 or 4 columns per tile,
FP32): the paper's Sec. 3.1 fused
z transform / tensor product / inverse z transform, checked through the C ABI
against the FP64 oracle element by element (rel-max <= 1e-5), against the
two-stage z kernel (variant 0) on the same plan, and on the edge cases of its
tiling: ragged column tiles (Kx not a multiple of 8), nz below L/2, one ky
row (Py = 1), the fold of ky and kz at their Nyquist rows, and plans that
cannot take it (Px = 1, FP64) falling back to the two-stage kernel; z
lengths 512 (2 x 16 x 16) and 256 (16 x 16)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1204_4302_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# (nx, ny, nz) with Pz = 512 (129 <= nz <= 256) and Pz = 256 (65 <= nz <= 128)
SHAPES = [
    (9, 17, 129),    # Kx = 17: three tiles, the last with one column; Py = 64
    (5, 3, 256),     # nz = L/2 exactly; Kx = 9: a tile of one column
    (20, 12, 200),   # nz between; Kx = 33
    (33, 1, 256),    # Py = 1: one ky row
    (16, 2, 140),    # Py = 4: ky = Py/2 on the fold
    (7, 30, 255),    # odd sizes
    (9, 17, 65),     # L = 256 from here
    (5, 3, 128),
    (20, 12, 100),
    (33, 1, 128),
    (7, 30, 127),
]


@pytest.mark.parametrize("zv", [6, 7])
@pytest.mark.parametrize("n", SHAPES)
def test_persistent_z_pass_matches_oracle_and_two_stage_kernel(n, zv):
    from paper_1204_4302_gb300.plan import Plan
    d = (2e-9, 1.5e-9, 1e-9)
    M = 8e5 * inputs.random_unit(n, seed=41)
    Href = oracle.field_fft(M, d)
    Eref = oracle.energy(M, Href, d)
    p = Plan(n, d, prec="f32")
    Mt = torch.tensor(M, dtype=torch.float32, device="cuda")
    p.set_variants(0, 0, 1)
    H0 = p.field(Mt).double().cpu().numpy()
    p.set_variants(zv, 0, 1)
    H6, E6 = p.field_energy(Mt)
    H6 = H6.double().cpu().numpy()
    assert _relmax(H6, Href) <= 1e-5
    assert _relmax(H6, H0) <= 2e-6
    assert abs(E6.item() - Eref) <= 1e-4 * abs(Eref)
    # twice in a row (the persistent CTAs restart from the same state)
    H6b = p.field(Mt).double().cpu().numpy()
    assert np.array_equal(H6, H6b)
    p.check_pipeline()
    p.close()


@pytest.mark.parametrize("zv", [6, 7])
def test_persistent_z_pass_adjoint_and_gradient(zv):
    """The adjoint (the same pipeline) and the gradient epilogue."""
    from paper_1204_4302_gb300.plan import Plan
    n, d, Ms = (12, 10, 180), (2e-9, 2e-9, 2e-9), 8e5
    m = inputs.random_unit(n, seed=43)
    Href = oracle.field_fft(Ms * m, d)
    p = Plan(n, d, prec="f32")
    p.set_variants(zv, 0, 1)
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    E, G = p.energy_grad(mt, Ms)
    Gref = -oracle.MU0 * d[0] * d[1] * d[2] * Ms * Href
    assert _relmax(G.double().cpu().numpy(), Gref) <= 1e-5
    a = torch.tensor(inputs.random_unit(n, seed=44), dtype=torch.float32, device="cuda")
    b = torch.tensor(inputs.random_unit(n, seed=45), dtype=torch.float32, device="cuda")
    Ka = p.field(a)
    Kb = p.field_adjoint(b)
    lhs = float((Ka.double() * b.double()).sum())
    rhs = float((a.double() * Kb.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1e-30) + 1e-6 * float(Ka.double().abs().max()) * a.numel() ** 0.5
    p.check_pipeline()
    p.close()


@pytest.mark.parametrize("n,prec", [((1, 1, 200), "f32"), ((6, 5, 130), "f64")])
def test_plans_the_persistent_pass_cannot_take_fall_back(n, prec):
    """Px = 1 (rows of one complex value: not a TMA box) and FP64 plans run
    the two-stage kernel when variant 6 is asked for."""
    from paper_1204_4302_gb300.plan import Plan
    d = (1e-9, 1e-9, 1e-9)
    M = 8e5 * inputs.random_unit(n, seed=47)
    Href = oracle.field_fft(M, d)
    dt = torch.float32 if prec == "f32" else torch.float64
    p = Plan(n, d, prec=prec)
    for zv in (6, 7):
        p.set_variants(zv, 0, 1)
        H = p.field(torch.tensor(M, dtype=dt, device="cuda")).double().cpu().numpy()
        assert _relmax(H, Href) <= (1e-5 if prec == "f32" else 1e-12)
    p.close()


def test_persistent_z_pass_large_cuboid_against_two_stage_kernel():
    """512 x 512 x 128 (padded 1024 x 1024 x 256, the large workload): L = 256
    forms against the two-stage kernel on the same plan."""
    from paper_1204_4302_gb300.plan import Plan
    n, d = (512, 512, 128), (1e-9, 1e-9, 1e-9)
    g = torch.Generator(device="cuda").manual_seed(6)
    M = torch.randn(3, 128, 512, 512, device="cuda", generator=g)
    M = 8e5 * M / M.norm(dim=0, keepdim=True)
    p = Plan(n, d, prec="f32")
    p.set_variants(0, 2, 1)
    H0, E0 = p.field_energy(M)
    for zv in (6, 7):
        p.set_variants(zv, 2, 1)
        H6, E6 = p.field_energy(M)
        rel = float((H6 - H0).abs().max() / H0.abs().max())
        assert rel <= 2e-6, (zv, rel)
        assert abs(E6.item() - E0.item()) <= 1e-5 * abs(E0.item())
    p.check_pipeline()
    p.close()


def test_persistent_z_pass_full_size_against_two_stage_kernel():
    """256^3 (padded 512^3, the headline grid), seeded random unit state:
    variant 6 against variant 0 on the same plan, and the energy."""
    from paper_1204_4302_gb300.plan import Plan
    n, d = (256, 256, 256), (2e-9, 2e-9, 2e-9)
    g = torch.Generator(device="cuda").manual_seed(5)
    M = torch.randn(3, 256, 256, 256, device="cuda", generator=g)
    M = 8e5 * M / M.norm(dim=0, keepdim=True)
    p = Plan(n, d, prec="f32")
    p.set_variants(0, 2, 1)
    H0, E0 = p.field_energy(M)
    for zv in (6, 7):
        p.set_variants(zv, 2, 1)
        H6, E6 = p.field_energy(M)
        rel = float((H6 - H0).abs().max() / H0.abs().max())
        assert rel <= 2e-6, (zv, rel)
        assert abs(E6.item() - E0.item()) <= 1e-5 * abs(E0.item())
    p.check_pipeline()
    p.close()
