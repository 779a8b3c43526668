"""Out-of-bounds writes, looked for without compute-sanitizer: with
DEMAG_DEBUG=1 every device buffer a plan allocates sits between two 4 KB
guard zones of 0xA5 bytes, and demag_check_pipeline scans them. Each test
runs the field, adjoint, energy and gradient entry points (and the SP
potential) on the mixed-radix grids (every stage radix the generic passes
instantiate), on power-of-two grids through every z-pass form, and on SP
plans, with the caller's M and H inside guard bands of their own (a sentinel
value before and after each tensor); then checks the guard zones and the
bands. The scan itself is tested by overwriting one guard byte from the
host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1204_4302_gb300 import inputs  # noqa: E402

BAND = 1024          # elements of sentinel before and after each caller tensor
SENTINEL = -12345.0


@pytest.fixture(scope="module", autouse=True)
def _built_debug():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()
    mp = pytest.MonkeyPatch()
    mp.setenv("DEMAG_DEBUG", "1")
    yield
    mp.undo()


def _banded(shape, dtype, fill=None):
    n = int(np.prod(shape))
    big = torch.full((n + 2 * BAND,), SENTINEL, dtype=dtype, device="cuda")
    view = big[BAND:BAND + n].view(shape)
    if fill is not None:
        view.copy_(fill)
    return big, view


def _bands_intact(big):
    return bool((big[:BAND] == SENTINEL).all()) and bool((big[-BAND:] == SENTINEL).all())


def _exercise(n, d, prec, pad=None, zv=None, method="dm"):
    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.plan import Plan
    dt = torch.float32 if prec == "f32" else torch.float64
    before = B.demag_debug_guard_count()
    p = Plan(n, d, prec=prec, pad=pad, method=method)
    assert B.demag_debug_guard_count() > before  # the plan's buffers are guarded
    if zv is not None:
        p.set_variants(zv, 0, 0)
    shape = (3, n[2], n[1], n[0])
    m = torch.tensor(inputs.random_unit(n, seed=sum(n)), dtype=dt, device="cuda")
    bigM, M = _banded(shape, dt, 8e5 * m)
    bigH, H = _banded(shape, dt)
    st = torch.cuda.current_stream().cuda_stream
    if method == "sp":
        bigP, P = _banded((n[2] + 1, n[1] + 1, n[0] + 1), dt)
        B.demag_sp_potential(p.handle, M.data_ptr(), P.data_ptr(), st)
        E = torch.empty((), dtype=torch.float64, device="cuda")
        B.demag_field_energy(p.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(), st)
        torch.cuda.synchronize()
        assert _bands_intact(bigP)
    else:
        E = torch.empty((), dtype=torch.float64, device="cuda")
        B.demag_field_energy(p.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(), st)
        bigA, A = _banded(shape, dt)
        B.demag_field_adjoint(p.handle, H.data_ptr(), A.data_ptr(), st)
        p.energy(M)
        bigG, G = _banded(shape, dt)
        E2 = torch.empty((), dtype=torch.float64, device="cuda")
        B.demag_energy_grad(p.handle, m.data_ptr(), None, 8e5, E2.data_ptr(), G.data_ptr(), None, st)
        torch.cuda.synchronize()
        assert _bands_intact(bigA) and _bands_intact(bigG)
    assert _bands_intact(bigM) and _bands_intact(bigH)
    assert torch.isfinite(H).all()
    p.check_pipeline()   # raises on an overwritten guard zone
    p.close()


MIXED = [((80, 24, 10), "smooth"), ((13, 9, 5), (42, 18, 10)), ((15, 11, 6), (30, 24, 14)),
         ((7, 20, 3), (16, 40, 6)), ((50, 3, 49), (100, 6, 98)), ((400, 4, 3), (800, 8, 6)),
         ((3, 300, 2), (6, 600, 4)), ((4, 3, 250), (8, 6, 500)), ((64, 16, 1), "smooth"), ((1, 1, 1), "smooth"),
         ((9, 9, 20), (18, 18, 40)), ((10, 10, 18), (20, 20, 36)), ((14, 14, 21), (28, 28, 42)),
         ((20, 27, 27), (40, 54, 54)), ((25, 25, 25), (50, 50, 50)), ((42, 42, 42), (84, 84, 84)),
         ((49, 49, 49), (98, 98, 98)), ((75, 80, 6), (150, 160, 12)), ((81, 81, 4), (162, 162, 8)),
         ((20, 20, 4), (40, 40, 8)), ((4, 4, 75), (8, 8, 150)), ((4, 4, 147), (8, 8, 294)),
         ((4, 4, 243), (8, 8, 486)), ((4, 4, 315), (8, 8, 630)), ((4, 4, 320), (8, 8, 640))]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,pad", MIXED)
def test_mixed_radix_grids_stay_in_bounds(n, pad, prec):
    _exercise(n, (1e-9, 1.1e-9, 0.9e-9), prec, pad=pad)


@pytest.mark.parametrize("zv", [0, 1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("n", [(33, 17, 5), (40, 6, 100), (9, 17, 129), (24, 24, 24), (20, 30, 16)])
def test_power_of_two_z_forms_stay_in_bounds(n, zv):
    _exercise(n, (2e-9, 1.5e-9, 1e-9), "f32", zv=zv)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,pad", [((20, 12, 7), None), ((15, 11, 6), "smooth"), ((33, 17, 5), None)])
def test_sp_plans_stay_in_bounds(n, pad, prec):
    _exercise(n, (1e-9, 1e-9, 2e-9), prec, pad=pad, method="sp")


def test_the_scan_finds_an_overwritten_guard_byte():
    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.plan import Plan
    p = Plan((8, 8, 8), (1e-9,) * 3, prec="f32")
    p.check_pipeline()
    B.demag_debug_poke_guard()
    with pytest.raises(B.DemagError) as ei:
        p.check_pipeline()
    assert ei.value.status == 7
    p.close()   # frees the poked block: the scan is clean again
    q = Plan((8, 8, 8), (1e-9,) * 3, prec="f32")
    q.check_pipeline()
    q.close()
