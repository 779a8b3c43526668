"""GPU parity of the mixed-radix passes: plans whose padded lengths are even
products of 2, 3, 5 and 7 instead of powers of two.

The zero-padded convolution of Sec. 3.1 is exact for every period P >= 2n - 1
per axis, so the field of such a plan equals the oracle's field (computed
with its own power-of-two period) up to rounding: same tolerances as the
power-of-two plans (rel-max FP64 <= 1e-12, FP32 <= 1e-5).
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


def _plan(n, d, prec, pad):
    from paper_1204_4302_gb300.plan import Plan
    return Plan(n, d, prec=prec, pad=pad)


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _smooth_pad(n):
    if n == 1:
        return 1
    p = 2 * n - 1
    while True:
        m = p
        for f in (2, 3, 5, 7):
            while m % f == 0:
                m //= f
        if m == 1 and p % 2 == 0:
            return p
        p += 1


# (n, d, pad): pad "smooth" = the smallest even 2,3,5,7-smooth length per axis
CASES = [
    ((80, 24, 10), (1e-9, 1e-9, 1e-9), "smooth"),         # 160 x 48 x 20: radix 8, 4, 5, 3
    ((13, 9, 5), (1e-9, 1.5e-9, 0.7e-9), (42, 18, 10)),   # radix 7 on x (L = 21), 3 x 3 on y, 5 on z
    ((15, 11, 6), (2e-9, 2e-9, 2e-9), (30, 24, 14)),      # odd x transform (L = 15), radix 7 on z
    ((7, 20, 3), (1e-9, 1e-9, 1e-9), (16, 40, 6)),        # power-of-two x with mixed y, z
    ((40, 36, 20), (1e-9, 1e-9, 1e-9), "smooth"),         # 80 x 72 x 40
    ((50, 3, 49), (1e-9, 1e-9, 1e-9), (100, 6, 98)),      # z length 98 = 2 7^2
    ((400, 4, 3), (1e-9, 1e-9, 1e-9), (800, 8, 6)),       # x transform of 400 points (the largest tile)
    ((3, 300, 2), (1e-9, 1e-9, 1e-9), (6, 600, 4)),       # y length 600
    ((4, 3, 250), (1e-9, 1e-9, 1e-9), (8, 6, 500)),       # z length 500
    ((64, 16, 1), (2e-9, 2e-9, 2e-9), "smooth"),          # film: Pz = 1
    ((1, 1, 1), (1e-9, 2e-9, 3e-9), "smooth"),            # single cell
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,d,pad", CASES)
def test_mixed_radix_field_matches_oracle(n, d, pad, prec):
    M = 8e5 * inputs.random_unit(n, seed=sum(n) + 7)
    Href = oracle.field_fft(M, d)
    plan = _plan(n, d, prec, pad)
    info = plan.info()
    want = tuple(_smooth_pad(v) for v in n) if pad == "smooth" else pad
    assert (info["px"], info["py"], info["pz"]) == want
    H = plan.field(torch.tensor(M, dtype=DT[prec], device="cuda"))
    torch.cuda.synchronize()
    assert _relmax(H.double().cpu().numpy(), Href) <= TOL[prec]
    plan.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_mixed_radix_energy_gradient_and_adjoint(prec):
    """Energy, dE/dm with a sphere mask, and the adjoint identity on a
    smooth-padded plan (every pass of the three entry points is mixed-radix)."""
    n, d = (26, 22, 12), (2e-9, 2e-9, 2e-9)   # padded 54 x 48 x 24
    Ms = 8e5
    w = inputs.sphere_mask(n, 10)
    m = inputs.random_unit(n, seed=31)
    M = Ms * w[None] * m
    Href = oracle.field_fft(M, d)
    Eref = oracle.energy(M, Href, d)
    Gref = -oracle.MU0 * d[0] * d[1] * d[2] * Ms * w[None] * Href
    plan = _plan(n, d, prec, "smooth")
    assert (plan.info()["px"], plan.info()["py"], plan.info()["pz"]) == (54, 48, 24)
    mt = torch.tensor(m, dtype=DT[prec], device="cuda")
    wt = torch.tensor(w, dtype=DT[prec], device="cuda")
    E, G = plan.energy_grad(mt, Ms, wt)
    torch.cuda.synchronize()
    assert abs(E.item() - Eref) <= 10 * TOL[prec] * abs(Eref)
    assert _relmax(G.double().cpu().numpy(), Gref) <= TOL[prec]
    a = torch.tensor(inputs.random_unit(n, seed=32), dtype=DT[prec], device="cuda")
    b = torch.tensor(inputs.random_unit(n, seed=33), dtype=DT[prec], device="cuda")
    Ka = plan.field(a).double()
    KTb = plan.field_adjoint(b).double()
    lhs = float((Ka * b.double()).sum())
    rhs = float((a.double() * KTb).sum())
    assert abs(lhs - rhs) <= 10 * TOL[prec] * float(Ka.abs().sum())
    plan.close()


def test_smooth_and_pow2_plans_agree():
    """Two periods of the same convolution: FP64 fields equal to rounding."""
    n, d = (33, 17, 9), (1e-9, 1e-9, 1e-9)
    M = torch.tensor(inputs.random_unit(n, seed=5), dtype=torch.float64, device="cuda")
    a = _plan(n, d, "f64", None)
    b = _plan(n, d, "f64", "smooth")
    assert (b.info()["px"], b.info()["py"], b.info()["pz"]) == (70, 36, 18)
    Ha = a.field(M).cpu().numpy()
    Hb = b.field(M).cpu().numpy()
    assert _relmax(Hb, Ha) <= 1e-13
    a.close()
    b.close()


def test_smooth_plan_tensor_spectrum_is_real():
    n = (21, 13, 11)
    plan = _plan(n, (1e-9, 1.1e-9, 0.9e-9), "f64", "smooth")
    assert plan.info()["tensor_imag_max"] < 1e-13
    plan.close()


def _point_source_field(src, mom, targets, d):
    out = np.zeros((len(targets), 3))
    for t, (ti, tj, tk) in enumerate(targets):
        for (si, sj, sk), mv in zip(src, mom):
            c = oracle.cell_tensor(((ti - si) * d[0], (tj - sj) * d[1], (tk - sk) * d[2]), d)
            N = np.array([[c[0], c[3], c[4]], [c[3], c[1], c[5]], [c[4], c[5], c[2]]])
            out[t] -= N @ mv
    return out


@pytest.mark.parametrize("n,d,P", [((200, 200, 40), (2e-9, 2e-9, 2e-9), (400, 400, 80)),
                                   ((300, 260, 100), (1e-9, 1e-9, 1e-9), (600, 540, 200))])
def test_mixed_radix_large_point_sources(n, d, P):
    """Large smooth-padded grids (powers of two would give 512 x 512 x 128 and
    1024 x 1024 x 256): point moments, sampled targets against direct sums of the
    oracle's cell tensor (sources included, so the maximum is sampled)."""
    rng = np.random.default_rng(sum(n))
    src = [tuple(int(rng.integers(0, v)) for v in n) for _ in range(16)] + [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1)]
    mom = [rng.standard_normal(3) for _ in src]
    targets = list(src) + [tuple(int(rng.integers(0, v)) for v in n) for _ in range(16)]
    ref = _point_source_field(src, mom, targets, d)
    for prec in ("f64", "f32"):
        M = torch.zeros((3, n[2], n[1], n[0]), dtype=DT[prec], device="cuda")
        for (i, j, k), mv in zip(src, mom):
            M[:, k, j, i] += torch.tensor(mv, dtype=DT[prec], device="cuda")
        plan = _plan(n, d, prec, "smooth")
        assert (plan.info()["px"], plan.info()["py"], plan.info()["pz"]) == P
        H = plan.field(M)
        idx = torch.tensor([[k, j, i] for (i, j, k) in targets], device="cuda")
        got = H[:, idx[:, 0], idx[:, 1], idx[:, 2]].T.double().cpu().numpy()
        assert _relmax(got, ref) <= TOL[prec], prec
        plan.close()
        del M, H
        torch.cuda.empty_cache()


def test_padding_autotuner_and_tuned_plan(tmp_path, monkeypatch):
    """The padding autotuner times every per-axis choice of power-of-two or
    smooth length; a plan created with pad="tuned" takes its choice (from the
    cache) and its field matches the oracle."""
    from paper_1204_4302_gb300 import binding as B
    monkeypatch.setenv("DEMAG_TUNE_CACHE", str(tmp_path / "tune.txt"))
    n, d = (70, 40, 20), (1e-9, 1e-9, 1e-9)
    P, ms_best, ms_pow2 = B.demag_tune_padding(*n, *d, B.DEMAG_F32, use_cache=True)
    assert P[0] in (256, 140) and P[1] in (128, 80) and P[2] in (64, 40)
    assert 0 < ms_best <= ms_pow2
    P2, mb2, mp2 = B.demag_tune_padding(*n, *d, B.DEMAG_F32, use_cache=True)  # from the cache file
    assert P2 == P and mb2 == pytest.approx(ms_best, abs=1e-6) and mp2 == pytest.approx(ms_pow2, abs=1e-6)
    plan = _plan(n, d, "f32", "tuned")
    assert (plan.info()["px"], plan.info()["py"], plan.info()["pz"]) == P
    M = 8e5 * inputs.random_unit(n, seed=77)
    H = plan.field(torch.tensor(M, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    assert _relmax(H, oracle.field_fft(M, d)) <= TOL["f32"]
    plan.close()


@pytest.mark.parametrize("pad", ["smooth", "tuned"])
def test_batch_with_mixed_radix_padding(pad, tmp_path, monkeypatch):
    """A batch of uneven grids padded to smooth lengths runs as a graph of
    per-state branches; every state's field and energy against the oracle."""
    from paper_1204_4302_gb300.batch import Batch
    monkeypatch.setenv("DEMAG_TUNE_CACHE", str(tmp_path / "tune.txt"))
    dims = [(33, 20, 9), (40, 36, 12), (17, 65, 5), (24, 24, 24)]
    cells = [(3e-9, 3e-9, 3e-9)] * len(dims)
    b = Batch(dims, cells, pad=pad)
    Ms = [8e5 * inputs.random_unit(n, seed=i) for i, n in enumerate(dims)]
    Hs, E = b.field([torch.tensor(m, dtype=torch.float32, device="cuda") for m in Ms], energies=True)
    torch.cuda.synchronize()
    if pad == "smooth":
        assert b.info()["mode"] == b.BRANCHES
    for m, h, e, d in zip(Ms, Hs, E.cpu().numpy(), cells):
        Href = oracle.field_fft(m, d)
        assert _relmax(h.double().cpu().numpy(), Href) <= TOL["f32"]
        Eref = oracle.energy(m, Href, d)
        assert abs(e - Eref) <= 10 * TOL["f32"] * abs(Eref)
    b.close()


# Every stage radix the mixed-radix passes instantiate (rows and columns: 2..16;
# the z pass: 5..32), each reached by the plan of some padded length here.
RADIX_CASES = [
    ((9, 9, 20), (18, 18, 40)),       # x 9 | y 6.3 | z 8.5
    ((10, 10, 18), (20, 20, 36)),     # x 10 | y 5.4 | z 6.6
    ((14, 14, 21), (28, 28, 42)),     # x 14 | y 7.4 | z 7.6
    ((20, 27, 27), (40, 54, 54)),     # x 5.4 | y 9.6 | z 9.6
    ((25, 25, 25), (50, 50, 50)),     # x 5.5 | y 10.5 | z 10.5
    ((42, 42, 42), (84, 84, 84)),     # x 7.6 | y 12.7 | z 12.7
    ((49, 49, 49), (98, 98, 98)),     # x 7.7 | y 14.7 | z 14.7
    ((75, 80, 6), (150, 160, 12)),    # x 15.5 | y 16.10 | z 12
    ((81, 81, 4), (162, 162, 8)),     # x 9.9 | y 9.9.2
    ((20, 20, 4), (40, 40, 8)),       # x 5.4 | y 8.5
    ((4, 4, 75), (8, 8, 150)),        # z 15.10
    ((4, 4, 80), (8, 8, 160)),        # z 16.10
    ((4, 4, 81), (8, 8, 162)),        # z 18.9
    ((4, 4, 100), (8, 8, 200)),       # z 20.10
    ((4, 4, 147), (8, 8, 294)),       # z 21.14
    ((4, 4, 192), (8, 8, 384)),       # z 24.16
    ((4, 4, 125), (8, 8, 250)),       # z 25.10
    ((4, 4, 243), (8, 8, 486)),       # z 27.18
    ((4, 4, 196), (8, 8, 392)),       # z 28.14
    ((4, 4, 315), (8, 8, 630)),       # z 30.21
    ((4, 4, 320), (8, 8, 640)),       # z 32.20
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,pad", RADIX_CASES)
def test_every_stage_radix_matches_oracle(n, pad, prec):
    d = (1e-9, 1.1e-9, 0.9e-9)
    M = 8e5 * inputs.random_unit(n, seed=sum(pad))
    Href = oracle.field_fft(M, d)
    plan = _plan(n, d, prec, pad)
    assert (plan.info()["px"], plan.info()["py"], plan.info()["pz"]) == pad
    H = plan.field(torch.tensor(M, dtype=DT[prec], device="cuda"))
    torch.cuda.synchronize()
    assert _relmax(H.double().cpu().numpy(), Href) <= TOL[prec]
    plan.close()


def test_batch_padding_autotuner_keeps_the_faster_padding():
    """demag_batch_autotune_padding times power-of-two and smooth padding of the
    same states and keeps the faster; the fields stay the oracle's."""
    from paper_1204_4302_gb300.batch import Batch
    dims = [(33, 20, 9), (40, 36, 12), (17, 65, 5), (24, 24, 24)]
    cells = [(3e-9, 3e-9, 3e-9)] * len(dims)
    b = Batch(dims, cells)
    t_pow2, t_smooth = b.autotune_padding(use_cache=False)
    assert t_pow2 > 0 and t_smooth > 0
    Ms = [8e5 * inputs.random_unit(n, seed=40 + i) for i, n in enumerate(dims)]
    for _ in range(2):                    # the first call after a rebuild builds the graphs
        Hs, E = b.field([torch.tensor(m, dtype=torch.float32, device="cuda") for m in Ms], energies=True)
    torch.cuda.synchronize()
    for m, h, e, d in zip(Ms, Hs, E.cpu().numpy(), cells):
        Href = oracle.field_fft(m, d)
        assert _relmax(h.double().cpu().numpy(), Href) <= TOL["f32"]
        assert abs(e - oracle.energy(m, Href, d)) <= 10 * TOL["f32"] * abs(oracle.energy(m, Href, d))
    b.close()
