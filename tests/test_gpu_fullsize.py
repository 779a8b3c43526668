"""Parity at the full sizes of the benchmark workloads.

Where the oracle can evaluate the whole field in seconds (the 512x128x4 film,
the 64^3 sphere, the 128^3 cube) the comparison is element by element. At
256^3 and 512x512x128 the oracle checks single outputs it can compute one by
one: fields of a few point sources (each target a short direct sum with the
oracle's cell tensor) and the closed-form field of a uniformly magnetized
body; plus properties that hold at any size (operator symmetry, FP32 vs
FP64 agreement).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1204_4302_gb300 import inputs  # noqa: E402

MS = 8e5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_film_512x128x4_fp32_elementwise():
    """Thin-film workload: vortex (in-plane curl, Feldtkeller core) + 5% noise."""
    from paper_1204_4302_gb300.plan import Plan
    n, d = (512, 128, 4), (2e-9, 2e-9, 2e-9)
    ext = tuple(a * b for a, b in zip(n, d))
    m = inputs.vortex_noise(n, ext, rc=0.14 * ext[0], noise=0.05, seed=2)
    M = MS * m
    Href = oracle.field_fft(M, d)
    p = Plan(n, d, prec="f32")
    H, E = p.field_energy(torch.tensor(M, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert _relmax(H.double().cpu().numpy(), Href) <= 1e-5
    Eref = oracle.energy(M, Href, d)
    assert abs(E.item() - Eref) <= 1e-5 * abs(Eref)
    p.close()


@pytest.mark.parametrize("state", ["uniform", "random"])
def test_sphere_64_masked_fp32_elementwise(state):
    """Sphere of radius 32 cells in 64^3 (staircase, paper Sec. 5.4), M = 0 outside."""
    from paper_1204_4302_gb300.plan import Plan
    n, d = (64, 64, 64), (2e-9, 2e-9, 2e-9)
    w = inputs.sphere_mask(n, 32)
    m = inputs.uniform(n, (0, 0, 1)) if state == "uniform" else inputs.random_unit(n, seed=3)
    M = MS * w[None] * m
    Href = oracle.field_fft(M, d)
    p = Plan(n, d, prec="f32")
    E, G = p.energy_grad(torch.tensor(m, dtype=torch.float32, device="cuda"), MS,
                         torch.tensor(w, dtype=torch.float32, device="cuda"))
    H = p.field(torch.tensor(M, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert _relmax(H.double().cpu().numpy(), Href) <= 1e-5
    Eref = oracle.energy(M, Href, d)
    assert abs(E.item() - Eref) <= 1e-5 * abs(Eref)
    Gref = -oracle.MU0 * d[0] * d[1] * d[2] * MS * w[None] * Href
    assert _relmax(G.double().cpu().numpy(), Gref) <= 1e-5
    p.close()


def test_cube_128_gradient_fp32_vs_fp64_oracle_and_fd():
    """Differentiation workload: E and dE/dm by the adjoint kernel behind
    autograd (FP32) against the FP64 oracle gradient element by element, and
    against central finite differences of the FP64 energy at 32 seeded probes."""
    from paper_1204_4302_gb300.autograd import demag_energy
    from paper_1204_4302_gb300.plan import Plan
    n, d = (128, 128, 128), (2e-9, 2e-9, 2e-9)
    m = inputs.random_unit(n, seed=5)
    Href = oracle.field_fft(MS * m, d)
    Gref = -oracle.MU0 * d[0] * d[1] * d[2] * MS * Href
    p32 = Plan(n, d, prec="f32")
    mt = torch.tensor(m, dtype=torch.float32, device="cuda", requires_grad=True)
    E = demag_energy(mt, MS, p32)
    E.backward()
    G = mt.grad.double().cpu().numpy()
    assert _relmax(G, Gref) <= 1e-5
    Eref = oracle.energy(MS * m, Href, d)
    assert abs(E.item() - Eref) <= 1e-5 * abs(Eref)
    p32.close()
    p64 = Plan(n, d, prec="f64")
    m64 = torch.tensor(m, device="cuda")
    rng = np.random.default_rng(5)
    h = 1e-3
    gmax = np.max(np.abs(Gref))
    for _ in range(32):
        c, k, j, i = (int(rng.integers(0, s)) for s in (3, n[2], n[1], n[0]))
        mp = m64.clone(); mp[c, k, j, i] += h
        mm = m64.clone(); mm[c, k, j, i] -= h
        fd = (p64.energy_grad(mp, MS, want_grad=False)[0].item() -
              p64.energy_grad(mm, MS, want_grad=False)[0].item()) / (2 * h)
        assert abs(fd - G[c, k, j, i]) <= 1e-5 * gmax, (c, k, j, i)
    p64.close()


def _sparse_sources(n, count, seed):
    rng = np.random.default_rng(seed)
    src = [tuple(int(rng.integers(0, v)) for v in n) for _ in range(count)]
    src += [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1)]
    mom = rng.standard_normal((len(src), 3))
    return src, mom


def _sparse_reference(src, mom, targets, d):
    """H at each target = -sum_sources N(target - source) M_source, with the
    oracle's cell tensor evaluated pair by pair."""
    out = np.zeros((len(targets), 3))
    for t, (ti, tj, tk) in enumerate(targets):
        acc = np.zeros(3)
        for (si, sj, sk), mv in zip(src, mom):
            R = ((ti - si) * d[0], (tj - sj) * d[1], (tk - sk) * d[2])
            c = oracle.cell_tensor(R, d)
            N = np.array([[c[0], c[3], c[4]], [c[3], c[1], c[5]], [c[4], c[5], c[2]]])
            acc -= N @ mv
        out[t] = acc
    return out


@pytest.mark.parametrize("n,d", [((256, 256, 256), (2e-9, 2e-9, 2e-9)),
                                 ((512, 512, 128), (1e-9, 1e-9, 1e-9))])
def test_full_size_point_sources(n, d):
    """A few point moments spread over the full grid: the field at sampled
    targets (sources, grid corners, random cells, far pairs) against direct
    sums of the oracle's tensor; FP64 to 1e-12, FP32 to 1e-5 (rel-max over
    the sampled targets, which include the source cells and so the maximum)."""
    from paper_1204_4302_gb300.plan import Plan
    src, mom = _sparse_sources(n, 24, seed=sum(n))
    rng = np.random.default_rng(1)
    targets = list(src) + [(0, n[1] - 1, 0), (n[0] - 1, 0, n[2] - 1), (n[0] // 2, n[1] // 2, n[2] // 2)]
    targets += [tuple(int(rng.integers(0, v)) for v in n) for _ in range(24)]
    ref = _sparse_reference(src, mom, targets, d)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        dt = torch.float32 if prec == "f32" else torch.float64
        M = torch.zeros((3, n[2], n[1], n[0]), dtype=dt, device="cuda")
        for (i, j, k), mv in zip(src, mom):
            M[:, k, j, i] += torch.tensor(mv, dtype=dt, device="cuda")
        p = Plan(n, d, prec=prec)
        H = p.field(M)
        idx = torch.tensor([[k, j, i] for (i, j, k) in targets], device="cuda")
        got = H[:, idx[:, 0], idx[:, 1], idx[:, 2]].T.double().cpu().numpy()
        assert _relmax(got, ref) <= tol, prec
        p.close()
        del M, H
        torch.cuda.empty_cache()


@pytest.mark.parametrize("n,d", [((256, 256, 256), (2e-9, 2e-9, 2e-9)),
                                 ((512, 512, 128), (1e-9, 1e-9, 1e-9))])
def test_full_size_uniform_body(n, d):
    """Uniform M: the cell-averaged field is exact on any grid (paper Sec. 5.1),
    H_cell = -N(cell, body) M from the oracle's two-box closed form."""
    from paper_1204_4302_gb300.plan import Plan
    mv = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    d = np.array(d)
    body_c = np.array(n) * d / 2
    body_e = np.array(n) * d
    rng = np.random.default_rng(2)
    cells = [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (n[0] // 2, n[1] // 2, n[2] // 2)]
    cells += [tuple(int(rng.integers(0, v)) for v in n) for _ in range(20)]
    ref = []
    for (i, j, k) in cells:
        t = oracle.box_tensor((np.array([i, j, k]) + 0.5) * d, d, body_c, body_e)
        N = np.array([[t[0], t[3], t[4]], [t[3], t[1], t[5]], [t[4], t[5], t[2]]])
        ref.append(-N @ mv)
    ref = np.array(ref)
    M = torch.empty((3, n[2], n[1], n[0]), dtype=torch.float32, device="cuda")
    for c in range(3):
        M[c] = float(mv[c])
    p = Plan(n, tuple(d), prec="f32")
    H = p.field(M)
    idx = torch.tensor([[k, j, i] for (i, j, k) in cells], device="cuda")
    got = H[:, idx[:, 0], idx[:, 1], idx[:, 2]].T.double().cpu().numpy()
    assert _relmax(got, ref) <= 1e-5
    p.close()


def test_large_forward_plus_adjoint_symmetry_and_precision():
    """512x512x128 smooth random state (Gaussian-filtered noise, 8 cells):
    <K a, b> = <a, K^T b> at full size, and FP32 within 1e-5 of FP64."""
    from paper_1204_4302_gb300.plan import Plan
    n, d = (512, 512, 128), (1e-9, 1e-9, 1e-9)
    a = torch.tensor(inputs.smooth_random(n, 8.0, seed=6), dtype=torch.float32, device="cuda")
    b = torch.tensor(inputs.random_unit(n, seed=7), dtype=torch.float32, device="cuda")
    p = Plan(n, d, prec="f32")
    Ka = p.field(a)
    KTb = p.field_adjoint(b)
    lhs = float((Ka.double() * b.double()).sum())
    rhs = float((a.double() * KTb.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float((Ka.double().abs() * b.double().abs()).sum())
    p.close()
    del KTb, b
    torch.cuda.empty_cache()
    p64 = Plan(n, d, prec="f64")
    K64 = p64.field(a.double())
    assert float((Ka.double() - K64).abs().max() / K64.abs().max()) <= 1e-5
    p64.close()
