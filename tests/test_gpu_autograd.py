"""Gradients: DemagField / DemagEnergy backward passes against central finite
differences and against the FP64 oracle's gradient dE/dm = -mu0 V Ms w H."""
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


def test_energy_gradient_vs_central_differences_f64():
    from paper_1204_4302_gb300.autograd import demag_energy
    from paper_1204_4302_gb300.plan import Plan
    n, d, Ms = (12, 10, 8), (2e-9, 2e-9, 2e-9), 8e5
    plan = Plan(n, d, prec="f64")
    m0 = torch.tensor(inputs.random_unit(n, seed=5), device="cuda", requires_grad=True)
    E = demag_energy(m0, Ms, plan)
    E.backward()
    g = m0.grad.detach().cpu().numpy()
    rng = np.random.default_rng(7)
    m = m0.detach().clone()
    h = 1e-4
    for _ in range(32):
        c, k, j, i = (int(rng.integers(0, s)) for s in (3, n[2], n[1], n[0]))
        mp = m.clone(); mp[c, k, j, i] += h
        mm = m.clone(); mm[c, k, j, i] -= h
        fd = (plan.energy_grad(mp, Ms, want_grad=False)[0].item() -
              plan.energy_grad(mm, Ms, want_grad=False)[0].item()) / (2 * h)
        # E is quadratic in m: central differences are exact up to rounding
        assert abs(fd - g[c, k, j, i]) <= 1e-6 * np.max(np.abs(g)), (c, k, j, i)
    plan.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_energy_gradient_vs_oracle(prec):
    from paper_1204_4302_gb300.autograd import demag_energy
    from paper_1204_4302_gb300.plan import Plan
    n, d, Ms = (16, 12, 10), (1e-9, 1e-9, 1e-9), 8e5
    dt = torch.float32 if prec == "f32" else torch.float64
    m = inputs.random_unit(n, seed=6)
    w = inputs.sphere_mask(n, 6)
    plan = Plan(n, d, prec=prec)
    mt = torch.tensor(m, dtype=dt, device="cuda", requires_grad=True)
    wt = torch.tensor(w, dtype=dt, device="cuda")
    E = demag_energy(mt, Ms, plan, w=wt)
    (3.0 * E).backward()   # upstream gradient 3 is applied on the device
    M = Ms * w[None] * m
    Href = oracle.field_fft(M, d)
    Gref = 3.0 * (-oracle.MU0 * d[0] * d[1] * d[2] * Ms * w[None] * Href)
    G = mt.grad.double().cpu().numpy()
    tol = 1e-5 if prec == "f32" else 1e-12
    assert np.max(np.abs(G - Gref)) / np.max(np.abs(Gref)) <= tol
    assert abs(E.item() - oracle.energy(M, Href, d)) <= 10 * tol * abs(E.item())
    plan.close()


def test_field_backward_is_adjoint():
    from paper_1204_4302_gb300.autograd import demag_field
    from paper_1204_4302_gb300.plan import Plan
    n, d = (10, 9, 7), (1e-9, 1e-9, 1e-9)
    plan = Plan(n, d, prec="f64")
    M = torch.tensor(inputs.random_unit(n, seed=1), device="cuda", requires_grad=True)
    C = torch.tensor(inputs.random_unit(n, seed=2), device="cuda")
    H = demag_field(M, plan)
    (H * C).sum().backward()
    # d/dM sum(C . K M) = K^T C = K C (self-adjoint)
    want = oracle.field_fft(C.cpu().numpy(), d)
    got = M.grad.cpu().numpy()
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 1e-12
    plan.close()


def test_field_gradcheck_small():
    from paper_1204_4302_gb300.autograd import DemagField
    from paper_1204_4302_gb300.plan import Plan
    plan = Plan((3, 2, 2), (1e-9, 1e-9, 1e-9), prec="f64")
    M = torch.randn(3, 2, 2, 3, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: DemagField.apply(x, plan), (M,), eps=1e-6, atol=1e-8)
    plan.close()
