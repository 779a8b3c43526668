"""CUDA-graph replay of plan calls: a captured call replays the same kernels,
so its results equal the directly launched call's bit for bit, for every
entry point, method and padding, across pointer changes (recapture, least
recently used eviction) and variant changes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1204_4302_gb300 import inputs  # noqa: E402

DT = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def _pair(n, d, prec, **kw):
    from paper_1204_4302_gb300.plan import Plan
    a = Plan(n, d, prec=prec, **kw)
    b = Plan(n, d, prec=prec, **kw)
    b.set_graphs(True)
    return a, b


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("pad", [None, "smooth"])
def test_graph_replay_equals_direct_launch(prec, pad):
    n, d = (20, 12, 7), (1e-9, 1.2e-9, 0.9e-9)
    a, b = _pair(n, d, prec, pad=pad)
    Ms = [torch.tensor(8e5 * inputs.random_unit(n, seed=s), dtype=DT[prec], device="cuda") for s in range(6)]
    w = torch.tensor(inputs.sphere_mask(n, 6), dtype=DT[prec], device="cuda")
    l0 = b.launch_count()
    for rep in range(3):                       # capture, then replays; 6 pointers > 4 slots: evictions
        for M in Ms:
            assert torch.equal(a.field(M), b.field(M))
            assert torch.equal(a.field_adjoint(M), b.field_adjoint(M))
            Ha, Ea = a.field_energy(M)
            Hb, Eb = b.field_energy(M)
            assert torch.equal(Ha, Hb) and Ea.item() == Eb.item()
            assert a.energy(M) == b.energy(M)
    Ea, Ga = a.energy_grad(Ms[0] / 8e5, 8e5, w)
    Eb, Gb = b.energy_grad(Ms[0] / 8e5, 8e5, w)
    torch.cuda.synchronize()
    assert Ea.item() == Eb.item() and torch.equal(Ga, Gb)
    assert b.launch_count() - l0 > 0
    # the replayed field is the oracle's
    Href = oracle.field_fft(Ms[1].double().cpu().numpy(), d)
    H = b.field(Ms[1]).double().cpu().numpy()
    tol = 1e-5 if prec == "f32" else 1e-12
    assert float(np.max(np.abs(H - Href)) / np.max(np.abs(Href))) <= tol
    a.close()
    b.close()


def test_graph_replay_counts_launches_and_follows_variants():
    n, d = (12, 40, 60), (2e-9, 2e-9, 2e-9)   # z length 128: several z variants
    a, b = _pair(n, d, "f32")
    M = torch.tensor(8e5 * inputs.random_unit(n, seed=3), dtype=torch.float32, device="cuda")
    H = torch.empty_like(M)
    l0 = a.launch_count()
    a.field(M, out=H)
    per_call = a.launch_count() - l0
    l1 = b.launch_count()
    for _ in range(3):
        b.field(M, out=H)
    assert b.launch_count() - l1 == 3 * per_call
    for z in (0, 1, 3, 5):
        a.set_variants(z, 0)
        b.set_variants(z, 0)
        assert torch.equal(a.field(M), b.field(M)), z
    b.set_timing(True)                         # timed calls launch directly
    assert torch.equal(a.field(M), b.field(M))
    b.set_timing(False)
    b.set_graphs(False)
    assert torch.equal(a.field(M), b.field(M))
    a.close()
    b.close()


def test_graph_replay_scalar_potential():
    from paper_1204_4302_gb300.plan import Plan
    n, d = (18, 10, 6), (1e-9, 1e-9, 1e-9)
    a = Plan(n, d, method="sp")
    b = Plan(n, d, method="sp")
    b.set_graphs(True)
    M = torch.tensor(8e5 * inputs.random_unit(n, seed=4), dtype=torch.float32, device="cuda")
    for _ in range(2):
        assert torch.equal(a.field(M), b.field(M))
        assert torch.equal(a.potential(M), b.potential(M))
    a.close()
    b.close()
