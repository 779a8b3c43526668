"""Batched states of uneven grid sizes: the persistent kernel, the
pass-batched launches and the graph of branches against the per-state plans
and against the oracle; the bounded
dependency wait of the persistent kernel made to run out on purpose (a
dependency that never completes), after which the GPU context keeps working."""
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


def _states(count, lo, hi, seed, d=3e-9):
    dims = inputs.batch_sizes(count, lo=lo, hi=hi, seed=seed)
    cells = [(d, d, d)] * count
    ms = [torch.tensor(8e5 * inputs.random_unit(n, seed=100 + i), dtype=torch.float32, device="cuda")
          for i, n in enumerate(dims)]
    return dims, cells, ms


@pytest.fixture(scope="module")
def small_batch():
    from paper_1204_4302_gb300.batch import Batch
    dims, cells, ms = _states(7, (17, 9, 3), (70, 40, 20), seed=4)
    dims[0] = (33, 33, 8)     # a few fixed corner shapes
    dims[1] = (64, 17, 2)
    ms[0] = torch.tensor(8e5 * inputs.random_unit(dims[0], seed=1), dtype=torch.float32, device="cuda")
    ms[1] = torch.tensor(8e5 * inputs.random_unit(dims[1], seed=2), dtype=torch.float32, device="cuda")
    b = Batch(dims, cells)
    yield b, dims, cells, ms
    b.close()


def test_persistent_matches_per_state_plans(small_batch):
    from paper_1204_4302_gb300.plan import Plan
    b, dims, cells, ms = small_batch
    assert b.info()["persistent_ok"]
    b.set_mode(b.PERSISTENT)
    Hs, E = b.field(ms, energies=True)
    b.status()
    torch.cuda.synchronize()
    for i, (n, d, m) in enumerate(zip(dims, cells, ms)):
        p = Plan(n, d, prec="f32")
        H, Ei = p.field_energy(m)
        torch.cuda.synchronize()
        # same tile functions in the same order: identical up to reassociation-free rounding
        rel = float((Hs[i] - H).abs().max() / H.abs().max())
        assert rel <= 1e-6, (i, rel)
        assert abs(E[i].item() - Ei.item()) <= 1e-6 * abs(Ei.item())
        p.close()


def test_batch_matches_oracle(small_batch):
    b, dims, cells, ms = small_batch
    for mode in (b.PERSISTENT, b.BRANCHES, b.PASSES):
        b.set_mode(mode)
        Hs, E = b.field(ms, energies=True)
        torch.cuda.synchronize()
        for i in (0, 1, 4):
            M = ms[i].double().cpu().numpy()
            Href = oracle.field_fft(M, cells[i])
            rel = np.max(np.abs(Hs[i].double().cpu().numpy() - Href)) / np.max(np.abs(Href))
            assert rel <= 1e-5, (mode, i, rel)
            Eref = oracle.energy(M, Href, cells[i])
            assert abs(E[i].item() - Eref) <= 1e-4 * abs(Eref)


def test_modes_agree_and_replay_is_stable(small_batch):
    b, dims, cells, ms = small_batch
    b.set_mode(b.PERSISTENT)
    H0, E0 = b.field(ms, energies=True)
    H0 = [h.clone() for h in H0]
    H0b, _ = b.field(ms, energies=True)           # graph replay, new outputs
    b.set_mode(b.BRANCHES)
    H1, E1 = b.field(ms, energies=True)
    H1 = [h.clone() for h in H1]
    b.set_mode(b.PASSES)
    H2, E2 = b.field(ms, energies=True)            # first call: direct launches, then captured
    H2 = [h.clone() for h in H2]
    H2b, E2b = b.field(ms, energies=True)          # graph replay
    torch.cuda.synchronize()
    for a, c, e, f, g in zip(H0, H0b, H1, H2, H2b):
        assert torch.equal(a, c)
        assert float((a - e).abs().max() / e.abs().max()) <= 1e-6
        assert torch.equal(a, f)                    # the same tile functions: identical fields
        assert torch.equal(f, g)
    assert torch.allclose(E0, E1, rtol=1e-6, atol=0)
    assert torch.equal(E0, E2) and torch.equal(E2, E2b)
    b.set_mode(b.PERSISTENT)


def test_pass_batched_timing_records_each_pass(small_batch):
    b, dims, cells, ms = small_batch
    b.set_mode(b.PASSES)
    ref, _ = b.field(ms)
    ref = [h.clone() for h in ref]
    b.set_timing(True)
    for _ in range(3):
        Hs, _ = b.field(ms)
    t, calls = b.get_timing()
    b.set_timing(False)
    assert calls == 3 and all(v > 0 for v in t)
    for a, c in zip(ref, Hs):
        assert torch.equal(a, c)
    b.set_mode(b.PERSISTENT)


def test_bounded_wait_times_out_and_context_survives(small_batch):
    from paper_1204_4302_gb300 import binding as B
    b, dims, cells, ms = small_batch
    b.set_mode(b.PERSISTENT)
    ref, _ = b.field(ms)
    ref = [h.clone() for h in ref]
    b.set_timeout(0.02, stall_state=2)   # state 2 never finishes its first pass
    b.field(ms)
    with pytest.raises(B.DemagError) as err:
        b.status()
    assert err.value.name == "DEMAG_ERR_TIMEOUT"
    b.set_timeout(2.0, stall_state=-1)
    Hs, _ = b.field(ms)
    b.status()
    torch.cuda.synchronize()
    for a, c in zip(ref, Hs):
        assert torch.equal(a, c)


def test_config_sized_batch_runs_persistent():
    """64 states between 32x32x8 and 128x128x32 cells of 3 nm (the batched
    workload's size range), persistent kernel vs branches on a subset."""
    from paper_1204_4302_gb300.batch import Batch
    dims, cells, ms = _states(64, (32, 32, 8), (128, 128, 32), seed=4)
    b = Batch(dims, cells)
    assert b.info()["persistent_ok"]
    b.set_mode(b.PERSISTENT)
    H0, E0 = b.field(ms, energies=True)
    b.status()
    H0 = [h.clone() for h in H0]
    b.set_mode(b.BRANCHES)
    H1, E1 = b.field(ms, energies=True)
    H1 = [h.clone() for h in H1]
    b.set_mode(b.PASSES)
    H2, E2 = b.field(ms, energies=True)
    torch.cuda.synchronize()
    for a, c, e in zip(H0, H1, H2):
        assert float((a - c).abs().max() / c.abs().max()) <= 1e-6
        assert torch.equal(a, e)
    assert torch.allclose(E0, E1, rtol=1e-6, atol=0)
    b.close()


def test_batch_autotune_chooses_a_mode(tmp_path, monkeypatch):
    from paper_1204_4302_gb300.batch import Batch
    monkeypatch.setenv("DEMAG_TUNE_CACHE", str(tmp_path / "tune.txt"))
    dims, cells, ms = _states(5, (17, 9, 3), (70, 40, 20), seed=8)
    b = Batch(dims, cells)
    tp, tb = b.autotune()
    assert tb > 0 and (tp > 0 or tp == -1)
    mode = b.info()["mode"]          # the fastest of persistent, branches, pass-batched
    assert mode in (0, 1, 2)
    if mode == 1 and tp > 0:
        assert tb <= tp
    if mode == 0:
        assert tp <= tb
    Hs, _ = b.field(ms)
    torch.cuda.synchronize()
    for i in (0, 3):
        Href = oracle.field_fft(ms[i].double().cpu().numpy(), cells[i])
        rel = np.max(np.abs(Hs[i].double().cpu().numpy() - Href)) / np.max(np.abs(Href))
        assert rel <= 1e-5
    b.close()
