"""Error paths under injected device-allocation failures (a host-side hook,
no GPU fault): every allocation of plan creation and tensor setup, for both
methods and precisions, fails once in turn; each failure is reported as
DEMAG_ERR_OOM, leaves no plan (creation) or a plan that is not set up
(setup), and nothing leaks; the next, un-failed attempt works."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1204_4302_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def _create(B, method, prec, n, d):
    if method == "sp":
        return B.demag_plan_create_sp(*n, *d, prec)
    return B.demag_plan_create(*n, *d, prec)


def test_each_allocation_failure_is_reported_and_freed():
    from paper_1204_4302_gb300 import binding as B
    n, d = (20, 12, 6), (1e-9, 1e-9, 1e-9)
    M = torch.tensor(8e5 * inputs.random_unit(n, seed=2), dtype=torch.float32, device="cuda")
    # warm-up: load every kernel once (module code and the runtime's local-memory
    # reservation are allocated on first use and kept, which is not a leak)
    for method in ("dm", "sp"):
        for prec in (B.DEMAG_F32, B.DEMAG_F64):
            h = _create(B, method, prec, n, d)
            B.demag_tensor_setup(h)
            Mw = M if prec == B.DEMAG_F32 else M.double()
            B.demag_field(h, Mw.data_ptr(), torch.empty_like(Mw).data_ptr())
            B.demag_plan_destroy(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for method in ("dm", "sp"):
        for prec in (B.DEMAG_F32, B.DEMAG_F64):
            failures = 0
            k = 1
            while True:
                B.demag_debug_fail_alloc(k)
                try:
                    h = _create(B, method, prec, n, d)
                except B.DemagError as e:
                    assert e.name == "DEMAG_ERR_OOM", (method, prec, k, str(e))
                    failures += 1
                    k += 1
                    continue
                try:
                    B.demag_tensor_setup(h)
                except B.DemagError as e:
                    assert e.name == "DEMAG_ERR_OOM", (method, prec, k, str(e))
                    with pytest.raises(B.DemagError) as e2:      # the plan is intact but not set up
                        B.demag_field(h, M.data_ptr(), torch.empty_like(M).data_ptr())
                    assert e2.value.name in ("DEMAG_ERR_NOT_SETUP", "DEMAG_ERR_INVALID_ARG")
                    B.demag_plan_destroy(h)
                    failures += 1
                    k += 1
                    continue
                B.demag_debug_fail_alloc(0)
                if prec == B.DEMAG_F32:
                    H = torch.empty_like(M)
                    B.demag_field(h, M.data_ptr(), H.data_ptr())
                    torch.cuda.synchronize()
                    assert torch.isfinite(H).all()
                B.demag_plan_destroy(h)
                break
            assert failures >= 8, (method, prec, failures)   # every buffer of creation and setup was hit
    B.demag_debug_fail_alloc(0)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < 8 << 20


def test_host_entry_allocation_failure():
    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.plan import Plan
    n = (16, 8, 4)
    p = Plan(n, (1e-9,) * 3)
    Mh = torch.tensor(8e5 * inputs.random_unit(n, seed=1), dtype=torch.float32).pin_memory()
    Hh = torch.empty_like(Mh).pin_memory()
    B.demag_debug_fail_alloc(1)
    with pytest.raises(B.DemagError) as e:
        B.demag_field_host(p.handle, Mh.data_ptr(), Hh.data_ptr())
    assert e.value.name == "DEMAG_ERR_OOM"
    B.demag_debug_fail_alloc(0)
    B.demag_field_host(p.handle, Mh.data_ptr(), Hh.data_ptr())
    ref = p.field(Mh.cuda()).cpu()
    assert torch.equal(ref, Hh)
    p.close()


def test_last_error_per_plan_and_per_thread():
    """demag_last_error(plan) keeps the latest failed call on that plan;
    demag_last_error(NULL) the calling thread's latest message."""
    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.plan import Plan
    p = Plan((8, 8, 8), (1e-9,) * 3, prec="f32")
    q = Plan((8, 8, 8), (1e-9,) * 3, prec="f32")
    assert B.demag_last_error(p.handle) == ""
    with pytest.raises(B.DemagError) as ei:
        B.demag_set_variants(p.handle, 99, 0)
    msg = B.demag_last_error(p.handle)
    assert msg and msg == B.demag_last_error() and msg in str(ei.value)
    assert B.demag_last_error(q.handle) == ""
    with pytest.raises(B.DemagError):
        B.demag_tg_plan_create(2, 2, 2, 1e-9, 1e-9, 1e-9, 1)   # plan-less failure
    assert B.demag_last_error() != msg
    assert B.demag_last_error(p.handle) == msg
    p.close()
    q.close()
