"""C ABI behaviour on the GPU: error statuses, timing, launch counts. Bad
pointers are rejected on the host before any kernel runs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def test_error_statuses():
    from paper_1204_4302_gb300 import binding as B
    n = (8, 6, 4)
    h = B.demag_plan_create(*n, 1e-9, 1e-9, 1e-9, B.DEMAG_F32)
    M = torch.zeros(3, 4, 6, 8, device="cuda")
    H = torch.zeros_like(M)
    with pytest.raises(B.DemagError) as e:
        B.demag_field(h, M.data_ptr(), H.data_ptr())
    assert e.value.name == "DEMAG_ERR_NOT_SETUP"
    B.demag_tensor_setup(h)
    B.demag_tensor_setup(h)  # idempotent
    with pytest.raises(B.DemagError) as e:
        B.demag_field(h, M.data_ptr(), M.data_ptr())
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"   # in place
    with pytest.raises(B.DemagError) as e:
        B.demag_field(h, M.data_ptr() + 4, H.data_ptr())
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"   # misaligned
    host = torch.zeros(3, 4, 6, 8)
    with pytest.raises(B.DemagError) as e:
        B.demag_field(h, host.data_ptr(), H.data_ptr())
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"   # host memory
    with pytest.raises(B.DemagError) as e:
        B.demag_energy_grad(h, M.data_ptr(), None, 1.0, None, None)
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"   # nothing to compute
    B.demag_field(h, M.data_ptr(), H.data_ptr())
    torch.cuda.synchronize()
    assert float(H.abs().max()) == 0.0
    B.demag_plan_destroy(h)


def test_info_and_launch_count():
    from paper_1204_4302_gb300.plan import Plan
    plan = Plan((40, 30, 5), (1e-9, 1e-9, 1e-9), prec="f32")
    info = plan.info()
    assert (info["px"], info["py"], info["pz"]) == (128, 64, 16)
    assert info["kx"] == 65
    assert info["launches_per_field"] == 5
    c0 = plan.launch_count()
    M = torch.randn(3, 5, 30, 40, device="cuda")
    plan.field(M)
    assert plan.launch_count() - c0 == 5
    plan.field_energy(M)
    assert plan.launch_count() - c0 == 11
    plan.close()


def test_timing_records_each_pass():
    from paper_1204_4302_gb300.plan import Plan
    plan = Plan((64, 64, 32), (1e-9, 1e-9, 1e-9), prec="f32")
    M = torch.randn(3, 32, 64, 64, device="cuda")
    plan.set_timing(True)
    for _ in range(70):   # more calls than the event ring holds
        plan.field(M)
    ms, cnt = plan.get_timing(6)
    assert cnt[:5] == [70] * 5
    assert all(v > 0 for v in ms[:5])
    plan.set_timing(False)
    plan.close()


def test_stream_ordering():
    """Work issued on a side stream stays ordered with the torch stream it came from."""
    from paper_1204_4302_gb300.plan import Plan
    plan = Plan((32, 32, 8), (1e-9, 1e-9, 1e-9), prec="f32")
    s = torch.cuda.Stream()
    M = torch.randn(3, 8, 32, 32, device="cuda")
    ref = plan.field(M)
    with torch.cuda.stream(s):
        M2 = M * 1.0
        H = plan.field(M2)
    torch.cuda.current_stream().wait_stream(s)
    assert torch.equal(H, ref)
    plan.close()
