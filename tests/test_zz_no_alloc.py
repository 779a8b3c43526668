"""The allocation-free energy entry point (demag_energy_noalloc), called
through the C ABI, against the regular energy of demag_field_energy on the
same field: two calls in a row, each within the energy tolerance the other
tests use (10x the field tolerance: 1e-4 relative in FP32, 1e-11 in FP64).

It exists for callers that cannot allocate device memory where they need
the energy (graph capture in the global mode, pool-only hosts, loops that
must not synchronise), so it keeps its partial sums in a fixed library-owned
device array. This file sorts last so that a run stopping at the first
failure has run every other test before it."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("f32", 1e-4), ("f64", 1e-11)])
def test_noalloc_energy_matches_regular_energy_twice(prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300 import build, inputs
    build.build()
    n = (40, 28, 12)
    d = (2e-9, 2e-9, 2e-9)
    code = B.DEMAG_F32 if prec == "f32" else B.DEMAG_F64
    dt = torch.float32 if prec == "f32" else torch.float64
    M = torch.tensor(8e5 * inputs.random_unit(n, seed=31), dtype=dt, device="cuda")
    H = torch.empty_like(M)
    E_ref = torch.empty((), dtype=torch.float64, device="cuda")
    plan = B.demag_plan_create(*n, *d, code)
    try:
        B.demag_tensor_setup(plan)
        B.demag_field_energy(plan, M.data_ptr(), H.data_ptr(), E_ref.data_ptr())
        torch.cuda.synchronize()
        ref = E_ref.item()
        got = []
        for _ in range(2):
            E = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
            B.demag_energy_noalloc(*n, *d, code, M.data_ptr(), H.data_ptr(), E.data_ptr())
            torch.cuda.synchronize()
            got.append(E.item())
        for e in got:
            assert abs(e - ref) <= tol * abs(ref), (e, ref)
        assert got[0] == got[1]
        # on a non-default stream, with the device's free memory unchanged
        side = torch.cuda.Stream()
        E2 = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        with torch.cuda.stream(side):
            B.demag_energy_noalloc(*n, *d, code, M.data_ptr(), H.data_ptr(), E2.data_ptr(), side.cuda_stream)
        side.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert E2.item() == got[0]
        # a grid beyond the fixed partial-sum array is refused, nothing launched
        with pytest.raises(B.DemagError) as err:
            B.demag_energy_noalloc(1024, 1024, 512, *d, code, M.data_ptr(), H.data_ptr(), E.data_ptr())
        assert err.value.name == "DEMAG_ERR_UNSUPPORTED"
    finally:
        B.demag_plan_destroy(plan)
