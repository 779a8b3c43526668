"""Tensor-spectrum files: a plan loaded from the file a set-up plan wrote
computes the same fields bit for bit (DM FP32/FP64, smooth padding, SP), keeps
its sizes, edges and setup residue, and a corrupted file is refused."""
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


@pytest.mark.parametrize("prec,pad,method", [("f32", None, "dm"), ("f64", None, "dm"), ("f32", "smooth", "dm"),
                                             ("f64", None, "sp"), ("f32", None, "sp")])
def test_saved_plan_reproduces_fields(tmp_path, prec, pad, method):
    from paper_1204_4302_gb300.plan import Plan
    n, d = (21, 13, 9), (1e-9, 1.3e-9, 0.8e-9)
    a = Plan(n, d, prec=prec, pad=pad, method=method)
    path = tmp_path / "plan.spec"
    a.save(str(path))
    b = Plan.load(str(path))
    ia, ib = a.info(), b.info()
    for k in ("nx", "ny", "nz", "px", "py", "pz", "prec", "method", "dx", "dy", "dz", "tensor_imag_max"):
        assert ia[k] == ib[k], k
    M = torch.tensor(8e5 * inputs.random_unit(n, seed=8), dtype=DT[prec], device="cuda")
    Ha, Hb = a.field(M), b.field(M)
    torch.cuda.synchronize()
    assert torch.equal(Ha, Hb)
    if method == "dm":
        Href = oracle.field_fft(M.double().cpu().numpy(), d)
        tol = 1e-5 if prec == "f32" else 1e-12
        assert float(np.max(np.abs(Hb.double().cpu().numpy() - Href)) / np.max(np.abs(Href))) <= tol
    a.close()
    b.close()


def test_corrupted_file_is_refused(tmp_path):
    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.plan import Plan
    a = Plan((16, 8, 4), (1e-9,) * 3)
    path = tmp_path / "plan.spec"
    a.save(str(path))
    raw = bytearray(path.read_bytes())
    raw[200] ^= 0x40                      # one bit of the table
    bad = tmp_path / "bad.spec"
    bad.write_bytes(bytes(raw))
    with pytest.raises(B.DemagError) as e:
        B.demag_plan_load(str(bad))
    assert e.value.name == "DEMAG_ERR_INVALID_ARG" and "checksum" in str(e.value)
    not_set_up = Plan((16, 8, 4), (1e-9,) * 3, setup=False)
    with pytest.raises(B.DemagError) as e:
        not_set_up.save(str(tmp_path / "x.spec"))
    assert e.value.name == "DEMAG_ERR_NOT_SETUP"
    a.close()
    not_set_up.close()
