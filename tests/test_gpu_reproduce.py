"""The paper-reproduction command (paper_1204_4302_gb300.reproduce): the DM
and SP energies of the paper's states from the CUDA path, against the values
the paper prints, and the convergence data behind its convergence figure."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def _digits_ok(value, printed, digits):
    mag = 10 ** (math.floor(math.log10(abs(printed))) - digits + 1)
    return abs(value - printed) <= 0.5 * mag


def test_states_match_the_printed_tables():
    from paper_1204_4302_gb300 import reproduce
    rows = {r["state"]: r for r in reproduce.run_states("f64")}
    cube = rows["cube_homogeneous"]
    assert cube["relerr_dm_vs_exact"] < 2.9e-9          # paper: 2.9e-9
    assert _digits_ok(cube["relerr_sp_vs_exact"], 1.1e-3, 2)
    for name in ("cube_flower", "cube_vortex", "film_homogeneous", "film_vortex"):
        p = rows[name]["paper"]
        assert _digits_ok(rows[name]["e_dm"], p["dm"], 4), name
        assert _digits_ok(rows[name]["e_sp"], p["sp"], 4), name
    # SP is a finite-difference approximation of the DM field: small but nonzero
    for name in ("cube_homogeneous", "cube_flower", "film_homogeneous"):
        assert 1e-4 < rows[name]["relerr_h"] < 1e-2, name
    sph = rows["sphere"]
    assert abs(sph["e_dm"] - math.pi / 36) / (math.pi / 36) < 0.02   # staircase at 40^3


def test_convergence_rows():
    from paper_1204_4302_gb300 import reproduce
    rows = reproduce.run_convergence("f64", sizes=(8, 16, 32))
    cube = [r for r in rows if r["state"] == "cube_homogeneous"]
    assert all(r["relerr_dm"] < 1e-9 for r in cube)          # DM is exact for uniform cells
    errs = [r["relerr_sp"] for r in cube]
    assert errs[0] > errs[1] > errs[2]                       # SP converges with the grid
    sph = [r for r in rows if r["state"] == "sphere"]
    assert sph[-1]["relerr_dm"] < sph[0]["relerr_dm"]
