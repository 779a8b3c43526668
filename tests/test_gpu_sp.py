"""Scalar-potential (SP) method on the GPU against the SP oracle.

The CUDA path (x and y forward passes, the SP z pass, one-component inverse
passes to the node potential, the finite-difference field) is compared with
the FP64 oracle element by element: the node potential and the field, FP64 to
1e-12 and FP32 to a bound derived from the arithmetic (below), on ragged
sizes that span several tiles, single layers, and the sizes whose padded
length is exactly 2n (the node rows then reach the middle of the period).

FP32 bound. The FFT convolution rounds the potential to about
eps32 * log2(Px Py Pz) relative to its largest value; the field divides
potential differences by one cell edge, so its error relative to the largest
field value is that amount times A = max|phi| / (max|H| min(d)), the ratio of
the potential's size to the field's size over one cell. The tests allow
4 eps32 log2(PxPyPz) (1 + A); measured errors are 3-6% of that bound
(e.g. 2e-5 for a uniformly magnetized 256^3 cube, A = 55; 4e-7 for random
states, A = 1.4).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1204_4302_gb300 import inputs  # noqa: E402

EPS32 = 2.0 ** -24
MS = 8e5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_4302_gb300 import build
    build.build()


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _fp32_bound(n, d, phi, H):
    P = [oracle.sp_padded_size(v) for v in n]
    A = float(np.max(np.abs(phi)) / (np.max(np.abs(H)) * min(d)))
    return 4 * EPS32 * math.log2(P[0] * P[1] * P[2]) * (1 + A)


SHAPES = [(1, 1, 1), (2, 3, 1), (5, 4, 3), (17, 9, 6), (16, 16, 8), (40, 33, 20), (64, 8, 4), (70, 5, 3),
          (33, 64, 17), (130, 6, 5), (9, 5, 40), (4, 3, 130), (128, 16, 16), (6, 200, 7)]


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sp_field_and_potential_match_oracle(n, prec):
    from paper_1204_4302_gb300.plan import Plan
    d = (2e-9, 1.5e-9, 2.5e-9)
    M = MS * inputs.random_unit(n, seed=sum(n))
    phi_ref = oracle.sp_potential_fft(M, d)
    H_ref = oracle.sp_field_from_potential(phi_ref, d)
    dt = torch.float32 if prec == "f32" else torch.float64
    p = Plan(n, d, prec=prec, method="sp")
    Mt = torch.tensor(M, dtype=dt, device="cuda")
    H = p.field(Mt).double().cpu().numpy()
    phi = p.potential(Mt).double().cpu().numpy()
    tol = 1e-12 if prec == "f64" else _fp32_bound(n, d, phi_ref, H_ref)
    assert _relmax(H, H_ref) <= tol, (n, prec, _relmax(H, H_ref), tol)
    assert _relmax(phi, phi_ref) <= (1e-12 if prec == "f64" else 8 * EPS32 * math.log2(
        np.prod([oracle.sp_padded_size(v) for v in n]))), n
    p.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sp_uniform_cube_and_energy(prec):
    """Uniform magnetization: the potential is that of a box (large, smooth),
    the case where the FP32 differences lose most; energy with the field."""
    from paper_1204_4302_gb300.plan import Plan
    n, d = (48, 40, 24), (1e-9, 1e-9, 1e-9)
    M = MS * inputs.uniform(n, (0.3, -0.4, 0.866))
    phi_ref = oracle.sp_potential_fft(M, d)
    H_ref = oracle.sp_field_from_potential(phi_ref, d)
    E_ref = oracle.energy(M, H_ref, d)
    dt = torch.float32 if prec == "f32" else torch.float64
    p = Plan(n, d, prec=prec, method="sp")
    H, E = p.field_energy(torch.tensor(M, dtype=dt, device="cuda"))
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "f64" else _fp32_bound(n, d, phi_ref, H_ref)
    assert _relmax(H.double().cpu().numpy(), H_ref) <= tol
    assert abs(E.item() - E_ref) <= (1e-12 if prec == "f64" else 1e-5) * abs(E_ref)
    assert abs(p.energy(torch.tensor(M, dtype=dt, device="cuda")) - E_ref) <= \
        (1e-12 if prec == "f64" else 1e-5) * abs(E_ref)
    p.close()


def test_sp_paper_energies_on_gpu():
    """The five SP energies the paper prints (cube homogeneous relative error,
    flower, vortex, thin-film homogeneous and vortex), computed by the CUDA
    path in FP64, to the printed digits."""
    import json
    import os
    from paper_1204_4302_gb300.plan import Plan
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_sp_energies.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        n = tuple(case["grid"])
        d = tuple(e / k for e, k in zip(case["extent"], n))
        ext = tuple(case["extent"])
        m = {"uniform_z": lambda: inputs.uniform(n, (0, 0, 1)),
             "flower": lambda: inputs.flower(n, ext),
             "vortex": lambda: inputs.vortex(n, ext, rc=0.14)}[case["state"]]()
        p = Plan(n, d, prec="f64", method="sp")
        H = p.field(torch.tensor(m, device="cuda")).cpu().numpy()
        p.close()
        e = oracle.energy_reduced(m, H, d)
        if "relerr_vs_exact" in case:
            val, ref = abs(e - case["exact"]) / case["exact"], case["relerr_vs_exact"]
        else:
            val, ref = e, case["e"]
        mag = 10 ** (math.floor(math.log10(abs(ref))) - case["digits"] + 1)
        assert abs(val - ref) <= 0.5 * mag, (case["name"], val)


def test_sp_info_and_unsupported_calls():
    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.plan import Plan
    n, d = (12, 10, 6), (1e-9, 1e-9, 1e-9)
    p = Plan(n, d, prec="f32", method="sp")
    info = p.info()
    assert info["method"] == B.DEMAG_METHOD_SP
    assert (info["px"], info["py"], info["pz"]) == (32, 32, 16)
    assert info["launches_per_field"] == 6
    assert info["tensor_imag_max"] < 1e-12 * 1e-9   # the kernel scales like a length
    M = torch.zeros((3, 6, 10, 12), device="cuda")
    with pytest.raises(B.DemagError) as e:
        p.field_adjoint(M)
    assert e.value.name == "DEMAG_ERR_UNSUPPORTED"
    with pytest.raises(B.DemagError) as e:
        p.energy_grad(M, 8e5)
    assert e.value.name == "DEMAG_ERR_UNSUPPORTED"
    before = p.launch_count()
    p.field(M)
    torch.cuda.synchronize()
    assert p.launch_count() - before == 6
    pd = Plan(n, d, prec="f32")
    with pytest.raises(B.DemagError):
        pd.potential(M)
    pd.close()
    p.close()


def test_sp_padding_choice_does_not_change_the_field():
    from paper_1204_4302_gb300.plan import Plan
    n, d = (10, 7, 5), (1e-9, 2e-9, 1e-9)
    M = torch.tensor(MS * inputs.random_unit(n, seed=9), device="cuda")
    a = Plan(n, d, prec="f64", method="sp").field(M)
    b = Plan(n, d, prec="f64", method="sp", pad=(64, 32, 32)).field(M)
    assert float((a - b).abs().max() / a.abs().max()) <= 1e-13


def test_sp_host_entry_point():
    from paper_1204_4302_gb300.plan import Plan
    n, d = (20, 12, 9), (1e-9, 1e-9, 1e-9)
    M = MS * inputs.random_unit(n, seed=4)
    p = Plan(n, d, prec="f64", method="sp")
    H = p.field_host(torch.tensor(M).pin_memory()).numpy()
    assert _relmax(H, oracle.sp_field(M, d)) <= 1e-12
    p.close()


def _corner_potential(src, mom, node, d):
    """Potential at one node by the direct sum over the sources (oracle kernel)."""
    acc = 0.0
    for (si, sj, sk), mv in zip(src, mom):
        R = ((node[0] - si - 0.5) * d[0], (node[1] - sj - 0.5) * d[1], (node[2] - sk - 0.5) * d[2])
        acc += float(np.dot(oracle.sp_kernel(R, d), mv))
    return acc


@pytest.mark.parametrize("n,d", [((256, 256, 256), (2e-9, 2e-9, 2e-9)),
                                 ((512, 512, 128), (1e-9, 1e-9, 1e-9))])
def test_sp_full_size_point_sources(n, d):
    """Full-size grids: a few point moments; at sampled cells (the sources,
    corners, random cells) the field from the node potentials of the direct
    sum with the oracle's kernel, differenced like the oracle does."""
    from paper_1204_4302_gb300.plan import Plan
    rng = np.random.default_rng(sum(n))
    src = [tuple(int(rng.integers(0, v)) for v in n) for _ in range(12)] + [(0, 0, 0)]
    mom = rng.standard_normal((len(src), 3))
    cells = list(src[:6]) + [(n[0] - 1, n[1] - 1, n[2] - 1), (n[0] // 2, 0, n[2] - 1)]
    cells += [tuple(int(rng.integers(0, v)) for v in n) for _ in range(8)]
    ref = []
    for (i, j, k) in cells:
        phi = np.zeros((2, 2, 2))
        for a in range(2):
            for b in range(2):
                for c in range(2):
                    phi[c, b, a] = _corner_potential(src, mom, (i + a, j + b, k + c), d)
        ref.append(oracle.sp_field_from_potential(phi, d)[:, 0, 0, 0])
    ref = np.array(ref)
    for prec in ("f64", "f32"):
        dt = torch.float32 if prec == "f32" else torch.float64
        M = torch.zeros((3, n[2], n[1], n[0]), dtype=dt, device="cuda")
        for (i, j, k), mv in zip(src, mom):
            M[:, k, j, i] += torch.tensor(mv, dtype=dt, device="cuda")
        p = Plan(n, d, prec=prec, method="sp")
        H = p.field(M)
        idx = torch.tensor([[k, j, i] for (i, j, k) in cells], device="cuda")
        got = H[:, idx[:, 0], idx[:, 1], idx[:, 2]].T.double().cpu().numpy()
        # point sources: the potential is no larger than the field over a cell
        tol = 1e-12 if prec == "f64" else 8 * EPS32 * math.log2(np.prod([oracle.sp_padded_size(v) for v in n])) * 4
        assert _relmax(got, ref) <= tol, (prec, _relmax(got, ref))
        p.close()
        del M, H
        torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [(17, 9, 20), (33, 64, 17), (40, 33, 64), (24, 20, 128), (9, 5, 100)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sp_tma_z_pass_variant(n, prec):
    """The persistent SP z pass with TMA-staged columns (z variant 5) gives the
    one-tile form's field and the oracle's, node rows reaching P/2 included."""
    from paper_1204_4302_gb300.plan import Plan
    d = (2e-9, 1.5e-9, 2.5e-9)
    M = MS * inputs.random_unit(n, seed=3 + sum(n))
    phi_ref = oracle.sp_potential_fft(M, d)
    H_ref = oracle.sp_field_from_potential(phi_ref, d)
    dt = torch.float32 if prec == "f32" else torch.float64
    p = Plan(n, d, prec=prec, method="sp")
    Mt = torch.tensor(M, dtype=dt, device="cuda")
    out = []
    for z in (0, 5):
        p.set_variants(z, 0)
        out.append(p.field(Mt).double().cpu().numpy())
    p.check_pipeline()
    tol = 1e-12 if prec == "f64" else _fp32_bound(n, d, phi_ref, H_ref)
    for H in out:
        assert _relmax(H, H_ref) <= tol
    assert np.array_equal(out[0], out[1])
    p.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,pad", [((17, 9, 6), "smooth"),                 # 36 x 18 x 12
                                   ((40, 33, 20), "smooth"),               # 80 x 70 x 40
                                   ((13, 11, 5), (30, 42, 10)),            # odd x transform (15), radix 7 on y
                                   ((70, 5, 100), (140, 12, 200)),         # z 200 = 20 . 10
                                   ((6, 100, 130), (12, 250, 270))])       # y 250, z 270 = 18 . 15
def test_sp_mixed_radix_padding_matches_oracle(n, pad, prec):
    """Scalar-potential plans on padded lengths that are products of 2, 3, 5, 7
    (the mixed-radix passes, including the SP z pass): field and node
    potential against the oracle (which pads to powers of two; every even
    period >= 2n gives the same convolution)."""
    from paper_1204_4302_gb300.plan import Plan
    d = (2e-9, 1.5e-9, 2.5e-9)
    M = MS * inputs.random_unit(n, seed=sum(n) + 3)
    phi_ref = oracle.sp_potential_fft(M, d)
    H_ref = oracle.sp_field_from_potential(phi_ref, d)
    dt = torch.float32 if prec == "f32" else torch.float64
    p = Plan(n, d, prec=prec, method="sp", pad=pad)
    info = p.info()
    P = (info["px"], info["py"], info["pz"])
    assert all(v >= 2 * m for v, m in zip(P, n)) and any(v & (v - 1) for v in P), P
    if pad != "smooth":
        assert P == pad
    Mt = torch.tensor(M, dtype=dt, device="cuda")
    H = p.field(Mt).double().cpu().numpy()
    phi = p.potential(Mt).double().cpu().numpy()
    tol = 1e-12 if prec == "f64" else _fp32_bound(n, d, phi_ref, H_ref)
    assert _relmax(H, H_ref) <= tol, (n, prec, _relmax(H, H_ref), tol)
    assert _relmax(phi, phi_ref) <= (1e-12 if prec == "f64" else 8 * EPS32 * math.log2(
        np.prod([oracle.sp_padded_size(v) for v in n]))), n
    p.close()
