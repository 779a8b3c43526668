"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every entry point include/demag.h declares, fails cleanly (a status,
not a crash) when no CUDA device is present, and the Python mirrors of its
structs have the C layout."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "demag.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(demag_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1204_4302_gb300 import build, binding
    build.build()
    return binding.load()


def test_exports_every_declared_symbol(lib):
    from paper_1204_4302_gb300 import binding
    declared = _declared()
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTS) == declared


def test_status_strings(lib):
    from paper_1204_4302_gb300 import binding
    for code, name in binding.STATUS.items():
        assert binding.demag_status_string(code) == name


def test_invalid_arguments_are_rejected_before_any_device_call(lib):
    from paper_1204_4302_gb300 import binding
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_create(0, 4, 4, 1.0, 1.0, 1.0)
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_create(4, 4, 4, -1.0, 1.0, 1.0)
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_create(513, 4, 4, 1.0, 1.0, 1.0)
    assert e.value.name == "DEMAG_ERR_UNSUPPORTED"
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_create_ex(8, 8, 8, 1.0, 1.0, 1.0, 0, 22, 0, 0)  # prime factor 11
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_create_ex(8, 8, 8, 1.0, 1.0, 1.0, 0, 8, 0, 0)  # below 2n - 1
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"
    with pytest.raises(binding.DemagError) as e:
        binding.demag_field(None, None, None)
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"
    with pytest.raises(binding.DemagError):
        binding.demag_energy(None, None)
    binding.demag_plan_destroy(None)
    assert binding.demag_launch_count(None) == 0


def test_padding_options_are_checked_before_any_device_call(lib):
    """Padded lengths: powers of two or even products of 2, 3, 5, 7, at least
    2n - 1 and at most 1024; pad_mode 0 (powers of two), 1 (smooth) or 2
    (tuned, without explicit lengths); batches take a pad_mode only."""
    from paper_1204_4302_gb300 import binding
    bad = [({"px": 26}, "DEMAG_ERR_INVALID_ARG"),        # 2 x 13
           ({"px": 21}, "DEMAG_ERR_INVALID_ARG"),        # odd
           ({"py": 14}, "DEMAG_ERR_INVALID_ARG"),        # below 2n - 1
           ({"pz": 1050}, "DEMAG_ERR_UNSUPPORTED"),      # 2 3 5^2 7 > 1024
           ({"pad_mode": 3}, "DEMAG_ERR_INVALID_ARG"),
           ({"pad_mode": -1}, "DEMAG_ERR_INVALID_ARG"),
           ({"pad_mode": 2, "px": 16}, "DEMAG_ERR_INVALID_ARG")]  # tuned: no explicit lengths
    for kw, status in bad:
        with pytest.raises(binding.DemagError) as e:
            binding.demag_plan_create_ex(8, 8, 8, 1.0, 1.0, 1.0, 0, **kw)
        assert e.value.name == status, kw
    # accepted by the argument checks (then the device decides)
    for kw in [{"px": 18}, {"py": 42, "pz": 30}, {"pad_mode": 1}, {"px": 1000, "pad_mode": 1}]:
        try:
            h = binding.demag_plan_create_ex(8, 8, 8, 1.0, 1.0, 1.0, 0, **kw)
        except binding.DemagError as e:
            assert e.name not in ("DEMAG_ERR_INVALID_ARG", "DEMAG_ERR_UNSUPPORTED"), kw
        else:
            binding.demag_plan_destroy(h)
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_create_sp(8, 8, 8, 1.0, 1.0, 1.0, 0, pad_mode=2)
    assert e.value.name == "DEMAG_ERR_UNSUPPORTED"
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_create_sp(8, 8, 8, 1.0, 1.0, 1.0, 0, px=14)     # even and smooth but below 2n
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"
    for kw in [{"pad_mode": 1}, {"px": 18, "pz": 20}]:   # accepted by the checks
        try:
            h = binding.demag_plan_create_sp(8, 8, 8, 1.0, 1.0, 1.0, 0, **kw)
        except binding.DemagError as e:
            assert e.name not in ("DEMAG_ERR_INVALID_ARG", "DEMAG_ERR_UNSUPPORTED"), kw
        else:
            binding.demag_plan_destroy(h)
    import ctypes
    lib_ = binding.load()
    d = (ctypes.c_int * 3)(8, 8, 8)
    c = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    h = ctypes.c_void_p()
    opt = binding.demag_options(16, 0, 0, 0)
    assert lib_.demag_batch_create_ex(1, d, c, 0, ctypes.byref(opt), ctypes.byref(h)) == 1
    best = binding.demag_options()
    assert lib_.demag_tune_padding(8, 8, 8, 1.0, 1.0, 1.0, 0, 0, None, None, None, None) == \
        1  # DEMAG_ERR_INVALID_ARG
    assert lib_.demag_tune_padding(0, 8, 8, 1.0, 1.0, 1.0, 0, 0, ctypes.byref(best), None, None, None) == \
        1  # DEMAG_ERR_INVALID_ARG


def _smooth_even(p):
    if p % 2:
        return False
    for f in (2, 3, 5, 7):
        while p % f == 0:
            p //= f
    return p == 1


def test_padded_lengths_rules(lib):
    """Default padding: the smallest power of two >= 2n - 1; smooth: the
    smallest even length >= 2n - 1 with prime factors 2, 3, 5, 7 (brute force
    here); 1 for a single cell; explicit lengths kept."""
    from paper_1204_4302_gb300 import binding
    for n in list(range(1, 70)) + [100, 130, 200, 255, 257, 300, 333, 400, 511, 512]:
        pw = 1 if n == 1 else 1 << (2 * n - 2).bit_length()
        sm = 1 if n == 1 else next(p for p in range(2 * n - 1, 4 * n) if _smooth_even(p))
        assert binding.demag_padded_lengths(n, 1, 1) == (pw, 1, 1), n
        assert binding.demag_padded_lengths(1, n, 1, pad_mode=1) == (1, sm, 1), n
        assert sm <= pw and sm >= 2 * n - 1
    assert binding.demag_padded_lengths(8, 8, 8, px=18, pz=30) == (18, 16, 30)
    assert binding.demag_padded_lengths(130, 130, 130, pad_mode=1) == (270, 270, 270)
    with pytest.raises(binding.DemagError) as e:
        binding.demag_padded_lengths(8, 8, 8, pad_mode=2)
    assert e.value.name == "DEMAG_ERR_UNSUPPORTED"
    with pytest.raises(binding.DemagError) as e:
        binding.demag_padded_lengths(8, 8, 8, px=22)
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"


def _spec_file(path, *, magic=b"DMGSPEC\0", version=1, method=0, prec=0, n=(4, 3, 2), P=(8, 8, 4), ntab=6,
               d=(1e-9, 1e-9, 1e-9), count=None, payload=None, checksum=None, extra=b""):
    """A tensor-spectrum file in the library's format (header + FP32 table)."""
    import struct
    kx = P[0] // 2 + 1
    want = ntab * (P[2] // 2 + 1) * (P[1] // 2 + 1) * kx
    if payload is None:
        payload = struct.pack(f"<{want}f", *[0.25 * (i % 7) for i in range(want)])

    def fnv(b):
        h = 1469598103934665603
        for c in b:
            h = ((h ^ c) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
        return h
    hdr = struct.pack("<8s10i3dd", magic, version, method, prec, *n, *P, ntab, *d, 0.0)
    hdr += b"\0" * ((-len(hdr)) % 8)
    hdr += struct.pack("<QQ", want if count is None else count, fnv(payload) if checksum is None else checksum)
    with open(path, "wb") as f:
        f.write(hdr + payload + extra)


def test_spectrum_files_are_validated_before_any_device_call(lib, tmp_path):
    """demag_plan_load checks magic, version, sizes, padded lengths, table size
    and checksum on the host; a file that passes reaches the device step
    (here: no CUDA device)."""
    from paper_1204_4302_gb300 import binding
    good = tmp_path / "good.spec"
    _spec_file(good)
    try:
        h = binding.demag_plan_load(str(good))
    except binding.DemagError as e:
        assert e.name == "DEMAG_ERR_CUDA", e      # every check passed; no device here
    else:
        binding.demag_plan_destroy(h)
    bad = {
        "missing": None,
        "magic": dict(magic=b"NOTSPEC\0"),
        "version": dict(version=2),
        "method": dict(method=5),
        "ntab": dict(ntab=3),
        "size": dict(n=(600, 3, 2)),
        "padding": dict(P=(6, 8, 4)),            # below 2n - 1 for nx = 4
        "odd padding": dict(P=(9, 8, 4)),
        "count": dict(count=12345),
        "checksum": dict(checksum=1),
        "trailing": dict(extra=b"x"),
        "edge": dict(d=(0.0, 1e-9, 1e-9)),
    }
    for name, kw in bad.items():
        path = tmp_path / f"{name.replace(' ', '_')}.spec"
        if kw is not None:
            _spec_file(path, **kw)
        with pytest.raises(binding.DemagError) as e:
            binding.demag_plan_load(str(path))
        assert e.value.name == "DEMAG_ERR_INVALID_ARG", name
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_save(None, str(tmp_path / "x.spec"))
    assert e.value.name == "DEMAG_ERR_INVALID_ARG"


def test_sp_plan_arguments_are_checked_before_any_device_call(lib):
    """Scalar-potential plans: padding must be a power of two >= 2n (not 2n - 1),
    z is built up to 256 cells, and the usual size and edge checks apply."""
    from paper_1204_4302_gb300 import binding
    cases = [((0, 4, 4, 1.0, 1.0, 1.0), {}, "DEMAG_ERR_INVALID_ARG"),
             ((4, 4, 4, 1.0, 0.0, 1.0), {}, "DEMAG_ERR_INVALID_ARG"),
             ((8, 8, 257, 1.0, 1.0, 1.0), {}, "DEMAG_ERR_UNSUPPORTED"),
             ((513, 8, 8, 1.0, 1.0, 1.0), {}, "DEMAG_ERR_UNSUPPORTED"),
             ((8, 8, 8, 1.0, 1.0, 1.0), {"px": 15}, "DEMAG_ERR_INVALID_ARG"),
             ((8, 8, 8, 1.0, 1.0, 1.0), {"py": 8}, "DEMAG_ERR_INVALID_ARG")]
    for args, pad, status in cases:
        with pytest.raises(binding.DemagError) as e:
            binding.demag_plan_create_sp(*args, 0, **pad)
        assert e.value.name == status, (args, pad)


def test_tg_plan_arguments_are_checked_before_any_device_call(lib):
    """Tensor-grid plans: at least 3 cells per axis (second-order one-sided
    differences), at most 512, CP rank 1..64, positive edges."""
    from paper_1204_4302_gb300 import binding
    cases = [((2, 8, 8, 1.0, 1.0, 1.0, 1), "DEMAG_ERR_INVALID_ARG"),
             ((8, 8, 8, 1.0, -1.0, 1.0, 1), "DEMAG_ERR_INVALID_ARG"),
             ((8, 8, 8, 1.0, 1.0, 1.0, 0), "DEMAG_ERR_INVALID_ARG"),
             ((8, 8, 8, 1.0, 1.0, 1.0, 65), "DEMAG_ERR_INVALID_ARG"),
             ((513, 8, 8, 1.0, 1.0, 1.0, 1), "DEMAG_ERR_UNSUPPORTED")]
    for args, status in cases:
        with pytest.raises(binding.DemagError) as e:
            binding.demag_tg_plan_create(*args)
        assert e.value.name == status, args


def test_no_device_gives_a_cuda_status():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1204_4302_gb300 import binding
    with pytest.raises(binding.DemagError) as e:
        binding.demag_plan_create(4, 4, 4, 1.0, 1.0, 1.0)
    assert e.value.name in ("DEMAG_ERR_CUDA", "DEMAG_ERR_OOM")


def test_plan_refuses_without_cuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1204_4302_gb300.batch import Batch
    from paper_1204_4302_gb300.plan import Plan
    from paper_1204_4302_gb300.tg import TGPlan
    with pytest.raises(RuntimeError):
        Plan((4, 4, 4), (1.0, 1.0, 1.0))
    with pytest.raises(RuntimeError):
        Plan((4, 4, 4), (1.0, 1.0, 1.0), method="sp", pad="smooth")
    with pytest.raises(RuntimeError):
        Plan.load("any.spec")
    with pytest.raises(RuntimeError):
        Batch([(4, 4, 4)], [(1.0, 1.0, 1.0)], pad="smooth")
    with pytest.raises(RuntimeError):
        TGPlan((4, 4, 4), (1.0, 1.0, 1.0), 1)


def test_inputs_module_is_independent():
    """The input generators import neither the library nor the oracle."""
    src = open(os.path.join(ROOT, "paper_1204_4302_gb300", "inputs.py")).read()
    assert "import oracle" not in src and "binding" not in src and "torch" not in src


def test_noalloc_capacity_is_checked_before_the_sizes_are_multiplied(lib):
    """Axes whose product overflows 64-bit integers (2^21 each: 3 * 2^63) and
    axes just beyond the fixed array are refused as unsupported before any
    device call, never wrapped to a small or negative size."""
    from paper_1204_4302_gb300 import binding
    for dims in ((1 << 21, 1 << 21, 1 << 21), (2 ** 31 - 1, 2 ** 31 - 1, 2 ** 31 - 1), (1024, 1024, 512)):
        with pytest.raises(binding.DemagError) as e:
            binding.demag_energy_noalloc(*dims, 1.0, 1.0, 1.0, binding.DEMAG_F32, None, None, None)
        assert e.value.name == "DEMAG_ERR_UNSUPPORTED", dims


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of demag_options and demag_info have the C layout
    (size and every field offset), checked with a C program compiled against
    include/demag.h."""
    import ctypes
    import shutil
    import subprocess
    from paper_1204_4302_gb300 import binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "demag.h"', "int main(void) {"]
    for st in (B.demag_options, B.demag_info):
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in (B.demag_options, B.demag_info):
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)
