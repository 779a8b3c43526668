"""Host-side pieces of the mixed-radix passes, checked on the CPU:
* the compile-time cosines and sines of 2 pi e / n (the in-register DFT
  twiddles) against the C library, for every n <= 32;
* the stage planner: radices multiply to L, respect the per-pass limit, and
  the plan has the fewest stages and then the smallest largest radix (brute
  force over all splits);
* the multiply-high division that replaces runtime divisions: exact for all
  divisors d <= 4096 over the operands the kernels use (grid columns below
  2^20 divided by slab widths <= 513; element and butterfly indices below
  2^14 divided by tile, stage and row sizes)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1204_4302_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "mixed_impl.cuh"
int main()
{
    for (int n = 3; n <= 32; ++n)
        for (int e = 0; e < n; ++e)
            printf("T %d %d %.17g %.17g\n", n, e, demag::ct_cos2pi(e, n), demag::ct_sin2pi(e, n));
    for (int L = 2; L < 2048; ++L)
        for (int maxr : {16, 32}) {
            demag::GenRadix g;
            if (!demag::gen_plan(L, 4096, g, maxr, 1)) continue;
            printf("P %d %d %d", L, maxr, g.n);
            for (int s = 0; s < g.n; ++s) printf(" %d", g.r[s]);
            printf("\n");
        }
    return 0;
}
"""


def _smooth(r):
    for f in (2, 3, 5, 7):
        while r % f == 0:
            r //= f
    return r == 1


def _best_split(L, maxr, depth=4):
    """(fewest stages, smallest largest radix) over all splits into radices <= maxr."""
    radices = [r for r in range(2, maxr + 1) if _smooth(r)]
    best = None

    def rec(m, cur):
        nonlocal best
        if m == 1:
            key = (len(cur), max(cur))
            if best is None or key < best:
                best = key
            return
        if len(cur) == depth:
            return
        for r in radices:
            if m % r == 0 and (not cur or r <= cur[-1]):
                rec(m // r, cur + [r])
    rec(L, [])
    return best


@pytest.fixture(scope="module")
def host_output(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("mixed_host")
    src = d / "t.cu"
    src.write_text(PROGRAM)
    exe = d / "t"
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC, str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=600)
    return subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.splitlines()


def test_compile_time_twiddles(host_output):
    """Against 30-digit values (a double-precision angle 2 pi e / n would itself
    be off by up to an ulp of 2 pi, ~9e-16 in the sine near the full turn)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    worst = 0.0
    for line in host_output:
        if not line.startswith("T "):
            continue
        _, n, e, c, s = line.split()
        a = 2 * mpmath.pi * int(e) / int(n)
        worst = max(worst, abs(float(c) - float(mpmath.cos(a))), abs(float(s) - float(mpmath.sin(a))))
    assert worst <= 2.5e-16, worst


def test_stage_plans_are_minimal(host_output):
    seen = 0
    for line in host_output:
        if not line.startswith("P "):
            continue
        f = [int(v) for v in line.split()[1:]]
        L, maxr, n, r = f[0], f[1], f[2], f[3:]
        assert len(r) == n and math.prod(r) == L, line
        assert all(2 <= v <= maxr and _smooth(v) for v in r), line
        assert (len(r), max(r)) == _best_split(L, maxr), line
        seen += 1
    smooth_lengths = [L for L in range(2, 2048) if _smooth(L)]
    assert seen >= len(smooth_lengths)        # every smooth length has a plan for radix 32
    planned = {int(l.split()[1]) for l in host_output if l.startswith("P ") and int(l.split()[2]) == 32}
    assert planned == set(smooth_lengths)


def test_multiply_high_division_is_exact():
    for d in range(2, 4097):
        m = ((1 << 32) + d - 1) // d
        # slab widths (<= 513) divide grid columns (< 2^20); tile, stage and row
        # divisors (< 4096) divide element and butterfly indices (< 2^14)
        nmax = min((1 << 32) // d, 1 << 20 if d <= 513 else 1 << 14)
        n = np.arange(0, nmax, dtype=np.uint64)
        q = (n * np.uint64(m)) >> np.uint64(32)
        assert np.array_equal(q, n // np.uint64(d)), d
