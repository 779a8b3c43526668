"""FP64 CPU oracle for the FFT demagnetization-tensor (DM) stray field.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. The GPU library never
calls it and shares no code with it: the tensor comes from ``newell.c`` (closed
form of Newell et al. 1993 for touching cells, tent-weighted Gauss-Legendre
quadrature of the point kernel for separated cells) and the convolution from
``numpy.fft`` in float64.

What is computed (paper Sec. 2 and Sec. 3.1):

* ``field_bruteforce``: H_a = -sum_b N(r_a - r_b) M_b over all cell pairs, every
  signed offset evaluated directly (Eq. "demag" discretised on cells, with the
  cell-averaged tensor described in Sec. 5.1).
* ``field_fft``: the same sum as a zero-padded FFT convolution (Eq.
  "convolution", applied to the matrix kernel as Sec. 3.1 describes for DM):
  pad every axis to P >= 2N - 1, place N at wrapped offsets, multiply the 3x3
  tensor spectrum with the magnetization spectrum, invert, crop.
* ``energy``: E = -(mu0/2) V sum_cells M.H (Sec. 2, energy e_d, read in SI
  units; the paper's values in units of mu0 Ms^2 follow with m = M/Ms).

Layout: M and H are float64 arrays of shape (3, nz, ny, nx) (x fastest).
The tensor table has shape (6, nz, ny, nx) in the order xx, yy, zz, xy, xz, yz.

The scalar-potential method (SP, Sec. 3.1, Eqs. "scpot" and "field") has its
own oracle in ``scalar_potential.c`` and the ``sp_*`` functions below: the
potential at the grid nodes as the sum over cells of M . S with the vector
kernel S of one homogeneously magnetized cell, by direct sum or by zero-padded
FFT convolution, and the field of each cell from the node potentials by
finite differences (the cell average of minus the gradient of the trilinear
interpolant). Potentials have shape (nz+1, ny+1, nx+1).

The tensor-grid method (TG, Sec. 3.2) has its oracle in ``tensor_grid.py``
(``oracle.tensor_grid``): sinc quadrature of the Gaussian representation of
1/r^3, closed-form Gaussian matrices, mode products for dense and CP
magnetization, the exact cell-centre potential for comparison, and the
second-order finite-difference field.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

MU0 = 4e-7 * math.pi  # exact SI value used by the library as well

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_SO = _BUILD / "liboracle.so"
_lib = None

COMPONENTS = ("xx", "yy", "zz", "xy", "xz", "yz")


_SOURCES = ("newell.c", "scalar_potential.c")


def build(force: bool = False) -> Path:
    """Compile the oracle's C sources into oracle/_build/liboracle.so with gcc (no fast-math)."""
    srcs = [_HERE / s for s in _SOURCES]
    if _SO.exists() and not force and all(_SO.stat().st_mtime >= s.stat().st_mtime for s in srcs):
        return _SO
    _BUILD.mkdir(exist_ok=True)
    tmp = _BUILD / f"liboracle.{os.getpid()}.so"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
           *[str(s) for s in srcs], "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(str(_SO))
    D = ctypes.c_double
    I = ctypes.c_int
    P = ctypes.c_void_p
    lib.oracle_box_tensor.argtypes = [P, P, P, P, P]
    lib.oracle_cell_tensor_closed.argtypes = [D, D, D, D, D, D, P]
    lib.oracle_cell_tensor_quad.argtypes = [D, D, D, D, D, D, I, I, I, P]
    lib.oracle_cell_tensor_quad.restype = I
    lib.oracle_cell_tensor.argtypes = [D, D, D, D, D, D, P]
    lib.oracle_gl_rule.argtypes = [I, P, P]
    lib.oracle_gl_rule.restype = I
    lib.oracle_tensor_octant.argtypes = [I, I, I, D, D, D, I, P]
    lib.oracle_tensor_octant.restype = I
    lib.oracle_tensor_signed.argtypes = [I, I, I, D, D, D, I, P]
    lib.oracle_tensor_signed.restype = I
    lib.oracle_field_bruteforce.argtypes = [I, I, I, P, P, P]
    lib.oracle_field_bruteforce.restype = I
    lib.oracle_field_at.argtypes = [I, I, I, P, P, I, P, P]
    lib.oracle_field_at.restype = I
    lib.oracle_sp_rect.argtypes = [D, D, D, D, D]
    lib.oracle_sp_rect.restype = D
    lib.oracle_sp_kernel_closed.argtypes = [D, D, D, D, D, D, P]
    lib.oracle_sp_kernel_quad.argtypes = [D, D, D, D, D, D, I, I, I, P]
    lib.oracle_sp_kernel_quad.restype = I
    lib.oracle_sp_kernel.argtypes = [D, D, D, D, D, D, P]
    lib.oracle_sp_kernel_nodes.argtypes = [I, I, I, D, D, D, I, P]
    lib.oracle_sp_kernel_nodes.restype = I
    lib.oracle_sp_potential_bruteforce.argtypes = [I, I, I, D, D, D, P, P]
    lib.oracle_sp_potential_bruteforce.restype = I
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    env = os.environ.get("ORACLE_THREADS")
    if env:
        return max(1, int(env))
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


# ----------------------------------------------------------------- tensor
def box_tensor(tc, td, sc, sd) -> np.ndarray:
    """Mutual tensor of a target box and a source box (closed form, 64 corner pairs)."""
    lib = _load()
    tc = np.ascontiguousarray(tc, dtype=np.float64)
    td = np.ascontiguousarray(td, dtype=np.float64)
    sc = np.ascontiguousarray(sc, dtype=np.float64)
    sd = np.ascontiguousarray(sd, dtype=np.float64)
    out = np.zeros(6)
    lib.oracle_box_tensor(_ptr(tc), _ptr(td), _ptr(sc), _ptr(sd), _ptr(out))
    return out


def cell_tensor_closed(R, d) -> np.ndarray:
    out = np.zeros(6)
    _load().oracle_cell_tensor_closed(float(R[0]), float(R[1]), float(R[2]),
                                      float(d[0]), float(d[1]), float(d[2]), _ptr(out))
    return out


def cell_tensor_quad(R, d, nodes=(0, 0, 0)) -> np.ndarray:
    out = np.zeros(6)
    rc = _load().oracle_cell_tensor_quad(float(R[0]), float(R[1]), float(R[2]),
                                         float(d[0]), float(d[1]), float(d[2]),
                                         int(nodes[0]), int(nodes[1]), int(nodes[2]), _ptr(out))
    if rc != 0:
        raise ValueError(f"quadrature not applicable at offset {R} (cells touch), rc={rc}")
    return out


def cell_tensor(R, d) -> np.ndarray:
    """The oracle's tensor entry N(R) for two cells of edges d at offset R."""
    out = np.zeros(6)
    _load().oracle_cell_tensor(float(R[0]), float(R[1]), float(R[2]),
                               float(d[0]), float(d[1]), float(d[2]), _ptr(out))
    return out


def gl_rule(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _load().oracle_gl_rule(int(n), _ptr(x), _ptr(w))
    return x, w


def tensor_octant(n, d, threads: int | None = None) -> np.ndarray:
    """Octant table (6, nz, ny, nx): entry [c, k, j, i] = N_c(i dx, j dy, k dz)."""
    nx, ny, nz = (int(v) for v in n)
    out = np.zeros((6, nz, ny, nx))
    rc = _load().oracle_tensor_octant(nx, ny, nz, float(d[0]), float(d[1]), float(d[2]),
                                      threads or default_threads(), _ptr(out))
    if rc != 0:
        raise ValueError(f"bad tensor arguments n={n} d={d}")
    return out


def tensor_signed(n, d, threads: int | None = None) -> np.ndarray:
    """Signed table (6, 2nz-1, 2ny-1, 2nx-1): every offset evaluated directly."""
    nx, ny, nz = (int(v) for v in n)
    out = np.zeros((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    rc = _load().oracle_tensor_signed(nx, ny, nz, float(d[0]), float(d[1]), float(d[2]),
                                      threads or default_threads(), _ptr(out))
    if rc != 0:
        raise ValueError(f"bad tensor arguments n={n} d={d}")
    return out


# ----------------------------------------------------------------- field
def _check_m(M: np.ndarray) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.float64)
    if M.ndim != 4 or M.shape[0] != 3:
        raise ValueError("M must have shape (3, nz, ny, nx)")
    return M


def field_bruteforce(M: np.ndarray, d, signed_table: np.ndarray | None = None) -> np.ndarray:
    """Direct O(N^2) pair sum with every signed offset evaluated directly."""
    M = _check_m(M)
    _, nz, ny, nx = M.shape
    tab = signed_table if signed_table is not None else tensor_signed((nx, ny, nz), d)
    tab = np.ascontiguousarray(tab, dtype=np.float64)
    H = np.zeros_like(M)
    rc = _load().oracle_field_bruteforce(nx, ny, nz, _ptr(tab), _ptr(M), _ptr(H))
    if rc != 0:
        raise ValueError("bruteforce failed")
    return H


def field_at(M: np.ndarray, octant: np.ndarray, cells) -> np.ndarray:
    """Direct sum at selected target cells; cells = [(x, y, z), ...]; returns (ncell, 3)."""
    M = _check_m(M)
    _, nz, ny, nx = M.shape
    octant = np.ascontiguousarray(octant, dtype=np.float64)
    if octant.shape != (6, nz, ny, nx):
        raise ValueError("octant table shape does not match M")
    c = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((c.shape[0], 3))
    rc = _load().oracle_field_at(nx, ny, nz, _ptr(octant), _ptr(M), int(c.shape[0]), _ptr(c), _ptr(out))
    if rc != 0:
        raise ValueError(f"field_at failed rc={rc}")
    return out


def padded_size(n: int) -> int:
    """Smallest power of two >= 2n - 1 (1 when n == 1)."""
    need = 2 * n - 1
    p = 1
    while p < need:
        p *= 2
    return p


_PARITY = {  # component -> axes (x=0, y=1, z=2) in which it is odd
    0: (), 1: (), 2: (), 3: (0, 1), 4: (0, 2), 5: (1, 2),
}


def wrapped_tensor(octant: np.ndarray, P) -> np.ndarray:
    """Place the octant table at wrapped offsets of a (6, Pz, Py, Px) array.

    Offset i >= 0 goes to index i, offset -i to index P - i; the other octants
    take the parity sign of each component. Entries at offsets no pair of
    cells realises stay zero."""
    _, nz, ny, nx = octant.shape
    Px, Py, Pz = (int(v) for v in P)
    if Px < 2 * nx - 1 or Py < 2 * ny - 1 or Pz < 2 * nz - 1:
        raise ValueError("padded size too small")
    W = np.zeros((6, Pz, Py, Px))
    for sz in (1, -1):
        for sy in (1, -1):
            for sx in (1, -1):
                # offsets with a negative sign start at 1 (offset 0 belongs to +)
                ix = np.arange(nx) if sx > 0 else np.arange(1, nx)
                iy = np.arange(ny) if sy > 0 else np.arange(1, ny)
                iz = np.arange(nz) if sz > 0 else np.arange(1, nz)
                if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
                    continue
                px = ix if sx > 0 else Px - ix
                py = iy if sy > 0 else Py - iy
                pz = iz if sz > 0 else Pz - iz
                sign = {0: sx, 1: sy, 2: sz}
                for c in range(6):
                    s = 1.0
                    for ax in _PARITY[c]:
                        s *= sign[ax]
                    W[c][np.ix_(pz, py, px)] = s * octant[c][np.ix_(iz, iy, ix)]
    return W


def _rfftn(a, s=None, axes=None, workers=None):
    """numpy.fft.rfftn, or scipy.fft.rfftn over `workers` threads (the same
    transform; used for grids where one thread would take minutes)."""
    if workers and workers > 1:
        import scipy.fft
        return scipy.fft.rfftn(a, s=s, axes=axes, workers=workers)
    return np.fft.rfftn(a, s=s, axes=axes)


def _irfftn(a, s=None, axes=None, workers=None):
    if workers and workers > 1:
        import scipy.fft
        return scipy.fft.irfftn(a, s=s, axes=axes, workers=workers)
    return np.fft.irfftn(a, s=s, axes=axes)


def tensor_spectrum(octant: np.ndarray, P, workers: int | None = None) -> np.ndarray:
    """Real-to-complex 3-D DFT of the wrapped tensor: (6, Pz, Py, Px//2+1) complex."""
    W = wrapped_tensor(octant, P)
    return _rfftn(W, axes=(1, 2, 3), workers=workers)


def field_fft(M: np.ndarray, d, P=None, octant: np.ndarray | None = None,
              spectrum: np.ndarray | None = None, workers: int | None = None) -> np.ndarray:
    """Zero-padded FFT convolution H = -N * M in float64 (numpy.fft; with
    workers > 1, scipy.fft's threaded transforms of the same definition)."""
    M = _check_m(M)
    _, nz, ny, nx = M.shape
    if P is None:
        P = (padded_size(nx), padded_size(ny), padded_size(nz))
    Px, Py, Pz = (int(v) for v in P)
    if spectrum is None:
        if octant is None:
            octant = tensor_octant((nx, ny, nz), d)
        spectrum = tensor_spectrum(octant, (Px, Py, Pz), workers=workers)
    Nh = spectrum
    Mh = _rfftn(M, s=(Pz, Py, Px), axes=(1, 2, 3), workers=workers)
    xx, yy, zz, xy, xz, yz = Nh
    Hh = np.empty_like(Mh)
    Hh[0] = -(xx * Mh[0] + xy * Mh[1] + xz * Mh[2])
    Hh[1] = -(xy * Mh[0] + yy * Mh[1] + yz * Mh[2])
    Hh[2] = -(xz * Mh[0] + yz * Mh[1] + zz * Mh[2])
    H = _irfftn(Hh, s=(Pz, Py, Px), axes=(1, 2, 3), workers=workers)
    return np.ascontiguousarray(H[:, :nz, :ny, :nx])


def energy(M: np.ndarray, H: np.ndarray, d) -> float:
    """E = -(mu0/2) V sum_cells M.H, summed exactly rounded (math.fsum)."""
    V = float(d[0]) * float(d[1]) * float(d[2])
    prod = (np.asarray(M, dtype=np.float64) * np.asarray(H, dtype=np.float64)).ravel()
    return -0.5 * MU0 * V * math.fsum(prod.tolist())


def energy_reduced(m: np.ndarray, h: np.ndarray, d) -> float:
    """Energy in units of mu0 Ms^2 (m = M/Ms, h = H/Ms): e = -(1/2) V sum m.h."""
    V = float(d[0]) * float(d[1]) * float(d[2])
    prod = (np.asarray(m, dtype=np.float64) * np.asarray(h, dtype=np.float64)).ravel()
    return -0.5 * V * math.fsum(prod.tolist())


def rel_errors(H: np.ndarray, Href: np.ndarray) -> dict:
    """rel-max = max|H - Href| / max|Href|; rel-RMS = ||H - Href||_2 / ||Href||_2;
    paper relerr (Sec. 5.1, Eq. "relerr") = sqrt(sum |H - Href|^2 / N_cells)."""
    H = np.asarray(H, dtype=np.float64)
    Href = np.asarray(Href, dtype=np.float64)
    diff = H - Href
    ncell = Href[0].size
    mref = float(np.max(np.abs(Href))) if Href.size else 0.0
    nref = float(np.linalg.norm(Href.ravel()))
    return {
        "rel_max": float(np.max(np.abs(diff))) / mref if mref > 0 else float(np.max(np.abs(diff), initial=0.0)),
        "rel_rms": float(np.linalg.norm(diff.ravel())) / nref if nref > 0 else float(np.linalg.norm(diff.ravel())),
        "paper_relerr": float(math.sqrt(float(np.sum(diff * diff)) / ncell)) if ncell else 0.0,
    }


# ----------------------------------------------------------------- SP method
def sp_rect(a, V, W, hv, hw) -> float:
    """Int over [-hv, hv] x [-hw, hw] of 1 / sqrt(a^2 + (V - v)^2 + (W - w)^2) (closed form)."""
    return float(_load().oracle_sp_rect(float(a), float(V), float(W), float(hv), float(hw)))


def sp_kernel_closed(R, d) -> np.ndarray:
    """S(R) of one cell of edges d by its face integrals (closed form)."""
    out = np.zeros(3)
    _load().oracle_sp_kernel_closed(*(float(v) for v in R), *(float(v) for v in d), _ptr(out))
    return out


def sp_kernel_quad(R, d, nodes=(0, 0, 0)) -> np.ndarray:
    """S(R) by Gauss-Legendre quadrature of (R - u) / |R - u|^3 over the cell."""
    out = np.zeros(3)
    rc = _load().oracle_sp_kernel_quad(*(float(v) for v in R), *(float(v) for v in d),
                                       int(nodes[0]), int(nodes[1]), int(nodes[2]), _ptr(out))
    if rc != 0:
        raise ValueError(f"quadrature not applicable at {R} (rc={rc})")
    return out


def sp_kernel(R, d) -> np.ndarray:
    """The oracle's S(R): closed form within 2.5 edges per axis, quadrature beyond."""
    out = np.zeros(3)
    _load().oracle_sp_kernel(*(float(v) for v in R), *(float(v) for v in d), _ptr(out))
    return out


def sp_kernel_nodes(n, d, threads: int | None = None) -> np.ndarray:
    """(3, nz, ny, nx): entry [c, k, j, i] = S_c((i+1/2) dx, (j+1/2) dy, (k+1/2) dz)."""
    nx, ny, nz = (int(v) for v in n)
    out = np.zeros((3, nz, ny, nx))
    rc = _load().oracle_sp_kernel_nodes(nx, ny, nz, float(d[0]), float(d[1]), float(d[2]),
                                        threads or default_threads(), _ptr(out))
    if rc != 0:
        raise ValueError(f"bad kernel arguments n={n} d={d}")
    return out


def sp_padded_size(n: int) -> int:
    """Smallest power of two >= 2n: node-minus-cell offsets take 2n values per axis."""
    p = 1
    while p < 2 * n:
        p *= 2
    return p


def sp_wrapped_kernel(table: np.ndarray, P) -> np.ndarray:
    """Place the half-integer octant table at wrapped offsets of a (3, Pz, Py, Px) array.

    Node i minus cell j = q in [-(n-1), n] on each axis, at distance (q - 1/2) d;
    q >= 1 reads table index q - 1, q <= 0 reads index -q with the parity sign
    (component a is odd along axis a). Offset q goes to index q mod P."""
    _, nz, ny, nx = table.shape
    n = (nx, ny, nz)
    Px, Py, Pz = (int(v) for v in P)
    for a, p in zip(n, (Px, Py, Pz)):
        if p < 2 * a:
            raise ValueError("padded size too small for the node offsets")
    W = np.zeros((3, Pz, Py, Px))
    t = [np.arange(a) for a in n]
    pos = [t[a] + 1 for a in range(3)]
    neg = [(-t[a]) % p for a, p in zip(range(3), (Px, Py, Pz))]
    for sz in (1, -1):
        for sy in (1, -1):
            for sx in (1, -1):
                px = pos[0] if sx > 0 else neg[0]
                py = pos[1] if sy > 0 else neg[1]
                pz = pos[2] if sz > 0 else neg[2]
                signs = (sx, sy, sz)
                for c in range(3):
                    W[c][np.ix_(pz, py, px)] = signs[c] * table[c]
    return W


def sp_potential_fft(M: np.ndarray, d, P=None, table: np.ndarray | None = None) -> np.ndarray:
    """Node potential phi = S * M (Eq. "scpot" with Eq. "convolution") by a
    zero-padded float64 FFT convolution; shape (nz+1, ny+1, nx+1)."""
    M = _check_m(M)
    _, nz, ny, nx = M.shape
    if P is None:
        P = (sp_padded_size(nx), sp_padded_size(ny), sp_padded_size(nz))
    Px, Py, Pz = (int(v) for v in P)
    if table is None:
        table = sp_kernel_nodes((nx, ny, nz), d)
    W = sp_wrapped_kernel(table, (Px, Py, Pz))
    Sh = np.fft.rfftn(W, axes=(1, 2, 3))
    Mh = np.fft.rfftn(M, s=(Pz, Py, Px), axes=(1, 2, 3))
    ph = Sh[0] * Mh[0] + Sh[1] * Mh[1] + Sh[2] * Mh[2]
    phi = np.fft.irfftn(ph, s=(Pz, Py, Px), axes=(0, 1, 2))
    return np.ascontiguousarray(phi[:nz + 1, :ny + 1, :nx + 1])


def sp_potential_bruteforce(M: np.ndarray, d) -> np.ndarray:
    """Node potential by the direct sum over cells, every pair evaluated on its own."""
    M = _check_m(M)
    _, nz, ny, nx = M.shape
    phi = np.zeros((nz + 1, ny + 1, nx + 1))
    rc = _load().oracle_sp_potential_bruteforce(nx, ny, nz, float(d[0]), float(d[1]), float(d[2]),
                                                _ptr(M), _ptr(phi))
    if rc != 0:
        raise ValueError("SP bruteforce failed")
    return phi


def sp_field_from_potential(phi: np.ndarray, d) -> np.ndarray:
    """H = -grad phi by finite differences (Eq. "field"): per cell, the average
    over its four edges along each axis of the node differences over the edge
    length (the cell average of -grad of the trilinear interpolant)."""
    phi = np.asarray(phi, dtype=np.float64)
    nz, ny, nx = (s - 1 for s in phi.shape)
    H = np.zeros((3, nz, ny, nx))
    ex = (phi[:, :, 1:] - phi[:, :, :-1]) / float(d[0])        # (nz+1, ny+1, nx)
    H[0] = -0.25 * (ex[:-1, :-1] + ex[:-1, 1:] + ex[1:, :-1] + ex[1:, 1:])
    ey = (phi[:, 1:, :] - phi[:, :-1, :]) / float(d[1])        # (nz+1, ny, nx+1)
    H[1] = -0.25 * (ey[:-1, :, :-1] + ey[:-1, :, 1:] + ey[1:, :, :-1] + ey[1:, :, 1:])
    ez = (phi[1:] - phi[:-1]) / float(d[2])                    # (nz, ny+1, nx+1)
    H[2] = -0.25 * (ez[:, :-1, :-1] + ez[:, :-1, 1:] + ez[:, 1:, :-1] + ez[:, 1:, 1:])
    return H


def sp_field(M: np.ndarray, d, P=None) -> np.ndarray:
    """SP stray field: FFT node potential, then the finite-difference field."""
    return sp_field_from_potential(sp_potential_fft(M, d, P), d)


from . import tensor_grid  # noqa: E402  (TG oracle, numpy only)
