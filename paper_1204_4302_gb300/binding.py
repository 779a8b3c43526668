"""ctypes binding of libdemag.so: the C entry points under the same names.

Argument marshalling only. Every computation runs in the library's CUDA
kernels; when the library is missing this module raises instead of falling
back to anything else. Pointers are passed as integers (device addresses,
e.g. ``tensor.data_ptr()``), streams as integer handles (``cudaStream_t``).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_long, c_size_t, c_void_p
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "_build" / "libdemag.so"

DEMAG_F32 = 0
DEMAG_F64 = 1

DEMAG_METHOD_DM = 0
DEMAG_METHOD_SP = 1
DEMAG_PAD_POW2 = 0
DEMAG_PAD_SMOOTH = 1
DEMAG_PAD_TUNED = 2

STATUS = {
    0: "DEMAG_OK",
    1: "DEMAG_ERR_INVALID_ARG",
    2: "DEMAG_ERR_NOT_SETUP",
    3: "DEMAG_ERR_OOM",
    4: "DEMAG_ERR_CUDA",
    5: "DEMAG_ERR_TIMEOUT",
    6: "DEMAG_ERR_UNSUPPORTED",
    7: "DEMAG_ERR_GUARD",
}

# Every symbol include/demag.h declares (the CPU tests check the export list).
EXPORTS = [
    "demag_plan_create", "demag_plan_create_ex", "demag_tensor_setup", "demag_field",
    "demag_field_adjoint", "demag_field_energy", "demag_energy", "demag_energy_grad",
    "demag_field_host", "demag_plan_info", "demag_set_timing", "demag_get_timing",
    "demag_launch_count", "demag_plan_destroy", "demag_last_error", "demag_status_string",
    "demag_energy_noalloc",
    "demag_batch_create", "demag_batch_create_ex", "demag_tune_padding", "demag_padded_lengths", "demag_set_graphs",
    "demag_plan_save", "demag_plan_load", "demag_debug_fail_alloc", "demag_debug_guard_count",
    "demag_debug_poke_guard", "demag_field_energy_host_async",
    "demag_batch_autotune_padding",
    "demag_batch_field", "demag_batch_set_mode", "demag_batch_set_timeout",
    "demag_batch_set_timing", "demag_batch_get_timing",
    "demag_batch_status", "demag_batch_info", "demag_batch_launch_count", "demag_batch_destroy",
    "demag_autotune", "demag_get_variants", "demag_set_variants", "demag_batch_autotune",
    "demag_set_spectral_energy",
    "demag_field_host_async", "demag_host_wait",
    "demag_plan_create_sp", "demag_sp_potential",
    "demag_get_x_variant", "demag_set_x_variant", "demag_check_pipeline",
    "demag_tg_plan_create", "demag_tg_field_cp", "demag_tg_potential_cp", "demag_tg_plan_info",
    "demag_tg_plan_destroy", "demag_tg_set_contraction", "demag_tg_get_contraction", "demag_tg_status",
    "demag_tg_set_timing", "demag_tg_get_timing", "demag_cp_als", "demag_tucker_als",
    "demag_tg_plan_create_tucker", "demag_tg_field_tucker", "demag_tg_potential_tucker",
]


class DemagError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{where}: {self.name}: {message}")


class demag_options(ctypes.Structure):
    _fields_ = [("px", c_int), ("py", c_int), ("pz", c_int), ("pad_mode", c_int)]


class demag_info(ctypes.Structure):
    _fields_ = [
        ("nx", c_int), ("ny", c_int), ("nz", c_int),
        ("px", c_int), ("py", c_int), ("pz", c_int),
        ("kx", c_int), ("prec", c_int),
        ("device_bytes", c_size_t),
        ("launches_per_field", c_int),
        ("tensor_imag_max", c_double),
        ("method", c_int),
        ("dx", c_double), ("dy", c_double), ("dz", c_double),
        ("energy_in_z", c_int),
    ]


_lib = None


def load(path: str | Path | None = None):
    """Load libdemag.so (built in-tree by ``paper_1204_4302_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise ImportError(
            f"{p} is missing: build the CUDA library first "
            "(python -m paper_1204_4302_gb300.build, or __graft_entry__.build())")
    lib = ctypes.CDLL(str(p))
    S = c_int
    P = c_void_p
    D = c_double
    I = c_int
    sig = {
        "demag_plan_create": (S, [I, I, I, D, D, D, I, POINTER(c_void_p)]),
        "demag_plan_create_ex": (S, [I, I, I, D, D, D, I, POINTER(demag_options), POINTER(c_void_p)]),
        "demag_tensor_setup": (S, [P, P]),
        "demag_field": (S, [P, P, P, P]),
        "demag_field_adjoint": (S, [P, P, P, P]),
        "demag_field_energy": (S, [P, P, P, P, P]),
        "demag_energy": (S, [P, P, POINTER(c_double), P]),
        "demag_energy_grad": (S, [P, P, P, D, P, P, P, P]),
        "demag_field_host": (S, [P, P, P, P]),
        "demag_plan_info": (S, [P, POINTER(demag_info)]),
        "demag_set_timing": (S, [P, I]),
        "demag_set_spectral_energy": (S, [P, I]),
        "demag_batch_set_timing": (S, [P, I]),
        "demag_batch_get_timing": (S, [P, POINTER(c_double), POINTER(c_long)]),
        "demag_set_graphs": (S, [P, I]),
        "demag_batch_autotune_padding": (S, [P, I, POINTER(c_double), POINTER(c_double), P]),
        "demag_field_energy_host_async": (S, [P, P, P, P, P]),
        "demag_debug_fail_alloc": (None, [ctypes.c_long]),
        "demag_debug_guard_count": (ctypes.c_long, []),
        "demag_debug_poke_guard": (S, []),
        "demag_plan_save": (S, [P, ctypes.c_char_p]),
        "demag_plan_load": (S, [ctypes.c_char_p, POINTER(c_void_p)]),
        "demag_get_timing": (S, [P, POINTER(c_double), POINTER(c_long), I]),
        "demag_launch_count": (c_long, [P]),
        "demag_plan_destroy": (None, [P]),
        "demag_last_error": (ctypes.c_char_p, [P]),
        "demag_status_string": (ctypes.c_char_p, [I]),
        "demag_energy_noalloc": (S, [I, I, I, D, D, D, I, P, P, P, P]),
        "demag_batch_create": (S, [I, P, P, I, POINTER(c_void_p)]),
        "demag_batch_create_ex": (S, [I, P, P, I, POINTER(demag_options), POINTER(c_void_p)]),
        "demag_padded_lengths": (S, [I, I, I, POINTER(demag_options), POINTER(c_int)]),
        "demag_tune_padding": (S, [I, I, I, D, D, D, I, I, POINTER(demag_options), POINTER(c_double),
                                   POINTER(c_double), P]),
        "demag_batch_field": (S, [P, P, P, P, P]),
        "demag_batch_set_mode": (S, [P, I]),
        "demag_batch_set_timeout": (S, [P, D, I]),
        "demag_batch_status": (S, [P, P]),
        "demag_batch_info": (S, [P, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                 POINTER(c_size_t)]),
        "demag_batch_launch_count": (c_long, [P]),
        "demag_batch_destroy": (None, [P]),
        "demag_autotune": (S, [P, I, POINTER(c_double), P]),
        "demag_get_variants": (S, [P, POINTER(c_int), POINTER(c_int)]),
        "demag_set_variants": (S, [P, I, I]),
        "demag_batch_autotune": (S, [P, I, POINTER(c_double), POINTER(c_double), P]),
        "demag_field_host_async": (S, [P, P, P, P]),
        "demag_host_wait": (S, [P]),
        "demag_plan_create_sp": (S, [I, I, I, D, D, D, I, POINTER(demag_options), POINTER(c_void_p)]),
        "demag_sp_potential": (S, [P, P, P, P]),
        "demag_get_x_variant": (S, [P, POINTER(c_int)]),
        "demag_set_x_variant": (S, [P, I]),
        "demag_check_pipeline": (S, [P]),
        "demag_tg_plan_create": (S, [I, I, I, D, D, D, I, I, POINTER(c_void_p)]),
        "demag_tg_field_cp": (S, [P, P, P, P, P, P, P, P]),
        "demag_tg_potential_cp": (S, [P, P, P, P, P, P, P]),
        "demag_tg_plan_info": (S, [P, POINTER(c_int), POINTER(c_size_t), POINTER(c_long)]),
        "demag_tg_plan_destroy": (None, [P]),
        "demag_tg_set_contraction": (S, [P, I]),
        "demag_tg_get_contraction": (S, [P, POINTER(c_int)]),
        "demag_tg_status": (S, [P, P]),
        "demag_tg_set_timing": (S, [P, I]),
        "demag_cp_als": (S, [I, I, I, P, I, I, P, P, P, P, P, P]),
        "demag_tg_plan_create_tucker": (S, [I, I, I, D, D, D, I, I, I, I, POINTER(c_void_p)]),
        "demag_tg_field_tucker": (S, [P, P, P, P, P, P, P, P]),
        "demag_tg_potential_tucker": (S, [P, P, P, P, P, P, P]),
        "demag_tucker_als": (S, [I, I, I, P, I, I, I, I, P, P, P, P, P, P]),
        "demag_tg_get_timing": (S, [P, POINTER(c_double), POINTER(c_long)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        msg = load().demag_last_error(None)
        raise DemagError(status, where, msg.decode() if msg else "")


def _p(v):
    return None if v is None or v == 0 else c_void_p(int(v))


# ------------------------------------------------------------------ entry points
def demag_plan_create(nx, ny, nz, dx, dy, dz, prec=DEMAG_F32):
    h = c_void_p()
    _check(load().demag_plan_create(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                    int(prec), ctypes.byref(h)), "demag_plan_create")
    return h.value


def demag_plan_create_ex(nx, ny, nz, dx, dy, dz, prec=DEMAG_F32, px=0, py=0, pz=0, pad_mode=0):
    h = c_void_p()
    opt = demag_options(int(px), int(py), int(pz), int(pad_mode))
    _check(load().demag_plan_create_ex(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                       int(prec), ctypes.byref(opt), ctypes.byref(h)),
           "demag_plan_create_ex")
    return h.value


def demag_plan_create_sp(nx, ny, nz, dx, dy, dz, prec=DEMAG_F32, px=0, py=0, pz=0, pad_mode=0):
    h = c_void_p()
    opt = demag_options(int(px), int(py), int(pz), int(pad_mode))
    _check(load().demag_plan_create_sp(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                       int(prec), ctypes.byref(opt), ctypes.byref(h)),
           "demag_plan_create_sp")
    return h.value


def demag_sp_potential(plan, M, phi, stream=0):
    _check(load().demag_sp_potential(_p(plan), _p(M), _p(phi), _p(stream)), "demag_sp_potential")


def demag_get_x_variant(plan) -> int:
    x = c_int()
    _check(load().demag_get_x_variant(_p(plan), ctypes.byref(x)), "demag_get_x_variant")
    return x.value


def demag_set_x_variant(plan, x):
    _check(load().demag_set_x_variant(_p(plan), int(x)), "demag_set_x_variant")


def demag_check_pipeline(plan):
    _check(load().demag_check_pipeline(_p(plan)), "demag_check_pipeline")


def demag_tg_plan_create(nx, ny, nz, dx, dy, dz, rank, prec=DEMAG_F32):
    h = c_void_p()
    _check(load().demag_tg_plan_create(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), int(rank),
                                       int(prec), ctypes.byref(h)), "demag_tg_plan_create")
    return h.value


def demag_tg_plan_create_tucker(nx, ny, nz, dx, dy, dz, r1, r2, r3, prec=DEMAG_F32):
    h = c_void_p()
    _check(load().demag_tg_plan_create_tucker(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), int(r1),
                                              int(r2), int(r3), int(prec), ctypes.byref(h)),
           "demag_tg_plan_create_tucker")
    return h.value


def demag_tg_field_tucker(plan, G, A, B_, C, H, E_dev, stream=0):
    _check(load().demag_tg_field_tucker(_p(plan), _p(G), _p(A), _p(B_), _p(C), _p(H), _p(E_dev), _p(stream)),
           "demag_tg_field_tucker")


def demag_tg_potential_tucker(plan, G, A, B_, C, phi, stream=0):
    _check(load().demag_tg_potential_tucker(_p(plan), _p(G), _p(A), _p(B_), _p(C), _p(phi), _p(stream)),
           "demag_tg_potential_tucker")


def demag_tg_field_cp(plan, lam, Ux, Uy, Uz, H, E_dev, stream=0):
    _check(load().demag_tg_field_cp(_p(plan), _p(lam), _p(Ux), _p(Uy), _p(Uz), _p(H), _p(E_dev), _p(stream)),
           "demag_tg_field_cp")


def demag_tg_potential_cp(plan, lam, Ux, Uy, Uz, phi, stream=0):
    _check(load().demag_tg_potential_cp(_p(plan), _p(lam), _p(Ux), _p(Uy), _p(Uz), _p(phi), _p(stream)),
           "demag_tg_potential_cp")


def demag_tg_plan_info(plan) -> dict:
    r = c_int()
    b = c_size_t()
    n = c_long()
    _check(load().demag_tg_plan_info(_p(plan), ctypes.byref(r), ctypes.byref(b), ctypes.byref(n)),
           "demag_tg_plan_info")
    return {"sinc_terms": r.value, "device_bytes": b.value, "launches": n.value}


def demag_tg_set_contraction(plan, contraction):
    _check(load().demag_tg_set_contraction(_p(plan), int(contraction)), "demag_tg_set_contraction")


def demag_tg_get_contraction(plan) -> int:
    c = ctypes.c_int(0)
    _check(load().demag_tg_get_contraction(_p(plan), ctypes.byref(c)), "demag_tg_get_contraction")
    return c.value


def demag_tg_set_timing(plan, enable):
    _check(load().demag_tg_set_timing(_p(plan), int(bool(enable))), "demag_tg_set_timing")


def demag_tg_get_timing(plan):
    ms = (c_double * 4)()
    calls = c_long()
    _check(load().demag_tg_get_timing(_p(plan), ms, ctypes.byref(calls)), "demag_tg_get_timing")
    return list(ms), calls.value


def demag_cp_als(nx, ny, nz, M, rank, iters, lam, Ux, Uy, Uz, relerr, stream=0):
    _check(load().demag_cp_als(int(nx), int(ny), int(nz), _p(M), int(rank), int(iters), _p(lam), _p(Ux), _p(Uy),
                               _p(Uz), _p(relerr), _p(stream)), "demag_cp_als")


def demag_tucker_als(nx, ny, nz, M, r1, r2, r3, iters, G, A, B, C, relerr, stream=0):
    _check(load().demag_tucker_als(int(nx), int(ny), int(nz), _p(M), int(r1), int(r2), int(r3), int(iters), _p(G),
                                   _p(A), _p(B), _p(C), _p(relerr), _p(stream)), "demag_tucker_als")


def demag_tg_status(plan, stream=0):
    _check(load().demag_tg_status(_p(plan), _p(stream)), "demag_tg_status")


def demag_tg_plan_destroy(plan):
    if plan:
        load().demag_tg_plan_destroy(_p(plan))


def demag_tensor_setup(plan, stream=0):
    _check(load().demag_tensor_setup(_p(plan), _p(stream)), "demag_tensor_setup")


def demag_field(plan, M, H, stream=0):
    _check(load().demag_field(_p(plan), _p(M), _p(H), _p(stream)), "demag_field")


def demag_field_adjoint(plan, G, out, stream=0):
    _check(load().demag_field_adjoint(_p(plan), _p(G), _p(out), _p(stream)), "demag_field_adjoint")


def demag_field_energy(plan, M, H, E_dev, stream=0):
    _check(load().demag_field_energy(_p(plan), _p(M), _p(H), _p(E_dev), _p(stream)), "demag_field_energy")


def demag_energy(plan, M, stream=0) -> float:
    e = c_double()
    _check(load().demag_energy(_p(plan), _p(M), ctypes.byref(e), _p(stream)), "demag_energy")
    return e.value


def demag_energy_grad(plan, m, w, Ms, E_dev, grad, gscale_dev=None, stream=0):
    _check(load().demag_energy_grad(_p(plan), _p(m), _p(w), float(Ms), _p(E_dev), _p(grad),
                                    _p(gscale_dev), _p(stream)), "demag_energy_grad")


def demag_field_host(plan, M_host, H_host, stream=0):
    _check(load().demag_field_host(_p(plan), _p(M_host), _p(H_host), _p(stream)), "demag_field_host")


def demag_field_host_async(plan, M_host, H_host, stream=0):
    _check(load().demag_field_host_async(_p(plan), _p(M_host), _p(H_host), _p(stream)), "demag_field_host_async")


def demag_host_wait(plan):
    _check(load().demag_host_wait(_p(plan)), "demag_host_wait")


def demag_plan_info(plan) -> dict:
    info = demag_info()
    _check(load().demag_plan_info(_p(plan), ctypes.byref(info)), "demag_plan_info")
    return {name: getattr(info, name) for name, _ in demag_info._fields_}


def demag_set_timing(plan, enable=True):
    _check(load().demag_set_timing(_p(plan), int(bool(enable))), "demag_set_timing")


def demag_set_spectral_energy(plan, enable=True):
    _check(load().demag_set_spectral_energy(_p(plan), int(bool(enable))), "demag_set_spectral_energy")


def demag_get_timing(plan, n=6):
    ms = (c_double * n)()
    cnt = (c_long * n)()
    _check(load().demag_get_timing(_p(plan), ms, cnt, int(n)), "demag_get_timing")
    return list(ms), list(cnt)


def demag_launch_count(plan) -> int:
    return int(load().demag_launch_count(_p(plan)))


def demag_plan_destroy(plan):
    if plan:
        load().demag_plan_destroy(_p(plan))


def demag_last_error(plan=None) -> str:
    """The calling thread's latest error message (plan None), or the latest
    failed call's on that plan."""
    m = load().demag_last_error(_p(plan))
    return m.decode() if m else ""


def demag_energy_noalloc(nx, ny, nz, dx, dy, dz, prec, M, H, E_dev, stream=0):
    """Energy of a field pair without any allocation (see include/demag.h)."""
    status = load().demag_energy_noalloc(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                         int(prec), _p(M), _p(H), _p(E_dev), _p(stream))
    if status != 0:
        raise DemagError(status, "demag_energy_noalloc", "see include/demag.h for the conditions")


def demag_batch_create(dims, cells, prec=DEMAG_F32, pad_mode=None):
    """dims: [(nx, ny, nz), ...]; cells: [(dx, dy, dz), ...]; pad_mode None
    (powers of two) or a DEMAG_PAD_* value (demag_batch_create_ex)."""
    n = len(dims)
    d = (c_int * (3 * n))(*[int(v) for t in dims for v in t])
    c = (c_double * (3 * n))(*[float(v) for t in cells for v in t])
    h = c_void_p()
    if pad_mode is None:
        _check(load().demag_batch_create(n, d, c, int(prec), ctypes.byref(h)), "demag_batch_create")
    else:
        opt = demag_options(0, 0, 0, int(pad_mode))
        _check(load().demag_batch_create_ex(n, d, c, int(prec), ctypes.byref(opt), ctypes.byref(h)),
               "demag_batch_create_ex")
    return h.value


def demag_plan_save(plan, path):
    _check(load().demag_plan_save(_p(plan), os.fsencode(path)), "demag_plan_save")


def demag_plan_load(path):
    h = c_void_p()
    _check(load().demag_plan_load(os.fsencode(path), ctypes.byref(h)), "demag_plan_load")
    return h.value


def demag_debug_guard_count() -> int:
    return int(load().demag_debug_guard_count())


def demag_debug_poke_guard():
    _check(load().demag_debug_poke_guard(), "demag_debug_poke_guard")


def demag_debug_fail_alloc(n):
    """Make the n-th next device allocation of the library fail (0 disarms)."""
    load().demag_debug_fail_alloc(int(n))


def demag_field_energy_host_async(plan, M_host, H_host, E_host, stream=0):
    _check(load().demag_field_energy_host_async(_p(plan), _p(M_host), _p(H_host), _p(E_host), _p(stream)),
           "demag_field_energy_host_async")


def demag_batch_autotune_padding(batch, use_cache=True, stream=0):
    """Keep the faster of power-of-two and smooth padding; returns (ms_pow2, ms_smooth)."""
    a, b = c_double(), c_double()
    _check(load().demag_batch_autotune_padding(_p(batch), 1 if use_cache else 0, ctypes.byref(a), ctypes.byref(b),
                                               _p(stream)), "demag_batch_autotune_padding")
    return a.value, b.value


def demag_set_graphs(plan, enable=True):
    _check(load().demag_set_graphs(_p(plan), 1 if enable else 0), "demag_set_graphs")


def demag_padded_lengths(nx, ny, nz, px=0, py=0, pz=0, pad_mode=0):
    """Padded lengths (px, py, pz) a DM plan takes with these options (no device)."""
    opt = demag_options(int(px), int(py), int(pz), int(pad_mode))
    P = (c_int * 3)()
    _check(load().demag_padded_lengths(int(nx), int(ny), int(nz), ctypes.byref(opt), P), "demag_padded_lengths")
    return tuple(P)


def demag_tune_padding(nx, ny, nz, dx, dy, dz, prec=DEMAG_F32, use_cache=True, stream=0):
    """Fastest padded lengths of a DM plan: ((px, py, pz), ms_best, ms_pow2)."""
    opt = demag_options()
    mb, mp = c_double(), c_double()
    _check(load().demag_tune_padding(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), int(prec),
                                     1 if use_cache else 0, ctypes.byref(opt), ctypes.byref(mb), ctypes.byref(mp),
                                     _p(stream)), "demag_tune_padding")
    return (opt.px, opt.py, opt.pz), mb.value, mp.value


def demag_batch_field(batch, M_ptrs, H_ptrs, E_dev=None, stream=0):
    n = len(M_ptrs)
    m = (c_void_p * n)(*[int(v) for v in M_ptrs])
    h = (c_void_p * n)(*[int(v) for v in H_ptrs])
    _check(load().demag_batch_field(_p(batch), m, h, _p(E_dev), _p(stream)), "demag_batch_field")


def demag_batch_set_mode(batch, mode):
    _check(load().demag_batch_set_mode(_p(batch), int(mode)), "demag_batch_set_mode")


def demag_batch_set_timeout(batch, seconds, stall_state=-1):
    _check(load().demag_batch_set_timeout(_p(batch), float(seconds), int(stall_state)), "demag_batch_set_timeout")


def demag_batch_status(batch, stream=0):
    _check(load().demag_batch_status(_p(batch), _p(stream)), "demag_batch_status")


def demag_batch_info(batch) -> dict:
    mode, ok, items, grid = c_int(), c_int(), c_int(), c_int()
    smem = c_size_t()
    _check(load().demag_batch_info(_p(batch), ctypes.byref(mode), ctypes.byref(ok), ctypes.byref(items),
                                   ctypes.byref(grid), ctypes.byref(smem)), "demag_batch_info")
    return {"mode": mode.value, "persistent_ok": bool(ok.value), "items": items.value, "grid": grid.value,
            "smem": smem.value}


def demag_batch_set_timing(batch, enable=True):
    _check(load().demag_batch_set_timing(_p(batch), int(bool(enable))), "demag_batch_set_timing")


def demag_batch_get_timing(batch):
    ms = (c_double * 6)()
    calls = c_long()
    _check(load().demag_batch_get_timing(_p(batch), ms, ctypes.byref(calls)), "demag_batch_get_timing")
    return list(ms), calls.value


def demag_batch_launch_count(batch) -> int:
    return int(load().demag_batch_launch_count(_p(batch)))


def demag_batch_destroy(batch):
    if batch:
        load().demag_batch_destroy(_p(batch))


def demag_autotune(plan, use_cache=True, stream=0) -> float:
    ms = c_double()
    _check(load().demag_autotune(_p(plan), int(bool(use_cache)), ctypes.byref(ms), _p(stream)), "demag_autotune")
    return ms.value


def demag_get_variants(plan):
    z, y = c_int(), c_int()
    _check(load().demag_get_variants(_p(plan), ctypes.byref(z), ctypes.byref(y)), "demag_get_variants")
    return z.value, y.value


def demag_set_variants(plan, z, y):
    _check(load().demag_set_variants(_p(plan), int(z), int(y)), "demag_set_variants")


def demag_batch_autotune(batch, use_cache=True, stream=0):
    a, b = c_double(), c_double()
    _check(load().demag_batch_autotune(_p(batch), int(bool(use_cache)), ctypes.byref(a), ctypes.byref(b),
                                       _p(stream)), "demag_batch_autotune")
    return a.value, b.value


def demag_status_string(s: int) -> str:
    return load().demag_status_string(int(s)).decode()
