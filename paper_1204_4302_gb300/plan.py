"""Torch-facing wrapper of a libdemag plan.

PyTorch only provides device memory and the current stream here; every
operation is one call into the C ABI (``binding``). Fields are tensors of
shape (3, nz, ny, nx), float32 for ``prec="f32"`` plans and float64 for
``prec="f64"``, contiguous, on the plan's CUDA device.
"""
from __future__ import annotations

import torch

from . import binding as B


class Plan:
    """Stray field of an nx x ny x nz grid of cells with edges (dx, dy, dz).

    method="dm": the demagnetization-tensor convolution (paper Sec. 3.1, Eq.
    "demag"); method="sp": the scalar-potential convolution at the grid nodes
    with the finite-difference field (Eqs. "scpot" and "field").

    pad: None or "pow2" pads each axis to the smallest power of two >= 2n - 1;
    "smooth" to the smallest even length >= 2n - 1 (SP: >= 2n) with prime
    factors 2, 3, 5 and 7 (mixed-radix passes); "tuned" (DM) to the per-axis choice of the
    two that the padding autotuner finds fastest (timed once, then cached);
    or explicit (px, py, pz)."""

    def __init__(self, n, d, prec: str = "f32", pad=None, device=None, setup: bool = True,
                 method: str = "dm"):
        if not torch.cuda.is_available():
            raise RuntimeError("libdemag needs a CUDA device; there is no CPU path")
        self.n = tuple(int(v) for v in n)
        self.d = tuple(float(v) for v in d)
        if prec not in ("f32", "f64"):
            raise ValueError("prec must be 'f32' or 'f64'")
        self.prec = prec
        if method not in ("dm", "sp"):
            raise ValueError("method must be 'dm' or 'sp'")
        self.method = method
        self.dtype = torch.float32 if prec == "f32" else torch.float64
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        nx, ny, nz = self.n
        code = B.DEMAG_F32 if prec == "f32" else B.DEMAG_F64
        self.handle = None
        with torch.cuda.device(self.device):
            if method == "sp":
                if pad == "smooth":
                    self.handle = B.demag_plan_create_sp(nx, ny, nz, *self.d, code, pad_mode=B.DEMAG_PAD_SMOOTH)
                else:
                    self.handle = B.demag_plan_create_sp(nx, ny, nz, *self.d, code,
                                                         *(pad if pad not in (None, "pow2") else (0, 0, 0)))
            elif pad is None or pad == "pow2":
                self.handle = B.demag_plan_create(nx, ny, nz, *self.d, code)
            elif pad == "smooth":
                self.handle = B.demag_plan_create_ex(nx, ny, nz, *self.d, code, pad_mode=B.DEMAG_PAD_SMOOTH)
            elif pad == "tuned":
                self.handle = B.demag_plan_create_ex(nx, ny, nz, *self.d, code, pad_mode=B.DEMAG_PAD_TUNED)
            else:
                self.handle = B.demag_plan_create_ex(nx, ny, nz, *self.d, code, *pad)
        self.shape = (3, nz, ny, nx)
        if setup:
            self.setup()

    # ------------------------------------------------------------------ basics
    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _field_arg(self, t: torch.Tensor, name: str) -> torch.Tensor:
        if not isinstance(t, torch.Tensor) or t.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if t.dtype != self.dtype:
            raise ValueError(f"{name} must be {self.dtype} for a {self.prec} plan")
        if tuple(t.shape) != self.shape:
            raise ValueError(f"{name} must have shape {self.shape}, got {tuple(t.shape)}")
        return t.contiguous()

    def _cell_arg(self, w):
        if w is None:
            return None
        nx, ny, nz = self.n
        if not isinstance(w, torch.Tensor) or w.device != self.device or w.dtype != self.dtype:
            raise ValueError(f"the cell weight must be a {self.dtype} tensor on {self.device}")
        if tuple(w.shape) != (nz, ny, nx):
            raise ValueError(f"the cell weight must have shape {(nz, ny, nx)}")
        return w.contiguous()

    def setup(self):
        with torch.cuda.device(self.device):
            B.demag_tensor_setup(self.handle, self._stream())

    def info(self) -> dict:
        return B.demag_plan_info(self.handle)

    def close(self):
        if self.handle:
            B.demag_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ ops
    def field(self, M: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """H = -N * M (paper Sec. 3.1, Eq. "demag")."""
        M = self._field_arg(M, "M")
        H = torch.empty_like(M) if out is None else self._field_arg(out, "out")
        B.demag_field(self.handle, M.data_ptr(), H.data_ptr(), self._stream())
        return H

    def potential(self, M: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """SP plans: node potential phi = S * M, shape (nz+1, ny+1, nx+1) (Eq. "scpot")."""
        M = self._field_arg(M, "M")
        nx, ny, nz = self.n
        shape = (nz + 1, ny + 1, nx + 1)
        if out is None:
            out = torch.empty(shape, dtype=self.dtype, device=self.device)
        elif tuple(out.shape) != shape or out.dtype != self.dtype or out.device != self.device:
            raise ValueError(f"out must be a {self.dtype} tensor of shape {shape} on {self.device}")
        B.demag_sp_potential(self.handle, M.data_ptr(), out.data_ptr(), self._stream())
        return out

    def field_adjoint(self, G: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        G = self._field_arg(G, "G")
        R = torch.empty_like(G) if out is None else self._field_arg(out, "out")
        B.demag_field_adjoint(self.handle, G.data_ptr(), R.data_ptr(), self._stream())
        return R

    def field_energy(self, M: torch.Tensor, out: torch.Tensor | None = None):
        """(H, E) with E a float64 device scalar, E = -(mu0/2) V sum M.H."""
        M = self._field_arg(M, "M")
        H = torch.empty_like(M) if out is None else self._field_arg(out, "out")
        E = torch.empty((), dtype=torch.float64, device=self.device)
        B.demag_field_energy(self.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(), self._stream())
        return H, E

    def energy(self, M: torch.Tensor) -> float:
        M = self._field_arg(M, "M")
        return B.demag_energy(self.handle, M.data_ptr(), self._stream())

    def energy_grad(self, m: torch.Tensor, Ms: float, w: torch.Tensor | None = None,
                    want_energy: bool = True, want_grad: bool = True,
                    gscale: torch.Tensor | None = None):
        """E and g * dE/dm for M = Ms * w * m, in one pass of the pipeline."""
        m = self._field_arg(m, "m")
        w = self._cell_arg(w)
        E = torch.empty((), dtype=torch.float64, device=self.device) if want_energy else None
        G = torch.empty_like(m) if want_grad else None
        if gscale is not None:
            if gscale.dtype != torch.float64 or gscale.numel() != 1 or gscale.device != self.device:
                raise ValueError("gscale must be a float64 device scalar")
            gscale = gscale.contiguous()
        B.demag_energy_grad(self.handle, m.data_ptr(), None if w is None else w.data_ptr(), float(Ms),
                            None if E is None else E.data_ptr(), None if G is None else G.data_ptr(),
                            None if gscale is None else gscale.data_ptr(), self._stream())
        return E, G

    def field_host(self, M_host, H_host=None):
        """End to end from host memory: copies in, computes, copies out, syncs.
        M_host / H_host: CPU tensors (pinned for full bandwidth)."""
        if M_host.device.type != "cpu" or M_host.dtype != self.dtype or tuple(M_host.shape) != self.shape:
            raise ValueError("M_host must be a CPU tensor of the plan's dtype and shape")
        M_host = M_host.contiguous()
        if H_host is None:
            H_host = torch.empty(self.shape, dtype=self.dtype, pin_memory=M_host.is_pinned())
        B.demag_field_host(self.handle, M_host.data_ptr(), H_host.data_ptr(), self._stream())
        return H_host

    def field_host_async(self, M_host, H_host):
        """Queue an end-to-end field evaluation of pinned host buffers; call
        host_wait() before reading H_host or changing M_host."""
        for t in (M_host, H_host):
            if t.device.type != "cpu" or t.dtype != self.dtype or tuple(t.shape) != self.shape or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors of the plan's dtype and shape")
        B.demag_field_host_async(self.handle, M_host.data_ptr(), H_host.data_ptr(), self._stream())

    def field_energy_host_async(self, M_host, H_host, E_host):
        """As field_host_async, with the energy written to E_host (a pinned
        float64 CPU tensor of one element) after host_wait()."""
        for t in (M_host, H_host):
            if t.device.type != "cpu" or t.dtype != self.dtype or tuple(t.shape) != self.shape or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors of the plan's dtype and shape")
        if E_host.device.type != "cpu" or E_host.dtype != torch.float64 or E_host.numel() != 1:
            raise ValueError("E_host must be a float64 CPU tensor of one element")
        B.demag_field_energy_host_async(self.handle, M_host.data_ptr(), H_host.data_ptr(), E_host.data_ptr(),
                                        self._stream())

    def host_wait(self):
        B.demag_host_wait(self.handle)

    # ------------------------------------------------------------------ tuning
    def autotune(self, use_cache: bool = True) -> float:
        """Pick the fastest kernel variants for this plan; returns ms per field call."""
        with torch.cuda.device(self.device):
            return B.demag_autotune(self.handle, use_cache, self._stream())

    def variants(self):
        return B.demag_get_variants(self.handle)

    def set_variants(self, z: int, y: int, x: int | None = None):
        B.demag_set_variants(self.handle, z, y)
        if x is not None:
            B.demag_set_x_variant(self.handle, x)

    def x_variant(self) -> int:
        return B.demag_get_x_variant(self.handle)

    def check_pipeline(self):
        """Raise DemagError(DEMAG_ERR_TIMEOUT) if a pipelined pass gave up waiting."""
        B.demag_check_pipeline(self.handle)

    # ------------------------------------------------------------------ timing
    def save(self, path):
        """Write the set-up tensor spectrum (and sizes) to a file (demag_plan_save)."""
        B.demag_plan_save(self.handle, path)

    @classmethod
    def load(cls, path, device=None):
        """A ready plan from a file written by save(): no tensor setup runs."""
        if not torch.cuda.is_available():
            raise RuntimeError("libdemag needs a CUDA device; there is no CPU path")
        self = cls.__new__(cls)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.handle = None
        with torch.cuda.device(self.device):
            self.handle = B.demag_plan_load(path)
        info = self.info()
        self.n = (info["nx"], info["ny"], info["nz"])
        self.d = (info["dx"], info["dy"], info["dz"])
        self.prec = "f32" if info["prec"] == B.DEMAG_F32 else "f64"
        self.method = "sp" if info["method"] == B.DEMAG_METHOD_SP else "dm"
        self.dtype = torch.float32 if self.prec == "f32" else torch.float64
        self.shape = (3, self.n[2], self.n[1], self.n[0])
        return self

    def set_graphs(self, enable: bool = True):
        """Replay each distinct call as one captured CUDA graph (see demag_set_graphs)."""
        B.demag_set_graphs(self.handle, enable)

    def set_spectral_energy(self, enable: bool = True):
        """Energies without a field by the Parseval sum in the z pass (default)
        or by the field pipeline (see demag_set_spectral_energy)."""
        B.demag_set_spectral_energy(self.handle, enable)

    def set_timing(self, enable: bool = True):
        B.demag_set_timing(self.handle, enable)

    def get_timing(self, n: int = 6):
        return B.demag_get_timing(self.handle, n)

    def launch_count(self) -> int:
        return B.demag_launch_count(self.handle)
