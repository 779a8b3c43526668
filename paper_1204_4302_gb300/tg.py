"""Torch-facing wrapper of the tensor-grid (TG) entry points (paper Sec. 3.2).

A magnetization in CP format (App. A): for each component p,
M^(p)[k, j, i] = sum_m lam[p, m] Ux[p, m, i] Uy[p, m, j] Uz[p, m, k].
Tensors: lam (3, r), Ux (3, r, nx), Uy (3, r, ny), Uz (3, r, nz), on the
plan's CUDA device, float32 or float64 as the plan. Every computation runs
in the library's CUDA kernels (argument marshalling only here).
"""
from __future__ import annotations

import torch

from . import binding as B


class TGPlan:
    """Cell-centre potential, field and energy of CP magnetizations on an
    nx x ny x nz grid of cells (dx, dy, dz)."""

    def __init__(self, n, d, rank=None, prec: str = "f32", device=None, tucker=None):
        """rank: CP rank; or tucker = (r1, r2, r3) for Tucker input (then
        field/potential take (G, A, B, C))."""
        if not torch.cuda.is_available():
            raise RuntimeError("libdemag needs a CUDA device; there is no CPU path")
        if prec not in ("f32", "f64"):
            raise ValueError("prec must be 'f32' or 'f64'")
        self.n = tuple(int(v) for v in n)
        self.d = tuple(float(v) for v in d)
        if (rank is None) == (tucker is None):
            raise ValueError("give a CP rank or Tucker ranks")
        self.tucker = None if tucker is None else tuple(int(v) for v in tucker)
        self.rank = int(rank) if tucker is None else self.tucker[0]
        self.prec = prec
        self.dtype = torch.float32 if prec == "f32" else torch.float64
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.handle = None
        with torch.cuda.device(self.device):
            pr = B.DEMAG_F32 if prec == "f32" else B.DEMAG_F64
            if self.tucker is None:
                self.handle = B.demag_tg_plan_create(*self.n, *self.d, self.rank, pr)
            else:
                self.handle = B.demag_tg_plan_create_tucker(*self.n, *self.d, *self.tucker, pr)

    def _factors(self, lam, Ux, Uy, Uz):
        nx, ny, nz = self.n
        if self.tucker is None:
            r = self.rank
            shapes = ((3, r), (3, r, nx), (3, r, ny), (3, r, nz))
            names = ("lam", "Ux", "Uy", "Uz")
        else:
            r1, r2, r3 = self.tucker
            shapes = ((3, r3, r2, r1), (3, r1, nx), (3, r2, ny), (3, r3, nz))
            names = ("G", "A", "B", "C")
        out = []
        for t, shp, nm in zip((lam, Ux, Uy, Uz), shapes, names):
            if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != self.dtype:
                raise ValueError(f"{nm} must be a {self.dtype} tensor on {self.device}")
            if tuple(t.shape) != shp:
                raise ValueError(f"{nm} must have shape {shp}, got {tuple(t.shape)}")
            out.append(t.contiguous())
        return out

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def field(self, lam, Ux, Uy, Uz, energy: bool = False):
        """H (3, nz, ny, nx), and E (float64 device scalar) when energy=True.
        CP: (lam, Ux, Uy, Uz); Tucker: (G, A, B, C)."""
        f = self._factors(lam, Ux, Uy, Uz)
        nx, ny, nz = self.n
        H = torch.empty((3, nz, ny, nx), dtype=self.dtype, device=self.device)
        E = torch.empty((), dtype=torch.float64, device=self.device) if energy else None
        fn = B.demag_tg_field_cp if self.tucker is None else B.demag_tg_field_tucker
        fn(self.handle, *(t.data_ptr() for t in f), H.data_ptr(), None if E is None else E.data_ptr(), self._stream())
        return (H, E) if energy else H

    def potential(self, lam, Ux, Uy, Uz):
        f = self._factors(lam, Ux, Uy, Uz)
        nx, ny, nz = self.n
        phi = torch.empty((nz, ny, nx), dtype=self.dtype, device=self.device)
        fn = B.demag_tg_potential_cp if self.tucker is None else B.demag_tg_potential_tucker
        fn(self.handle, *(t.data_ptr() for t in f), phi.data_ptr(), self._stream())
        return phi

    def info(self) -> dict:
        return B.demag_tg_plan_info(self.handle)

    CUDA_CORES = 0
    TENSOR_CORES = 1

    def set_contraction(self, contraction: int):
        """0: the dense contraction on the CUDA cores; 1 (FP32 default): on the
        tensor cores, three TF32 products per term."""
        B.demag_tg_set_contraction(self.handle, contraction)

    def contraction(self) -> int:
        return B.demag_tg_get_contraction(self.handle)

    def set_timing(self, enable: bool = True):
        """Per-stage event timing (factor transforms, operand preparation,
        contraction, differences + energy) of the following calls."""
        B.demag_tg_set_timing(self.handle, enable)

    def get_timing(self):
        """(ms per stage summed over the timed calls, number of calls)."""
        return B.demag_tg_get_timing(self.handle)

    def status(self):
        """Raises (DEMAG_ERR_TIMEOUT) if a bounded wait of the tensor-core
        contraction ran out since the last check; synchronises the stream."""
        B.demag_tg_status(self.handle, self._stream())

    def close(self):
        if self.handle:
            B.demag_tg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
