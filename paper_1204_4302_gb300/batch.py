"""Torch-facing wrapper of a libdemag batch: many independent states of
uneven grid sizes evaluated by one graph launch (see include/demag.h)."""
from __future__ import annotations

import torch

from . import binding as B


class Batch:
    PERSISTENT = 0
    BRANCHES = 1
    PASSES = 2

    PAD = {None: None, "pow2": 0, "smooth": 1, "tuned": 2}

    def __init__(self, dims, cells, prec: str = "f32", pad=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libdemag needs a CUDA device; there is no CPU path")
        self.dims = [tuple(int(v) for v in t) for t in dims]
        self.cells = [tuple(float(v) for v in t) for t in cells]
        self.dtype = torch.float32 if prec == "f32" else torch.float64
        self.device = torch.device("cuda", torch.cuda.current_device())
        if pad not in self.PAD:
            raise ValueError("pad must be None, 'pow2', 'smooth' or 'tuned'")
        self.handle = B.demag_batch_create(self.dims, self.cells, B.DEMAG_F32 if prec == "f32" else B.DEMAG_F64,
                                           self.PAD[pad])
        self.n = len(self.dims)

    def shapes(self):
        return [(3, nz, ny, nx) for (nx, ny, nz) in self.dims]

    def field(self, Ms, Hs=None, energies: bool = False):
        """Ms: list of (3, nz, ny, nx) tensors; returns (Hs, E) with E a float64
        device tensor of n energies (or None)."""
        if len(Ms) != self.n:
            raise ValueError("one magnetization per state")
        Ms = [m.contiguous() for m in Ms]
        for m, shp in zip(Ms, self.shapes()):
            if tuple(m.shape) != shp or m.dtype != self.dtype or m.device != self.device:
                raise ValueError(f"state magnetization must be {self.dtype} {shp} on {self.device}")
        if Hs is None:
            Hs = [torch.empty_like(m) for m in Ms]
        E = torch.empty(self.n, dtype=torch.float64, device=self.device) if energies else None
        B.demag_batch_field(self.handle, [m.data_ptr() for m in Ms], [h.data_ptr() for h in Hs],
                            None if E is None else E.data_ptr(),
                            torch.cuda.current_stream(self.device).cuda_stream)
        return Hs, E

    def autotune(self, use_cache: bool = True):
        """Tune every state's plan and choose the fastest batch mode (persistent,
        branches, pass-batched); returns (ms per call persistent, ms per call
        branches)."""
        return B.demag_batch_autotune(self.handle, use_cache, torch.cuda.current_stream(self.device).cuda_stream)

    def autotune_padding(self, use_cache: bool = True):
        """Keep the faster of power-of-two and smooth padding (rebuilding the
        plans when needed); returns (ms per call power-of-two, smooth)."""
        return B.demag_batch_autotune_padding(self.handle, use_cache, torch.cuda.current_stream(self.device).cuda_stream)

    def set_mode(self, mode: int):
        B.demag_batch_set_mode(self.handle, mode)

    def set_timeout(self, seconds: float, stall_state: int = -1):
        B.demag_batch_set_timeout(self.handle, seconds, stall_state)

    def status(self):
        B.demag_batch_status(self.handle, torch.cuda.current_stream(self.device).cuda_stream)

    def info(self) -> dict:
        return B.demag_batch_info(self.handle)

    def set_timing(self, enable: bool = True):
        """Per-pass event timing of the pass-batched mode (see demag_batch_set_timing)."""
        B.demag_batch_set_timing(self.handle, enable)

    def get_timing(self):
        """(ms per pass summed over the timed calls, number of calls)."""
        return B.demag_batch_get_timing(self.handle)

    def launch_count(self) -> int:
        return B.demag_batch_launch_count(self.handle)

    def close(self):
        if self.handle:
            B.demag_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
