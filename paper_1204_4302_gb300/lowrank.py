"""Torch-facing wrappers of the low-rank entry points (paper Sec. 3.2,
"Low-Rank Magnetization"): CP-ALS and Tucker-ALS of the magnetization
components on the GPU, FP64 (see include/demag.h). Every computation runs in
the library's CUDA kernels (argument marshalling only here)."""
from __future__ import annotations

import torch

from . import binding as B


def _dev_f64(t, name, shape, device):
    if not isinstance(t, torch.Tensor) or t.device != device or t.dtype != torch.float64:
        raise ValueError(f"{name} must be a float64 tensor on {device}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.contiguous().clone()


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


def cp_als(M: torch.Tensor, rank: int, init, iters: int):
    """M: (3, nz, ny, nx) float64 on a CUDA device; init = (Ux, Uy, Uz) with
    Ux (3, rank, nx), Uy (3, rank, ny), Uz (3, rank, nz) (Ux is not read).
    Returns (lam (3, rank), Ux, Uy, Uz, relerr) with relerr Eq. "relr" (a float)."""
    if not torch.cuda.is_available():
        raise RuntimeError("libdemag needs a CUDA device; there is no CPU path")
    _, nz, ny, nx = M.shape
    dev = M.device
    M = _dev_f64(M, "M", M.shape, dev)
    Ux = _dev_f64(init[0], "Ux", (3, rank, nx), dev)
    Uy = _dev_f64(init[1], "Uy", (3, rank, ny), dev)
    Uz = _dev_f64(init[2], "Uz", (3, rank, nz), dev)
    lam = torch.empty((3, rank), dtype=torch.float64, device=dev)
    err = torch.empty((), dtype=torch.float64, device=dev)
    B.demag_cp_als(nx, ny, nz, M.data_ptr(), rank, iters, lam.data_ptr(), Ux.data_ptr(), Uy.data_ptr(),
                   Uz.data_ptr(), err.data_ptr(), _stream(dev))
    return lam, Ux, Uy, Uz, float(err.item())


def tucker_als(M: torch.Tensor, ranks, init, iters: int):
    """M: (3, nz, ny, nx) float64 on a CUDA device; ranks = (r1, r2, r3);
    init = (A, B, C) with A (3, r1, nx), B (3, r2, ny), C (3, r3, nz) (A is
    not read). Returns (G (3, r3, r2, r1), A, B, C, relerr)."""
    if not torch.cuda.is_available():
        raise RuntimeError("libdemag needs a CUDA device; there is no CPU path")
    _, nz, ny, nx = M.shape
    r1, r2, r3 = (int(v) for v in ranks)
    dev = M.device
    M = _dev_f64(M, "M", M.shape, dev)
    A = _dev_f64(init[0], "A", (3, r1, nx), dev)
    Bf = _dev_f64(init[1], "B", (3, r2, ny), dev)
    C = _dev_f64(init[2], "C", (3, r3, nz), dev)
    G = torch.empty((3, r3, r2, r1), dtype=torch.float64, device=dev)
    err = torch.empty((), dtype=torch.float64, device=dev)
    B.demag_tucker_als(nx, ny, nz, M.data_ptr(), r1, r2, r3, iters, G.data_ptr(), A.data_ptr(), Bf.data_ptr(),
                       C.data_ptr(), err.data_ptr(), _stream(dev))
    return G, A, Bf, C, float(err.item())
