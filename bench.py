#!/usr/bin/env python
"""Benchmark of the FFT demagnetization-tensor (DM) stray field on GB300.

One step = one pass of the field pipeline with the fused energy, i.e.
H = -N * M and E = -(mu0/2) V sum M.H on a 256^3 grid (2 nm cubic cells,
seeded random unit m, Ms = 8e5 A/m) in FP32 (FFTs and spectral product in
FP32, tensor set up in FP64). The tensor setup runs once per geometry before
the timed region (the method's setup/apply split) and is reported as
setup_ms. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (numpy FFT convolution) on a
bounded sample grid of the same workload, on the host cores.
Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(independent magnetization states, no data-path collective); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "stray-field cells/s at 256^3 FP32 (field + energy step), vs plain FP64 on 1 GB300"
N_GRID = (256, 256, 256)
CELL = (2e-9, 2e-9, 2e-9)
MS = 8e5
SEED = 1
MU0 = 4e-7 * math.pi
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
PASS_NAMES = ["x_fwd", "y_fwd", "z_conv", "y_inv", "x_inv", "energy"]
STATES = 40          # independent 256^3 states per step (about 1 s per 20 steps)
L2_BYTES = 129 << 20  # GB300 L2: working sets below it are not HBM-bound
FP64_TFLOPS = 1.25   # nominal GB300 FP64 rate (the FP64 form's ALU ceiling)
# FP32 CUDA-core rate: 152 SMs x 128 FMA lanes x 2 flops x 2.07 GHz
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def pass_bytes(n, P, elem=4, energy=True):
    """Algorithmic HBM bytes of each kernel per launch (the data each pass must
    read and write once): spectra are complex (2 elem), the tensor spectrum is
    6 real octant arrays; energy: the last pass also reads M (false where the
    energy is taken in the z pass, demag_info.energy_in_z)."""
    nx, ny, nz = n
    Px, Py, Pz = P
    Kx = Px // 2 + 1
    c = 2 * elem
    cells = nx * ny * nz
    s1 = 3 * nz * ny * Kx * c
    s2 = 3 * nz * Py * Kx * c
    nh = 6 * (Pz // 2 + 1) * (Py // 2 + 1) * Kx * elem
    return {
        "x_fwd": 3 * cells * elem + s1,
        "y_fwd": s1 + s2,
        "z_conv": 2 * s2 + nh,
        "y_inv": s2 + s1,
        "x_inv": s1 + 3 * cells * elem + (3 * cells * elem if energy else 0),  # reads S1 (and M), writes H
    }


def fft_flops(L: int) -> float:
    """Flops of one complex FFT of length L (the 5 L log2 L count)."""
    return 5.0 * L * math.log2(L) if L > 1 else 0.0


def step_flops(n, P) -> float:
    """Arithmetic of one field step as the 5 L log2 L count of its transforms
    (pruned: the forward passes run on the physical rows, the x pair-packed
    R2C as a half-length complex transform) plus the 3x3 product (36 flops per
    frequency). An estimate for the ALU ceiling, not an instruction count."""
    nx, ny, nz = n
    Px, Py, Pz = P
    Kx = Px // 2 + 1
    x = 3 * nz * ny * fft_flops(Px // 2)           # forward and inverse x: 2x this
    y = 3 * nz * Kx * fft_flops(Py)                # forward and inverse y: 2x this
    z = 3 * Py * Kx * fft_flops(Pz)                # forward and inverse z: 2x this
    prod = 36.0 * Pz * Py * Kx
    return 2 * (x + y + z) + prod


SP_PASS_NAMES = ["x_fwd", "y_fwd", "sp_z", "y_inv", "x_inv", "sp_grad"]


def sp_pass_bytes(n, P, elem=4):
    """Algorithmic HBM bytes per launch of the scalar-potential pipeline: the
    forward passes as for DM; the SP z pass reads three spectra and the three
    real kernel tables and writes one spectrum of nz + 1 rows; the inverse
    passes move one component; the field stencil reads the node potential and
    M (for the energy) and writes H."""
    nx, ny, nz = n
    Px, Py, Pz = P
    Kx = Px // 2 + 1
    c = 2 * elem
    cells = nx * ny * nz
    nodes = (nx + 1) * (ny + 1) * (nz + 1)
    s1 = 3 * nz * ny * Kx * c
    s2 = 3 * nz * Py * Kx * c
    phi_hat = (nz + 1) * Py * Kx * c
    phi_y = (nz + 1) * (ny + 1) * Kx * c
    tab = 3 * (Pz // 2 + 1) * (Py // 2 + 1) * Kx * elem
    return {
        "x_fwd": 3 * cells * elem + s1,
        "y_fwd": s1 + s2,
        "sp_z": s2 + tab + phi_hat,
        "y_inv": phi_hat + phi_y,
        "x_inv": phi_y + nodes * elem,
        "sp_grad": nodes * elem + 3 * cells * elem + 3 * cells * elem,
    }


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest value of x over all ranks (the slowest rank's time); x itself
    without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Units all ranks processed divided by the slowest rank's time (cells/s)."""
    return world * cells_per_rank * steps / (ms_max / 1e3)


# The sources that define the field-step kernels of the DM and SP pipelines
# and their launch shapes (the per-kernel DRAM traffic in profiles/traffic.json
# is valid while these are unchanged).
STEP_KERNEL_SOURCES = ("fft_engine.cuh", "fft2.cuh", "xpipe.cuh", "zws.cuh", "sp.cuh", "passes_impl.cuh", "passes_f32.cu",
                       "passes_f64.cu", "plan.h")


def source_hash() -> str:
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1204_4302_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    try:
        with open(PEAKS) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def load_tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 burst rate scaled by the
    nominal GB300 TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s), or the fallback
    bf16 figure scaled the same way."""
    try:
        with open(PEAKS) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
        src = "measured bf16 burst x 1.1/2.25 (nominal TF32/bf16 ratio)"
    except (OSError, KeyError, ValueError):
        bf16, src = 1900.0, "fallback bf16 1.9 PF/s x 1.1/2.25 (nominal TF32/bf16 ratio)"
    return bf16 * 1.1 / 2.25, src


def load_traffic(kernel: str, n, src_hash: str):
    """DRAM bytes per launch of a kernel from a committed ncu summary, scaled to
    this workload, or None if absent or taken on an older kernel source."""
    try:
        with open(TRAFFIC) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = t.get(kernel)
    if not ent or ent.get("source_hash") != src_hash:
        return None
    cells = n[0] * n[1] * n[2]
    return ent["bytes_per_cell"] * cells


# --------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1204_4302_gb300 import inputs
    from paper_1204_4302_gb300.plan import Plan

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n = N_GRID
    cells = n[0] * n[1] * n[2]
    S = args.states
    # independent states per rank (replicas of the method, distinct inputs):
    # state 0 from the shared numpy generator (the oracle tests' state), the
    # others from seeded device generators
    m_np = inputs.random_unit(n, seed=SEED + rank)
    M = torch.tensor(MS * m_np, dtype=torch.float32, device=dev)
    Ms_list = [M]
    for i in range(1, S):
        g = torch.Generator(device=dev).manual_seed(1000003 * (rank + 1) + i)
        mi = torch.randn(3, n[2], n[1], n[0], device=dev, generator=g)
        Ms_list.append(MS * mi / mi.norm(dim=0, keepdim=True))
        del mi

    t0 = time.perf_counter()
    plan = Plan(n, CELL, prec="f32", device=dev, pad=None if args.pad == "pow2" else args.pad)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    if args.variants:
        z, y, x = (int(v) for v in args.variants.split(","))
        plan.set_variants(z, y, x)
    tuned_ms = None if (args.no_tune or args.variants) else plan.autotune(use_cache=False)
    variants = plan.variants()
    info = plan.info()
    P = (info["px"], info["py"], info["pz"])
    H = torch.empty_like(M)
    Hb = [H, torch.empty_like(M)]
    Es = torch.empty(S, dtype=torch.float64, device=dev)
    E = Es[0]
    st = torch.cuda.current_stream(dev)

    from paper_1204_4302_gb300 import binding as B

    def step():
        # one step: field + energy of every state of the batch
        for i, Mi in enumerate(Ms_list):
            B.demag_field_energy(plan.handle, Mi.data_ptr(), Hb[i & 1].data_ptr(), Es[i:].data_ptr(),
                                 st.cuda_stream)

    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launches0 = plan.launch_count()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(args.steps):
        step()
    ev1.record(st)
    ev1.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = plan.launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(ms, dist, dev)
    ms_per_step = ms / args.steps
    ms_per_field = ms_per_step / S
    value = whole_job_rate(cells * S, world, args.steps, ms)

    # per-pass times from a separate run (event timing adds events per call;
    # the headline above ran without them)
    plan.set_timing(True)
    for _ in range(max(20, args.steps)):
        B.demag_field_energy(plan.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(), st.cuda_stream)
    torch.cuda.synchronize()
    pass_ms, pass_n = plan.get_timing(6)
    plan.set_timing(False)

    # energy sanity (device value, read after timing)
    B.demag_field_energy(plan.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(), st.cuda_stream)
    E_val = float(E.item())

    # ---------------------------------------------------------------- roofline
    peak, peak_kind = load_peaks()
    pb = pass_bytes(n, P, 4, energy=not plan.info()["energy_in_z"])
    avg = {nm: (pass_ms[i] / pass_n[i] if pass_n[i] else None) for i, nm in enumerate(PASS_NAMES[:5])}
    per_pass = {}
    for nm in PASS_NAMES[:5]:
        if avg[nm]:
            gbs = pb[nm] / (avg[nm] * 1e-3) / 1e9
            per_pass[nm] = {"ms": round(avg[nm], 4), "bytes": pb[nm], "gbs": round(gbs, 1),
                            "frac": round(gbs / peak, 3)}
    dominant = max(per_pass, key=lambda k: per_pass[k]["ms"]) if per_pass else "z_conv"
    src_hash = source_hash()
    traffic = load_traffic(dominant, n, src_hash)
    roof = {
        "bound": "hbm",
        "kernel": dominant,
        "achieved": per_pass.get(dominant, {}).get("gbs"),
        "peak": peak,
        "unit": "GB/s",
        "frac": per_pass.get(dominant, {}).get("frac"),
        "traffic": traffic,
        "peak_source": peak_kind,
        "algorithmic_bytes": pb[dominant],
    }

    # ------------------------------------------------ FP64 form and FP32 error
    f64 = None
    if not args.skip_f64:
        plan64 = Plan(n, CELL, prec="f64", device=dev)
        M64 = M.double()
        H64 = torch.empty_like(M64)
        E64 = torch.empty((), dtype=torch.float64, device=dev)
        from paper_1204_4302_gb300 import binding as B
        for _ in range(2):
            B.demag_field_energy(plan64.handle, M64.data_ptr(), H64.data_ptr(), E64.data_ptr(), st.cuda_stream)
        torch.cuda.synchronize()
        k64 = max(3, args.steps // 4)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(k64):
            B.demag_field_energy(plan64.handle, M64.data_ptr(), H64.data_ptr(), E64.data_ptr(), st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        diff = (H.double() - H64)
        rel_max = float(diff.abs().max() / H64.abs().max())
        rel_rms = float(diff.norm() / H64.norm())
        b64 = sum(pass_bytes(n, P, 8).values())
        fl64 = step_flops(n, P)
        f64 = {"ms_per_field": round(ms64, 4), "cells_per_s": cells / (ms64 / 1e3),
               "speedup_f32_over_f64": round(ms64 / ms_per_field, 2),
               "f32_rel_max_err_vs_f64": rel_max, "f32_rel_rms_err_vs_f64": rel_rms,
               "energy_rel_diff": abs(E_val - float(E64.item())) / abs(float(E64.item())),
               # the FP64 form's two ceilings: HBM bytes of its passes and its
               # FFT + product arithmetic against the FP64 rate
               "hbm": {"bytes": b64, "gbs": round(b64 / (ms64 * 1e-3) / 1e9, 1),
                       "frac": round(b64 / (ms64 * 1e-3) / 1e9 / peak, 3), "peak_gbs": peak},
               "fp64": {"flops": fl64, "tflops": round(fl64 / (ms64 * 1e-3) / 1e12, 3),
                        "frac": round(fl64 / (ms64 * 1e-3) / 1e12 / FP64_TFLOPS, 3), "peak_tflops": FP64_TFLOPS,
                        "peak_source": "nominal GB300 FP64 rate (not measured)"}}
        plan64.close()
        del M64, H64

    # ------------------------------------------------ gradient (adjoint) timing
    grad = None
    if not args.skip_grad:
        m32 = torch.tensor(m_np, dtype=torch.float32, device=dev)
        G = torch.empty_like(m32)
        from paper_1204_4302_gb300 import binding as B
        for _ in range(2):
            B.demag_energy_grad(plan.handle, m32.data_ptr(), None, MS, E.data_ptr(), G.data_ptr(), None,
                                st.cuda_stream)
        torch.cuda.synchronize()
        kg = max(3, args.steps // 2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(kg):
            B.demag_energy_grad(plan.handle, m32.data_ptr(), None, MS, E.data_ptr(), G.data_ptr(), None,
                                st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        grad = {"ms_per_step": round(e0.elapsed_time(e1) / kg, 4)}
        del m32, G

    # ------------------------------------------------ end to end (host buffers)
    e2e = None
    if not args.skip_e2e:
        # end to end through the public API from pinned host buffers: every
        # step uploads its M and downloads its H; streamed calls overlap one
        # step's copies with the neighbouring steps' fields
        NH = min(4, S)
        Mh = [Ms_list[i].cpu().pin_memory() for i in range(NH)]
        Hh = [torch.empty_like(Mh[0]).pin_memory() for _ in range(2)]
        Eh = [torch.zeros(1, dtype=torch.float64).pin_memory() for _ in range(2)]

        def e2e_step(step_idx):
            # the step's S states: each uploaded from pinned host memory,
            # field + energy computed, H and E downloaded (streamed calls)
            for i in range(S):
                plan.field_energy_host_async(Mh[i % NH], Hh[(step_idx * S + i) % 2], Eh[(step_idx * S + i) % 2])

        e2e_step(0)
        plan.host_wait()
        barrier()
        ke = max(2, args.steps)
        t0 = time.perf_counter()
        for i in range(ke):
            e2e_step(i)
        plan.host_wait()
        barrier()
        te = (time.perf_counter() - t0) / ke
        tmax = max_over_ranks(te, dist, dev)
        plan.field_energy_host_async(Mh[0], Hh[0], Eh[0])
        plan.host_wait()
        e2e_energy_rel = abs(float(Eh[0].item()) - E_val) / abs(E_val)
        # the same calls one at a time (upload, field, download, synchronise)
        from paper_1204_4302_gb300 import binding as B
        t1 = time.perf_counter()
        for i in range(3):
            B.demag_field_host(plan.handle, Mh[0].data_ptr(), Hh[0].data_ptr(), st.cuda_stream)
        ts = (time.perf_counter() - t1) / 3
        nbytes = 3 * cells * 4
        e2e = {"value": world * cells * S / tmax, "unit": "cells/s", "h2d_bytes_per_step": nbytes * S,
               "d2h_bytes_per_step": (nbytes + 8) * S, "ms_per_step": round(tmax * 1e3, 4),
               "mode": f"streamed demag_field_energy_host_async calls, {S} states per step (field + energy, "
                       "H and E downloaded), pinned buffers",
               "energy_rel_diff_vs_device_step": e2e_energy_rel,
               "ms_per_field_synchronous_field_only": round(ts * 1e3, 4)}
        del Mh, Hh

    # energy without a field (minimisation loops): the spectral (Parseval) sum
    # against the field pipeline's energy, same states
    energy_only = None
    if not args.skip_grad:
        def estep():
            for i, Mi in enumerate(Ms_list):
                B.demag_energy_grad(plan.handle, Mi.data_ptr(), None, 1.0, Es[i:].data_ptr(), None, None,
                                    st.cuda_stream)
        res = {}
        for route in (True, False):
            plan.set_spectral_energy(route)
            estep()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(max(2, args.steps // 2)):
                estep()
            e1.record(st)
            e1.synchronize()
            res[route] = (e0.elapsed_time(e1) / max(2, args.steps // 2) / S, float(Es[0].item()))
        plan.set_spectral_energy(True)
        energy_only = {"ms_per_energy_spectral": round(res[True][0], 4),
                       "ms_per_energy_field_pipeline": round(res[False][0], 4),
                       "cells_per_s_spectral": cells / (res[True][0] / 1e3),
                       "speedup_spectral": round(res[False][0] / res[True][0], 3),
                       "energy_rel_diff": abs(res[True][1] - res[False][1]) / abs(res[False][1]),
                       "ms_per_field_energy_step": round(ms_per_field, 4)}

    batch = None
    if not args.skip_batch:
        batch = run_batch(args, dev, rank, peak)

    sp = None
    if not args.skip_sp:
        sp = run_sp(args, dev, M, H, peak)
        sp["speedup_over_dm"] = round(ms_per_field / sp["ms_per_step"], 3)

    tgr = None
    if not args.skip_tg:
        tgr = run_tg(args, dev, peak)

    padding = None
    if not args.skip_padding:
        padding = run_padding(args, dev)

    configs = None
    if not args.skip_configs:
        configs = run_configs(args, dev, peak)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        cpu = cpu_baseline(args.ref_sample, args.cpu_headline)

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value,
            "unit": "cells/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_per_step, 4),
            "ms_per_field": round(ms_per_field, 5),
            "states_per_step": S,
            "timed_region_s": round(ms / 1e3, 3),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic (seeded random unit magnetization)",
            "config": {"workload": f"DM stray field + energy, 256x256x256 cells of 2 nm, padded 512^3, FP32 "
                                   f"FFT/product, FP64 tensor setup; {S} independent states per step",
                       "states_per_step": S,
                       "grid": list(n), "padded": list(P), "cell_m": list(CELL), "Ms": MS,
                       "parallelism": f"replicas x{world} (independent states)",
                       "l2": "inputs and spectra (~2 GB) larger than L2, no flush needed"},
            "gpu_launches": launches,
            "setup_ms": round(setup_ms, 1),
            "autotune": {"z_variant": variants[0], "y_variant": variants[1], "x_variant": plan.x_variant(),
                         "ms_per_field_energy": None if tuned_ms is None else round(tuned_ms, 4)},
            "batch": batch,
            "scalar_potential": sp,
            "tensor_grid": tgr,
            "padding": padding,
            "configs": configs,
            "energy_J": E_val,
            "energy_only": energy_only,
            "passes": per_pass,
            "roofline": roof,
            "clocks": clocks,
            "e2e": e2e,
            "plain_f64": f64,
            "gradient": grad,
            "cpu_baseline": cpu,
            "source_hash": src_hash,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    plan.close()


def run_sp(args, dev, M, H_dm, peak):
    """The scalar-potential method (paper Sec. 3.1) on the same state: FP32
    field + energy per step, per-pass times and HBM fractions, and its FP32
    error against the FP64 SP path. (Its field differs from the DM field by the
    finite-difference error, which for a random state is of order one and for
    the paper's smooth states about 1e-3; the tests check the latter.)"""
    import torch

    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.plan import Plan

    n = N_GRID
    cells = n[0] * n[1] * n[2]
    st = torch.cuda.current_stream(dev)
    plan = Plan(n, CELL, prec="f32", device=dev, method="sp")
    if args.variants:
        plan.set_variants(0, int(args.variants.split(",")[1]), int(args.variants.split(",")[2]))
    tuned = None if (args.no_tune or args.variants) else plan.autotune(use_cache=False)
    info = plan.info()
    P = (info["px"], info["py"], info["pz"])
    H = torch.empty_like(M)
    E = torch.empty((), dtype=torch.float64, device=dev)

    def step():
        B.demag_field_energy(plan.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(), st.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    k = max(5, args.steps)
    plan.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(k):
        step()
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / k
    pass_ms, pass_n = plan.get_timing(7)
    plan.set_timing(False)
    pb = sp_pass_bytes(n, P, 4)
    passes = {}
    for i, nm in enumerate(SP_PASS_NAMES):
        if pass_n[i]:
            t = pass_ms[i] / pass_n[i]
            gbs = pb[nm] / (t * 1e-3) / 1e9
            passes[nm] = {"ms": round(t, 4), "bytes": pb[nm], "gbs": round(gbs, 1), "frac": round(gbs / peak, 3)}
    out = {"ms_per_step": round(ms, 4), "cells_per_s": cells / (ms / 1e3), "passes": passes,
           "y_variant": plan.variants()[1], "energy_J": float(E.item()),
           "speedup_over_dm": None}
    plan.close()
    if not args.skip_f64:
        p64 = Plan(n, CELL, prec="f64", device=dev, method="sp")
        H64 = p64.field(M.double())
        out["f32_rel_max_err_vs_f64"] = float((H.double() - H64).abs().max() / H64.abs().max())
        p64.close()
        del H64
    del H
    torch.cuda.empty_cache()
    return out


def run_tg(args, dev, peak):
    """The tensor-grid method (paper Sec. 3.2) on the same grid for CP
    magnetizations of rank 1 (a uniform body, exact) and rank 8 (seeded random
    factors): field + energy per step with the dense contraction on the tensor
    cores (the FP32 default) and on the CUDA cores, the per-stage times, the
    contraction's tensor-pipe rate against the TF32 peak, and the FP32 error
    of the rank-8 field against the FP64 TG path."""
    import numpy as np
    import torch

    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300.tg import TGPlan

    n = N_GRID
    cells = n[0] * n[1] * n[2]
    st = torch.cuda.current_stream(dev)
    tf32_peak, tf32_src = load_tf32_peak()
    out = {}
    rng = np.random.default_rng(SEED)
    for r in (1, 8):
        if r == 1:
            lam = np.array([[0.3], [-0.5], [0.8]]) * MS
            U = [np.ones((3, 1, v)) for v in n]
        else:
            lam = MS * rng.standard_normal((3, r)) / r
            U = [rng.standard_normal((3, r, v)) for v in n]
        f32 = [torch.tensor(a, dtype=torch.float32, device=dev) for a in [lam] + U]
        plan = TGPlan(n, CELL, r, prec="f32", device=dev)
        H = torch.empty((3, n[2], n[1], n[0]), dtype=torch.float32, device=dev)
        E = torch.empty((), dtype=torch.float64, device=dev)
        R = plan.info()["sinc_terms"]
        K = 3 * R * r
        # the dense block-CP contraction Phi[k][j][i] = sum_K Z[K][k] Y[K][j] X[K][i]
        # over K = 3 R r terms: 2 cells K flops (the step's dominant arithmetic)
        fl = 2.0 * cells * K

        def step():
            B.demag_tg_field_cp(plan.handle, *(t.data_ptr() for t in f32), H.data_ptr(), E.data_ptr(),
                                st.cuda_stream)

        def timed():
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            k = max(5, args.steps)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(k):
                step()
            e1.record(st)
            e1.synchronize()
            return e0.elapsed_time(e1) / k

        def stages():
            plan.set_timing(True)
            for _ in range(3):
                step()
            ms, calls = plan.get_timing()
            plan.set_timing(False)
            return [v / calls for v in ms]

        ent = {"rank": r, "sinc_terms": R, "terms_K": K, "flops_contraction": fl}
        for name, c in (("tensor_cores", TGPlan.TENSOR_CORES), ("cuda_cores", TGPlan.CUDA_CORES)):
            plan.set_contraction(c)
            ms = timed()
            sg = stages()
            sub = {"ms_per_step": round(ms, 4), "cells_per_s": cells / (ms / 1e3),
                   "stage_ms": {"factor_transforms": round(sg[0], 4), "operand_prep": round(sg[1], 4),
                                "contraction": round(sg[2], 4), "differences_energy": round(sg[3], 4)}}
            if c == TGPlan.TENSOR_CORES:
                plan.status()
                t = 3 * fl / (sg[2] * 1e-3) / 1e12
                sub["roofline"] = {"bound": "tensor", "kernel": "k_tg_mma", "achieved": round(t, 1),
                                   "peak": round(tf32_peak, 1), "unit": "TFLOP/s", "frac": round(t / tf32_peak, 3),
                                   "peak_source": tf32_src,
                                   "flops": "3 TF32 products per term (hi hi, hi lo, lo hi): 3 x 2 cells K",
                                   "fp32_equivalent_tflops": round(fl / (sg[2] * 1e-3) / 1e12, 1)}
                ent["energy_J"] = float(E.item())
            else:
                t = fl / (sg[2] * 1e-3) / 1e12
                sub["alu"] = {"bound": "alu", "kernel": "k_tg_dense", "achieved": round(t, 2),
                              "peak": round(FP32_TFLOPS, 1), "unit": "TFLOP/s", "frac": round(t / FP32_TFLOPS, 3),
                              "peak_source": "FP32 CUDA cores: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (derived)"}
            ent[name] = sub
        plan.set_contraction(TGPlan.TENSOR_CORES)
        ent["ms_per_step"] = ent["tensor_cores"]["ms_per_step"]
        ent["cells_per_s"] = ent["tensor_cores"]["cells_per_s"]
        if r == 8 and not args.skip_f64:
            step()
            p64 = TGPlan(n, CELL, r, prec="f64", device=dev)
            H64 = p64.field(*[torch.tensor(a, dtype=torch.float64, device=dev) for a in [lam] + U])
            ent["f32_rel_max_err_vs_f64"] = float((H.double() - H64).abs().max() / H64.abs().max())
            plan.set_contraction(TGPlan.CUDA_CORES)
            step()
            ent["f32_cuda_cores_rel_max_err_vs_f64"] = float((H.double() - H64).abs().max() / H64.abs().max())
            p64.close()
            del H64
        plan.close()
        out[f"rank{r}"] = ent
        del H, f32
        torch.cuda.empty_cache()
    return out


def run_batch(args, dev, rank, peak):
    """64 independent states of uneven sizes (32..128 x 32..128 x 8..32 cells of
    3 nm, seeded random unit m), FP32, one graph launch per batch call."""
    import torch

    from paper_1204_4302_gb300 import inputs
    from paper_1204_4302_gb300.batch import Batch
    saved_cache = os.environ.get("DEMAG_TUNE_CACHE")
    dims = inputs.batch_sizes(64, lo=(32, 32, 8), hi=(128, 128, 32), seed=4)
    d = 3e-9
    cells = [(d, d, d)] * len(dims)
    ms = [torch.tensor(MS * inputs.random_unit(nn, seed=1000 * rank + i), dtype=torch.float32, device=dev)
          for i, nn in enumerate(dims)]
    hs = [torch.empty_like(m) for m in ms]
    b = Batch(dims, cells)
    t_p, t_b = b.autotune(use_cache=False)
    E = torch.empty(len(dims), dtype=torch.float64, device=dev)
    from paper_1204_4302_gb300 import binding as B
    st = torch.cuda.current_stream(dev)
    mp, hp = [m.data_ptr() for m in ms], [h.data_ptr() for h in hs]
    for _ in range(3):
        B.demag_batch_field(b.handle, mp, hp, E.data_ptr(), st.cuda_stream)
    torch.cuda.synchronize()
    k = max(5, args.steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = b.launch_count()
    e0.record(st)
    for _ in range(k):
        B.demag_batch_field(b.handle, mp, hp, E.data_ptr(), st.cuda_stream)
    e1.record(st)
    e1.synchronize()
    b.status()
    ms_call = e0.elapsed_time(e1) / k
    def time_modes():
        """Every batch mode timed on the batch's current padding, the
        pass-batched mode's per-pass event times; the tuned mode restored."""
        tuned_mode = b.info()["mode"]
        mode_ms = {}
        for mode, name in ((0, "persistent"), (2, "pass_batched"), (1, "branches")):
            try:
                b.set_mode(mode)
            except B.DemagError:
                continue
            for _ in range(3):
                B.demag_batch_field(b.handle, mp, hp, E.data_ptr(), st.cuda_stream)
            e0.record(st)
            for _ in range(k):
                B.demag_batch_field(b.handle, mp, hp, E.data_ptr(), st.cuda_stream)
            e1.record(st)
            e1.synchronize()
            mode_ms[name] = round(e0.elapsed_time(e1) / k, 4)
        pass_times = None
        try:
            b.set_mode(2)
            b.set_timing(True)
            for _ in range(k):
                B.demag_batch_field(b.handle, mp, hp, E.data_ptr(), st.cuda_stream)
            tms, calls = b.get_timing()
            b.set_timing(False)
            pass_times = [t / max(calls, 1) for t in tms]
        except B.DemagError:
            pass
        b.set_mode(tuned_mode)
        return mode_ms, pass_times

    modes_pow2 = time_modes()
    launches_per_call = (b.launch_count() - l0) / k
    cells_total = sum(a * bb * c for a, bb, c in dims)
    info = b.info()
    # the batch's padding autotuner: the same states with smooth padding, each
    # configuration's modes tuned; the faster is kept and timed again
    t0 = time.perf_counter()
    pad_pow2, pad_smooth = b.autotune_padding(use_cache=False)
    t_padtune = time.perf_counter() - t0
    for _ in range(3):
        B.demag_batch_field(b.handle, mp, hp, E.data_ptr(), st.cuda_stream)
    e0.record(st)
    for _ in range(k):
        B.demag_batch_field(b.handle, mp, hp, E.data_ptr(), st.cuda_stream)
    e1.record(st)
    e1.synchronize()
    b.status()
    ms_autotuned = e0.elapsed_time(e1) / k
    mode_autotuned = b.info()["mode"]
    modes_kept = time_modes()
    # the per-state padding tuner (each state's lengths timed alone; no cache)
    ms_pad = {}
    for pad in ("tuned",):
        t0 = time.perf_counter()
        os.environ["DEMAG_TUNE_CACHE"] = os.path.join(tempfile.gettempdir(), f"demag_bench_tune_{os.getpid()}.txt")
        bs = Batch(dims, cells, pad=pad)
        t_create = time.perf_counter() - t0
        bs.autotune(use_cache=False)
        for _ in range(3):
            B.demag_batch_field(bs.handle, mp, hp, E.data_ptr(), st.cuda_stream)
        e0.record(st)
        for _ in range(k):
            B.demag_batch_field(bs.handle, mp, hp, E.data_ptr(), st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        bs.status()
        ms_pad[pad] = (e0.elapsed_time(e1) / k, t_create)
        bs.close()
    try:
        os.remove(os.environ["DEMAG_TUNE_CACHE"])
    except OSError:
        pass
    if saved_cache is None:
        os.environ.pop("DEMAG_TUNE_CACHE", None)
    else:
        os.environ["DEMAG_TUNE_CACHE"] = saved_cache
    # algorithmic bytes of every pass of every state (kept padding: the whole
    # call's fraction; power-of-two padding: the pass-batched per-pass ones)
    def batch_bytes(pad_mode):
        tot = 0
        per = {nm: 0 for nm in PASS_NAMES[:5]}
        for nn in dims:
            pbs = pass_bytes(nn, tuple(B.demag_padded_lengths(*nn, pad_mode=pad_mode)), 4)
            tot += sum(pbs.values())
            for nm in per:
                per[nm] += pbs[nm]
        return tot, per

    kept_mode = B.DEMAG_PAD_SMOOTH if pad_smooth < pad_pow2 else B.DEMAG_PAD_POW2
    bytes_total, _ = batch_bytes(kept_mode)
    gbs_call = bytes_total / (ms_autotuned * 1e-3) / 1e9
    mode_ms_pow2, pass_times = modes_pow2
    mode_ms_kept, _ = modes_kept
    passes_batched = None
    if pass_times:
        bytes_p2, bytes_pass = batch_bytes(B.DEMAG_PAD_POW2)
        passes_batched = {"padding": "pow2"}
        for i, nm in enumerate(PASS_NAMES[:5]):
            t = pass_times[i]
            gbs = bytes_pass[nm] / (t * 1e-3) / 1e9
            passes_batched[nm] = {"ms": round(t, 4), "bytes": bytes_pass[nm], "gbs": round(gbs, 1),
                                  "frac": round(gbs / peak, 3)}
        passes_batched["energy"] = {"ms": round(pass_times[5], 4)}
        tp2 = sum(pass_times)
        passes_batched["whole_call_frac"] = round(bytes_p2 / (tp2 * 1e-3) / 1e9 / peak, 3)
    out = {"workload": "64 states, 32..128 x 32..128 x 8..32 cells of 3 nm, FP32, field + energy",
           "cells": cells_total,
           "hbm": {"bytes_per_call": bytes_total, "gbs": round(gbs_call, 1),
                   "frac_whole_call": round(gbs_call / peak, 3),
                   "note": "all passes of all states over the kept mode's time per call"},
           "ms_per_call_by_mode_pow2_padding": mode_ms_pow2,
           "ms_per_call_by_mode_kept_padding": mode_ms_kept,
           "passes_pass_batched": passes_batched, "mode": {0: "persistent", 1: "graph branches", 2: "pass-batched launches"}[mode_autotuned],
           "padding": "smooth" if pad_smooth < pad_pow2 else "pow2",
           # the configuration the autotuners keep (modes, then padding)
           "ms_per_call": round(ms_autotuned, 4), "cells_per_s": cells_total / (ms_autotuned / 1e3),
           "ms_per_call_pow2_padding": round(ms_call, 4), "cells_per_s_pow2_padding": cells_total / (ms_call / 1e3),
           "ms_persistent": round(t_p, 4), "ms_branches": round(t_b, 4),
           "padding_autotuner": {"ms_pow2": round(pad_pow2, 4), "ms_smooth": round(pad_smooth, 4),
                                 "kept": "smooth" if pad_smooth < pad_pow2 else "pow2",
                                 "ms_per_call_after": round(ms_autotuned, 4), "s_tuning": round(t_padtune, 2)},
           "ms_per_call_tuned_padding": round(ms_pad["tuned"][0], 4),
           "s_create_tuned_padding": round(ms_pad["tuned"][1], 2),
           "graph_launches_per_call": launches_per_call,
           "persistent_items": info["items"], "persistent_grid": info["grid"]}
    b.close()
    return out


def run_padding(args, dev):
    """Padded lengths that are not powers of two (mixed-radix passes): grids
    just above a power of two, FP32 field + energy per call with each plan
    autotuned, padded to powers of two and to the smallest even 2,3,5,7-smooth
    lengths; plus the padding autotuner's choice."""
    import torch

    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300 import inputs
    from paper_1204_4302_gb300.plan import Plan
    st = torch.cuda.current_stream(dev)
    out = []
    for n in ((130, 130, 130), (300, 260, 100), (100, 100, 100)):
        M = torch.tensor(MS * inputs.random_unit(n, seed=SEED), dtype=torch.float32, device=dev)
        H = torch.empty_like(M)
        E = torch.empty((), dtype=torch.float64, device=dev)
        row = {"grid": list(n)}
        for pad in ("pow2", "smooth"):
            plan = Plan(n, CELL, pad=pad, device=dev)
            plan.autotune(use_cache=False)
            for _ in range(max(3, args.warmup)):
                B.demag_field_energy(plan.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(), st.cuda_stream)
            torch.cuda.synchronize()
            k = max(10, args.steps)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(k):
                B.demag_field_energy(plan.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(), st.cuda_stream)
            e1.record(st)
            e1.synchronize()
            info = plan.info()
            row[pad] = {"padded": [info["px"], info["py"], info["pz"]], "ms_per_call": round(e0.elapsed_time(e1) / k, 4)}
            plan.close()
        P, mb, mp = B.demag_tune_padding(*n, *CELL, B.DEMAG_F32, use_cache=False, stream=st.cuda_stream)
        row["tuned"] = {"padded": list(P), "ms_per_call": round(mb, 4)}
        row["speedup_tuned_over_pow2"] = round(row["pow2"]["ms_per_call"] / row["tuned"]["ms_per_call"], 3)
        out.append(row)
        del M, H
        torch.cuda.empty_cache()
    return out


def run_configs(args, dev, peak):
    """The other workloads of the method's benchmark set, each on its own plan
    (autotuned): the 16^3 cube (FP64 and FP32), the 512x128x4 thin film
    (vortex + 5% noise), the 64^3 grid with a radius-32 sphere mask, the 128^3
    energy + gradient, and the 512x512x128 smooth state (forward field plus
    adjoint). Time per call from CUDA events (the small grids are L2
    resident: launch- and latency-bound, no HBM roofline), cells/s, and the
    FP32 field's rel-max error against the FP64 plan of the same call."""
    import numpy as np
    import torch

    from paper_1204_4302_gb300 import binding as B
    from paper_1204_4302_gb300 import inputs
    from paper_1204_4302_gb300.plan import Plan
    st = torch.cuda.current_stream(dev)

    def timed(fn, k):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(k):
            fn()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    def relmax(a, b):
        return float((a.double() - b.double()).abs().max() / b.double().abs().max())

    out = []
    k = max(20, args.steps)
    specs = [
        ("cube 16^3, 1 nm, random unit m, field + energy", (16, 16, 16), (1e-9,) * 3,
         MS * inputs.random_unit((16, 16, 16), seed=1), None, "field"),
        ("thin film 512x128x4, 2 nm, vortex + 5% noise, field + energy", (512, 128, 4), (2e-9,) * 3,
         MS * inputs.vortex_noise((512, 128, 4), (1024e-9, 256e-9, 8e-9), rc=0.14 * 1024e-9, noise=0.05, seed=2),
         None, "field"),
        ("sphere of radius 32 cells in 64^3, 2 nm, M = 0 outside, field + energy", (64, 64, 64), (2e-9,) * 3,
         MS * inputs.sphere_mask((64, 64, 64), 32)[None] * inputs.random_unit((64, 64, 64), seed=3), None, "field"),
        ("cube 128^3, 2 nm, energy + dE/dm", (128, 128, 128), (2e-9,) * 3,
         inputs.random_unit((128, 128, 128), seed=5), None, "grad"),
        ("cuboid 512x512x128, 1 nm, smooth state, field + adjoint", (512, 512, 128), (1e-9,) * 3,
         MS * inputs.smooth_random((512, 512, 128), 8, seed=6), None, "fwdadj"),
    ]
    for name, n, d, Mnp, _, kind in specs:
        cells = n[0] * n[1] * n[2]
        row = {"workload": name, "grid": list(n)}
        res = {}
        for prec in ("f32", "f64"):
            dt = torch.float32 if prec == "f32" else torch.float64
            plan = Plan(n, d, prec=prec, device=dev)
            if prec == "f32":
                plan.autotune(use_cache=False)
            M = torch.tensor(Mnp, dtype=dt, device=dev)
            H = torch.empty_like(M)
            E = torch.empty((), dtype=torch.float64, device=dev)
            if kind == "field":
                fn = lambda: B.demag_field_energy(plan.handle, M.data_ptr(), H.data_ptr(), E.data_ptr(),  # noqa: E731
                                                  st.cuda_stream)
            elif kind == "grad":
                fn = lambda: B.demag_energy_grad(plan.handle, M.data_ptr(), None, MS, E.data_ptr(),  # noqa: E731
                                                 H.data_ptr(), None, st.cuda_stream)
            else:
                H2 = torch.empty_like(M)
                fn = lambda: (B.demag_field(plan.handle, M.data_ptr(), H.data_ptr(), st.cuda_stream),  # noqa: E731
                              B.demag_field_adjoint(plan.handle, H.data_ptr(), H2.data_ptr(), st.cuda_stream))
            ms = timed(fn, k if prec == "f32" else max(3, k // 4))
            if prec == "f32":
                plan.set_graphs(True)          # the same calls replayed as one captured graph each
                ms_graph = timed(fn, k)
                plan.set_graphs(False)
                # per-pass event times (separate run) and, for working sets
                # larger than L2, each pass's fraction of the HBM peak
                plan.set_timing(True)
                timed(fn, k)
                pms, pn = plan.get_timing(6)
                plan.set_timing(False)
                pinfo = plan.info()
                Pp = (pinfo["px"], pinfo["py"], pinfo["pz"])
                pbytes = pass_bytes(n, Pp, 4, energy=kind != "fwdadj" and not pinfo["energy_in_z"])
                work = sum(pbytes.values()) * (2 if kind == "fwdadj" else 1)
                passes = {}
                for i, nm in enumerate(PASS_NAMES[:5]):
                    if pn[i]:
                        t = pms[i] / pn[i]
                        gbs = pbytes[nm] / (t * 1e-3) / 1e9
                        passes[nm] = {"ms": round(t, 4), "gbs": round(gbs, 1)}
                        if work > L2_BYTES:
                            passes[nm]["frac"] = round(gbs / peak, 3)
            fn()
            torch.cuda.synchronize()
            res[prec] = (ms, H.clone(), E.item() if kind != "fwdadj" else None)
            info = plan.info()
            plan.close()
            del M
        ms32, H32, E32 = res["f32"]
        ms64, H64, E64 = res["f64"]
        row.update({"padded": [info["px"], info["py"], info["pz"]], "ms_per_call_f32": round(ms32, 4),
                    "cells_per_s_f32": cells / (ms32 / 1e3), "ms_per_call_f32_graph": round(ms_graph, 4),
                    "cells_per_s_f32_graph": cells / (ms_graph / 1e3), "ms_per_call_f64": round(ms64, 4),
                    "speedup_f32_over_f64": round(ms64 / ms32, 2),
                    "f32_rel_max_err_vs_f64": relmax(H32, H64),
                    "energy_rel_diff_f32_f64": abs(E32 - E64) / abs(E64) if E64 else None,
                    "passes_f32": passes, "hbm_roofline_quoted": work > L2_BYTES,
                    "output": {"field": "H", "grad": "dE/dm", "fwdadj": "H (the adjoint runs after it)"}[kind]})
        out.append(row)
        del res, H32, H64
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------- oracle side
def _cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                v = ln.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    return v
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_sample(k: int, workers: int):
    """The oracle's field + energy on a k^3 grid of the same workload (same
    cell, same state recipe), its FFTs threaded over `workers` cores; the
    tensor table and spectrum are set up once (untimed, the method's setup /
    apply split). Returns a callable that runs one evaluation."""
    import oracle
    from paper_1204_4302_gb300 import inputs
    n = (k, k, k)
    M = MS * inputs.random_unit(n, seed=SEED)
    P = tuple(oracle.padded_size(v) for v in n)
    t0 = time.perf_counter()
    spec = oracle.tensor_spectrum(oracle.tensor_octant(n, CELL, threads=workers), P, workers=workers)
    setup_s = time.perf_counter() - t0

    def run():
        H = oracle.field_fft(M, CELL, P=P, spectrum=spec, workers=workers)
        return oracle.energy(M, H, CELL)
    return run, k ** 3, setup_s


def _time_oracle(run, reps_max: int, budget_s: float):
    run()
    t0 = time.perf_counter()
    reps = 0
    while True:
        run()
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= reps_max:
            break
    return (time.perf_counter() - t0) / reps, reps


def cpu_baseline(k: int, k_head: int):
    """The FP64 oracle timed on the host cores: on the bounded sample the
    reference arm times per step (k^3) and on the headline grid (k_head^3)."""
    cores = _host_cores()
    model = _cpu_model()
    run, cells, setup_s = _oracle_sample(k, cores)
    dt, reps = _time_oracle(run, 5, 10.0)
    out = {"value": cells / dt, "unit": "cells/s", "cores": cores, "kind": "oracle", "cpu_model": model,
           "sample": f"FP64 oracle (numpy / threaded scipy FFT convolution + fsum energy) field + energy on a "
                     f"{k}^3 grid of the same workload (2 nm cells, random unit m), FFTs over {cores} cores, "
                     f"tensor spectrum set up once ({setup_s:.1f} s, untimed); {reps} runs, {dt:.2f} s each; the "
                     f"reference arm times the same sample per step"}
    del run
    if k_head and k_head != k:
        run, cells_h, setup_h = _oracle_sample(k_head, cores)
        dth, reps_h = _time_oracle(run, 2, 20.0)
        out["headline_grid"] = {"grid": [k_head] * 3, "value": cells_h / dth, "unit": "cells/s",
                                "s_per_field": round(dth, 3), "runs": reps_h, "setup_s": round(setup_h, 1),
                                "cores": cores}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    k = args.ref_sample
    cores = _host_cores()
    run, cells, setup_s = _oracle_sample(k, cores)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    dt = (time.perf_counter() - t0) / args.steps
    value = cells / dt
    sample = (f"FP64 oracle field + energy per step on a {k}^3 grid of the same workload, FFTs over {cores} "
              f"cores, tensor spectrum set up once ({setup_s:.1f} s, untimed)")
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "cells/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded random unit magnetization)",
        "config": {"workload": "DM stray field + energy, 256x256x256 cells of 2 nm (bounded sample, see cpu_baseline)",
                   "grid": list(N_GRID), "sample_grid": [k, k, k]},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "cpu_model": _cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


PASS_KERNELS = {"x_fwd": "k_x_fwd_tma", "y_fwd": "k_col3", "z_conv": "k_z_ws", "y_inv": "k_col3", "x_inv": "k_x_inv2"}


def write_traffic(logs, command, workload):
    """profiles/traffic.json from ncu CSV logs (--metrics dram__bytes_read.sum,
    dram__bytes_write.sum,gpu__time_duration.sum, one or two launches per log
    of the 256^3 step): per pass its kernel's DRAM bytes per launch and per
    cell, keyed by the hash of the step-kernel sources. The y passes share a
    kernel template: the first captured k_col3 launch of a log is the forward
    pass, the second the inverse one."""
    import csv as _csv
    launches = []  # (kernel name, {metric: value}) in capture order
    for path in logs:
        with open(path) as fh:
            rows = [r for r in _csv.reader(line for line in fh if line.startswith('"'))]
        head, body = rows[0], rows[1:]
        ki, ii, mi, vi = head.index("Kernel Name"), head.index("ID"), head.index("Metric Name"), head.index("Metric Value")
        by_id = {}
        for r in body:
            ent = by_id.setdefault(r[ii], (r[ki], {}))
            ent[1][r[mi]] = float(r[vi].replace(",", ""))
        launches += [by_id[k] for k in sorted(by_id, key=int)]
    cells = N_GRID[0] * N_GRID[1] * N_GRID[2]
    out, col3 = {}, [l for l in launches if "k_col3" in l[0]]
    for name, pat in PASS_KERNELS.items():
        if pat == "k_col3":
            pick = col3[0] if name == "y_fwd" and col3 else (col3[1] if len(col3) > 1 else None)
        else:
            pick = next((l for l in launches if pat in l[0]), None)
        if pick is None:
            continue
        kname, m = pick
        rd, wr = m["dram__bytes_read.sum"], m["dram__bytes_write.sum"]
        short = kname.split("(")[0].replace("void ", "").replace("demag::", "").strip()
        out[name] = {"kernel": short, "source_hash": source_hash(), "dram_read_bytes": rd, "dram_write_bytes": wr,
                     "bytes_per_cell": (rd + wr) / cells, "ncu_ms": m["gpu__time_duration.sum"] / 1e6,
                     "workload": workload, "command": command}
    with open(TRAFFIC, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: v["bytes_per_cell"] for k, v in out.items()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--states", type=int, default=STATES, help="independent states per step")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-sample", type=int, default=128,
                    help="grid edge of the oracle sample per reference step (and of cpu_baseline.value)")
    ap.add_argument("--cpu-headline", type=int, default=256,
                    help="grid edge of the oracle timed on the headline grid (0: skip)")
    ap.add_argument("--skip-f64", action="store_true")
    ap.add_argument("--skip-grad", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-padding", action="store_true")
    ap.add_argument("--skip-configs", action="store_true")
    ap.add_argument("--skip-sp", action="store_true", help="skip the scalar-potential method leg")
    ap.add_argument("--skip-tg", action="store_true", help="skip the tensor-grid method leg")
    ap.add_argument("--no-tune", action="store_true", help="default kernel variants (for profiling runs)")
    ap.add_argument("--pad", choices=["pow2", "smooth"], default="pow2",
                    help="padded lengths of the headline plan (smooth: mixed-radix passes; for profiling runs)")
    ap.add_argument("--variants", default="", help="fixed z,y,x kernel variants instead of autotuning")
    ap.add_argument("--grid", default="", help="grid edge n (cubic) or nx,ny,nz (default 256^3, the headline; "
                                               "other grids are for profiling runs)")
    ap.add_argument("--write-traffic", nargs="+", default=None, metavar="NCU_CSV",
                    help="write profiles/traffic.json from ncu CSV logs of the step kernels and exit "
                         "(with --traffic-command, the command that produced them)")
    ap.add_argument("--traffic-command", default="")
    args = ap.parse_args()
    if args.write_traffic:
        write_traffic(args.write_traffic, args.traffic_command,
                      "256^3 FP32 field + energy, padded 512^3, z variant 6, y 2, x 1")
        return
    if args.warmup < 3:
        args.warmup = 3
    global N_GRID
    if args.grid:
        g = [int(v) for v in args.grid.split(",")]
        N_GRID = tuple(g) if len(g) == 3 else (g[0],) * 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
