"""Reproduction of the paper's stray-field experiments (Sec. 5) on the GPU.

    python -m paper_1204_4302_gb300.reproduce [--prec f64|f32] [--convergence] [--json]

States (unit edge length, magnetization normalised, energies in mu0 Ms^2):
  * homogeneously magnetized cube, 40^3 cells (Sec. 5.1; exact e = 1/6),
  * flower state in the cube, a = c = 1, b = 2 (Sec. 5.2, Eq. "flower_mag"),
  * Feldtkeller vortex in the cube, r_c = 0.14 (Sec. 5.2, Eq. "config1"),
  * homogeneous and vortex thin film 1 x 1 x 0.1, 80 x 80 x 8 cells,
    magnetized out of plane (Sec. 5.3),
  * homogeneous sphere of radius 0.5 on a staircase grid (Sec. 5.4; the paper
    shows only its convergence figure).
For each state the DM and SP energies come from the library's CUDA path,
next to the values the paper prints, together with the paper's field error
of SP against DM (Eq. "relerr": root mean square over cells of the field
difference, in units of Ms) and the mean and largest angle between the two
fields. --convergence adds energy against grid size for the cube (exact 1/6)
and the sphere (continuum value pi/36), the data behind the paper's
convergence figure, which the text does not print. --lowrank adds the data
of the paper's low-rank figure (Sec. 3.2), also not printed: the relative
error (Eq. "relr") of CP and Tucker approximations found by ALS on the GPU
from seeded random initial guesses, for the flower (a = c = 0.5, b = 1) and
vortex (r_c = 1/2) cube states, against the rank at N = 100^3 cells and
against N at rank 5.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import inputs
from .plan import Plan

MU0 = 4e-7 * math.pi

# Energies printed in the paper (mu0 Ms^2, unit edge): (table, DM, SP). For the
# homogeneous cube the table gives relative errors to the exact 1/6.
PAPER = {
    "cube_homogeneous": ("Table cube_homo", {"dm_relerr": 2.9e-9, "sp_relerr": 1.1e-3}),
    "cube_flower": ("Table cube_flower", {"dm": 1.528e-1, "sp": 1.526e-1}),
    "cube_vortex": ("Table cube_vortex", {"dm": 2.189e-2, "sp": 2.163e-2}),
    "film_homogeneous": ("Table thin_homo", {"dm": 4.025e-2, "sp": 4.021e-2}),
    "film_vortex": ("Table thin_vortex", {"dm": 1.569e-3, "sp": 1.555e-3}),
}


def state(name: str, n=None):
    """(grid, cell edges, m) of one of the paper's states."""
    if name.startswith("cube") or name == "sphere":
        n = n or (40, 40, 40)
        ext = (1.0, 1.0, 1.0)
    else:
        n = n or (80, 80, 8)
        ext = (1.0, 1.0, 0.1)
    d = tuple(e / k for e, k in zip(ext, n))
    if name.endswith("homogeneous"):
        m = inputs.uniform(n, (0, 0, 1))
    elif name == "cube_flower":
        m = inputs.flower(n, ext)
    elif name.endswith("vortex"):
        m = inputs.vortex(n, ext, rc=0.14)
    elif name == "sphere":
        m = inputs.uniform(n, (0, 0, 1)) * inputs.sphere_mask(n, n[0] / 2)[None]
    else:
        raise KeyError(name)
    return tuple(n), d, m


def fields(n, d, m, prec: str):
    """H / Ms of both methods and their energies e = E / (mu0 Ms^2)."""
    dt = torch.float32 if prec == "f32" else torch.float64
    M = torch.tensor(m, dtype=dt, device="cuda")
    out = {}
    for method in ("dm", "sp"):
        p = Plan(n, d, prec=prec, method=method)
        H, E = p.field_energy(M)
        torch.cuda.synchronize()
        out[method] = (H.double(), float(E.item()) / MU0)
        p.close()
    return out


def field_errors(Hdm: torch.Tensor, Hsp: torch.Tensor) -> dict:
    """Paper Eq. "relerr" (RMS over cells of |H_DM - H_SP|) and field angles."""
    ncell = Hdm[0].numel()
    diff = Hdm - Hsp
    relerr = math.sqrt(float((diff * diff).sum()) / ncell)
    ndm = Hdm.norm(dim=0)
    nsp = Hsp.norm(dim=0)
    live = (ndm > 0) & (nsp > 0)
    cosang = ((Hdm * Hsp).sum(0)[live] / (ndm[live] * nsp[live])).clamp(-1.0, 1.0)
    ang = torch.rad2deg(torch.arccos(cosang))
    return {"relerr_h": relerr, "angle_mean_deg": float(ang.mean()) if ang.numel() else 0.0,
            "angle_max_deg": float(ang.max()) if ang.numel() else 0.0}


def run_states(prec: str = "f64") -> list[dict]:
    rows = []
    for name in ("cube_homogeneous", "cube_flower", "cube_vortex", "film_homogeneous", "film_vortex", "sphere"):
        n, d, m = state(name)
        f = fields(n, d, m, prec)
        row = {"state": name, "grid": list(n), "e_dm": f["dm"][1], "e_sp": f["sp"][1]}
        row.update(field_errors(f["dm"][0], f["sp"][0]))
        if name in PAPER:
            table, vals = PAPER[name]
            row["paper"] = dict(vals, source=table)
            if name == "cube_homogeneous":
                row["relerr_dm_vs_exact"] = abs(row["e_dm"] - 1 / 6) * 6
                row["relerr_sp_vs_exact"] = abs(row["e_sp"] - 1 / 6) * 6
        rows.append(row)
    return rows


def run_convergence(prec: str = "f64", sizes=(8, 16, 24, 32, 48, 64, 96)) -> list[dict]:
    rows = []
    for k in sizes:
        for name, exact in (("cube_homogeneous", 1 / 6), ("sphere", math.pi / 36)):
            n, d, m = state(name, (k, k, k))
            f = fields(n, d, m, prec)
            rows.append({"state": name, "n": k, "e_dm": f["dm"][1], "e_sp": f["sp"][1],
                         "relerr_dm": abs(f["dm"][1] - exact) / exact, "relerr_sp": abs(f["sp"][1] - exact) / exact})
    return rows


def lowrank_errors(m: np.ndarray, rank: int, seed: int = 5, cp_iters: int = 100, tucker_iters: int = 10) -> dict:
    """Eq. "relr" of the CP-ALS and Tucker-ALS (ranks r, r, r) approximations
    of a (3, nz, ny, nx) state, from seeded random initial guesses."""
    from . import lowrank
    nz, ny, nx = m.shape[1:]
    M = torch.tensor(m, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(seed)
    init = [torch.tensor(rng.standard_normal((3, rank, v)), dtype=torch.float64, device="cuda") for v in (nx, ny, nz)]
    *_, e_cp = lowrank.cp_als(M, rank, init, cp_iters)
    tr = tuple(min(rank, v) for v in (nx, ny, nz))
    init_t = [f[:, :r] for f, r in zip(init, tr)]
    *_, e_tk = lowrank.tucker_als(M, tr, init_t, tucker_iters)
    return {"cp": e_cp, "tucker": e_tk}


def lowrank_states(n):
    ext = (1.0, 1.0, 1.0)
    return {"flower": inputs.flower(n, ext, a=0.5, b=1.0, c=0.5), "vortex": inputs.vortex(n, ext, rc=0.5)}


def run_lowrank(ranks=range(1, 11), sizes=(10, 20, 40, 60, 80, 100), n_rank_sweep=100, rank_n_sweep=5) -> dict:
    by_rank, by_n = [], []
    for name, m in lowrank_states((n_rank_sweep,) * 3).items():
        for r in ranks:
            by_rank.append(dict(state=name, n=n_rank_sweep, rank=r, **lowrank_errors(m, r)))
    for k in sizes:
        for name, m in lowrank_states((k,) * 3).items():
            by_n.append(dict(state=name, n=k, rank=rank_n_sweep, **lowrank_errors(m, rank_n_sweep)))
    return {"by_rank": by_rank, "by_n": by_n}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--prec", choices=["f32", "f64"], default="f64")
    ap.add_argument("--convergence", action="store_true")
    ap.add_argument("--lowrank", action="store_true")
    ap.add_argument("--json", action="store_true")
    args = ap.parse_args()
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is needed (the library has no CPU path)")
    out = {"states": run_states(args.prec)}
    if args.convergence:
        out["convergence"] = run_convergence(args.prec)
    if args.lowrank:
        out["lowrank"] = run_lowrank()
    if args.json:
        print(json.dumps(out))
        return
    print(f"{'state':18s} {'e_DM':>12s} {'e_SP':>12s} {'paper DM':>10s} {'paper SP':>10s} "
          f"{'relerr h':>9s} {'ang mean':>9s} {'ang max':>8s}")
    for r in out["states"]:
        p = r.get("paper", (None, {}))
        vals = p if isinstance(p, dict) else {}
        pd = vals.get("dm", vals.get("dm_relerr", float("nan")))
        ps = vals.get("sp", vals.get("sp_relerr", float("nan")))
        print(f"{r['state']:18s} {r['e_dm']:12.6e} {r['e_sp']:12.6e} {pd:10.4g} {ps:10.4g} "
              f"{r['relerr_h']:9.2e} {r['angle_mean_deg']:9.2e} {r['angle_max_deg']:8.2f}")
    if args.convergence:
        print(f"\n{'state':18s} {'n':>4s} {'e_DM':>12s} {'e_SP':>12s} {'err DM':>9s} {'err SP':>9s}")
        for r in out["convergence"]:
            print(f"{r['state']:18s} {r['n']:4d} {r['e_dm']:12.6e} {r['e_sp']:12.6e} "
                  f"{r['relerr_dm']:9.2e} {r['relerr_sp']:9.2e}")
    if args.lowrank:
        print(f"\n{'state':8s} {'N':>7s} {'rank':>4s} {'relerr CP':>10s} {'relerr Tucker':>13s}")
        for r in out["lowrank"]["by_rank"] + out["lowrank"]["by_n"]:
            print(f"{r['state']:8s} {r['n'] ** 3:7d} {r['rank']:4d} {r['cp']:10.3e} {r['tucker']:13.3e}")


if __name__ == "__main__":
    main()
