"""Timing of the 3-D path: python -m paper_1406_1864_gb300.bench3d [options].

Models the seeded 3-D dipping-layer workload (workloads.dipping3d: surface
receivers every cell, shots on a grid at depth 2), times forward modelling
(per-level step time and algorithmic bandwidth at 16 B per padded
point-step per shot) and one snapshot-checkpointed gradient per snapshot
precision, with CUDA events on the library's stream, after fwi_autotune has
picked the step variants (``--no-autotune``: the defaults), and from the
gradient's phase times an upper bound of the backward step per level (20 B
of fields per padded point-step per shot: psi^{m+1}, psi^{m+2}, psi^m, the
imaging factor q^{m-1} kept by the re-propagation, c2). With ``--hmax H``
also the offset-Hessian diagonal (offsets 0..H): its forward phase against
that of the illumination pass (the same steps without the sums) gives the
sums' time per level (4 B per physical point-step per shot: u^n read once
more). Prints one JSON line.
Defaults: the 200 x 400 x 400, 8-shot, nt 3000 workload in shot groups of 4.
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    import torch

    from . import fwi, workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--nz", type=int, default=200)
    ap.add_argument("--ny", type=int, default=400)
    ap.add_argument("--nx", type=int, default=400)
    ap.add_argument("--shots", type=int, default=8)
    ap.add_argument("--nt", type=int, default=3000)
    ap.add_argument("--shot-group", type=int, default=4)
    ap.add_argument("--snap", default="f32,bf16")
    ap.add_argument("--no-autotune", action="store_true", help="default step variants (no fwi_autotune)")
    ap.add_argument("--variants", default="", help="F,B: pin the forward and backward step variants "
                    "(fwi_autotune_set) instead of autotuning")
    ap.add_argument("--segments", default="0,0", help="F,B: z-segments per column with --variants "
                    "(0: chosen from the items and resident CTAs)")
    ap.add_argument("--hmax", type=int, default=-1, help=">= 0: also time the offset-Hessian diagonal")
    args = ap.parse_args()
    p = W.dipping3d(nz=args.nz, ny=args.ny, nx=args.nx, nt=args.nt, ns=args.shots)
    grid, geom = fwi.from_problem(p)
    ws = fwi.Workspace()
    grp = fwi.Options(shot_group=args.shot_group)
    npad = (p.nz + 2 * p.sponge) * (p.ny + 2 * p.sponge) * (p.nx + 2 * p.sponge)
    g = min(p.nshots, args.shot_group or p.nshots)
    tiles = "default"
    if args.variants:
        fv, bv = (int(x) for x in args.variants.split(","))
        fs, bs = (int(x) for x in args.segments.split(","))
        tiles = {"forward_variant": fv, "forward_chunk": fs, "backward_variant": bv, "backward_chunk": bs}
        fwi.autotune_set(grid, geom, fwi.Options(ckpt="snapshot", shot_group=args.shot_group), tiles)
    elif not args.no_autotune:  # step variants timed on this problem (not timed)
        tiles = fwi.autotune(grid, geom, torch.as_tensor(p.v_init, device="cuda"),
                             fwi.Options(ckpt="snapshot", shot_group=args.shot_group), ws=ws)
    fwi.profile(True)
    torch.cuda.synchronize()
    d_obs = fwi.forward(grid, geom, torch.as_tensor(p.v_true, device="cuda"), ws=ws, opts=grp)
    ph = fwi.last_phase_times()
    us = 1e3 * ph["forward_ms"] / max(1, ph["forward_launches"])
    out = {"workload": f"dipping3d {p.nz}x{p.ny}x{p.nx}, {p.nshots} shots, nt {p.nt}, {p.nrec} receivers",
           "shot_group": g, "tiles": tiles, "forward_us_per_level": us,
           "forward_alg_GBps": 16 * npad * g / (us * 1e-6) / 1e9, "gradients": {}}
    v = torch.as_tensor(p.v_init, device="cuda")
    for snap in args.snap.split(","):
        o = fwi.Options(ckpt="snapshot", snap=snap, shot_group=args.shot_group)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fwi.adjoint_gradient(grid, geom, v, d_obs, o, ws=ws)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["gradients"][snap] = {"seconds": dt, "Gpts_per_s": p.phys_points * p.nt * p.nshots / dt / 1e9,
                                  "workspace_GB": fwi.workspace_bytes(grid, geom, o, "gradient") / 1e9}
        # backward step per level: the 3-D gradient's first phase spans the
        # time loops of all shot groups (forward passes, the segments'
        # re-propagation, the backward steps, residuals and snapshot copies);
        # the forward and re-propagation steps are counted at the forward
        # pass's step time, the rest is put on the nt - 1 backward steps per
        # group (an upper bound of the backward step time)
        ph = fwi.last_phase_times()
        groups = -(-p.nshots // g)
        n_bwd = (p.nt - 1) * groups
        n_rep = ph["adjoint_launches"] - n_bwd
        if n_bwd > 0 and n_rep >= 0:
            bus = (1e3 * ph["forward_ms"] - (ph["forward_launches"] + n_rep) * us) / n_bwd
            out["gradients"][snap]["backward_us_per_level_est"] = bus
            out["gradients"][snap]["backward_alg_GBps_est"] = 20 * npad * g / (bus * 1e-6) / 1e9
    if args.hmax >= 0:
        runs = {"illumination": lambda: fwi.illumination(grid, geom, v, grp, ws=ws),
                "offset_hessian": lambda: fwi.offset_hessian_diag(
                    grid, geom, v, fwi.Options(hmax=args.hmax, shot_group=args.shot_group), ws=ws)}
        ms = {}
        for name, run in runs.items():
            for _ in range(2):  # the first call warms up
                run()
                torch.cuda.synchronize()
            ms[name] = fwi.last_phase_times()["forward_ms"]
        levels = max(1, (p.nt - 1) * -(-p.nshots // g))
        ous = 1e3 * (ms["offset_hessian"] - ms["illumination"]) / levels
        out["offset_hessian"] = {"hmax": args.hmax, "forward_phase_ms": ms["offset_hessian"],
                                 "illumination_forward_phase_ms": ms["illumination"],
                                 "sums_us_per_level_est": ous,
                                 "sums_alg_GBps_est": 4 * p.phys_points * g / (ous * 1e-6) / 1e9 if ous > 0 else None}
    fwi.profile(False)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
