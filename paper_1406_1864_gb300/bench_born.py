"""Timing of Born modelling, Gauss-Newton Hessian-vector products and the
extended operators: python -m paper_1406_1864_gb300.bench_born [options].

On the seeded dipping-layer workload (workloads.dipping, default 300 x 1000,
96 shots, nt 4000, dv = v_true - v_init; --shots and --nt give smaller cases
of the same model), times fwi_born and
fwi_gauss_newton_hvp with CUDA events on the library's stream (phase times of
the library's profiler: the Born pass, the backward pass). The Born step
moves 24 B per padded point-step per shot at the least: u^n and du^n read
once (halo tiles), u^{n-1} and du^{n-1} read, u^{n+1} and du^{n+1} written;
the backward step 28 B (its own figure). With --hext H (> 0) also
fwi_extended_born and fwi_extended_migration with offsets -H..H (a random
dv_ext and a random adjoint source): the same 24 B / 28 B
per point-step (the 2 H + 1 planes of D~ and of the image are read or added
once per tile and chunk of shots). Prints one JSON line with the
per-level step times, the algorithmic bandwidth and its fraction of the
measured copy bandwidth (MEASURED_PEAKS.json at the repository root, burst
figure), and the whole-call throughput in physical point-steps per second.
"""
from __future__ import annotations

import argparse
import json
import os

BORN_BYTES = 24
BWD_BYTES = 28


def hbm_peak():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def main():
    import torch

    from . import fwi, workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--shots", type=int, default=96)
    ap.add_argument("--nt", type=int, default=4000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--hext", type=int, default=4)
    args = ap.parse_args()
    p = W.dipping(ns=args.shots, nt=args.nt)
    grid, geom = fwi.from_problem(p)
    ws = fwi.Workspace()
    v = torch.as_tensor(p.v_init, device="cuda")
    dv = torch.as_tensor((p.v_true - p.v_init).astype("float32"), device="cuda")
    npad = (p.nz + 2 * p.sponge) * (p.nx + 2 * p.sponge)
    peak, kind = hbm_peak()
    fwi.profile(True)
    res = {}
    calls = [("born", lambda: fwi.born(grid, geom, v, dv, ws=ws)),
             ("gn_hvp", lambda: fwi.gauss_newton_hvp(grid, geom, v, dv, ws=ws))]
    if args.hext > 0:
        gen = torch.Generator(device="cuda").manual_seed(3)
        dve = 20.0 * torch.randn((2 * args.hext + 1,) + tuple(v.shape), device="cuda", generator=gen)
        adj = torch.randn((p.nshots, p.nt, p.nrec), device="cuda", generator=gen)
        calls += [("extended_born", lambda: fwi.extended_born(grid, geom, v, dve, ws=ws)),
                  ("extended_migration", lambda: fwi.extended_migration(grid, geom, v, adj, args.hext, ws=ws))]
    for name, fn in calls:
        for _ in range(args.warmup):
            fn()
        best = None
        for _ in range(args.reps):
            torch.cuda.synchronize()
            fn()
            ph = fwi.last_phase_times()
            if best is None or ph["forward_ms"] + ph["adjoint_ms"] + ph["other_ms"] < best["total"]:
                best = dict(ph, total=ph["forward_ms"] + ph["adjoint_ms"] + ph["other_ms"])
        us_b = 1e3 * best["forward_ms"] / max(1, best["forward_launches"])
        fb = 16 if name == "extended_migration" else BORN_BYTES   # its forward pass is the plain step
        r = {"call_ms": best["total"], "forward_us_per_level": us_b,
             "forward_alg_GBps": fb * npad * p.nshots / (us_b * 1e-6) / 1e9,
             "Gpts_per_s": p.nz * p.nx * p.nt * p.nshots / (best["total"] * 1e-3) / 1e9}
        r["forward_frac"] = r["forward_alg_GBps"] / peak
        if best["adjoint_launches"]:
            us_a = 1e3 * best["adjoint_ms"] / best["adjoint_launches"]
            r["bwd_us_per_level"] = us_a
            r["bwd_alg_GBps"] = BWD_BYTES * npad * p.nshots / (us_a * 1e-6) / 1e9
            r["bwd_frac"] = r["bwd_alg_GBps"] / peak
        res[name] = r
    fwi.profile(False)
    print(json.dumps({"workload": f"dipping {p.nz}x{p.nx}, {p.nshots} shots, nt {p.nt}, {p.nrec} receivers",
                      "peak_GBps": peak, "peak_kind": kind, **res}), flush=True)


if __name__ == "__main__":
    main()
