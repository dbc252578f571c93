"""Timing of Born modelling and Gauss-Newton Hessian-vector products:
python -m paper_1406_1864_gb300.bench_born [options].

On the seeded dipping-layer workload (workloads.dipping, default 300 x 1000,
96 shots, nt 4000, dv = v_true - v_init; --shots and --nt give smaller cases
of the same model), times fwi_born and
fwi_gauss_newton_hvp with CUDA events on the library's stream (phase times of
the library's profiler: the Born pass, the backward pass). The Born step
moves 24 B per padded point-step per shot at the least: u^n and du^n read
once (halo tiles), u^{n-1} and du^{n-1} read, u^{n+1} and du^{n+1} written;
the backward step 28 B (its own figure). Prints one JSON line with the
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
    for name, fn in (("born", fwi.born), ("gn_hvp", fwi.gauss_newton_hvp)):
        for _ in range(args.warmup):
            fn(grid, geom, v, dv, ws=ws)
        best = None
        for _ in range(args.reps):
            torch.cuda.synchronize()
            fn(grid, geom, v, dv, ws=ws)
            ph = fwi.last_phase_times()
            if best is None or ph["forward_ms"] + ph["adjoint_ms"] + ph["other_ms"] < best["total"]:
                best = dict(ph, total=ph["forward_ms"] + ph["adjoint_ms"] + ph["other_ms"])
        us_b = 1e3 * best["forward_ms"] / max(1, best["forward_launches"])
        r = {"call_ms": best["total"], "born_us_per_level": us_b,
             "born_alg_GBps": BORN_BYTES * npad * p.nshots / (us_b * 1e-6) / 1e9,
             "Gpts_per_s": p.nz * p.nx * p.nt * p.nshots / (best["total"] * 1e-3) / 1e9}
        r["born_frac"] = r["born_alg_GBps"] / peak
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
