"""The batched, autograd-checkpointed, reduced-precision-snapshot gradient
against the plain per-shot FP32 gradient on the same GPU:
python -m paper_1406_1864_gb300.bench_forms [options].

Workload: the seeded dipping-layer model at 400 x 1200 cells, 64 shots,
600 receivers, nt 5000 (workloads "dipping_400x1200_64shots"), OLS misfit,
starting model v_init, observed data modelled on v_true. Forms, each timed
with CUDA events around the whole gradient (after one untimed run):

* per_shot_f32: one fwi_adjoint_gradient call per shot (sponge checkpoints,
  FP32), the 64 gradients summed;
* batched_f32: one fwi_adjoint_gradient call over all shots;
* autograd_<snap>: autograd.traces (forward with checkpoints, backward =
  the hand-written adjoint) over all shots and the OLS loss in FP64, with
  sqrt(nt) snapshot checkpoints stored as F32, bfloat16 or scaled float16.

Reports Gpts/s (physical points x nt x shots per second), the speed-up over
the per-shot form, and each gradient's relative L2 difference from the
per-shot form's, as one JSON line.
"""
from __future__ import annotations

import argparse
import json


def main():
    import torch

    from . import autograd, fwi, workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="dipping_400x1200_64shots")
    ap.add_argument("--nt", type=int, default=0, help="0: the workload's")
    ap.add_argument("--shots", type=int, default=0, help="0: the workload's")
    args = ap.parse_args()
    p = W.workload(args.workload)
    if args.nt or args.shots:
        p = W.dipping(nz=p.nz, nx=p.nx, nt=args.nt or p.nt, ns=args.shots or p.nshots, nrec=p.nrec,
                      name=p.name)
    grid, geom = fwi.from_problem(p)
    ws = fwi.Workspace()
    d_obs = fwi.forward(grid, geom, torch.as_tensor(p.v_true, device="cuda"), ws=ws)
    v = torch.as_tensor(p.v_init, device="cuda")
    units = p.nz * p.nx * p.nt * p.nshots
    ols = fwi.Options(misfit="ols", precond="none")

    def timed(fn):
        fn()  # untimed: first-call set-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), g

    def per_shot():
        g = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        for s in range(p.nshots):
            r = fwi.adjoint_gradient(grid, geom.subset(s, s + 1), v, d_obs[s:s + 1].contiguous(), ols,
                                     want_pre=False, want_illum=False, ws=ws)
            g += r["grad"].double()
        return g

    def batched():
        return fwi.adjoint_gradient(grid, geom, v, d_obs, ols, want_pre=False, want_illum=False, ws=ws)["grad"]

    def auto(snap):
        def run():
            vv = v.clone().requires_grad_(True)
            d = autograd.traces(vv, grid, geom, fwi.Options(ckpt="snapshot", snap=snap))
            (0.5 * ((d.double() - d_obs.double()) ** 2).sum()).backward()
            return vv.grad
        return run

    res = {}
    ms, g_ref = timed(per_shot)
    g_ref = g_ref.double()
    res["per_shot_f32"] = {"ms": ms}
    forms = [("batched_f32", batched)] + [(f"autograd_{s}", auto(s)) for s in ("f32", "bf16", "f16s")]
    for name, fn in forms:
        ms, g = timed(fn)
        res[name] = {"ms": ms, "rel_diff_vs_per_shot": float(torch.linalg.vector_norm(g.double() - g_ref) /
                                                               torch.linalg.vector_norm(g_ref))}
    for r in res.values():
        r["Gpts_per_s"] = units / (r["ms"] * 1e-3) / 1e9
        r["speedup_vs_per_shot"] = res["per_shot_f32"]["ms"] / r["ms"]
    print(json.dumps({"workload": f"{p.name}: {p.nz}x{p.nx}, {p.nshots} shots, nt {p.nt}, {p.nrec} receivers",
                      "forms": res}), flush=True)


if __name__ == "__main__":
    main()
