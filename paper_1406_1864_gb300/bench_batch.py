"""Throughput of the uneven multi-model batch against one call per model:
python -m paper_1406_1864_gb300.bench_batch [options].

Workload: three independent models of the seeded dipping-layer generator at
200 x 400, 350 x 900 and 500 x 1500 cells, 32 shots each, nx / 2 receivers,
nt 4000 (workloads.uneven_batch), starting model v_init, observed data
modelled on v_true. Gradient options: OLS misfit with the illumination
preconditioner (``--variant plain``, default) or the time-integral misfit
with the offset Hessian |h| <= 10 and offset preconditioning
(``--variant full``). Forms, each timed with CUDA events around the whole
work after one untimed run, inputs resident on the GPU:

* batch_direct: one fwi_batch_gradient call, every time level of the three
  models in one launch per step kind;
* batch_graph: the same batch recorded once as a CUDA graph (fwi_exec) and
  replayed;
* separate_direct: one fwi_adjoint_gradient call per model, in sequence;
* separate_graph: one recorded graph per model, replayed in sequence.

Before the timing, fwi_autotune picks tiles for each model's shape; the
batch runs with the choice of its first model. Reports Gpts/s (physical
points x nt x shots per second, summed over the models) and ms per gradient
of each form, and the largest relative L2 difference between the batched
and the separate gradients, as one JSON line.
"""
from __future__ import annotations

import argparse
import json


def main():
    import torch

    from . import fwi, workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--variant", choices=["plain", "full"], default="plain")
    ap.add_argument("--nt", type=int, default=4000)
    ap.add_argument("--shots", type=int, default=32)
    ap.add_argument("--repeats", type=int, default=3)
    args = ap.parse_args()
    probs = W.uneven_batch(nt=args.nt, ns=args.shots)
    if args.variant == "full":
        opts = fwi.Options(misfit="integral", illum="u2", hmax=10, precond="offset")
    else:
        opts = fwi.Options(misfit="ols", illum="u2", hmax=-1, precond="illum")
    grids, geoms, vs, dobs = [], [], [], []
    for p in probs:
        grid, geom = fwi.from_problem(p)
        grids.append(grid)
        geoms.append(geom)
        vs.append(torch.as_tensor(p.v_init, device="cuda"))
        dobs.append(fwi.forward(grid, geom, torch.as_tensor(p.v_true, device="cuda")))
    units = sum(p.nz * p.nx * p.nt * p.nshots for p in probs)
    ws = fwi.Workspace()  # direct calls and the batch graph (grows to the batch's size)
    tiles = [fwi.autotune(g, ge, v, opts, ws=ws) for g, ge, v in zip(grids, geoms, vs)]

    def timed(fn):
        fn()  # untimed: first-call set-up
        torch.cuda.synchronize()
        best = None
        for _ in range(args.repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best, out

    def batch_direct():
        return fwi.batch_gradient(grids, geoms, vs, dobs, opts, ws=ws)

    def separate_direct():
        return [fwi.adjoint_gradient(g, ge, v, d, opts, ws=ws) for g, ge, v, d in zip(grids, geoms, vs, dobs)]

    forms = {}
    ms, out_b = timed(batch_direct)
    forms["batch_direct"] = ms
    grads_b = [o["grad"].clone() for o in out_b]
    ms, out_s = timed(separate_direct)
    forms["separate_direct"] = ms
    grads_s = [o["grad"].clone() for o in out_s]
    bgraph = fwi.GradientGraph(grids, geoms, vs, dobs, opts, ws=ws)
    forms["batch_graph"], _ = timed(bgraph.run)
    bgraph.close()
    del bgraph
    # one graph per model, each bound to its own workspace
    sgraphs = [fwi.GradientGraph([g], [ge], [v], [d], opts, ws=fwi.Workspace()) for g, ge, v, d in zip(grids, geoms,
                                                                                                      vs, dobs)]
    forms["separate_graph"], _ = timed(lambda: [sg.run() for sg in sgraphs])
    for sg in sgraphs:
        sg.close()
    diff = max(float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))
               for a, b in zip(grads_b, grads_s))
    line = {
        "workload": "uneven batch: " + ", ".join(f"{p.nz}x{p.nx}" for p in probs)
                    + f", {args.shots} shots each, nt {args.nt}",
        "variant": args.variant, "units_gpts": units / 1e9,
        "forms": {k: {"ms": v, "gpts_s": units / (v * 1e-3) / 1e9} for k, v in forms.items()},
        "speedup_batch_graph_vs_separate_graph": forms["separate_graph"] / forms["batch_graph"],
        "max_rel_l2_batch_vs_separate": diff, "tiles_per_model": tiles,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
