"""Convergence experiments after the paper's two examples, on the seeded
dipping-layer model (the paper's Marmousi model is not available):
python -m paper_1406_1864_gb300.convergence [options].

* Example 1 (Sec. 2.1): starting model v(z) = 1500 + z (m/s, z in m), L-BFGS,
  the OLS misfit against the time-integral misfit of Eq. 2, both with the
  illumination preconditioner (Eq. 1); 200 iterations in the paper.
* Example 2 (Sec. 3.1): starting model the true model Gaussian-smoothed,
  PRCG without preconditioner, with the illumination (Eq. 1) and with the
  offset-Hessian diagonal (Sec. 3, hmax 10); 270 iterations in the paper.
  Also the receiver-inclusive forms (fwi_receiver_factor): the illumination
  times Plessix and Mulder's factor, and the offset Hessian times the
  receiver Green's-function correlations (recomputed every 10 gradients).

Defaults: 150 x 460 cells of 20 m (3 km x 9.2 km), 80 shots at 20 m depth,
receivers at 20 m depth on every cell (full aperture), 1.2 s recording
(nt 800 at dt 1.5 ms; --record sets it: reflections from the bottom of the
model arrive after about 2.5 s), Ricker f0 6 Hz. Reports per iteration the
misfit (relative to the first), the relative model error ||v - v_true|| /
||v_0 - v_true|| over the whole model, over its upper and lower halves, and
over the depth band from a quarter to half of the model depth (0.75 - 1.5
km: the deepest part a 1.2 s recording constrains; below about v T / 2 the
forward and back-propagated fields do not meet and the gradient is zero),
and gradient and misfit-evaluation counts, as one JSON line (and into
--out).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def problem(nz=150, nx=460, dx=20.0, dt=1.5e-3, nt=800, ns=80, f0=6.0, seed=0, example=1):
    from . import workloads as W
    p = W.dipping(nz=nz, nx=nx, dx=dx, dt=dt, nt=nt, ns=ns, nrec=nx, rec_step=1, f0=f0, seed=seed, sponge=20,
                  name="dipping_convergence")
    if example == 1:
        z = np.arange(nz, dtype=np.float64)[:, None] * dx
        p.v_init = np.broadcast_to(1500.0 + z, (nz, nx)).astype(np.float32).copy()
    else:
        p.v_init = W.smooth(p.v_true, 300.0 / dx).astype(np.float32)
    p.vref = float(max(p.v_true.max(), p.v_init.max()))
    return p


def run(p, configs, iters, max_update):
    import torch

    from . import fwi, inversion as I
    grid, geom = fwi.from_problem(p)
    v_true = torch.as_tensor(p.v_true, device="cuda")
    d_obs = fwi.forward(grid, geom, v_true)
    v0 = torch.as_tensor(p.v_init, device="cuda")
    z0, z1 = p.nz // 4, p.nz // 2
    bands = {"deep_band": (z0, z1), "upper_half": (0, p.nz // 2), "lower_half": (p.nz // 2, p.nz)}
    e0b = {k: float(torch.linalg.vector_norm((v0[a:b] - v_true[a:b]).double())) for k, (a, b) in bands.items()}
    ws = fwi.Workspace()
    out = {}
    for name, method, opts, recv in configs:
        err_b = {k: [1.0] for k in bands}

        def cb(k, x, ev, h):
            for kb, (a, b) in bands.items():
                err_b[kb].append(float(torch.linalg.vector_norm((x[a:b] - v_true[a:b]).double())) / e0b[kb])
        obj = I.FwiObjective(grid, geom, d_obs, opts, ws=ws, mute_top=I.default_mute(geom), receiver=recv,
                             receiver_every=10)
        lo, hi = I.velocity_bounds(grid, v0)
        hist = I.History(model_error=[1.0])
        e0 = float(torch.linalg.vector_norm((v0 - v_true).double()))

        def cb2(k, x, ev, h):
            h.model_error.append(float(torch.linalg.vector_norm((x - v_true).double())) / e0)
            cb(k, x, ev, h)
        kw = dict(max_update=max_update, project=lambda x: x.clamp(lo, hi), callback=cb2)
        opt = I.LBFGS(obj.value_grad, obj.value, **kw) if method == "lbfgs" else I.PRCG(obj.value_grad, obj.value,
                                                                                          **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v, hist = opt.run(v0.clone(), iters, hist)
        torch.cuda.synchronize()
        m = np.asarray(hist.misfit)
        out[name] = {"method": method, "misfit": (m / m[0]).tolist(), "model_error": hist.model_error,
                     "model_error_deep_band": err_b["deep_band"], "model_error_upper_half": err_b["upper_half"],
                     "model_error_lower_half": err_b["lower_half"], "gradients": obj.n_gradients,
                     "misfits": obj.n_misfits, "seconds": time.perf_counter() - t0}
    return out


def main():
    from . import fwi
    ap = argparse.ArgumentParser()
    ap.add_argument("--example", type=int, choices=(1, 2), default=1)
    ap.add_argument("--iters", type=int, default=0, help="0: the paper's count (200 / 270)")
    ap.add_argument("--shots", type=int, default=80)
    ap.add_argument("--max-update", type=float, default=50.0)
    ap.add_argument("--record", type=float, default=1.2, help="recording length in s (dt 1.5 ms)")
    ap.add_argument("--f0", type=float, default=6.0, help="Ricker peak frequency in Hz")
    ap.add_argument("--out", default="")
    ap.add_argument("--only", default="", help="comma-separated configuration names")
    args = ap.parse_args()
    p = problem(ns=args.shots, example=args.example, nt=int(round(args.record / 1.5e-3)), f0=args.f0)
    if args.example == 1:
        iters = args.iters or 200
        configs = [("ols", "lbfgs", fwi.Options(misfit="ols", precond="illum"), None),
                   ("time_integral", "lbfgs", fwi.Options(misfit="integral", precond="illum"), None)]
    else:
        iters = args.iters or 270
        configs = [("none", "prcg", fwi.Options(precond="none"), None),
                   ("illumination", "prcg", fwi.Options(precond="illum"), None),
                   ("offset_hessian", "prcg", fwi.Options(precond="offset", hmax=10), None),
                   ("illumination_plessix_mulder", "prcg", fwi.Options(precond="illum"), "pm"),
                   ("offset_hessian_receiver", "prcg", fwi.Options(precond="offset", hmax=10), "green")]
    if args.only:
        keep = set(args.only.split(","))
        configs = [c for c in configs if c[0] in keep]
    res = run(p, configs, iters, args.max_update)
    line = {"example": args.example, "workload": f"dipping {p.nz}x{p.nx}, dx {p.dx} m, {p.nshots} shots, "
            f"nt {p.nt}, dt {p.dt}, f0 {args.f0} Hz, max update {args.max_update} m/s", "iterations": iters,
            "results": res}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(line, f)
    summary = {k: {"misfit": round(v["misfit"][-1], 4), "model_error": round(v["model_error"][-1], 4),
                   "deep_band": round(v["model_error_deep_band"][-1], 4),
                   "upper_half": round(v["model_error_upper_half"][-1], 4),
                   "lower_half": round(v["model_error_lower_half"][-1], 4), "gradients": v["gradients"],
                   "misfits": v["misfits"], "seconds": round(v["seconds"], 1)} for k, v in res.items()}
    print(json.dumps({"example": args.example, "iterations": iters, "final": summary}), flush=True)


if __name__ == "__main__":
    main()
