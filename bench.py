#!/usr/bin/env python
"""Benchmark of the preconditioned FWI gradient on GB300.

One step = one call of fwi_adjoint_gradient over the whole batch of shots:
forward modelling of every shot (source injection, receiver extraction,
illumination and offset-Hessian accumulation, sponge checkpoints), misfit and
adjoint source, back-propagation with reverse reconstruction, zero-lag
imaging, fold and preconditioning -- every step of the hot path.

Default workload: 2-D model of 300 x 1000 cells (dx 10 m), six dipping layers
1500-4500 m/s plus a Gaussian body, 96 shots at z = 20 m, 500 receivers at
z = 10 m, 8 Hz Ricker, dt 0.8 ms, nt 4000, 20-cell sponge; time-integral
residual misfit and offset-Hessian diagonal |h| <= 10 (``--variant full``), or
OLS misfit with illumination preconditioning only (``--variant plain``).

Metric: Gpts/s = nz * nx * nt * shots / step time (model points, not padded),
summed over all GPUs. With N GPUs (one process each, torchrun) the batch is
N times the per-GPU batch: each rank models its own 96 shots and one NCCL
all-reduce sums the gradient, illumination, offset Hessian and misfit before
preconditioning (weak scaling; paper_1406_1864_gb300/distributed.py).

Prints one JSON line on rank 0. ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0

# bytes per padded point-step per shot that each time-loop kernel must move:
# forward: read u^n, u^{n-1}, c2, write u^{n+1}; backward: reconstruction
# (read u^{m-1}, u^m, write u^{m-2}), adjoint (read psi^{m+1}, psi^{m+2},
# write psi^m) and c2 shared by both.
ALG_BYTES = {"forward": 16, "adjoint": 28}

# the metric of both arms (this implementation and the reference arm)
METRIC = "FWI gradient Gpts/s (fwd+adj+imaging, preconditioned)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="dipping_300x1000_96shots")
    ap.add_argument("--variant", choices=["full", "plain"], default="full")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default tile variants (no fwi_autotune)")
    ap.add_argument("--tiles", default="", help="F,FC,B,BC: pin the forward / backward tile variants and shot "
                    "chunks (fwi_autotune_set) instead of autotuning")
    ap.add_argument("--profile-region", action="store_true",
                    help="cudaProfilerStart/Stop around the timed steps (ncu --profile-from-start off)")
    ap.add_argument("--no-graph", action="store_true",
                    help="call fwi_adjoint_gradient directly instead of replaying the recorded gradient")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU-baseline sample time")
    ap.add_argument("--shots", type=int, default=0, help="use only the first N shots (profiling)")
    ap.add_argument("--nt", type=int, default=0, help="use only the first N time levels (profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_workload(args):
    from paper_1406_1864_gb300 import workloads as W
    prob = W.workload(args.workload)
    if args.shots:
        prob = prob.subset(list(range(min(args.shots, prob.nshots))))
    if args.nt:
        prob = prob.with_nt(args.nt)
    return prob


def options_for(variant):
    from paper_1406_1864_gb300 import fwi
    if variant == "full":
        return fwi.Options(misfit="integral", illum="u2", hmax=10, precond="offset")
    return fwi.Options(misfit="ols", illum="u2", hmax=-1, precond="illum")


# --------------------------------------------------------------- CPU oracle
def oracle_sample(prob, variant, seconds, cores):
    """Time the FP64 oracle on a bounded sample of the workload: the first
    ``k`` shots and the first ``nt_s`` time levels (same grid and geometry).
    Returns (Gpts/s, sample description, seconds)."""
    import oracle
    oracle.build()
    k = max(1, min(prob.nshots, cores))
    # per-thread oracle rate ~2e7 padded point-steps/s for a gradient step;
    # choose nt_s for the target time, bounded by memory (history of u kept)
    npad = (prob.nz + 2 * prob.sponge) * (prob.nx + 2 * prob.sponge)
    nt_s = int(max(50, min(prob.nt, seconds * 1.5e7 / npad)))
    nt_s = min(nt_s, int(1.5e9 / (npad * 8)))  # <= 1.5 GB of history per shot
    sub = prob.subset(list(range(0, prob.nshots, max(1, prob.nshots // k)))[:k]).with_nt(nt_s)
    g = oracle.Grid.of(sub)
    w = sub.wavelet.astype(np.float64)
    d_obs = oracle.forward(g, sub.v_true, sub.src, sub.rec, w, nthreads=cores)["seis"]
    misfit = "integral" if variant == "full" else "ols"
    hmax = 10 if variant == "full" else None
    t0 = time.perf_counter()
    oracle.fwi_gradient(g, sub.v_init, sub.src, sub.rec, w, d_obs, misfit=misfit, hmax=hmax,
                        nthreads=cores)
    dt = time.perf_counter() - t0
    pts = sub.nz * sub.nx * sub.nt * sub.nshots
    desc = (f"{sub.nshots} shots x {nt_s} steps of the {prob.nz}x{prob.nx} grid "
            f"({'time-integral misfit, hmax 10' if variant == 'full' else 'OLS'}), FP64, "
            f"OpenMP over shots")
    return pts / dt / 1e9, desc, dt


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    prob = load_workload(args)
    cores = os.cpu_count() or 1
    per = max(2.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(prob, args.variant, per, cores)
    vals, times, desc = [], [], ""
    for _ in range(args.steps):
        v, desc, dt = oracle_sample(prob, args.variant, per, cores)
        vals.append(v)
        times.append(dt)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "variant": args.variant},
            "cpu_baseline": {"value": value, "unit": "Gpts/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the
    timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = self.proc.communicate()[0]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in (self.out or "").strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def read_peak():
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    """Hash of the sources the 2-D step kernels are compiled from (their file,
    the device helpers and the argument blocks)."""
    h = hashlib.sha256()
    for f in ("fwi_step2d.cu", "fwi_device.cuh", "fwi_args.h"):
        with open(os.path.join(ROOT, "paper_1406_1864_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when it is missing or the kernel source changed since the capture."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        e = t[kernel]
        if e.get("source_hash") != kernel_source_hash() or e.get("workload") != workload:
            return None
        return float(e["bytes_per_launch"])
    except (OSError, KeyError, ValueError, TypeError):
        return None


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1406_1864_gb300 import fwi, workloads as W
    prob = load_workload(args)
    grid, geom = fwi.from_problem(prob)
    opts = options_for(args.variant)
    dev = torch.device("cuda", local)
    v_true = torch.as_tensor(prob.v_true, device=dev)
    v = torch.as_tensor(prob.v_init, device=dev)
    ws = fwi.Workspace(dev)
    d_obs = fwi.forward(grid, geom, v_true, ws=ws)           # observed data (not timed)
    del v_true
    out = None
    graph = None
    phase_box = []
    tiles = None
    if args.tiles:
        fv, fc, bv, bc = (int(x) for x in args.tiles.split(","))
        tiles = {"forward_variant": fv, "forward_chunk": fc, "backward_variant": bv, "backward_chunk": bc}
        fwi.autotune_set(grid, geom, opts, tiles)
    elif not args.no_autotune:  # tile variants timed on this problem (not timed)
        tiles = fwi.autotune(grid, geom, v, opts, ws=ws)

    if world > 1:
        # the global batch: every rank's shard is this per-GPU batch
        from paper_1406_1864_gb300 import distributed as D
        gsrc = np.concatenate([prob.src] * world)
        grec = np.concatenate([prob.rec] * world)

        def compute(grid_, sub, v_, d_, o_):
            r = fwi.adjoint_gradient(grid_, sub, v_, d_, o_, want_pre=False, ws=ws)
            phase_box.append(fwi.last_phase_times())
            return r

        def gradient(v_, d_, wav_):
            gg = fwi.Geometry(gsrc, grec, torch.cat([wav_] * world))
            return D.sharded_gradient(grid, gg, v_, d_, opts, rank=rank, world=world, compute=compute)
    elif not args.no_graph:
        # the gradient recorded once as a CUDA graph on these buffers (inputs
        # are updated in place: v, d_obs, the wavelet), replayed every step
        fwi.profile(True)  # phase events recorded into the graph
        graph = fwi.GradientGraph([grid], [geom], [v], [d_obs], opts, ws=ws)

        def gradient(v_, d_, wav_, d_obs_ready=None):
            assert v_ is v and d_ is d_obs and wav_ is geom.wavelet
            r = graph.run(d_obs_ready=d_obs_ready)[0]
            phase_box.append(fwi.last_phase_times())
            return r
    else:
        def gradient(v_, d_, wav_):
            nonlocal out
            out = fwi.adjoint_gradient(grid, fwi.Geometry(prob.src, prob.rec, wav_), v_, d_, opts, ws=ws,
                                       out=out)
            phase_box.append(fwi.last_phase_times())
            return out

    def step():
        nonlocal out
        out = gradient(v, d_obs, geom.wavelet)

    for _ in range(args.warmup):
        step()
    fwi.profile(True)
    phases = []
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if args.profile_region:
            torch.cuda.profiler.start()
        e0.record()
        for _ in range(args.steps):
            step()
            phases.append(phase_box[-1])
        e1.record()
        barrier()
        if args.profile_region:
            torch.cuda.profiler.stop()
    fwi.profile(False)
    ms = e0.elapsed_time(e1) / args.steps
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    units = prob.phys_points * prob.nt * prob.nshots
    value = world * units / (ms * 1e-3) / 1e9

    # end to end: host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_v = torch.as_tensor(prob.v_init).pin_memory()
        h_obs = d_obs.cpu().pin_memory()
        h_wav = geom.wavelet.cpu().pin_memory()
        hosts = {k: torch.empty(t.shape, dtype=t.dtype).pin_memory() for k, t in out.items()}
        # the step's own input buffers receive each step's host inputs
        d_v, d_o, d_w = v, d_obs, geom.wavelet
        h2d = h_v.numel() * 4 + h_obs.numel() * 4 + h_wav.numel() * 4
        d2h = sum(t.numel() * t.element_size() for t in hosts.values())
        # with the recorded graph, the observed traces are copied on a side
        # stream while the forward pass runs (the misfit waits for them)
        upload = torch.cuda.Stream() if graph is not None else None
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(args.steps):
            d_v.copy_(h_v, non_blocking=True)
            d_w.copy_(h_wav, non_blocking=True)
            if upload is not None:
                upload.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(upload):
                    d_o.copy_(h_obs, non_blocking=True)
                r = gradient(d_v, d_o, d_w, d_obs_ready=upload)
            else:
                d_o.copy_(h_obs, non_blocking=True)
                r = gradient(d_v, d_o, d_w)
            for k, t in r.items():
                hosts[k].copy_(t, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        f1.record()
        barrier()
        ems = f0.elapsed_time(f1) / args.steps
        if dist is not None:
            t = torch.tensor([ems], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        e2e = {"value": world * units / (ems * 1e-3) / 1e9, "unit": "Gpts/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": ems}

    # roofline of the dominant time-loop kernel, from the phase events
    fwd_ms = statistics.median(p["forward_ms"] for p in phases)
    adj_ms = statistics.median(p["adjoint_ms"] for p in phases)
    nf = phases[0]["forward_launches"]
    na = phases[0]["adjoint_launches"]
    dom, tms, nl = ("adjoint", adj_ms, na) if adj_ms >= fwd_ms else ("forward", fwd_ms, nf)
    npad = (prob.nz + 2 * prob.sponge) * (prob.nx + 2 * prob.sponge)
    bytes_per_launch = ALG_BYTES[dom] * npad * prob.nshots
    per_launch_s = tms / nl * 1e-3
    achieved = bytes_per_launch / per_launch_s / 1e9
    peak, peak_kind = read_peak()
    kname = "k_bwd_step" if dom == "adjoint" else ("k_fwd_step<offset Hessian>" if opts.hmax >= 0
                                                   else "k_fwd_step")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": read_traffic(kname, args.workload),
            "kernel": kname, "peak_source": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s",
            "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": per_launch_s * 1e3,
            "phase_ms": {"forward": fwd_ms, "adjoint": adj_ms,
                         "other": statistics.median(p["other_ms"] for p in phases)},
            "launches_per_step": {"forward": nf, "adjoint": na,
                                  "other": phases[0]["other_launches"]}}
    # the whole step against the method's minimum traffic: 44 B per padded
    # point-step per shot (forward 16 + backward 28), at the same peak
    t_min_ms = 44.0 * npad * prob.nt * prob.nshots / (peak * 1e9) * 1e3
    step_roof = {"bytes_per_padded_point_step": 44, "t_min_ms": t_min_ms, "ms_per_step": ms,
                 "frac": t_min_ms / ms}
    launches = sum(p["forward_launches"] + p["adjoint_launches"] + p["other_launches"] for p in phases)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        val, desc, _ = oracle_sample(prob, args.variant, args.cpu_seconds, cores)
        cpu = {"value": val, "unit": "Gpts/s", "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload + (f" (first {prob.nshots} shots, nt {prob.nt})"
                                                    if (args.shots or args.nt) else ""),
                       "variant": args.variant,
                       "grid": [prob.nz, prob.nx], "dx_m": prob.dx, "dt_s": prob.dt, "nt": prob.nt,
                       "shots": prob.nshots, "receivers": prob.nrec, "sponge": prob.sponge,
                       "misfit": opts.misfit, "offset_hessian_hmax": opts.hmax,
                       "precond": opts.precond, "tiles": tiles or "default",
                       "graph": world == 1 and not args.no_graph,
                       "parallelism": "1 GPU" if world == 1 else
                       f"shots x{world} (each GPU {prob.nshots} shots; NCCL all-reduce of the sums)",
                       "l2": "inputs larger than L2 (wavefields of all shots ~0.6 GB per step)"},
            "roofline": roof, "step_roofline": step_roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
