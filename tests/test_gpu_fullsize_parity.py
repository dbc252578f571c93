"""Oracle parity in the benchmark's own launch configuration.

The benchmark times the full preconditioned gradient of the 300 x 1000-cell
dipping model with all 96 shots: the time-integral misfit of Eq. 2, the
offset-Hessian diagonal for |h| <= 10 (Sec. 3), the shot illumination of
Eq. 1 and offset preconditioning (Sec. 3.1). Its launches cover the whole
padded grid with every shot: the plain forward step in two-shot items and
the offset-Hessian sums of all 96 shots per tile after it (the split
variant), shot chunks of 8 per tile, more tile chunks than resident CTAs (so
CTAs take a second chunk), items that span chunk boundaries. Here the same grid, shots,
receivers and options run with nt cut to 300, so that the FP64 oracle can
compute every output point by point (about 0.85 GB of wavefield history per
shot and thread), and the outputs are compared element by element:

  - with the benchmark's tile choice pinned (forward variant 4, the split
    one, chunk 8; backward variant 0, chunk 8), called directly, sponge
    checkpoints; and with the fused offset-Hessian step (forward variant 2,
    chunk 16);
  - with the autotuner's own choice, through the recorded CUDA graph the
    benchmark replays, sponge checkpoints;
  - with F32 snapshot checkpoints (the forward field re-propagated bit for
    bit), the benchmark's tiles.

Tolerances (relative L2, FP32 against FP64): gradient, illumination and
every offset-Hessian slice 1e-4; misfit 1e-5. The preconditioned gradient
g / (P + eps max P) magnifies poorly illuminated cells by up to 1/eps = 1000.
With sponge checkpoints the backward pass rebuilds u by reverse time
stepping, whose FP32 rounding leaves a noise floor (about 1e-7 of the
largest field values) in cells the forward field barely reached; there the
oracle's gradient is ~1e-17 and the GPU's its noise. So in sponge mode the
preconditioned gradient is checked against the FP64 division of the GPU's
own gradient and offset scale (1e-5: the division and the water level in
this launch configuration), and against the oracle with snapshot
checkpoints, where the forward field is exact (1e-4).
"""
import os

import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NT = 300
HMAX = 10
TOL_GRAD = 1e-4
TOL_MISFIT = 1e-5
TOL_DIV = 1e-5  # FP32 division against FP64 of the same inputs
BENCH_TILES = {"forward_variant": 4, "forward_chunk": 8, "backward_variant": 0, "backward_chunk": 8}
FUSED_TILES = {"forward_variant": 2, "forward_chunk": 16, "backward_variant": 0, "backward_chunk": 8}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case(oracle_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    torch.cuda.set_device(0)
    p = W.workload("dipping_300x1000_96shots").with_nt(NT)
    assert p.nshots == 96 and (p.nz, p.nx) == (300, 1000)
    g = oracle_mod.Grid.of(p)
    w = p.wavelet.astype(np.float64)
    threads = min(16, os.cpu_count() or 1)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, w, nthreads=threads)["seis"].astype(np.float32)
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, w, d_obs.astype(np.float64), misfit="integral",
                                  hmax=HMAX, nthreads=threads)
    return p, d_obs, ref


def opts():
    from paper_1406_1864_gb300 import fwi
    return fwi.Options(misfit="integral", illum="u2", hmax=HMAX, precond="offset")


def compare(res, ref, pre_vs_oracle):
    got = {k: (v.cpu().numpy().astype(np.float64) if hasattr(v, "cpu") else v) for k, v in res.items()}
    errs = {
        "grad": rel(got["grad"], ref["grad"][:, 0, :]),
        "illum": rel(got["illum"], ref["illum"][:, 0, :]),
        "offh": rel(got["offh"], ref["offh"][:, :, 0, :]),
        "misfit": abs(float(got["misfit"]) - ref["J"]) / abs(ref["J"]),
    }
    # every offset on its own, not only the sum over offsets
    for h in range(HMAX + 1):
        errs[f"offh[{h}]"] = rel(got["offh"][h], ref["offh"][h, :, 0, :])
    # the offset preconditioning of the GPU's own gradient and scale, in FP64
    P = np.abs(got["offh"][0]) + 2.0 * np.sum(np.abs(got["offh"][1:]), axis=0)
    errs["grad_pre/own"] = rel(got["grad_pre"], got["grad"] / (P + 1e-3 * P.max()))
    if pre_vs_oracle:
        errs["grad_pre"] = rel(got["grad_pre"], ref["grad_pre_offset"][:, 0, :])
    for k, e in errs.items():
        tol = TOL_MISFIT if k == "misfit" else (TOL_DIV if k == "grad_pre/own" else TOL_GRAD)
        assert e <= tol, (k, e, errs)
    return errs


@pytest.mark.parametrize("tiles", [BENCH_TILES, FUSED_TILES], ids=["split", "fused"])
def test_bench_tiles_direct_call(case, tiles):
    import torch
    from paper_1406_1864_gb300 import fwi
    p, d_obs, ref = case
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(p.v_init, device="cuda")
    d = torch.as_tensor(d_obs, device="cuda")
    try:
        fwi.autotune_set(grid, geom, opts(), tiles)
        res = fwi.adjoint_gradient(grid, geom, v, d, opts())
        torch.cuda.synchronize()
    finally:
        fwi.autotune_reset()
    compare(res, ref, pre_vs_oracle=False)


def test_autotuned_recorded_graph(case):
    import torch
    from paper_1406_1864_gb300 import fwi
    p, d_obs, ref = case
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(p.v_init, device="cuda")
    d = torch.as_tensor(d_obs, device="cuda")
    ws = fwi.Workspace()
    try:
        fwi.autotune(grid, geom, v, opts(), ws=ws)
        graph = fwi.GradientGraph([grid], [geom], [v], [d], opts(), ws=ws)
        for _ in range(2):  # a replay sees the same inputs and rewrites every output
            res = graph.run()[0]
            torch.cuda.synchronize()
            compare(res, ref, pre_vs_oracle=False)
    finally:
        fwi.autotune_reset()


def test_bench_tiles_snapshot_checkpoints(case):
    import torch
    from paper_1406_1864_gb300 import fwi
    p, d_obs, ref = case
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(p.v_init, device="cuda")
    d = torch.as_tensor(d_obs, device="cuda")
    o = opts()
    o.ckpt, o.snap = "snapshot", "f32"
    try:
        fwi.autotune_set(grid, geom, o, BENCH_TILES)
        res = fwi.adjoint_gradient(grid, geom, v, d, o)
        torch.cuda.synchronize()
    finally:
        fwi.autotune_reset()
    compare(res, ref, pre_vs_oracle=True)
