"""Snapshot checkpoints (options.ckpt = 'snapshot') against the FP64 oracle.

In this mode the forward pass keeps the whole state (u^n, u^{n-1}) every K
levels instead of every level's sponge cells, and the adjoint pass re-runs
each K-level segment forward from its snapshot before back-propagating
through it. With F32 snapshots the re-run reproduces the forward wavefield,
so the gradient meets the same 1e-4 bound as the sponge mode. With 16-bit
snapshots (bfloat16, or float16 after scaling by the max-abs) the restored
state carries the rounding of the format, and the bound on the gradient is
1e-2 (relative L2), as for any lossy wavefield storage.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_SEIS = 1e-5
TOL_GRAD = 1e-4
TOL_GRAD_16 = 1e-2


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    torch.cuda.set_device(0)
    return torch


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(nt=300, ns=3):
    # padded 51 x 97: ragged against every tile shape
    return W.dipping(nz=37, nx=83, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=20, rec_step=4, f0=15.0,
                     seed=2, sponge=7)


@pytest.fixture(scope="module")
def ref_case(oracle_mod):
    p = problem()
    g = oracle_mod.Grid.of(p)
    w64 = p.wavelet.astype(np.float64)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, w64)["seis"].astype(np.float32)
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, w64, d_obs.astype(np.float64), hmax=2)
    return p, d_obs, ref


def gradient(torch, p, d_obs, **kw):
    from paper_1406_1864_gb300 import fwi
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    opts = fwi.Options(hmax=2, **kw)
    res = fwi.adjoint_gradient(grid, geom, v, torch.as_tensor(d_obs, device="cuda"), opts)
    torch.cuda.synchronize()
    return {k: t.cpu().numpy() for k, t in res.items()}


@pytest.mark.parametrize("interval", [0, 1, 7, 299, 1000])
def test_f32_snapshot_gradient(torch_cuda, ref_case, interval):
    """Exact snapshots: every output as in the sponge mode, for intervals that
    divide nt-1 or not, one level per segment, and one segment for all."""
    p, d_obs, ref = ref_case
    out = gradient(torch_cuda, p, d_obs, ckpt="snapshot", snap="f32", snap_interval=interval)
    assert rel(out["grad"], ref["grad"][:, 0, :]) <= TOL_GRAD
    assert rel(out["illum"], ref["illum"][:, 0, :]) <= TOL_GRAD
    assert rel(out["offh"], ref["offh"][:, :, 0, :]) <= TOL_GRAD
    assert abs(float(out["misfit"]) - ref["J"]) / ref["J"] <= 1e-5


def test_f32_snapshot_matches_sponge_mode(torch_cuda, ref_case):
    p, d_obs, _ = ref_case
    a = gradient(torch_cuda, p, d_obs, ckpt="snapshot", snap="f32")
    b = gradient(torch_cuda, p, d_obs, ckpt="sponge")
    assert rel(a["grad"], b["grad"]) <= 2e-5
    assert np.array_equal(a["illum"], b["illum"])
    # the misfit is summed with double atomics: equal up to their order
    assert abs(float(a["misfit"]) - float(b["misfit"])) <= 1e-12 * float(b["misfit"])


@pytest.mark.parametrize("prec", ["bf16", "f16s"])
def test_16bit_snapshot_gradient(torch_cuda, ref_case, prec):
    p, d_obs, ref = ref_case
    out = gradient(torch_cuda, p, d_obs, ckpt="snapshot", snap=prec)
    e = rel(out["grad"], ref["grad"][:, 0, :])
    assert e <= TOL_GRAD_16, (prec, e)
    # the forward outputs do not depend on the checkpoints
    assert rel(out["illum"], ref["illum"][:, 0, :]) <= TOL_GRAD
    # the scaled half-precision format keeps 3 more mantissa bits than bfloat16
    if prec == "f16s":
        bf = gradient(torch_cuda, p, d_obs, ckpt="snapshot", snap="bf16")
        assert e < rel(bf["grad"], ref["grad"][:, 0, :])


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_snapshot_forward_save_adjoint_apply(torch_cuda, oracle_mod, prec):
    """forward(save) + adjoint_apply with snapshot checkpoints, random adjoint
    source (the autograd path), including nt = 2 and 3."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    for nt in (2, 3, 160):
        p = problem(nt=nt, ns=2)
        p.wavelet[:] = np.random.default_rng(nt).standard_normal(p.wavelet.shape).astype(np.float32)
        grid, geom = fwi.from_problem(p)
        v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
        opts = fwi.Options(ckpt="snapshot", snap=prec)
        adj = np.random.default_rng(1).standard_normal((p.nshots, nt, p.nrec)).astype(np.float32)
        ws = fwi.Workspace()
        fwi.forward(grid, geom, v, save=True, ws=ws, opts=opts)
        gr = fwi.adjoint_apply(grid, geom, v, torch.as_tensor(adj, device="cuda"), ws,
                               opts=opts).cpu().numpy()
        gref = oracle_mod.gradient_for_adjoint_source(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                                                      p.wavelet.astype(np.float64),
                                                      adj.astype(np.float64))["grad"][:, 0, :]
        if np.linalg.norm(gref) == 0:
            assert np.abs(gr).max() == 0
        else:
            assert rel(gr, gref) <= (TOL_GRAD if prec == "f32" else TOL_GRAD_16), (prec, nt)
