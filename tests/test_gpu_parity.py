"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over the whole array): traces 1e-5; gradient,
illumination, offset-Hessian diagonal and preconditioned gradients 1e-4; the
misfit 1e-5. Inputs are identical on both sides: the float32 model, wavelet and
observed traces, the latter modelled by the oracle on the true model.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_SEIS = 1e-5
TOL_GRAD = 1e-4


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


def ragged_problem(nt=300, ns=3):
    """Ragged sizes (padded 51 x 97: not multiples of the 64-wide tiles or of
    4), sources and receivers on the model edges and corners."""
    p = W.dipping(nz=37, nx=83, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=20, rec_step=4, f0=15.0,
                  seed=2, sponge=7)
    src = p.src.copy()
    src[0] = [0, 0, 0]
    if ns > 1:
        src[1] = [36, 0, 82]
    rec = p.rec.copy()
    rec[:, 0] = [0, 0, 0]
    rec[:, 1] = [36, 0, 82]
    rec[:, 2] = [36, 0, 0]
    rec[:, 3] = [0, 0, 82]
    rec[:, 4] = rec[:, 5]          # two receivers on one cell
    p.src, p.rec = src, rec
    return p


def gpu_inputs(torch, p):
    from paper_1406_1864_gb300 import fwi
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    return fwi, grid, geom, v


def observed(oracle_mod, p):
    g = oracle_mod.Grid.of(p)
    d = oracle_mod.forward(g, p.v_true, p.src, p.rec, p.wavelet.astype(np.float64))["seis"]
    return d.astype(np.float32)


def check_gradient(torch, oracle_mod, p, misfit="ols", hmax=None, illum="u2", precond="illum"):
    g = oracle_mod.Grid.of(p)
    d_obs = observed(oracle_mod, p)
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, p.wavelet.astype(np.float64),
                                  d_obs.astype(np.float64), misfit=misfit, hmax=hmax,
                                  illum_utt=(illum == "utt2"))
    fwi, grid, geom, v = gpu_inputs(torch, p)
    opts = fwi.Options(misfit=misfit, illum=illum, hmax=-1 if hmax is None else hmax,
                       precond=precond)
    res = fwi.adjoint_gradient(grid, geom, v, torch.as_tensor(d_obs, device="cuda"), opts)
    torch.cuda.synchronize()
    out = {k: t.cpu().numpy() for k, t in res.items()}
    errs = {"grad": rel(out["grad"], ref["grad"][:, 0, :]),
            "illum": rel(out["illum"], ref["illum"][:, 0, :]),
            "misfit": abs(float(out["misfit"]) - ref["J"]) / ref["J"]}
    if precond == "illum":
        errs["grad_pre"] = rel(out["grad_pre"], ref["grad_pre_illum"][:, 0, :])
    if hmax is not None:
        errs["offh"] = rel(out["offh"], ref["offh"][:, :, 0, :])
        if precond == "offset":
            errs["grad_pre"] = rel(out["grad_pre"], ref["grad_pre_offset"][:, 0, :])
    for k, e in errs.items():
        tol = 1e-5 if k == "misfit" else TOL_GRAD
        assert e <= tol, (k, e, errs)
    return errs, out, ref


def test_forward_traces_two_layer(torch_cuda, oracle_mod):
    """The 100 x 200, 4-shot, nt = 1000 two-layer workload: traces."""
    torch = torch_cuda
    p = W.two_layer()
    fwi, grid, geom, v = gpu_inputs(torch, p)
    seis = fwi.forward(grid, geom, v).cpu().numpy()
    ref = oracle_mod.forward(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                             p.wavelet.astype(np.float64))["seis"]
    assert rel(seis, ref) <= TOL_SEIS


def test_gradient_two_layer(torch_cuda, oracle_mod):
    """The 100 x 200, 4-shot, nt = 1000 two-layer workload: raw gradient,
    illumination and illumination-preconditioned gradient, OLS misfit."""
    check_gradient(torch_cuda, oracle_mod, W.two_layer())


def test_ragged_edges_and_corners(torch_cuda, oracle_mod):
    p = ragged_problem()
    torch = torch_cuda
    fwi, grid, geom, v = gpu_inputs(torch, p)
    seis = fwi.forward(grid, geom, v).cpu().numpy()
    ref = oracle_mod.forward(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                             p.wavelet.astype(np.float64))["seis"]
    assert rel(seis, ref) <= TOL_SEIS
    check_gradient(torch, oracle_mod, p)


def test_time_integral_misfit(torch_cuda, oracle_mod):
    p = W.two_layer(nz=60, nx=90, nt=700, ns=3, nrec=90, sponge=12)
    check_gradient(torch_cuda, oracle_mod, p, misfit="integral")


@pytest.mark.parametrize("hmax", [0, 3, 10, 12])
def test_offset_hessian(torch_cuda, oracle_mod, hmax):
    p = ragged_problem(nt=250, ns=2)
    errs, out, ref = check_gradient(torch_cuda, oracle_mod, p, hmax=hmax, precond="offset")
    # the h = 0 slice is Eq. 1's illumination
    assert rel(out["offh"][0], out["illum"]) <= 1e-6


@pytest.mark.parametrize("hmax", [0, 3, 12])
def test_offset_hessian_split_variants(torch_cuda, oracle_mod, hmax):
    """The split offset-Hessian variants (the plain step, then k_offh_level
    per level), pinned with fwi_autotune_set on the ragged grid (sponge 7:
    the rows are copied 4 bytes at a time) and on a grid with an 8-cell
    sponge (16-byte copies), against the oracle: gradient, illumination,
    every offset slice, offset-preconditioned gradient (1e-4)."""
    from paper_1406_1864_gb300 import fwi
    N_FWD_FUSED = 3  # split variants follow the fused ones
    for p in (ragged_problem(nt=250, ns=3),
              W.dipping(nz=41, nx=131, dx=10.0, dt=1e-3, nt=240, ns=5, nrec=30, rec_step=4, f0=15.0, seed=4,
                        sponge=8)):
        grid, geom = fwi.from_problem(p)
        opts = fwi.Options(hmax=hmax, precond="offset")
        try:
            for fv in (N_FWD_FUSED, N_FWD_FUSED + 1):
                fwi.autotune_set(grid, geom, opts, {"forward_variant": fv, "forward_chunk": 3,
                                                     "backward_variant": 0, "backward_chunk": 8})
                check_gradient(torch_cuda, oracle_mod, p, hmax=hmax, precond="offset")
        finally:
            fwi.autotune_reset()


def test_offset_hessian_entry_point(torch_cuda, oracle_mod):
    torch = torch_cuda
    p = W.dipping(nz=50, nx=140, nt=400, ns=4, nrec=70, f0=12.0, seed=5, sponge=10)
    fwi, grid, geom, v = gpu_inputs(torch, p)
    H = fwi.offset_hessian_diag(grid, geom, v, fwi.Options(hmax=10)).cpu().numpy()
    ref = oracle_mod.forward(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                             p.wavelet.astype(np.float64), hmax=10)["offh"][:, :, 0, :]
    assert rel(H, ref) <= TOL_GRAD
    I = fwi.illumination(grid, geom, v, fwi.Options()).cpu().numpy()
    assert rel(I, H[0]) <= 1e-6
    Iu = fwi.illumination(grid, geom, v, fwi.Options(illum="utt2")).cpu().numpy()
    refu = oracle_mod.forward(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                              p.wavelet.astype(np.float64), illum=True, illum_utt=True)["illum"][:, 0, :]
    assert rel(Iu, refu) <= TOL_GRAD


def test_illumination_utt_in_gradient(torch_cuda, oracle_mod):
    p = W.two_layer(nz=50, nx=80, nt=500, ns=2, nrec=80, sponge=10)
    check_gradient(torch_cuda, oracle_mod, p, illum="utt2")


def test_adjoint_apply_random_source(torch_cuda, oracle_mod):
    """forward(save) + adjoint_apply equals the oracle's J^T applied to a
    random adjoint source (the autograd backward path)."""
    torch = torch_cuda
    p = ragged_problem(nt=220)
    fwi, grid, geom, v = gpu_inputs(torch, p)
    rng = np.random.default_rng(0)
    adj = rng.standard_normal((p.nshots, p.nt, p.nrec)).astype(np.float32)
    ws = fwi.Workspace()
    seis = fwi.forward(grid, geom, v, save=True, ws=ws)
    gr = fwi.adjoint_apply(grid, geom, v, torch.as_tensor(adj, device="cuda"), ws).cpu().numpy()
    ref = oracle_mod.gradient_for_adjoint_source(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                                                 p.wavelet.astype(np.float64),
                                                 adj.astype(np.float64))["grad"][:, 0, :]
    assert rel(gr, ref) <= TOL_GRAD
    ref_s = oracle_mod.forward(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                               p.wavelet.astype(np.float64))["seis"]
    assert rel(seis.cpu().numpy(), ref_s) <= TOL_SEIS


def test_single_shot_and_two_levels(torch_cuda, oracle_mod):
    torch = torch_cuda
    for nt in (2, 3, 40):
        p = W.two_layer(nz=20, nx=30, nt=nt, ns=1, nrec=30, sponge=5)
        p.wavelet[:] = np.random.default_rng(nt).standard_normal(p.wavelet.shape).astype(np.float32)
        fwi, grid, geom, v = gpu_inputs(torch, p)
        seis = fwi.forward(grid, geom, v).cpu().numpy()
        ref = oracle_mod.forward(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                                 p.wavelet.astype(np.float64))["seis"]
        if np.linalg.norm(ref) == 0:
            assert np.abs(seis).max() == 0
        else:
            assert rel(seis, ref) <= TOL_SEIS, nt
        adj = np.random.default_rng(1).standard_normal(seis.shape).astype(np.float32)
        ws = fwi.Workspace()
        fwi.forward(grid, geom, v, save=True, ws=ws)
        gr = fwi.adjoint_apply(grid, geom, v, torch.as_tensor(adj, device="cuda"), ws).cpu().numpy()
        gref = oracle_mod.gradient_for_adjoint_source(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                                                      p.wavelet.astype(np.float64),
                                                      adj.astype(np.float64))["grad"][:, 0, :]
        if np.linalg.norm(gref) == 0:
            assert np.abs(gr).max() == 0
        else:
            assert rel(gr, gref) <= TOL_GRAD, nt


def test_no_receivers(torch_cuda):
    """nrec = 0: nothing to fit, the gradient is exactly zero."""
    torch = torch_cuda
    p = W.two_layer(nz=20, nx=30, nt=50, ns=2, nrec=1, sponge=5)
    p.rec = p.rec[:, :0, :]
    fwi, grid, geom, v = gpu_inputs(torch, p)
    d = torch.zeros((2, 50, 0), device="cuda")
    res = fwi.adjoint_gradient(grid, geom, v, d, fwi.Options())
    assert float(res["misfit"]) == 0.0
    assert float(res["grad"].abs().max()) == 0.0
    assert float(res["illum"].min()) >= 0.0


def test_status_errors(torch_cuda):
    from paper_1406_1864_gb300 import _lib as L
    torch = torch_cuda
    p = W.two_layer(nz=20, nx=30, nt=50, ns=1, nrec=5, sponge=5)
    fwi, grid, geom, v = gpu_inputs(torch, p)
    fast = v * 4.0  # v dt / dx = 1.2: unstable
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward(grid, geom, fast)
    assert e.value.status == L.FWI_ERR_CFL
    neg = v.clone()
    neg[3, 4] = -1.0
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward(grid, geom, neg)
    assert e.value.status == L.FWI_ERR_INVALID_ARG
    # the library still works after an error
    seis = fwi.forward(grid, geom, v)
    assert torch.isfinite(seis).all()


def test_precondition_entry_point(torch_cuda):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    grid = fwi.Grid(30, 50, 10.0, 1e-3, 10)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((30, 50)).astype(np.float32)
    I = rng.random((30, 50)).astype(np.float32)
    H = rng.standard_normal((4, 30, 50)).astype(np.float32)
    out = fwi.precondition(grid, torch.as_tensor(g, device="cuda"), torch.as_tensor(I, device="cuda"),
                           "illum", 1e-3).cpu().numpy()
    ref = g / (I + 1e-3 * I.max())
    assert rel(out, ref) <= 1e-6
    out = fwi.precondition(grid, torch.as_tensor(g, device="cuda"), torch.as_tensor(H, device="cuda"),
                           "offset", 1e-2).cpu().numpy()
    Po = np.abs(H[0]) + 2 * np.abs(H[1:]).sum(0)
    assert rel(out, g / (Po + 1e-2 * Po.max())) <= 1e-6


def test_sharded_gradient_one_rank(torch_cuda):
    """distributed.sharded_gradient with one rank (library compute, then the
    precondition entry point) equals one fwi_adjoint_gradient call."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import distributed as D
    p = ragged_problem(nt=200)
    fwi, grid, geom, v = gpu_inputs(torch, p)
    d_obs = fwi.forward(grid, geom, torch.as_tensor(np.ascontiguousarray(p.v_true), device="cuda"))
    for precond, hmax in (("illum", -1), ("offset", 4)):
        opts = fwi.Options(hmax=hmax, precond=precond)
        ref = fwi.adjoint_gradient(grid, geom, v, d_obs, opts)
        got = D.sharded_gradient(grid, geom, v, d_obs, opts, rank=0, world=1)
        for k in ("grad", "illum", "grad_pre") + (("offh",) if hmax >= 0 else ()):
            assert rel(got[k].cpu().numpy(), ref[k].cpu().numpy()) <= 1e-6, (precond, k)
        assert abs(float(got["misfit"]) - float(ref["misfit"])) <= 1e-12 * float(ref["misfit"])


def test_hessian_v6_prefactor(torch_cuda, oracle_mod):
    """hess_v6: the illumination, offset Hessian and preconditioned
    gradients with H_a's diagonal prefactor 4 / v^6 (Sec. 3)."""
    torch = torch_cuda
    p = ragged_problem(ns=2)
    g = oracle_mod.Grid.of(p)
    d_obs = observed(oracle_mod, p)
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, p.wavelet.astype(np.float64), d_obs.astype(np.float64),
                                  hmax=4, hess_v6=True)
    fwi, grid, geom, v = gpu_inputs(torch, p)
    for precond, key in (("illum", "grad_pre_illum"), ("offset", "grad_pre_offset")):
        r = fwi.adjoint_gradient(grid, geom, v, torch.as_tensor(d_obs, device="cuda"),
                                 fwi.Options(hmax=4, precond=precond, hess_v6=True))
        assert rel(r["illum"].cpu(), ref["illum"][:, 0, :]) <= TOL_GRAD
        assert rel(r["offh"].cpu(), ref["offh"][:, :, 0, :]) <= TOL_GRAD
        assert rel(r["grad_pre"].cpu(), ref[key][:, 0, :]) <= TOL_GRAD, precond
    il = fwi.illumination(grid, geom, v, fwi.Options(hess_v6=True))
    assert rel(il.cpu(), ref["illum"][:, 0, :]) <= TOL_GRAD

