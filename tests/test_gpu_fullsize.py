"""Full-size checks, in the launch configuration the benchmark times.

300 x 1000 cells, 96 shots, nt 4000 (the benchmark workload):
  - traces of three sampled shots against the FP64 oracle, which models those
    shots one by one (relative L2 <= 1e-5 per shot);
  - the gradient of all 96 shots against central finite differences of the
    misfit along smooth directions (the discrete adjoint is exact, so they
    agree at any size up to the O(eps^2) term and FP32 rounding);
  - the gradient and illumination of all shots against the sums over three
    launches of 32 shots each (sums over shots: Sec. 2 and Eq. 1);
  - with the offset Hessian (hmax 10), H(x, 0) = I(x) (Sec. 3 reduces to
    Eq. 1 at zero offset).
400 x 1200 cells, 64 shots, nt 5000 (autograd and snapshot checkpoints):
  - F32 snapshots give the sponge-mode gradient; bfloat16 and scaled float16
    snapshots stay within 1e-2 of it (the reduced-precision bound);
  - the autograd gradient against central finite differences along eight
    seeded smooth random directions (white noise smoothed over 5 cells,
    1% of the mean velocity).
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def c2(torch_cuda):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = W.workload("dipping_300x1000_96shots")
    grid, geom = fwi.from_problem(p)
    ws = fwi.Workspace()
    v_true = torch.as_tensor(p.v_true, device="cuda")
    d_obs = fwi.forward(grid, geom, v_true, ws=ws)
    v = torch.as_tensor(p.v_init, device="cuda")
    return p, grid, geom, v, d_obs, ws


def misfit_ols(torch, fwi, grid, geom, v, d_obs, ws):
    d = fwi.forward(grid, geom, v, ws=ws)
    return 0.5 * float(((d.double() - d_obs.double()) ** 2).sum())


def test_c2_traces_of_sampled_shots(c2, oracle_mod):
    p, grid, geom, v, d_obs, ws = c2
    shots = [0, 47, 95]
    g = oracle_mod.Grid.of(p)
    ref = oracle_mod.forward(g, p.v_true, p.src[shots], p.rec[shots], p.wavelet[shots].astype(np.float64),
                             nthreads=len(shots))["seis"]
    got = d_obs.cpu().numpy()[shots]
    for i, s in enumerate(shots):
        assert rel(got[i], ref[i]) <= 1e-5, (s, rel(got[i], ref[i]))


def test_c2_gradient_against_finite_differences(torch_cuda, c2):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, d_obs, ws = c2
    res = fwi.adjoint_gradient(grid, geom, v, d_obs, fwi.Options(misfit="ols"), ws=ws)
    g = res["grad"].cpu().numpy().astype(np.float64)
    J0 = float(res["misfit"])
    assert abs(J0 - misfit_ols(torch, fwi, grid, geom, v, d_obs, ws)) <= 1e-6 * J0
    v0 = p.v_init.astype(np.float64)
    eps = 2.0  # m/s times a unit-max direction
    for seed in (0, 1):
        dv = W.smooth_perturbation(v0.shape, seed, sigma_cells=20.0)
        jp = misfit_ols(torch, fwi, grid, geom, torch.as_tensor((v0 + eps * dv).astype(np.float32), device="cuda"),
                        d_obs, ws)
        jm = misfit_ols(torch, fwi, grid, geom, torch.as_tensor((v0 - eps * dv).astype(np.float32), device="cuda"),
                        d_obs, ws)
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(g * dv))
        assert abs(fd - an) <= 5e-3 * max(abs(an), 0.05 * np.linalg.norm(g) * np.linalg.norm(dv)), (seed, fd, an)


def test_c2_sum_over_shot_subsets(torch_cuda, c2):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, d_obs, ws = c2
    opts = fwi.Options(misfit="ols", precond="none")
    full = fwi.adjoint_gradient(grid, geom, v, d_obs, opts, ws=ws)
    acc = {k: torch.zeros_like(full[k]) for k in ("grad", "illum", "misfit")}
    for s0 in range(0, 96, 32):
        sub = fwi.adjoint_gradient(grid, geom.subset(s0, s0 + 32), v, d_obs[s0:s0 + 32].contiguous(), opts, ws=ws)
        for k in acc:
            acc[k] += sub[k]
    # each cell's sums are FP32 atomic additions of ~5e4 partial sums (4000
    # launches x 12 shot chunks), added in another order by the subsets:
    # rounding of order sqrt(5e4) * 6e-8 ~ 1e-5; the stated bound is 1e-4
    assert rel(acc["grad"].cpu(), full["grad"].cpu()) <= 1e-4
    assert rel(acc["illum"].cpu(), full["illum"].cpu()) <= 1e-4
    assert abs(float(acc["misfit"]) - float(full["misfit"])) <= 1e-9 * float(full["misfit"])


def test_c3_zero_offset_hessian_is_illumination(torch_cuda, c2):
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, d_obs, ws = c2
    res = fwi.adjoint_gradient(grid, geom, v, d_obs, fwi.Options(misfit="integral", hmax=10, precond="offset"),
                               ws=ws)
    offh, illum = res["offh"].cpu().numpy(), res["illum"].cpu().numpy()
    assert np.isfinite(res["grad_pre"].cpu().numpy()).all()
    assert rel(offh[0], illum) <= 1e-6
    # Cauchy-Schwarz along x: |H(x, h)| <= sqrt(I(x + h) I(x - h))
    for h in (1, 5, 10):
        lhs = np.abs(offh[h][:, h:-h])
        rhs = np.sqrt(illum[:, 2 * h:] * illum[:, :-2 * h])
        assert (lhs <= rhs * (1 + 1e-5) + 1e-30).all(), h


@pytest.fixture(scope="module")
def c4(torch_cuda):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = W.workload("dipping_400x1200_64shots")
    grid, geom = fwi.from_problem(p)
    ws = fwi.Workspace()
    d_obs = fwi.forward(grid, geom, torch.as_tensor(p.v_true, device="cuda"), ws=ws)
    return p, grid, geom, torch.as_tensor(p.v_init, device="cuda"), d_obs, ws


def test_c4_snapshot_precisions(torch_cuda, c4):
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, d_obs, ws = c4
    grads = {}
    for ck, sp in (("sponge", "f32"), ("snapshot", "f32"), ("snapshot", "bf16"), ("snapshot", "f16s")):
        r = fwi.adjoint_gradient(grid, geom, v, d_obs, fwi.Options(ckpt=ck, snap=sp), ws=ws)
        grads[(ck, sp)] = r["grad"].cpu().numpy()
    ref = grads[("sponge", "f32")]
    assert rel(grads[("snapshot", "f32")], ref) <= 1e-5
    e_bf, e_fs = rel(grads[("snapshot", "bf16")], ref), rel(grads[("snapshot", "f16s")], ref)
    assert e_bf <= 1e-2 and e_fs <= 1e-2, (e_bf, e_fs)
    assert e_fs < e_bf


def test_c4_autograd_finite_differences_8_directions(torch_cuda, c4):
    torch = torch_cuda
    from paper_1406_1864_gb300 import autograd, fwi
    p, grid, geom, v, d_obs, ws = c4
    opts = fwi.Options(ckpt="snapshot", snap="f32")
    vv = v.clone().requires_grad_(True)
    d = autograd.traces(vv, grid, geom, opts)
    (0.5 * ((d.double() - d_obs.double()) ** 2).sum()).backward()
    g = vv.grad.cpu().numpy().astype(np.float64)
    v0 = p.v_init.astype(np.float64)
    amp = 0.01 * float(v0.mean())
    eps = 0.1  # the step is 0.1% of the mean velocity at the direction's peak
    errs = []
    for seed in range(8):
        dv = W.smooth_perturbation(v0.shape, seed, sigma_cells=5.0, amplitude=amp)
        jp = misfit_ols(torch, fwi, grid, geom, torch.as_tensor((v0 + eps * dv).astype(np.float32), device="cuda"),
                        d_obs, ws)
        jm = misfit_ols(torch, fwi, grid, geom, torch.as_tensor((v0 - eps * dv).astype(np.float32), device="cuda"),
                        d_obs, ws)
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(g * dv))
        errs.append(abs(fd - an) / max(abs(an), 0.05 * np.linalg.norm(g) * np.linalg.norm(dv)))
    assert max(errs) <= 1e-2, errs

