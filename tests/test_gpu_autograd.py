"""Forward modelling as a torch autograd operation (paper_1406_1864_gb300.autograd).

- OLS misfit written in torch: loss.backward() gives the gradient of
  fwi_adjoint_gradient(misfit = OLS) and the same misfit value.
- The time-integral misfit of Eq. 2 written with torch.cumsum: its autograd
  gradient equals the library's own Eq. 2 gradient.
- The autograd gradient against central finite differences of the forward
  modelling along smooth perturbations of v (the discrete adjoint is exact).
- The same with snapshot checkpoints, and against the FP64 oracle.
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
def case(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = W.dipping(nz=45, nx=90, dx=10.0, dt=1e-3, nt=400, ns=3, nrec=45, rec_step=2, f0=15.0,
                  seed=5, sponge=10)
    g = oracle_mod.Grid.of(p)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, p.wavelet.astype(np.float64))["seis"]
    grid, geom = fwi.from_problem(p)
    return p, grid, geom, torch.as_tensor(d_obs.astype(np.float32), device="cuda")


def test_ols_autograd_equals_adjoint_gradient(torch_cuda, case):
    torch = torch_cuda
    from paper_1406_1864_gb300 import autograd, fwi
    p, grid, geom, d_obs = case
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda").requires_grad_(True)
    d = autograd.traces(v, grid, geom)
    loss = 0.5 * ((d.double() - d_obs.double()) ** 2).sum()
    loss.backward()
    ref = fwi.adjoint_gradient(grid, geom, v.detach(), d_obs, fwi.Options(misfit="ols"))
    assert rel(v.grad.cpu().numpy(), ref["grad"].cpu().numpy()) <= 1e-5
    assert abs(loss.item() - float(ref["misfit"])) <= 1e-6 * loss.item()


def test_time_integral_autograd_equals_library(torch_cuda, case):
    """Eq. 2 in torch: y = dt * cumsum(u - d) along time, J = 1/2 |y|^2."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import autograd, fwi
    p, grid, geom, d_obs = case
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda").requires_grad_(True)
    d = autograd.traces(v, grid, geom)
    y = grid.dt * torch.cumsum(d.double() - d_obs.double(), dim=1)
    loss = 0.5 * (y * y).sum()
    loss.backward()
    ref = fwi.adjoint_gradient(grid, geom, v.detach(), d_obs, fwi.Options(misfit="integral"))
    assert rel(v.grad.cpu().numpy(), ref["grad"].cpu().numpy()) <= 1e-5
    assert abs(loss.item() - float(ref["misfit"])) <= 1e-5 * loss.item()


def smooth_directions(nz, nx, k=8, seed=0):
    rng = np.random.default_rng(seed)
    z = np.linspace(0, 1, nz)[:, None]
    x = np.linspace(0, 1, nx)[None, :]
    out = []
    for _ in range(k):
        a, b = rng.uniform(0.5, 3.0, 2)
        pz, px = rng.uniform(0, 2 * np.pi, 2)
        out.append((np.sin(np.pi * a * z + pz) * np.cos(np.pi * b * x + px)).astype(np.float64))
    return out


@pytest.mark.parametrize("ckpt", ["sponge", "snapshot"])
def test_autograd_against_finite_differences(torch_cuda, case, ckpt):
    torch = torch_cuda
    from paper_1406_1864_gb300 import autograd, fwi
    p, grid, geom, d_obs = case
    opts = fwi.Options(ckpt=ckpt)
    v0 = np.ascontiguousarray(p.v_init).astype(np.float64)
    v = torch.as_tensor(v0.astype(np.float32), device="cuda").requires_grad_(True)

    def misfit(vv):
        with torch.no_grad():
            d = fwi.forward(grid, geom, torch.as_tensor(vv.astype(np.float32), device="cuda"))
            return 0.5 * float(((d.double() - d_obs.double()) ** 2).sum())

    d = autograd.traces(v, grid, geom, opts)
    (0.5 * ((d.double() - d_obs.double()) ** 2).sum()).backward()
    g = v.grad.cpu().numpy().astype(np.float64)
    h = 5.0  # m/s on a ~2000-4000 m/s model
    errs = []
    for dv in smooth_directions(p.nz, p.nx):
        fd = (misfit(v0 + h * dv) - misfit(v0 - h * dv)) / (2 * h)
        an = float(np.sum(g * dv))
        # relative, with a floor for directions nearly orthogonal to g
        errs.append(abs(fd - an) / max(abs(an), 0.05 * np.linalg.norm(g) * np.linalg.norm(dv)))
    assert max(errs) <= 5e-3, errs


def test_snapshot_autograd_against_oracle(torch_cuda, oracle_mod, case):
    torch = torch_cuda
    from paper_1406_1864_gb300 import autograd, fwi
    p, grid, geom, d_obs = case
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda").requires_grad_(True)
    d = autograd.Propagator(grid, geom, fwi.Options(ckpt="snapshot", snap="f16s"))(v)
    (0.5 * ((d - d_obs) ** 2).sum()).backward()
    g = oracle_mod.Grid.of(p)
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, p.wavelet.astype(np.float64),
                                  d_obs.cpu().numpy().astype(np.float64))
    assert rel(v.grad.cpu().numpy(), ref["grad"][:, 0, :]) <= 1e-2


def test_backward_twice_is_refused(torch_cuda, case):
    torch = torch_cuda
    from paper_1406_1864_gb300 import autograd
    p, grid, geom, d_obs = case
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda").requires_grad_(True)
    d = autograd.traces(v, grid, geom)
    loss = (d * d).sum()
    loss.backward(retain_graph=True)
    with pytest.raises(RuntimeError, match="consumed"):
        loss.backward()
