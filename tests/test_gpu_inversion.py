"""The outer inversion loops driven by the library (GPU) and, for parity, the
same loops driven by the FP64 oracle.

* The first two iterates of PRCG (illumination preconditioner, OLS misfit),
  of L-BFGS (offset-Hessian preconditioner, time-integral misfit of Eq. 2,
  hmax 3) and of truncated Gauss-Newton (three CG products per step) from the library's gradients, misfits and preconditioner
  against the same loops over the oracle's (relative L2 of the model update
  <= 1e-3: the line searches take the same branches, the steps then agree to
  the gradients' FP32 rounding).
* Ten iterations of each (also with the receiver factors of a fixed spread:
  Plessix-Mulder's, the receiver Green's functions) on a dipping-layer
  model: the misfit decreases at
  every iteration and by a quarter at least over the ten, the velocities stay
  within the projection bounds, the muted rows stay fixed, and fwi_misfit
  agrees with the gradient call's misfit. (The model error is reported, not
  asserted: early FWI iterations from a smooth model may add reflectivity
  that raises the L2 model error while the data fit improves.)
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


def problem():
    return W.dipping(nz=40, nx=96, dx=10.0, dt=1e-3, nt=500, ns=4, nrec=48, rec_step=2, f0=12.0, seed=4,
                     sponge=10)


class OracleObjective:
    """The misfit, gradient and diagonal preconditioner of the FP64 oracle,
    on torch float64 CPU tensors."""

    def __init__(self, oracle_mod, p, d_obs, misfit, precond, hmax, eps=1e-3):
        self.o, self.p, self.d_obs = oracle_mod, p, d_obs
        self.g = oracle_mod.Grid.of(p)
        self.w = p.wavelet.astype(np.float64)
        self.misfit, self.precond, self.hmax, self.eps = misfit, precond, hmax, eps

    def value(self, v):
        seis = self.o.forward(self.g, v.numpy(), self.p.src, self.p.rec, self.w)["seis"]
        if self.misfit == "ols":
            return self.o.misfit_ols(seis, self.d_obs)[0]
        return self.o.misfit_time_integral(seis, self.d_obs, self.p.dt)[0]

    def value_grad(self, v):
        import torch
        from paper_1406_1864_gb300 import inversion as I
        r = self.o.fwi_gradient(self.g, v.numpy(), self.p.src, self.p.rec, self.w, self.d_obs, misfit=self.misfit,
                                hmax=self.hmax if self.precond == "offset" else None, eps=self.eps)
        P = r["illum"][:, 0, :] if self.precond == "illum" else self.o.offset_scale(r["offh"])[:, 0, :]
        g = torch.as_tensor(r["grad"][:, 0, :])
        return I.Evaluation(r["J"], g, lambda q: torch.as_tensor(self.o.precondition(q.numpy(), P, self.eps)))

    def hvp(self, v, q):
        """J^T W^T W J q from the oracle's Born modelling and adjoint imaging."""
        import torch
        jq = self.o.born(self.g, v.numpy(), q.numpy(), self.p.src, self.p.rec, self.w)
        if self.misfit == "integral":
            jq = self.o.time_integral_adjoint(self.o.time_integral(jq, self.p.dt), self.p.dt)
        hq = self.o.gradient_for_adjoint_source(self.g, v.numpy(), self.p.src, self.p.rec, self.w, jq)["grad"]
        return torch.as_tensor(hq[:, 0, :])


@pytest.mark.parametrize("method,misfit,precond,hmax", [("prcg", "ols", "illum", -1),
                                                        ("lbfgs", "integral", "offset", 3),
                                                        ("gauss_newton", "ols", "illum", -1)])
def test_first_iterates_against_oracle_loop(torch_cuda, oracle_mod, method, misfit, precond, hmax):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi, inversion as I
    p = problem()
    g = oracle_mod.Grid.of(p)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, p.wavelet.astype(np.float64))["seis"].astype(np.float32)
    grid, geom = fwi.from_problem(p)
    opts = fwi.Options(misfit=misfit, precond=precond, hmax=hmax)
    lo, hi = I.velocity_bounds(grid, torch.as_tensor(p.v_init))
    seen_g, seen_o = [], []

    def make(o, cb):
        kw = dict(max_update=40.0, project=lambda x: x.clamp(lo, hi), callback=cb)
        if method == "gauss_newton":
            return I.GaussNewton(o.value_grad, o.value, o.hvp, cg_iters=3, **kw)
        return (I.LBFGS if method == "lbfgs" else I.PRCG)(o.value_grad, o.value, **kw)
    obj = I.FwiObjective(grid, geom, torch.as_tensor(d_obs, device="cuda"), opts)
    make(obj, lambda k, x, ev, h: seen_g.append(x.cpu().double())).run(torch.as_tensor(p.v_init, device="cuda"), 2)
    ob = OracleObjective(oracle_mod, p, d_obs.astype(np.float64), misfit, precond, hmax)
    make(ob, lambda k, x, ev, h: seen_o.append(x.clone())).run(torch.as_tensor(p.v_init.astype(np.float64)), 2)
    v0 = torch.as_tensor(p.v_init.astype(np.float64))
    assert len(seen_g) == len(seen_o) == 2
    for k, (a, b) in enumerate(zip(seen_g, seen_o)):
        err = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b - v0))
        assert err <= 1e-3, (k, err)


@pytest.mark.parametrize("method,misfit,precond,hmax,recv", [("lbfgs", "ols", "illum", -1, None),
                                                             ("prcg", "integral", "offset", 4, None),
                                                             ("prcg", "ols", "illum", -1, "pm"),
                                                             ("lbfgs", "ols", "offset", 2, "green"),
                                                             ("gauss_newton", "integral", "illum", -1, None)])
def test_ten_iterations_decrease_misfit(torch_cuda, method, misfit, precond, hmax, recv):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi, inversion as I
    p = problem()
    grid, geom = fwi.from_problem(p)
    v_true = torch.as_tensor(p.v_true, device="cuda")
    d_obs = fwi.forward(grid, geom, v_true)
    opts = fwi.Options(misfit=misfit, precond=precond, hmax=hmax)
    v0 = torch.as_tensor(p.v_init, device="cuda")
    v, h = I.invert(grid, geom, d_obs, v0, opts, method=method, iters=10, max_update=40.0, v_true=v_true,
                    receiver=recv, receiver_every=3)
    m = np.array(h.misfit)
    assert len(m) == 11 and (np.diff(m) < 0).all(), m
    assert m[-1] < 0.75 * m[0], m
    lo, hi = I.velocity_bounds(grid, v0)
    assert float(v.min()) >= lo and float(v.max()) <= hi
    mute = I.default_mute(geom)
    assert torch.equal(v[:mute], v0[:mute])  # the muted rows stay fixed
    r = fwi.adjoint_gradient(grid, geom, v, d_obs, opts)
    J = float(fwi.misfit(grid, geom, v, d_obs, opts))
    assert abs(J - float(r["misfit"])) <= 1e-12 * J


def test_moving_spread_plessix_mulder_preconditioner(torch_cuda):
    """PRCG preconditioned by Plessix and Mulder's per-shot Hessian for an
    end-on spread that moves with the shots (fwi_plessix_mulder_hessian as
    the scale): the misfit decreases at every iteration; a fixed-spread-only
    receiver factor is not used."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi, inversion as I
    p = problem()
    rec = np.zeros((p.nshots, 16, 3), np.int32)
    src = p.src.copy()
    for s in range(p.nshots):
        x0 = 20 + 18 * s
        src[s] = [2, 0, x0]
        rec[s, :, 0] = 1
        rec[s, :, 2] = np.arange(x0 - 17, x0 - 1)
    p.src, p.rec = src, rec
    grid, geom = fwi.from_problem(p)
    v_true = torch.as_tensor(p.v_true, device="cuda")
    d_obs = fwi.forward(grid, geom, v_true)
    opts = fwi.Options(misfit="ols", precond="illum")
    obj = I.FwiObjective(grid, geom, d_obs, opts, receiver="pm", mute_top=I.default_mute(geom))
    assert not obj.fixed_spread and obj.recv is None
    v, h = I.invert(grid, geom, d_obs, torch.as_tensor(p.v_init, device="cuda"), opts, method="prcg", iters=5,
                    max_update=40.0, receiver="pm", receiver_every=2)
    m = np.array(h.misfit)
    assert len(m) == 6 and (np.diff(m) < 0).all(), m
