"""Pins of the oracle's adjoint and gradient.

* Source-to-trace operator F (linear in the wavelet): <F f, d> = <f, F^T d>.
* Born operator of Eq. 4 against central differences of the forward map, and
  the Jacobian dot test <J dv, dd> = <dv, J^T dd>, where J^T is the adjoint
  imaging (zero-lag cross-correlation of Sec. 2).
* Gradient of the OLS misfit (Sec. 2) and of the time-integral misfit (Eq. 2)
  against central finite differences of the misfit itself, along smooth random
  directions and along directions confined to the model edge (these reach the
  sponge through the edge replication, so they pin the fold of the padded-grid
  gradient into the edge cells).
* A planted mistake (wrong sign of the adjoint source) must fail the FD check.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W


def small_problem(ns=2, nt=260, nz=30, nx=44, sponge=8, seed=3):
    p = W.dipping(nz=nz, nx=nx, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=22, rec_step=2, f0=15.0,
                  seed=seed, sponge=sponge)
    return p


def grid_of(oracle_mod, p):
    return oracle_mod.Grid.of(p)


def test_source_to_trace_dot(oracle_mod):
    p = small_problem()
    g = grid_of(oracle_mod, p)
    rng = np.random.default_rng(11)
    f = rng.standard_normal((p.nshots, p.nt))
    d = rng.standard_normal((p.nshots, p.nt, p.nrec))
    Ff = oracle_mod.forward(g, p.v_true, p.src, p.rec, f)["seis"]
    Ftd = oracle_mod.gradient_for_adjoint_source(g, p.v_true, p.src, p.rec, f, d,
                                                 want_psi_src=True)["psi_src"]
    lhs, rhs = np.sum(Ff * d), np.sum(f * Ftd)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_born_matches_finite_difference(oracle_mod):
    p = small_problem(ns=1)
    g = grid_of(oracle_mod, p)
    w = p.wavelet.astype(np.float64)
    v = p.v_init.astype(np.float64)
    dv = W.smooth_perturbation(v.shape, seed=5, sigma_cells=3.0, amplitude=1.0)
    eps = 1e-2
    fp = oracle_mod.forward(g, v + eps * dv, p.src, p.rec, w)["seis"]
    fm = oracle_mod.forward(g, v - eps * dv, p.src, p.rec, w)["seis"]
    fd = (fp - fm) / (2 * eps)
    b = oracle_mod.born(g, v, dv, p.src, p.rec, w)
    assert np.linalg.norm(b - fd) <= 1e-6 * np.linalg.norm(b)


def test_jacobian_dot(oracle_mod):
    p = small_problem()
    g = grid_of(oracle_mod, p)
    w = p.wavelet.astype(np.float64)
    v = p.v_init.astype(np.float64)
    rng = np.random.default_rng(7)
    dv = rng.standard_normal(v.shape)
    dd = rng.standard_normal((p.nshots, p.nt, p.nrec))
    Jdv = oracle_mod.born(g, v, dv, p.src, p.rec, w)
    JTdd = oracle_mod.gradient_for_adjoint_source(g, v, p.src, p.rec, w, dd)["grad"].reshape(v.shape)
    lhs, rhs = np.sum(Jdv * dd), np.sum(dv * JTdd)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _directions(shape):
    nz, nx = shape
    dirs = [W.smooth_perturbation(shape, seed=s, sigma_cells=3.0) for s in range(3)]
    edge = np.zeros(shape)
    edge[:, 0] = 1.0          # left edge column: replicated into the left sponge
    edge[-1, :] += 0.5        # bottom row and the bottom-right corner block
    dirs.append(edge)
    return dirs


@pytest.mark.parametrize("misfit", ["ols", "integral"])
def test_gradient_finite_difference(oracle_mod, misfit):
    p = small_problem()
    g = grid_of(oracle_mod, p)
    w = p.wavelet.astype(np.float64)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, w)["seis"]
    v = p.v_init.astype(np.float64)

    def J(vv):
        s = oracle_mod.forward(g, vv, p.src, p.rec, w)["seis"]
        if misfit == "ols":
            return oracle_mod.misfit_ols(s, d_obs)[0]
        return oracle_mod.misfit_time_integral(s, d_obs, p.dt)[0]

    res = oracle_mod.fwi_gradient(g, v, p.src, p.rec, w, d_obs, misfit=misfit)
    grad = res["grad"].reshape(v.shape)
    assert abs(res["J"] - J(v)) <= 1e-12 * res["J"]
    for dvec in _directions(v.shape):
        eps = 0.5
        fd = (J(v + eps * dvec) - J(v - eps * dvec)) / (2 * eps)
        an = float(np.sum(grad * dvec))
        assert abs(fd - an) <= 1e-6 * abs(an), (misfit, fd, an)


def test_planted_sign_error_fails_fd(oracle_mod):
    """A wrong sign on the adjoint source (a plausible slip) breaks the FD
    check: the check has the power to see it."""
    p = small_problem(ns=1)
    g = grid_of(oracle_mod, p)
    w = p.wavelet.astype(np.float64)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, w)["seis"]
    v = p.v_init.astype(np.float64)
    s = oracle_mod.forward(g, v, p.src, p.rec, w)["seis"]
    _, r = oracle_mod.misfit_ols(s, d_obs)
    bad = oracle_mod.gradient_for_adjoint_source(g, v, p.src, p.rec, w, -r)["grad"].reshape(v.shape)
    dvec = W.smooth_perturbation(v.shape, seed=0, sigma_cells=3.0)
    eps = 0.5
    Jp = oracle_mod.misfit_ols(oracle_mod.forward(g, v + eps * dvec, p.src, p.rec, w)["seis"], d_obs)[0]
    Jm = oracle_mod.misfit_ols(oracle_mod.forward(g, v - eps * dvec, p.src, p.rec, w)["seis"], d_obs)[0]
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - np.sum(bad * dvec)) > 0.5 * abs(fd)


def test_time_integral_operator_adjoint(oracle_mod):
    """C and C^T of Eq. 2's weighting are transposes: <C r, y> = <r, C^T y>."""
    rng = np.random.default_rng(2)
    r = rng.standard_normal((3, 50, 4))
    y = rng.standard_normal((3, 50, 4))
    dt = 1e-3
    lhs = np.sum(oracle_mod.time_integral(r, dt) * y)
    rhs = np.sum(r * oracle_mod.time_integral_adjoint(y, dt))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # and C r of a constant is the ramp dt*(n+1)
    ramp = oracle_mod.time_integral(np.ones((1, 5, 1)), 0.5)[0, :, 0]
    assert np.allclose(ramp, 0.5 * np.arange(1, 6))
