"""Pins of the oracle's 3-D path (25-point Laplacian, source f / dx^3), the
reference of the 3-D GPU tests:

* source-to-trace dot test <F f, d> = <f, F^T d> (1e-12);
* Jacobian dot test <J dv, dd> = <dv, J^T dd> (1e-12), J the Born operator;
* gradient of the OLS and time-integral misfits against central finite
  differences of the misfit along smooth directions and an edge direction
  that reaches the sponge (1e-6);
* illumination (Eq. 1) and the offset-Hessian diagonal (Sec. 3) against
  brute-force sums over the dumped field.
A planted mistake (a wrong sign of the adjoint source) fails the FD check.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W


def tiny3d(ns=2, nt=180):
    """10 x 9 x 11 cells of the layered 3-D model (up to 5.1 km/s), dt 0.5 ms:
    v dt / dx <= 0.26, inside the 3-D stability limit."""
    return W.dipping3d(nz=10, ny=9, nx=11, dx=10.0, dt=5e-4, nt=nt, ns=ns, rec_step=3, f0=20.0, seed=2,
                       sponge=4)


def test_3d_source_to_trace_and_jacobian_dot(oracle_mod):
    p = tiny3d()
    g = oracle_mod.Grid.of(p)
    rng = np.random.default_rng(4)
    f = rng.standard_normal((p.nshots, p.nt))
    d = rng.standard_normal((p.nshots, p.nt, p.nrec))
    Ff = oracle_mod.forward(g, p.v_true, p.src, p.rec, f)["seis"]
    Ftd = oracle_mod.gradient_for_adjoint_source(g, p.v_true, p.src, p.rec, f, d, want_psi_src=True)["psi_src"]
    lhs, rhs = np.sum(Ff * d), np.sum(f * Ftd)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)
    w = p.wavelet.astype(np.float64)
    v = p.v_init.astype(np.float64)
    dv = rng.standard_normal(v.shape)
    Jdv = oracle_mod.born(g, v, dv, p.src, p.rec, w)
    JTd = oracle_mod.gradient_for_adjoint_source(g, v, p.src, p.rec, w, d)["grad"].reshape(v.shape)
    lhs, rhs = np.sum(Jdv * d), np.sum(dv * JTd)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _smooth3(shape, seed):
    from scipy.ndimage import gaussian_filter
    r = np.random.default_rng(seed).standard_normal(shape)
    s = gaussian_filter(r, 2.0, mode="nearest")
    return s / np.abs(s).max()


@pytest.mark.parametrize("misfit", ["ols", "integral"])
def test_3d_gradient_finite_difference(oracle_mod, misfit):
    p = tiny3d()
    g = oracle_mod.Grid.of(p)
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
    edge = np.zeros(v.shape)
    edge[:, :, 0] = 1.0       # x = 0 face: replicated into the sponge
    edge[-1, -1, :] += 0.5    # a bottom edge line and its corner
    for dvec in (_smooth3(v.shape, 0), _smooth3(v.shape, 1), edge):
        eps = 0.5
        fd = (J(v + eps * dvec) - J(v - eps * dvec)) / (2 * eps)
        an = float(np.sum(grad * dvec))
        assert abs(fd - an) <= 1e-6 * abs(an), (misfit, fd, an)


def test_3d_planted_sign_error_fails_fd(oracle_mod):
    p = tiny3d(ns=1)
    g = oracle_mod.Grid.of(p)
    w = p.wavelet.astype(np.float64)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, w)["seis"]
    v = p.v_init.astype(np.float64)
    _, r = oracle_mod.misfit_ols(oracle_mod.forward(g, v, p.src, p.rec, w)["seis"], d_obs)
    bad = oracle_mod.gradient_for_adjoint_source(g, v, p.src, p.rec, w, -r)["grad"].reshape(v.shape)
    dvec = _smooth3(v.shape, 3)
    eps = 0.5
    Jp = oracle_mod.misfit_ols(oracle_mod.forward(g, v + eps * dvec, p.src, p.rec, w)["seis"], d_obs)[0]
    Jm = oracle_mod.misfit_ols(oracle_mod.forward(g, v - eps * dvec, p.src, p.rec, w)["seis"], d_obs)[0]
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - np.sum(bad * dvec)) > 0.5 * abs(fd)


def test_3d_illumination_brute_force(oracle_mod):
    p = tiny3d(ns=1)
    g = oracle_mod.Grid.of(p)
    P = p.sponge
    out = oracle_mod.forward(g, p.v_init, p.src, p.rec, p.wavelet, illum=True, dump_shot=0)
    u = out["dump"]                                   # [nt, nzp, nyp, nxp]
    I = np.sum(u[:, P:P + p.nz, P:P + p.ny, P:P + p.nx] ** 2, axis=0) * p.dt
    assert np.allclose(out["illum"], I, rtol=1e-12, atol=0)


def test_3d_offset_hessian_brute_force(oracle_mod):
    """Sec. 3's offset-Hessian diagonal in 3-D, H(x, h) = sum_n u(x + h e_x)
    u(x - h e_x) dt, against explicit shifts of the dumped field with zeros
    outside the padded grid (hmax 6 reaches past the 4-cell sponge); H(x, 0)
    is the illumination of Eq. 1; the same products shifted along y instead
    of x do not match (the offset axis is pinned)."""
    p = tiny3d(ns=1)
    g = oracle_mod.Grid.of(p)
    P, hmax = p.sponge, 6
    out = oracle_mod.forward(g, p.v_init, p.src, p.rec, p.wavelet, illum=True, hmax=hmax, dump_shot=0)
    u = out["dump"]                                   # [nt, nzp, nyp, nxp]
    Z = hmax
    up = np.pad(u, ((0, 0), (0, 0), (Z, Z), (Z, Z)))  # zero outside the padded grid along y and x
    zs = slice(P, P + p.nz)

    def at(dy, dx):
        return up[:, zs, P + Z + dy:P + Z + dy + p.ny, P + Z + dx:P + Z + dx + p.nx]

    H = out["offh"]
    assert H.shape == (hmax + 1, p.nz, p.ny, p.nx)
    for h in range(hmax + 1):
        ref = np.sum(at(0, h) * at(0, -h), axis=0) * p.dt
        assert np.allclose(H[h], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), h
    assert np.allclose(H[0], out["illum"], rtol=1e-12, atol=0)
    wrong = np.sum(at(2, 0) * at(-2, 0), axis=0) * p.dt
    assert np.abs(wrong - H[2]).max() > 1e-2 * np.abs(H[2]).max()
