"""Pins of the oracle's receiver side of the diagonal Hessian (Sec. 1).

* Plessix and Mulder's factor is the integral over the receiver line of the
  inverse distance, int_{x_min}^{x_max} dxi / sqrt((xi - x)^2 + z^2), whose
  antiderivative is asinh((xi - x)/z): checked against adaptive quadrature of
  that integral at cells inside, at the ends of and outside the spread, and
  against its limits (spread narrower than the depth: (x_max - x_min) / z;
  symmetric about the spread's centre; positive).
* The receiver Green's-function correlations equal a brute-force sum of
  shifted products of the dumped wavefield of a source at the receiver, add
  up over receivers, and at h = 0 equal the illumination of sources at the
  receivers (Eq. 1's form on the receiver side).
* Plessix and Mulder's per-shot Hessian reduces, for one spread shared by
  all shots, to the factor times the illumination of all shots.
A planted mistake (z not floored at the receiver row) must fail a pin.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W


def _quad_factor(x, z, xmin, xmax):
    from scipy.integrate import quad
    val, err = quad(lambda xi: 1.0 / np.sqrt((xi - x) ** 2 + z ** 2), xmin, xmax, epsabs=0, epsrel=1e-12,
                    limit=200)
    return val


def test_plessix_mulder_factor_is_the_inverse_distance_integral(oracle_mod):
    nz, nx, dx = 30, 50, 10.0
    rec = np.zeros((12, 3), np.int32)
    rec[:, 0] = 2
    rec[:, 2] = np.arange(10, 34, 2)           # spread x = 100 .. 320 m
    F = oracle_mod.plessix_mulder_factor(nz, nx, dx, rec)
    xmin, xmax, zr = 100.0, 320.0, 2.0
    for i, j in [(10, 20), (2, 5), (0, 0), (29, 49), (5, 10), (5, 32), (17, 40), (3, 21)]:
        z = max(abs(i - zr) * dx, 0.5 * dx)
        ref = _quad_factor(j * dx, z, xmin, xmax)
        assert abs(F[i, j] - ref) <= 1e-10 * ref, (i, j, F[i, j], ref)
    assert (F > 0).all()
    # symmetric about the spread's centre (x = 210 m = column 21)
    assert np.allclose(F[:, 21 - 8], F[:, 21 + 8], rtol=1e-12)
    # far below a short spread: (x_max - x_min) / z
    short = np.array([[0, 0, 20], [0, 0, 21]], np.int32)
    G = oracle_mod.plessix_mulder_factor(4000, 42, 1.0, short)
    assert abs(G[3999, 20] - 1.0 / 3999.0) <= 1e-6 / 3999.0 * 1e2


def test_planted_unfloored_depth_fails(oracle_mod, monkeypatch):
    """Without the floor at dx / 2 the factor at the receiver row is infinite
    or NaN, which the quadrature pin rejects."""
    real = np.maximum
    monkeypatch.setattr(oracle_mod.np, "maximum", lambda a, b: a)
    rec = np.array([[2, 0, 10], [2, 0, 30]], np.int32)
    with np.errstate(divide="ignore", invalid="ignore"):
        F = oracle_mod.plessix_mulder_factor(10, 40, 10.0, rec)
    monkeypatch.setattr(oracle_mod.np, "maximum", real)
    ref = _quad_factor(200.0, 5.0, 100.0, 300.0)
    assert not (abs(F[2, 20] - ref) <= 1e-10 * ref)


def _spread_problem(nrec=3):
    p = W.dipping(nz=24, nx=34, dx=10.0, dt=1e-3, nt=200, ns=1, nrec=nrec, rec_step=9, f0=15.0, sponge=6,
                  seed=5)
    return p


def test_receiver_green_factor_brute_force_and_sum(oracle_mod):
    p = _spread_problem()
    g = oracle_mod.Grid.of(p)
    P = p.sponge
    w0 = p.wavelet[0].astype(np.float64)
    rec = p.rec[0]
    R = oracle_mod.receiver_green_factor(g, p.v_init, rec, w0, hmax=3)
    parts = []
    for r in range(rec.shape[0]):
        one = oracle_mod.forward(g, p.v_init, rec[r:r + 1], np.zeros((1, 0, 3), np.int32), w0[None, :],
                                 dump_shot=0, illum=True)
        u = one["dump"][:, :, 0, :]
        Hr = []
        for h in range(4):
            up = np.zeros_like(u)
            um = np.zeros_like(u)
            up[:, :, :u.shape[2] - h] = u[:, :, h:]
            um[:, :, h:] = u[:, :, :u.shape[2] - h]
            Hr.append(np.sum(up * um, axis=0)[P:P + p.nz, P:P + p.nx] * p.dt)
        parts.append(np.array(Hr))
        assert np.allclose(Hr[0], one["illum"][:, 0, :], rtol=1e-12, atol=0)
    assert np.allclose(R[:, :, 0, :], np.sum(parts, axis=0), rtol=1e-10, atol=1e-30)


@pytest.mark.parametrize("h", [0, 2])
def test_receiver_green_factor_is_symmetric_positive_at_zero_offset(oracle_mod, h):
    p = _spread_problem(nrec=2)
    g = oracle_mod.Grid.of(p)
    R = oracle_mod.receiver_green_factor(g, p.v_init, p.rec[0], p.wavelet[0], hmax=2)
    if h == 0:
        assert (R[0] >= 0).all() and R[0].max() > 0
    else:
        I = R[0, :, 0, :]
        lhs = np.abs(R[h, :, 0, h:-h])
        rhs = np.sqrt(I[:, 2 * h:] * I[:, :-2 * h])
        assert (lhs <= rhs * (1 + 1e-12) + 1e-300).all()


def test_plessix_mulder_hessian_fixed_spread_is_factor_times_illumination(oracle_mod):
    """With one spread for all shots the per-shot sum factors: the asinh
    factor times the illumination of all shots."""
    p = W.dipping(nz=20, nx=30, dx=10.0, dt=1e-3, nt=120, ns=3, nrec=10, rec_step=3, f0=15.0, sponge=5, seed=2)
    g = oracle_mod.Grid.of(p)
    w = p.wavelet.astype(np.float64)
    H = oracle_mod.plessix_mulder_hessian(g, p.v_init, p.src, p.rec, w)
    il = oracle_mod.forward(g, p.v_init, p.src, p.rec, w, illum=True)["illum"]
    F = oracle_mod.plessix_mulder_factor(p.nz, p.nx, p.dx, p.rec[0])
    assert np.allclose(H[:, 0, :], F * il[:, 0, :], rtol=1e-12, atol=0)

