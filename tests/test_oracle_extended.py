"""Pins of the oracle's extended Born modelling (Eq. 5) and extended
migration (Eq. 6), horizontal subsurface offsets h = -he..he.

* Dot test: <B_ext dv, dd> = <dv, M_ext dd> to 1e-12 (M_ext is B_ext's
  adjoint, folds included).
* At h = 0 alone the extended operators are the plain ones: Born modelling
  (Eq. 4) and the gradient's imaging (Sec. 2).
* The offset convention of Eq. 5 (the incident field at x + h scatters from
  x - h): the extended Born traces of one spike dv(x0, h0) equal plain
  forward modelling with a point source at x0 - h0 driven by the background
  field's q = L u + s at x0 + h0, taken from the dumped background wavefield
  as its second time difference over c2 (the leapfrog update where the
  damping is zero), so no stencil is retyped here.
A planted mistake (the scatterer at x + h instead of x - h) fails the spike pin.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W


def small(ns=2, nt=220, seed=3):
    return W.dipping(nz=26, nx=40, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=14, rec_step=3, f0=15.0, sponge=6,
                     seed=seed)


def test_extended_dot_test(oracle_mod):
    p = small()
    g = oracle_mod.Grid.of(p)
    w = p.wavelet.astype(np.float64)
    he = 3
    rng = np.random.default_rng(1)
    dv = rng.standard_normal((2 * he + 1, p.nz, 1, p.nx))
    dd = rng.standard_normal((p.nshots, p.nt, p.nrec))
    Bdv = oracle_mod.extended_born(g, p.v_init, dv, p.src, p.rec, w, he)
    Mdd = oracle_mod.extended_migration(g, p.v_init, p.src, p.rec, w, dd, he)
    lhs, rhs = float(np.sum(Bdv * dd)), float(np.sum(dv * Mdd))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_zero_offset_reduces_to_plain_operators(oracle_mod):
    p = small()
    g = oracle_mod.Grid.of(p)
    w = p.wavelet.astype(np.float64)
    he = 2
    rng = np.random.default_rng(2)
    dv0 = rng.standard_normal((p.nz, p.nx))
    dv = np.zeros((2 * he + 1, p.nz, 1, p.nx))
    dv[he, :, 0, :] = dv0
    B = oracle_mod.extended_born(g, p.v_init, dv, p.src, p.rec, w, he)
    ref = oracle_mod.born(g, p.v_init, dv0, p.src, p.rec, w)
    assert np.linalg.norm(B - ref) <= 1e-12 * np.linalg.norm(ref)
    dd = rng.standard_normal((p.nshots, p.nt, p.nrec))
    M = oracle_mod.extended_migration(g, p.v_init, p.src, p.rec, w, dd, he)
    gref = oracle_mod.gradient_for_adjoint_source(g, p.v_init, p.src, p.rec, w, dd)["grad"]
    assert np.linalg.norm(M[he] - gref) <= 1e-12 * np.linalg.norm(gref)


def _spike_check(oracle_mod, h0, scatter_sign=-1):
    p = small(ns=1, nt=240)
    g = oracle_mod.Grid.of(p)
    w = p.wavelet.astype(np.float64)
    P = p.sponge
    he = 3
    iz0, ix0 = 14, 20
    A = 7.0
    dv = np.zeros((2 * he + 1, p.nz, 1, p.nx))
    dv[h0 + he, iz0, 0, ix0] = A
    B = oracle_mod.extended_born(g, p.v_init, dv, p.src, p.rec, w, he)
    # background field at x0 + h0 (padded), q = (u^{n+1} - 2 u^n + u^{n-1}) / c2
    dump = oracle_mod.forward(g, p.v_init, p.src, p.rec, w, dump_shot=0)["dump"][:, :, 0, :]
    v = p.v_init.astype(np.float64)
    xs = (iz0 + P, ix0 + h0 + P)
    u = dump[:, xs[0], xs[1]]
    um1 = np.concatenate([[0.0], u[:-1]])
    up1 = np.concatenate([u[1:], [0.0]])
    q = (up1 - 2 * u + um1) / (v[iz0, ix0 + h0] * p.dt) ** 2
    S = 2.0 * v[iz0, ix0] * A * p.dt ** 2 * q             # scattering source strength at level n
    iy = ix0 + scatter_sign * h0                           # the scatterer
    f = S * p.dx ** 2 / (v[iz0, iy] * p.dt) ** 2           # forward injects c2 f / dx^2
    f[-1] = 0.0
    F = oracle_mod.forward(g, p.v_init, np.array([[iz0, 0, iy]]), p.rec, f[None, :])["seis"]
    return np.linalg.norm(B - F) / np.linalg.norm(B)


@pytest.mark.parametrize("h0", [2, -3, 1])
def test_extended_born_offset_convention(oracle_mod, h0):
    assert _spike_check(oracle_mod, h0) <= 1e-10


def test_planted_scatterer_at_plus_h_fails(oracle_mod):
    assert _spike_check(oracle_mod, 2, scatter_sign=+1) > 1e-3
