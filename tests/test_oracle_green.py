"""Pins of the oracle's forward modelling against closed forms.

The paper's forward engine is the constant-density acoustic wave equation
1/v^2 u_tt - lap u = delta(x - x_s) f(t) (Sec. 2). In a homogeneous medium its
solution is the free-space Green's function convolved with f:
  2-D: u(r, t) = 1/(2 pi) int_0^{acosh(vt/r)} f(t - (r/v) cosh theta) dtheta
  3-D: u(r, t) = f(t - r/v) / (4 pi r)
These are independent of the oracle's code, so they pin its scale (source
normalisation 1/dx^d), sign, Laplacian weights and time stepping. Halving dx and
dt together must cut the error by about 4 (second order in time dominates).
"""
import numpy as np
import pytest
from scipy.integrate import quad

from paper_1406_1864_gb300 import workloads as W


def green2d_trace(r, v, t, f0):
    def f(tt):
        return float(W.ricker(1, 1.0, f0, t0=1.5 / f0 - tt)[0]) if tt > -1 else 0.0

    out = np.zeros_like(t)
    for n, tn in enumerate(t):
        if v * tn <= r:
            continue
        top = np.arccosh(v * tn / r)
        out[n] = quad(lambda th: f(tn - (r / v) * np.cosh(th)), 0.0, top, limit=400)[0] / (2 * np.pi)
    return out


def run_2d(oracle_mod, dx, dt, T, off_m, n_cells=160, f0=10.0, v=2000.0):
    nt = int(round(T / dt)) + 1
    nz = nx = n_cells
    c = nz // 2
    off = int(round(off_m / dx))
    p = W.homogeneous(nz, nx, v=v, dx=dx, dt=dt, nt=nt, src=[[c, 0, c]],
                      rec=[[c, 0, c + off]], f0=f0, sponge=20)
    g = oracle_mod.Grid.of(p)
    seis = oracle_mod.forward(g, p.v_init, p.src, p.rec, p.wavelet.astype(np.float64))["seis"]
    t = np.arange(nt) * dt
    return t, seis[0, :, 0]


def test_green_2d_homogeneous(oracle_mod):
    dx, dt, T, off = 10.0, 1e-3, 0.6, 300.0
    t, u = run_2d(oracle_mod, dx, dt, T, off)
    ref = green2d_trace(off, 2000.0, t, 10.0)
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert err < 2e-2, err
    # same polarity and peak within one sample
    assert abs(int(np.argmax(np.abs(u))) - int(np.argmax(np.abs(ref)))) <= 1
    assert np.sign(u[np.argmax(np.abs(u))]) == np.sign(ref[np.argmax(np.abs(ref))])


def test_green_2d_convergence(oracle_mod):
    T, off = 0.5, 300.0
    t1, u1 = run_2d(oracle_mod, 10.0, 1e-3, T, off, n_cells=120)
    t2, u2 = run_2d(oracle_mod, 5.0, 5e-4, T, off, n_cells=240)
    r1 = green2d_trace(off, 2000.0, t1, 10.0)
    r2 = green2d_trace(off, 2000.0, t2, 10.0)
    e1 = np.linalg.norm(u1 - r1) / np.linalg.norm(r1)
    e2 = np.linalg.norm(u2 - r2) / np.linalg.norm(r2)
    assert 3.0 < e1 / e2 < 5.5, (e1, e2)


def test_green_3d_homogeneous(oracle_mod):
    dx, dt, v, f0 = 10.0, 1e-3, 2000.0, 10.0
    n, P = 44, 12
    c = n // 2
    off = 15
    nt = 331
    p = W.homogeneous(n, n, v=v, dx=dx, dt=dt, nt=nt, src=[[c, c, c]], rec=[[c, c, c + off]],
                      f0=f0, sponge=P, ny=n, ndim=3)
    g = oracle_mod.Grid.of(p)
    u = oracle_mod.forward(g, p.v_init, p.src, p.rec, p.wavelet.astype(np.float64),
                           nthreads=1)["seis"][0, :, 0]
    t = np.arange(nt) * dt
    r = off * dx
    ref = W.ricker(nt, dt, f0, t0=1.5 / f0 + r / v) / (4 * np.pi * r)
    # compare before the first reflection off the sponge can come back
    first_return = (2 * (c + P) - off) * dx / v
    m = t < first_return
    err = np.linalg.norm(u[m] - ref[m]) / np.linalg.norm(ref[m])
    assert err < 2e-2, err


def test_sponge_absorbs(oracle_mod):
    """The 20-cell sponge absorbs: a trace recorded 10 cells from the sponge
    differs from the same trace on a domain large enough that nothing comes
    back by less than 10% of the direct wave (the damping has the right sign
    and strength); a 5-cell sponge reflects several times more."""
    def trace(n, P, nt=600):
        c = n // 2
        p = W.homogeneous(n, n, v=2000.0, dx=10.0, dt=1e-3, nt=nt, src=[[c, 0, c]],
                          rec=[[c, 0, c + 30], [c - 30, 0, c + 30]], sponge=P)
        return oracle_mod.forward(oracle_mod.Grid.of(p), p.v_init, p.src, p.rec,
                                  p.wavelet.astype(np.float64))["seis"][0]

    ref = trace(300, 20)
    r20 = np.abs(trace(80, 20) - ref).max() / np.abs(ref).max()
    r5 = np.abs(trace(80, 5) - ref).max() / np.abs(ref).max()
    assert r20 < 0.1, r20
    assert r5 > 4 * r20, (r5, r20)
    n = 80
    p = W.homogeneous(n, n, sponge=20)
    eta = oracle_mod.eta(oracle_mod.Grid.of(p))
    assert np.all(eta[20:20 + n, 0, 20:20 + n] == 0.0)
    assert eta.min() == 0.0 and eta[0, 0, 0] == eta.max() > 0
