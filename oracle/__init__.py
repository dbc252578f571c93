"""Plain FP64 CPU oracle of the preconditioned time-domain FWI gradient.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product path (``paper_1406_1864_gb300``) never imports it and shares no code
with it; both receive their inputs from the seeded generators in
``paper_1406_1864_gb300.workloads``, which hold none of the method's arithmetic.

The wave propagation, adjoint imaging and Born operator are plain C loops in
``fwi_oracle.c`` (double precision, OpenMP over shots). This module holds the
parts that are clearest in numpy, each following the paper:

* OLS misfit J = 1/2 sum_s sum_r sum_t (u - d)^2 and its adjoint source, the
  residual (Sec. 2, first misfit);
* the time-integral misfit J = 1/2 || int_0^t (u - d) dtau ||^2 (Eq. 2), with
  the integral read as the inclusive rectangle rule dt * sum_{k<=n}, and its
  adjoint source C^T C r (reverse cumulative sum);
* the gradient preconditioning of Sec. 3 / Fig. 5: g / (P + eps max P) with P the
  shot illumination (Eq. 1) or the offset-Hessian diagonal summed over offsets;
* (in C) extended Born modelling and extended migration with horizontal
  subsurface offsets (Eq. 5, Eq. 6);
* the receiver side of the diagonal Hessian for a fixed spread (Sec. 1):
  Plessix and Mulder's factor asinh((x_max - x)/z) - asinh((x_min - x)/z),
  and the receiver Green's-function correlations sum_r sum_t G_r(x+h)
  G_r(x-h) dt (the offset-Hessian pass with sources at the receivers).

Parity pins: none of these functions is trusted on its own; tests/test_oracle_*
check them against closed forms (2-D Green's function), adjoint dot products,
central finite differences, the cumulative-source identity of Sec. 2 and brute
force sums over dumped wavefields. The offset-preconditioner scale is pinned
against explicit sums over every negative and positive offset, and the
water-level division against hand cases with exact quotients. The
integral-misfit gradient is pinned
exactly against the OLS gradient of the integrated wavefield (Sec. 2), and
Eq. 3's form of it, -sum int u v dt with v = (2/v^3) dLambda/dt (Lambda the
back-propagated integrated residual), holds exactly in the discrete scheme's
undamped interior with a forward time difference.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwi_oracle.c")
_LIB = os.path.join(_HERE, "libfwi_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/libfwi_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i, d, p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        grid = [i, i, i, i, i, d, d, i, d, d]
        lib.oracle_forward.argtypes = grid + [p, i, p, p, i, p, p, p, i, i, p, p, i, i]
        lib.oracle_gradient.argtypes = grid + [p, i, p, p, i, p, p, p, p, p, i]
        lib.oracle_born.argtypes = grid + [p, p, i, p, p, i, p, p, i]
        lib.oracle_eta.argtypes = [i, i, i, i, i, d, d, d, p]
        lib.oracle_ext_born.argtypes = grid + [p, p, i, i, p, p, i, p, p, i]
        lib.oracle_ext_migration.argtypes = grid + [p, i, p, p, i, p, p, i, p, i]
        for f in (lib.oracle_forward, lib.oracle_gradient, lib.oracle_born, lib.oracle_eta, lib.oracle_ext_born,
                  lib.oracle_ext_migration):
            f.restype = i
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Grid:
    """Discretisation of one model: physical nz x ny x nx (ny=1 in 2-D)."""
    ndim: int
    nz: int
    ny: int
    nx: int
    dx: float
    dt: float
    nt: int
    sponge: int = 20
    vref: float = 3000.0
    refl: float = 0.05

    @classmethod
    def of(cls, prob) -> "Grid":
        return cls(prob.ndim, prob.nz, prob.ny, prob.nx, prob.dx, prob.dt, prob.nt,
                   prob.sponge, prob.vref, prob.refl)

    def args(self):
        return (self.ndim, self.nz, self.ny, self.nx, self.sponge, float(self.dx),
                float(self.dt), self.nt, float(self.vref), float(self.refl))

    @property
    def padded_shape(self):
        P = self.sponge
        nyp = self.ny + 2 * P if self.ndim == 3 else 1
        return (self.nz + 2 * P, nyp, self.nx + 2 * P)


def _geom(src, rec, wav, nt):
    src = np.ascontiguousarray(src, dtype=np.int32).reshape(-1, 3)
    ns = src.shape[0]
    rec = np.ascontiguousarray(rec, dtype=np.int32).reshape(ns, -1, 3)
    wav = np.ascontiguousarray(wav, dtype=np.float64).reshape(ns, nt)
    return src, rec, wav, ns, rec.shape[1]


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"{name}: invalid arguments (code {rc})")


# weights of the 8th-order second difference (the C oracle's W8)
_W8 = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


def stability_limit(ndim: int) -> float:
    """Largest v dt / dx for which leapfrog with the 8th-order Laplacian is
    stable: (v dt / dx)^2 ndim |s(pi)| <= 4, s the symbol of the 1-D second
    difference, s(pi) = w0 + 2 sum_k (-1)^k w_k."""
    s_pi = _W8[0] + 2.0 * sum((-1) ** k * w for k, w in enumerate(_W8) if k > 0)
    return 2.0 / np.sqrt(ndim * abs(s_pi))


def _check_stable(grid: Grid, v):
    c = float(np.max(v)) * grid.dt / grid.dx
    if not c <= stability_limit(grid.ndim):
        raise ValueError(f"v dt / dx = {c:.4f} above the {grid.ndim}-D stability limit "
                         f"{stability_limit(grid.ndim):.4f}: the oracle would model noise")


def forward(grid: Grid, v, src, rec, wav, *, illum=False, illum_utt=False, hmax=None,
            dump_shot=None, nthreads=0):
    """Forward modelling of every shot.

    Returns a dict with ``seis`` [ns, nt, nrec] and, on request, ``illum``
    [nz, ny, nx] (Eq. 1 as sum_s sum_n u^2 dt, or u_tt^2 dt), ``offh``
    [hmax+1, nz, ny, nx] (offset-Hessian diagonal, Sec. 3) and ``dump``
    [nt, nzp, nyp, nxp] (every time level of one shot, padded grid).
    """
    lib = _load()
    src, rec, wav, ns, nrec = _geom(src, rec, wav, grid.nt)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(grid.nz, grid.ny, grid.nx)
    _check_stable(grid, v)
    seis = np.zeros((ns, grid.nt, nrec))
    out = {"seis": seis}
    il = np.zeros((grid.nz, grid.ny, grid.nx)) if illum else None
    oh = np.zeros((hmax + 1, grid.nz, grid.ny, grid.nx)) if hmax is not None else None
    dump = np.zeros((grid.nt,) + grid.padded_shape) if dump_shot is not None else None
    rc = lib.oracle_forward(*grid.args(), _ptr(v), ns, _ptr(src), _ptr(wav), nrec, _ptr(rec),
                            _ptr(seis), _ptr(il), int(illum_utt), int(hmax or 0), _ptr(oh),
                            _ptr(dump), int(dump_shot or 0), int(nthreads))
    _check(rc, "oracle_forward")
    if il is not None:
        out["illum"] = il
    if oh is not None:
        out["offh"] = oh
    if dump is not None:
        out["dump"] = dump
    return out


def gradient_for_adjoint_source(grid: Grid, v, src, rec, wav, adj, *, want_pad=False,
                                want_psi_src=False, nthreads=0):
    """Gradient w.r.t. the physical velocity of sum a^n(r) d^n(r) for a given
    adjoint source ``adj`` [ns, nt, nrec] (Sec. 2 zero-lag cross-correlation,
    as the exact derivative of the discrete scheme). Returns a dict with
    ``grad`` [nz, ny, nx], and optionally ``grad_pad`` (padded, before the
    fold) and ``psi_src`` [ns, nt] (adjoint of the source-to-trace map)."""
    lib = _load()
    src, rec, wav, ns, nrec = _geom(src, rec, wav, grid.nt)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(grid.nz, grid.ny, grid.nx)
    _check_stable(grid, v)
    adj = np.ascontiguousarray(adj, dtype=np.float64).reshape(ns, grid.nt, nrec)
    grad = np.zeros((grid.nz, grid.ny, grid.nx))
    gpad = np.zeros(grid.padded_shape) if want_pad else None
    psi = np.zeros((ns, grid.nt)) if want_psi_src else None
    rc = lib.oracle_gradient(*grid.args(), _ptr(v), ns, _ptr(src), _ptr(wav), nrec, _ptr(rec),
                             _ptr(adj), _ptr(grad), _ptr(gpad), _ptr(psi), int(nthreads))
    _check(rc, "oracle_gradient")
    out = {"grad": grad}
    if gpad is not None:
        out["grad_pad"] = gpad
    if psi is not None:
        out["psi_src"] = psi
    return out


def born(grid: Grid, v, dv, src, rec, wav, nthreads=0):
    """Born modelling, Eq. 4: traces' derivative along the velocity change dv."""
    lib = _load()
    src, rec, wav, ns, nrec = _geom(src, rec, wav, grid.nt)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(grid.nz, grid.ny, grid.nx)
    _check_stable(grid, v)
    dv = np.ascontiguousarray(dv, dtype=np.float64).reshape(grid.nz, grid.ny, grid.nx)
    dseis = np.zeros((ns, grid.nt, nrec))
    rc = lib.oracle_born(*grid.args(), _ptr(v), _ptr(dv), ns, _ptr(src), _ptr(wav), nrec,
                         _ptr(rec), _ptr(dseis), int(nthreads))
    _check(rc, "oracle_born")
    return dseis


def extended_born(grid: Grid, v, dv_ext, src, rec, wav, he, nthreads=0):
    """Extended Born modelling, Eq. 5: traces [ns, nt, nrec] of the extended
    perturbation dv_ext [2 he + 1, nz, ny, nx] (horizontal subsurface offsets
    h = -he..he): the incident field at x + h scatters from x - h."""
    lib = _load()
    src, rec, wav, ns, nrec = _geom(src, rec, wav, grid.nt)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(grid.nz, grid.ny, grid.nx)
    _check_stable(grid, v)
    dv_ext = np.ascontiguousarray(dv_ext, dtype=np.float64).reshape(2 * he + 1, grid.nz, grid.ny, grid.nx)
    dseis = np.zeros((ns, grid.nt, nrec))
    rc = lib.oracle_ext_born(*grid.args(), _ptr(v), _ptr(dv_ext), int(he), ns, _ptr(src), _ptr(wav), nrec,
                             _ptr(rec), _ptr(dseis), int(nthreads))
    _check(rc, "oracle_ext_born")
    return dseis


def extended_migration(grid: Grid, v, src, rec, wav, adj, he, nthreads=0):
    """Extended migration, Eq. 6, the adjoint of extended_born: the image
    [2 he + 1, nz, ny, nx] of the adjoint source adj [ns, nt, nrec]."""
    lib = _load()
    src, rec, wav, ns, nrec = _geom(src, rec, wav, grid.nt)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(grid.nz, grid.ny, grid.nx)
    _check_stable(grid, v)
    adj = np.ascontiguousarray(adj, dtype=np.float64).reshape(ns, grid.nt, nrec)
    image = np.zeros((2 * he + 1, grid.nz, grid.ny, grid.nx))
    rc = lib.oracle_ext_migration(*grid.args(), _ptr(v), ns, _ptr(src), _ptr(wav), nrec, _ptr(rec), _ptr(adj),
                                  int(he), _ptr(image), int(nthreads))
    _check(rc, "oracle_ext_migration")
    return image


def eta(grid: Grid):
    """Sponge damping profile on the padded grid."""
    lib = _load()
    out = np.zeros(grid.padded_shape)
    rc = lib.oracle_eta(grid.ndim, grid.nz, grid.ny, grid.nx, grid.sponge, float(grid.dx),
                        float(grid.vref), float(grid.refl), _ptr(out))
    _check(rc, "oracle_eta")
    return out


# ------------------------------------------ receiver side of the Hessian (Sec. 1)

def plessix_mulder_factor(nz, nx, dx, rec):
    """Plessix and Mulder's receiver factor of the diagonal Hessian for one
    receiver spread (Sec. 1): asinh((x_max - x)/z) - asinh((x_min - x)/z) at
    every model cell, x = j dx, x_min / x_max the spread's extent (m), z the
    depth (m) below the receivers' mean row, floored at dx / 2. rec: [nrec, 3]
    (z, y, x) cells of the spread. Returns [nz, nx] float64."""
    rec = np.asarray(rec).reshape(-1, 3)
    x_min, x_max = rec[:, 2].min() * dx, rec[:, 2].max() * dx
    zr = rec[:, 0].mean()
    z = np.maximum(np.abs(np.arange(nz, dtype=np.float64) - zr) * dx, 0.5 * dx)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :] * dx
    return np.arcsinh((x_max - x) / z) - np.arcsinh((x_min - x) / z)


def plessix_mulder_hessian(grid: Grid, v, src, rec, wav, illum_utt=False, nthreads=0):
    """Plessix and Mulder's approximate diagonal Hessian (Sec. 1) for any
    acquisition: sum over shots of the shot's illumination (Eq. 1's form,
    sum_n u^2 dt or u_tt^2 dt) times the asinh factor of the shot's own
    receiver spread. Returns [nz, ny, nx]."""
    src = np.asarray(src).reshape(-1, 3)
    ns = src.shape[0]
    rec = np.asarray(rec).reshape(ns, -1, 3)
    wav = np.asarray(wav, np.float64).reshape(ns, -1)
    out = np.zeros((grid.nz, grid.ny, grid.nx))
    for s in range(ns):
        il = forward(grid, v, src[s:s + 1], rec[s:s + 1], wav[s:s + 1], illum=True, illum_utt=illum_utt,
                     nthreads=nthreads)["illum"]
        out += plessix_mulder_factor(grid.nz, grid.nx, grid.dx, rec[s])[:, None, :] * il
    return out


def receiver_green_factor(grid: Grid, v, rec, wav0, hmax=0, nthreads=0):
    """Receiver Green's-function correlations of a fixed spread (the
    receiver sum of H_a, Sec. 1 / Sec. 3): sum_r sum_n G_r(x + h) G_r(x - h) dt,
    h = 0..hmax, G_r the wavefield of a source at receiver r with the wavelet
    wav0 [nt]. Returns [hmax + 1, nz, ny, nx]."""
    rec = np.asarray(rec).reshape(-1, 3)
    wav = np.repeat(np.asarray(wav0, np.float64).reshape(1, -1), rec.shape[0], axis=0)
    none = np.zeros((rec.shape[0], 0, 3), np.int32)
    return forward(grid, v, rec, none, wav, hmax=hmax, nthreads=nthreads)["offh"]


# ---------------------------------------------------------------- misfits (Sec. 2)

def misfit_ols(seis, d_obs):
    """OLS misfit with W_d = I (Sec. 2): J = 1/2 sum r^2, r = u - d.
    Returns (J, adjoint source dJ/du = r)."""
    r = np.asarray(seis, dtype=np.float64) - np.asarray(d_obs, dtype=np.float64)
    return 0.5 * float(np.sum(r * r)), r


def time_integral(r, dt):
    """(C r)^n = dt * sum_{k<=n} r^k along the time axis (axis 1) -- the
    data weighting W_d u = int_0^t u dtau of Eq. 2, inclusive rectangle rule."""
    return dt * np.cumsum(r, axis=1)


def time_integral_adjoint(y, dt):
    """(C^T y)^n = dt * sum_{k>=n} y^k: the transpose of time_integral."""
    return dt * np.cumsum(y[:, ::-1, :], axis=1)[:, ::-1, :]


def misfit_time_integral(seis, d_obs, dt):
    """Time-integral residual misfit, Eq. 2: J = 1/2 || C (u - d) ||^2.
    Returns (J, adjoint source C^T C (u - d))."""
    r = np.asarray(seis, dtype=np.float64) - np.asarray(d_obs, dtype=np.float64)
    y = time_integral(r, dt)
    return 0.5 * float(np.sum(y * y)), time_integral_adjoint(y, dt)


# ------------------------------------------------------- preconditioning (Sec. 3)

def offset_scale(offh):
    """Per-point scale from the offset-Hessian diagonal H(x, h), h = 0..hmax:
    sum over |h| <= hmax of |H(x, h)| (H is even in h)."""
    offh = np.asarray(offh, dtype=np.float64)
    return np.abs(offh[0]) + 2.0 * np.sum(np.abs(offh[1:]), axis=0)


def precondition(grad, P, eps=1e-3):
    """Diagonal scaling of the gradient: g / (P + eps * max P)."""
    P = np.asarray(P, dtype=np.float64)
    return np.asarray(grad, dtype=np.float64) / (P + eps * P.max())


def fwi_gradient(grid: Grid, v, src, rec, wav, d_obs, *, misfit="ols", hmax=None,
                 illum_utt=False, eps=1e-3, hess_v6=False, nthreads=0):
    """The whole preconditioned gradient of one model: forward modelling,
    misfit, adjoint source, adjoint imaging, illumination / offset-Hessian
    preconditioners. Returns a dict of float64 arrays and the misfit J."""
    fw = forward(grid, v, src, rec, wav, illum=True, illum_utt=illum_utt, hmax=hmax,
                 nthreads=nthreads)
    if misfit == "ols":
        J, adj = misfit_ols(fw["seis"], d_obs)
    elif misfit == "integral":
        J, adj = misfit_time_integral(fw["seis"], d_obs, grid.dt)
    else:
        raise ValueError(misfit)
    g = gradient_for_adjoint_source(grid, v, src, rec, wav, adj, nthreads=nthreads)["grad"]
    # H_a's diagonal carries 4 omega^4 / (v^3(x) v^3(y)) (Sec. 3): at y = x, 4 / v(x)^6
    w6 = 4.0 / np.asarray(v, np.float64).reshape(grid.nz, grid.ny, grid.nx) ** 6 if hess_v6 else 1.0
    illum = fw["illum"] * w6
    out = {"seis": fw["seis"], "J": J, "grad": g, "illum": illum, "grad_pre_illum": precondition(g, illum, eps)}
    if hmax is not None:
        out["offh"] = fw["offh"] * w6
        out["grad_pre_offset"] = precondition(g, offset_scale(out["offh"]), eps)
    return out
