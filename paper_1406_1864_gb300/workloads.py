"""Seeded synthetic workloads: velocity models, acquisition geometry, wavelets.

This module produces INPUTS only and holds none of the method's arithmetic (no
propagation, misfit, imaging or Hessian). It is the one module that both the
CUDA path's tests / bench and the CPU oracle receive their inputs from.

The paper's experiments use the Marmousi model (Sec. 2.1, Sec. 3.1), which is
not available here; the generators below stand in for it with models of the
same velocity range (1.5-4.5 km/s), layered and dipping structure with a
high-velocity body, a smooth starting model and surface acquisition.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass
class Problem:
    """One modelling problem: grid, acquisition and models (float32)."""
    name: str
    ndim: int
    nz: int
    ny: int
    nx: int
    dx: float
    dt: float
    nt: int
    src: np.ndarray            # [ns, 3] int32 physical (z, y, x); y = 0 in 2-D
    rec: np.ndarray            # [ns, nrec, 3] int32
    wavelet: np.ndarray        # [ns, nt] float32 source time function f_s(t_n)
    v_true: np.ndarray         # [nz, nx] or [nz, ny, nx] float32 (m/s)
    v_init: np.ndarray         # same shape, starting model
    sponge: int = 20
    vref: float = 0.0          # damping reference speed (m/s); set by generators
    refl: float = 0.05         # sponge strength: eta_max = 3 vref ln(1/refl) / (2 P dx)
    meta: dict = field(default_factory=dict)

    @property
    def nshots(self) -> int:
        return int(self.src.shape[0])

    @property
    def nrec(self) -> int:
        return int(self.rec.shape[1])

    @property
    def phys_points(self) -> int:
        return self.nz * self.ny * self.nx

    @property
    def shape(self):
        return (self.nz, self.nx) if self.ndim == 2 else (self.nz, self.ny, self.nx)

    def courant(self) -> float:
        return float(max(self.v_true.max(), self.v_init.max()) * self.dt / self.dx)

    def subset(self, shots) -> "Problem":
        """The same problem restricted to some shots."""
        shots = np.asarray(shots)
        return replace(self, src=self.src[shots].copy(), rec=self.rec[shots].copy(),
                       wavelet=self.wavelet[shots].copy())

    def with_nt(self, nt: int) -> "Problem":
        """The same problem with fewer (or more) time levels."""
        f0 = self.meta.get("f0", 10.0)
        w = np.repeat(ricker(nt, self.dt, f0)[None, :], self.nshots, axis=0)
        return replace(self, nt=nt, wavelet=w.astype(np.float32))


def ricker(nt: int, dt: float, f0: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet with peak frequency f0, delayed by t0 = 1.5 / f0."""
    t0 = 1.5 / f0 if t0 is None else t0
    a = (np.pi * f0 * (np.arange(nt) * dt - t0)) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float64)


def _surface_geometry(nx: int, ns: int, nrec: int, src_row: int, rec_row: int,
                      rec_step: int = 1, ny: int = 1):
    sx = np.floor((np.arange(ns) + 0.5) * nx / ns).astype(np.int32)
    src = np.zeros((ns, 3), np.int32)
    src[:, 0] = src_row
    src[:, 2] = sx
    rx = (np.arange(nrec) * rec_step).astype(np.int32)
    if rx.max() >= nx:
        raise ValueError("receivers do not fit the grid")
    rec = np.zeros((ns, nrec, 3), np.int32)
    rec[:, :, 0] = rec_row
    rec[:, :, 2] = rx[None, :]
    return src, rec


def two_layer(nz=100, nx=200, dx=10.0, dt=1e-3, nt=1000, ns=4, nrec=200, f0=10.0,
              sponge=20, name="two_layer") -> Problem:
    """Two flat layers 2000 / 3000 m/s (interface at mid depth), starting model
    a 1-D linear gradient 2000 -> 3000 m/s; shots at z = 20 m evenly spaced,
    receivers on the surface row."""
    z = np.arange(nz)
    v_true = np.where(z[:, None] < nz // 2, 2000.0, 3000.0) * np.ones((1, nx))
    v_init = (2000.0 + 1000.0 * z / max(nz - 1, 1))[:, None] * np.ones((1, nx))
    src, rec = _surface_geometry(nx, ns, nrec, src_row=min(2, nz - 1), rec_row=0,
                                 rec_step=max(1, nx // nrec))
    w = np.repeat(ricker(nt, dt, f0)[None, :], ns, axis=0)
    return Problem(name, 2, nz, 1, nx, dx, dt, nt, src, rec, w.astype(np.float32),
                   v_true.astype(np.float32), v_init.astype(np.float32), sponge=sponge,
                   vref=3000.0, meta={"f0": f0})


def dipping_layers_model(nz, nx, dx, seed=0, vels=(1500, 2100, 2700, 3300, 3900, 4500),
                         max_dip_deg=8.0, body_sigma_m=200.0, body_dv=600.0):
    """Layered model with dipping interfaces and a Gaussian high-velocity body.

    len(vels) layers; len(vels)-1 interfaces at evenly spaced mean depths with
    dips drawn from U(-max_dip, max_dip); the body's centre is drawn uniformly
    from the middle third of the model in each direction."""
    rng = np.random.default_rng(seed)
    nl = len(vels)
    z = np.arange(nz)[:, None].astype(np.float64)
    x = np.arange(nx)[None, :].astype(np.float64)
    dips = np.deg2rad(rng.uniform(-max_dip_deg, max_dip_deg, nl - 1))
    depths = (np.arange(1, nl) * nz / nl)
    layer = np.zeros((nz, nx), np.int64)
    for d, a in zip(depths, dips):
        layer += (z >= d + np.tan(a) * (x - nx / 2.0)).astype(np.int64)
    v = np.asarray(vels, np.float64)[layer]
    zc = rng.uniform(nz / 3.0, 2.0 * nz / 3.0)
    xc = rng.uniform(nx / 3.0, 2.0 * nx / 3.0)
    s = body_sigma_m / dx
    v += body_dv * np.exp(-((z - zc) ** 2 + (x - xc) ** 2) / (2.0 * s * s))
    return v


def smooth(v, sigma_cells):
    """Gaussian-smoothed copy of a model (edge values extended)."""
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(np.asarray(v, np.float64), sigma_cells, mode="nearest")


def dipping(nz=300, nx=1000, dx=10.0, dt=8e-4, nt=4000, ns=96, nrec=500, rec_step=2,
            f0=8.0, seed=0, sponge=20, name="dipping") -> Problem:
    """Six dipping layers 1500-4500 m/s plus a Gaussian body (sigma 200 m,
    +600 m/s); starting model the true model smoothed with sigma = 300 m; shots
    at z = 20 m, receivers at z = 10 m every ``rec_step`` cells."""
    v_true = dipping_layers_model(nz, nx, dx, seed=seed)
    v_init = smooth(v_true, 300.0 / dx)
    nrec = min(nrec, (nx - 1) // rec_step + 1)
    src, rec = _surface_geometry(nx, ns, nrec, src_row=min(2, nz - 1), rec_row=min(1, nz - 1),
                                 rec_step=rec_step)
    w = np.repeat(ricker(nt, dt, f0)[None, :], ns, axis=0)
    vref = float(max(v_true.max(), v_init.max()))
    return Problem(name, 2, nz, 1, nx, dx, dt, nt, src, rec, w.astype(np.float32),
                   v_true.astype(np.float32), v_init.astype(np.float32), sponge=sponge,
                   vref=vref, meta={"f0": f0, "seed": seed})


def homogeneous(nz, nx, v=2000.0, dx=10.0, dt=1e-3, nt=400, src=None, rec=None, f0=10.0,
                sponge=20, ny=1, ndim=2, name="homogeneous") -> Problem:
    """Constant-velocity medium with explicit source/receiver coordinates."""
    shape = (nz, nx) if ndim == 2 else (nz, ny, nx)
    vv = np.full(shape, v, np.float32)
    src = np.asarray(src if src is not None else [[nz // 2, ny // 2 if ndim == 3 else 0, nx // 2]],
                     np.int32).reshape(-1, 3)
    ns = src.shape[0]
    rec = np.asarray(rec if rec is not None else [[0, 0, 0]], np.int32).reshape(1, -1, 3)
    rec = np.repeat(rec, ns, axis=0) if rec.shape[0] == 1 else rec.reshape(ns, -1, 3)
    w = np.repeat(ricker(nt, dt, f0)[None, :], ns, axis=0)
    return Problem(name, ndim, nz, ny if ndim == 3 else 1, nx, dx, dt, nt, src, rec,
                   w.astype(np.float32), vv, vv.copy(), sponge=sponge, vref=float(v),
                   meta={"f0": f0})


def smooth_perturbation(shape, seed, sigma_cells=5.0, amplitude=1.0):
    """White noise (seeded) smoothed by a Gaussian of sigma_cells, scaled to a
    max-abs of ``amplitude``: a smooth random direction in model space."""
    rng = np.random.default_rng(seed)
    p = smooth(rng.standard_normal(shape), sigma_cells)
    return (amplitude * p / np.abs(p).max()).astype(np.float64)


# ------------------------------------------------------------------ named workloads

def dipping_layers_model3d(nz, ny, nx, dx, seed=0, vels=(1500, 2100, 2700, 3300, 3900, 4500),
                           max_dip_deg=8.0, body_sigma_m=200.0, body_dv=600.0):
    """3-D counterpart of dipping_layers_model: planar interfaces dipping in x
    and y (dips from U(-max_dip, max_dip) each) at evenly spaced mean depths,
    plus a Gaussian body centred in the middle third of each axis."""
    rng = np.random.default_rng(seed)
    nl = len(vels)
    z = np.arange(nz)[:, None, None].astype(np.float64)
    y = np.arange(ny)[None, :, None].astype(np.float64)
    x = np.arange(nx)[None, None, :].astype(np.float64)
    dips = np.deg2rad(rng.uniform(-max_dip_deg, max_dip_deg, (nl - 1, 2)))
    depths = np.arange(1, nl) * nz / nl
    layer = np.zeros((nz, ny, nx), np.int64)
    for d, (ax, ay) in zip(depths, dips):
        layer += (z >= d + np.tan(ax) * (x - nx / 2.0) + np.tan(ay) * (y - ny / 2.0)).astype(np.int64)
    v = np.asarray(vels, np.float64)[layer]
    c = [rng.uniform(n / 3.0, 2.0 * n / 3.0) for n in (nz, ny, nx)]
    s = body_sigma_m / dx
    v += body_dv * np.exp(-((z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2) / (2.0 * s * s))
    return v


def dipping3d(nz=200, ny=400, nx=400, dx=12.5, dt=1e-3, nt=3000, ns=8, rec_step=1, f0=8.0, seed=0,
              sponge=20, smooth_m=300.0, name="dipping3d") -> Problem:
    """3-D layered model with a Gaussian body; starting model smoothed over
    smooth_m; ns shots at depth 2 cells on a regular (y, x) grid; receivers on
    the top model row every rec_step cells in y and x (400 x 400 by default)."""
    v_true = dipping_layers_model3d(nz, ny, nx, dx, seed=seed)
    v_init = smooth(v_true, smooth_m / dx)
    gy = int(np.floor(np.sqrt(ns)))
    while ns % gy:
        gy -= 1
    gx = ns // gy
    sy = np.floor((np.arange(gy) + 0.5) * ny / gy).astype(np.int32)
    sx = np.floor((np.arange(gx) + 0.5) * nx / gx).astype(np.int32)
    src = np.zeros((ns, 3), np.int32)
    src[:, 0] = min(2, nz - 1)
    src[:, 1] = np.repeat(sy, gx)
    src[:, 2] = np.tile(sx, gy)
    ry, rx = np.meshgrid(np.arange(0, ny, rec_step), np.arange(0, nx, rec_step), indexing="ij")
    one = np.stack([np.zeros(ry.size, np.int32), ry.ravel().astype(np.int32), rx.ravel().astype(np.int32)], 1)
    rec = np.repeat(one[None], ns, axis=0)
    w = np.repeat(ricker(nt, dt, f0)[None, :], ns, axis=0)
    vref = float(max(v_true.max(), v_init.max()))
    return Problem(name, 3, nz, ny, nx, dx, dt, nt, src, rec, w.astype(np.float32), v_true.astype(np.float32),
                   v_init.astype(np.float32), sponge=sponge, vref=vref, meta={"f0": f0, "seed": seed})


def uneven_batch(nt=4000, ns=32, sizes=((200, 400), (350, 900), (500, 1500)), seed=1) -> list:
    """Independent models of uneven sizes sharing nt: the dipping-layer
    generator at each size (its own seed), ns shots and nx / 2 receivers each."""
    return [dipping(nz=nz, nx=nx, nt=nt, ns=ns, nrec=nx // 2, seed=seed + k, name=f"dipping_{nz}x{nx}")
            for k, (nz, nx) in enumerate(sizes)]


def workload(name: str) -> Problem:
    """The named workloads of the benchmark suite (full sizes)."""
    if name == "two_layer_100x200":
        return two_layer()
    if name == "dipping_300x1000_96shots":
        return dipping()
    if name == "dipping3d_200x400x400_8shots":
        return dipping3d()
    if name == "dipping_400x1200_64shots":
        return dipping(nz=400, nx=1200, nt=5000, ns=64, nrec=600, name="dipping_400x1200_64shots")
    raise KeyError(name)
