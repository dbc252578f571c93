"""Python binding of the C ABI (include/fwi.h): argument marshalling only.

Every step of the path runs in libfwi's CUDA kernels. PyTorch supplies device
memory (the workspace and outputs are torch CUDA tensors) and the stream; the
functions below fill the C structs, pass raw pointers and raise FwiError on a
non-OK status.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from ._lib import FwiError  # noqa: F401  (re-export)

OPS = {"forward": L.FWI_OP_FORWARD, "forward_save": L.FWI_OP_FORWARD_SAVE,
       "gradient": L.FWI_OP_GRADIENT, "illumination": L.FWI_OP_ILLUMINATION,
       "offset_hessian": L.FWI_OP_OFFSET_HESSIAN, "precondition": L.FWI_OP_PRECONDITION,
       "born": L.FWI_OP_BORN, "gn_hvp": L.FWI_OP_GN_HVP, "misfit": L.FWI_OP_MISFIT,
       "receiver_factor": L.FWI_OP_RECEIVER_FACTOR, "precondition_receiver": L.FWI_OP_PRECONDITION_RECEIVER,
       "extended_born": L.FWI_OP_EXT_BORN, "extended_migration": L.FWI_OP_EXT_MIGRATION,
       "pm_hessian": L.FWI_OP_PM_HESSIAN}


@dataclass
class Grid:
    """fwi_grid: physical nz x nx (2-D) or nz x ny x nx (ndim = 3) model,
    spacing dx (m), step dt (s), nt levels."""
    nz: int
    nx: int
    dx: float
    dt: float
    nt: int
    sponge: int = 20
    vref: float = 3000.0
    refl: float = 0.05
    ny: int = 1
    ndim: int = 2

    def c(self) -> L.FwiGrid:
        return L.FwiGrid(self.ndim, self.nz, self.ny, self.nx, self.dx, self.dt, self.nt, self.sponge,
                         self.vref, self.refl)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.ndim == 3 else (self.nz, self.nx)


class Geometry:
    """fwi_geometry: src [ns,3] and rec [ns,nrec,3] int32 host arrays of
    (z, y, x) model cells, wavelet [ns, nt] float32 CUDA tensor."""

    def __init__(self, src, rec, wavelet: torch.Tensor):
        self.src = np.ascontiguousarray(src, dtype=np.int32).reshape(-1, 3)
        ns = self.src.shape[0]
        self.rec = np.ascontiguousarray(rec, dtype=np.int32).reshape(ns, -1, 3)
        if not (isinstance(wavelet, torch.Tensor) and wavelet.is_cuda and wavelet.dtype == torch.float32):
            raise TypeError("wavelet must be a float32 CUDA tensor")
        self.wavelet = wavelet.contiguous()

    @property
    def nshots(self) -> int:
        return self.src.shape[0]

    @property
    def nrec(self) -> int:
        return self.rec.shape[1]

    def c(self) -> L.FwiGeometry:
        return L.FwiGeometry(self.nshots, self.nrec, self.src.ctypes.data, self.rec.ctypes.data,
                             self.wavelet.data_ptr())

    def subset(self, s0: int, s1: int) -> "Geometry":
        """Shots [s0, s1) (the wavelet rows are a view of this geometry's)."""
        return Geometry(self.src[s0:s1], self.rec[s0:s1], self.wavelet[s0:s1])


@dataclass
class Options:
    """fwi_options: misfit 'ols' | 'integral', illum 'u2' | 'utt2', hmax
    (-1 = no offset Hessian), precond 'none' | 'illum' | 'offset', eps;
    ckpt 'sponge' | 'snapshot', snap 'f32' | 'bf16' | 'f16s', snap_interval
    (0 = ceil(sqrt(nt)))."""
    misfit: str = "ols"
    illum: str = "u2"
    hmax: int = -1
    precond: str = "illum"
    eps: float = 1e-3
    ckpt: str = "sponge"
    snap: str = "f32"
    snap_interval: int = 0
    shot_group: int = 0
    hess_v6: bool = False

    def c(self) -> L.FwiOptions:
        m = {"ols": L.FWI_MISFIT_OLS, "integral": L.FWI_MISFIT_TIME_INTEGRAL}[self.misfit]
        i = {"u2": L.FWI_ILLUM_U2, "utt2": L.FWI_ILLUM_UTT2}[self.illum]
        p = {"none": L.FWI_PRECOND_NONE, "illum": L.FWI_PRECOND_ILLUM,
             "offset": L.FWI_PRECOND_OFFSET}[self.precond]
        k = {"sponge": L.FWI_CKPT_SPONGE, "snapshot": L.FWI_CKPT_SNAPSHOT}[self.ckpt]
        sp = {"f32": L.FWI_SNAP_F32, "bf16": L.FWI_SNAP_BF16, "f16s": L.FWI_SNAP_F16S}[self.snap]
        return L.FwiOptions(m, i, int(self.hmax), p, float(self.eps), k, sp, int(self.snap_interval),
                            int(self.shot_group), int(bool(self.hess_v6)))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, name: str, shape=None, dtype=torch.float32):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def workspace_bytes(grid: Grid, geom: Geometry, opts: Options | None, op: str) -> int:
    n = ctypes.c_size_t(0)
    g, ge = grid.c(), geom.c()
    o = opts.c() if opts is not None else None
    L.check(L.load().fwi_workspace_bytes(ctypes.byref(g), ctypes.byref(ge),
                                         ctypes.byref(o) if o is not None else None,
                                         OPS[op], ctypes.byref(n)), "fwi_workspace_bytes")
    return int(n.value)


class Workspace:
    """A reusable device workspace (grows on demand)."""

    def __init__(self, device=None):
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = None
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf


def _ws(ws, nbytes):
    if ws is None:
        ws = Workspace()
    buf = ws.get(nbytes) if isinstance(ws, Workspace) else ws
    return buf, buf.numel()


def forward(grid: Grid, geom: Geometry, v: torch.Tensor, *, save=False, out=None, ws=None,
            opts: Options | None = None, stream=None) -> torch.Tensor:
    """fwi_forward: traces [ns, nt, nrec] of every shot."""
    _dev(v, "v", grid.shape)
    seis = out if out is not None else torch.empty((geom.nshots, grid.nt, geom.nrec),
                                                   dtype=torch.float32, device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "forward_save" if save else "forward"))
    g, ge = grid.c(), geom.c()
    o = opts.c() if opts is not None else None
    L.check(L.load().fwi_forward(ctypes.byref(g), ctypes.byref(ge),
                                 ctypes.byref(o) if o is not None else None, _ptr(v), _ptr(seis),
                                 int(bool(save)), _ptr(buf), nb, _stream(stream)), "fwi_forward")
    return seis


def adjoint_apply(grid: Grid, geom: Geometry, v: torch.Tensor, adj_src: torch.Tensor, ws, *,
                  out=None, opts: Options | None = None, stream=None) -> torch.Tensor:
    """fwi_adjoint_apply: gradient of <adj_src, traces> w.r.t. v, after
    forward(save=True) on the same workspace."""
    _dev(v, "v", grid.shape)
    _dev(adj_src, "adj_src", (geom.nshots, grid.nt, geom.nrec))
    grad = out if out is not None else torch.empty(grid.shape, dtype=torch.float32, device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "forward_save"))
    g, ge = grid.c(), geom.c()
    o = opts.c() if opts is not None else None
    L.check(L.load().fwi_adjoint_apply(ctypes.byref(g), ctypes.byref(ge),
                                       ctypes.byref(o) if o is not None else None, _ptr(v),
                                       _ptr(adj_src), _ptr(grad), _ptr(buf), nb, _stream(stream)),
            "fwi_adjoint_apply")
    return grad


def adjoint_gradient(grid: Grid, geom: Geometry, v: torch.Tensor, d_obs: torch.Tensor,
                     opts: Options | None = None, *, want_pre=True, want_illum=True,
                     want_offh=None, ws=None, out=None, stream=None) -> dict:
    """fwi_adjoint_gradient: the whole preconditioned gradient.
    Returns dict(grad, grad_pre?, misfit (0-d float64 CUDA tensor), illum?, offh?)."""
    opts = opts or Options()
    _dev(v, "v", grid.shape)
    _dev(d_obs, "d_obs", (geom.nshots, grid.nt, geom.nrec))
    dev = v.device
    want_offh = opts.hmax >= 0 if want_offh is None else want_offh
    o = out or {}
    res = {"grad": o.get("grad", torch.empty(grid.shape, dtype=torch.float32, device=dev)),
           "misfit": o.get("misfit", torch.zeros((), dtype=torch.float64, device=dev))}
    if want_pre:
        res["grad_pre"] = o.get("grad_pre", torch.empty(grid.shape, dtype=torch.float32, device=dev))
    if want_illum:
        res["illum"] = o.get("illum", torch.empty(grid.shape, dtype=torch.float32, device=dev))
    if want_offh:
        res["offh"] = o.get("offh", torch.empty((opts.hmax + 1,) + grid.shape, dtype=torch.float32,
                                                device=dev))
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "gradient"))
    g, ge, oc = grid.c(), geom.c(), opts.c()
    L.check(L.load().fwi_adjoint_gradient(
        ctypes.byref(g), ctypes.byref(ge), ctypes.byref(oc), _ptr(v), _ptr(d_obs), _ptr(res["grad"]),
        _ptr(res.get("grad_pre")), _ptr(res["misfit"]), _ptr(res.get("illum")), _ptr(res.get("offh")),
        _ptr(buf), nb, _stream(stream)), "fwi_adjoint_gradient")
    return res


def batch_workspace_bytes(grids, geoms, opts: Options) -> int:
    n = len(grids)
    g = (L.FwiGrid * n)(*[x.c() for x in grids])
    ge = (L.FwiGeometry * n)(*[x.c() for x in geoms])
    oc = opts.c()
    nb = ctypes.c_size_t(0)
    L.check(L.load().fwi_batch_workspace_bytes(n, g, ge, ctypes.byref(oc), ctypes.byref(nb)),
            "fwi_batch_workspace_bytes")
    return int(nb.value)


def _batch_args(grids, geoms, vs, d_obs, opts, want_pre, want_illum, want_offh):
    """Output tensors and ctypes arrays of a call over several models."""
    n = len(grids)
    if not (len(geoms) == len(vs) == len(d_obs) == n):
        raise ValueError("grids, geoms, vs and d_obs must have the same length")
    want_offh = opts.hmax >= 0 if want_offh is None else want_offh
    res = []
    for g, ge, v, d in zip(grids, geoms, vs, d_obs):
        _dev(v, "v", g.shape)
        _dev(d, "d_obs", (ge.nshots, g.nt, ge.nrec))
        r = {"grad": torch.empty(g.shape, dtype=torch.float32, device=v.device)}
        if want_pre:
            r["grad_pre"] = torch.empty(g.shape, dtype=torch.float32, device=v.device)
        if want_illum:
            r["illum"] = torch.empty(g.shape, dtype=torch.float32, device=v.device)
        if want_offh:
            r["offh"] = torch.empty((opts.hmax + 1,) + g.shape, dtype=torch.float32, device=v.device)
        res.append(r)
    misfit = torch.zeros(n, dtype=torch.float64, device=vs[0].device)
    for k, r in enumerate(res):
        r["misfit"] = misfit[k]

    def ptrs(key=None, src=None):
        vals = [t.data_ptr() for t in src] if src is not None else [r[key].data_ptr() if key in r else None
                                                                     for r in res]
        return (ctypes.c_void_p * n)(*vals)

    c = {"g": (L.FwiGrid * n)(*[x.c() for x in grids]), "ge": (L.FwiGeometry * n)(*[x.c() for x in geoms]),
         "o": opts.c(), "v": ptrs(src=vs), "d": ptrs(src=d_obs), "grad": ptrs("grad"),
         "pre": ptrs("grad_pre") if want_pre else None, "ill": ptrs("illum") if want_illum else None,
         "off": ptrs("offh") if want_offh else None, "misfit": misfit}
    return res, c


def batch_gradient(grids, geoms, vs, d_obs, opts: Options | None = None, *, want_pre=True,
                   want_illum=True, want_offh=None, ws=None, stream=None) -> list:
    """fwi_batch_gradient: the gradients of several independent models of
    different sizes (same nt), every time level of all models in one launch.
    Returns one dict per model, as adjoint_gradient."""
    opts = opts or Options()
    res, c = _batch_args(grids, geoms, vs, d_obs, opts, want_pre, want_illum, want_offh)
    buf, nb = _ws(ws, batch_workspace_bytes(grids, geoms, opts))
    L.check(L.load().fwi_batch_gradient(len(grids), c["g"], c["ge"], ctypes.byref(c["o"]), c["v"], c["d"],
                                        c["grad"], c["pre"], _ptr(c["misfit"]), c["ill"], c["off"], _ptr(buf),
                                        nb, _stream(stream)), "fwi_batch_gradient")
    return res


class GradientGraph:
    """fwi_exec: the gradient of one or several models recorded once as a CUDA
    graph, bound to fixed buffers, and replayed by run(). Inputs: the tensors
    `vs` and `d_obs` given here (update them in place between runs). Outputs:
    the same dicts, rewritten by every run. The graph runs on its own stream,
    ordered after the caller's current stream and before its next work."""

    def __init__(self, grids, geoms, vs, d_obs, opts: Options | None = None, *, want_pre=True,
                 want_illum=True, want_offh=None, ws=None):
        opts = opts or Options()
        self.inputs = (list(vs), list(d_obs))
        self.results, c = _batch_args(grids, geoms, vs, d_obs, opts, want_pre, want_illum, want_offh)
        self._c = c  # keep the ctypes arrays alive with the graph
        self.buf, nb = _ws(ws, batch_workspace_bytes(grids, geoms, opts))
        self.stream = torch.cuda.Stream(device=vs[0].device)
        self.stream.wait_stream(torch.cuda.current_stream())
        h = ctypes.c_void_p(0)
        L.check(L.load().fwi_exec_gradient_create(len(grids), c["g"], c["ge"], ctypes.byref(c["o"]), c["v"],
                                                  c["d"], c["grad"], c["pre"], _ptr(c["misfit"]), c["ill"],
                                                  c["off"], _ptr(self.buf), nb, _stream(self.stream),
                                                  ctypes.byref(h)), "fwi_exec_gradient_create")
        self._h = h

    def run(self, d_obs_ready=None) -> list:
        """Replay the gradient. d_obs_ready: a stream on which the observed
        traces are being written (e.g. copied from the host): the forward pass
        starts at once and the misfit waits for that stream's work queued so
        far (fwi_exec_input_ready), so the upload overlaps the forward pass;
        later work on that stream is ordered after this run."""
        if not self._h:
            raise RuntimeError("the graph was closed")
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        if d_obs_ready is not None:
            L.check(L.load().fwi_exec_input_ready(self._h, _stream(d_obs_ready)), "fwi_exec_input_ready")
        L.check(L.load().fwi_exec_run(self._h, _stream(self.stream)), "fwi_exec_run")
        cur.wait_stream(self.stream)
        if d_obs_ready is not None:
            d_obs_ready.wait_stream(self.stream)
        return self.results

    def close(self):
        if self._h:
            L.load().fwi_exec_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def illumination(grid: Grid, geom: Geometry, v: torch.Tensor, opts: Options | None = None, *,
                 ws=None, stream=None) -> torch.Tensor:
    """fwi_illumination: sum_s sum_n u^2 dt (or u_tt^2 dt), [nz, nx]."""
    opts = opts or Options()
    _dev(v, "v", grid.shape)
    out = torch.empty(grid.shape, dtype=torch.float32, device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "illumination"))
    g, ge, oc = grid.c(), geom.c(), opts.c()
    L.check(L.load().fwi_illumination(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(oc), _ptr(v),
                                      _ptr(out), _ptr(buf), nb, _stream(stream)), "fwi_illumination")
    return out


def misfit(grid: Grid, geom: Geometry, v: torch.Tensor, d_obs: torch.Tensor, opts: Options | None = None, *,
           ws=None, out=None, stream=None) -> torch.Tensor:
    """fwi_misfit: the misfit J (0-d float64 CUDA tensor) of v against d_obs,
    forward modelling only (OLS, or Eq. 2 with misfit="integral")."""
    _dev(v, "v", grid.shape)
    _dev(d_obs, "d_obs", (geom.nshots, grid.nt, geom.nrec))
    J = out if out is not None else torch.zeros((), dtype=torch.float64, device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "misfit"))
    g, ge = grid.c(), geom.c()
    o = opts.c() if opts is not None else None
    L.check(L.load().fwi_misfit(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(o) if o is not None else None,
                                _ptr(v), _ptr(d_obs), _ptr(J), _ptr(buf), nb, _stream(stream)), "fwi_misfit")
    return J


def extended_born(grid: Grid, geom: Geometry, v: torch.Tensor, dv_ext: torch.Tensor, *, ws=None, out=None,
                  stream=None) -> torch.Tensor:
    """fwi_extended_born (Eq. 5): traces [ns, nt, nrec] of the extended
    perturbation dv_ext [2 hext + 1, nz, nx] (plane k: offset k - hext)."""
    _dev(v, "v", grid.shape)
    hext = (dv_ext.shape[0] - 1) // 2
    _dev(dv_ext, "dv_ext", (2 * hext + 1,) + grid.shape)
    d = out if out is not None else torch.empty((geom.nshots, grid.nt, geom.nrec), dtype=torch.float32,
                                                device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, None, "extended_born"))
    g, ge = grid.c(), geom.c()
    L.check(L.load().fwi_extended_born(ctypes.byref(g), ctypes.byref(ge), None, int(hext), _ptr(v), _ptr(dv_ext),
                                       _ptr(d), _ptr(buf), nb, _stream(stream)), "fwi_extended_born")
    return d


def extended_migration(grid: Grid, geom: Geometry, v: torch.Tensor, adj_src: torch.Tensor, hext: int, *, ws=None,
                       out=None, stream=None) -> torch.Tensor:
    """fwi_extended_migration (Eq. 6): the image [2 hext + 1, nz, nx] of the
    adjoint source adj_src [ns, nt, nrec] (plane k: offset k - hext)."""
    _dev(v, "v", grid.shape)
    _dev(adj_src, "adj_src", (geom.nshots, grid.nt, geom.nrec))
    img = out if out is not None else torch.empty((2 * hext + 1,) + grid.shape, dtype=torch.float32,
                                                  device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, None, "extended_migration"))
    g, ge = grid.c(), geom.c()
    L.check(L.load().fwi_extended_migration(ctypes.byref(g), ctypes.byref(ge), None, int(hext), _ptr(v),
                                            _ptr(adj_src), _ptr(img), _ptr(buf), nb, _stream(stream)),
            "fwi_extended_migration")
    return img


def selftest_wait(limit_us: int = 1000, stream=None) -> int:
    """fwi_selftest_wait: one warp's bounded wait on an mbarrier nothing
    arrives at. Returns the status code, FWI_ERR_TIMEOUT when the mechanism
    works (the wait gave up, the kernel reported it, the context is usable)."""
    buf = torch.empty(256, dtype=torch.uint8, device="cuda")
    return int(L.load().fwi_selftest_wait(int(limit_us), _ptr(buf), 256, _stream(stream)))


def born(grid: Grid, geom: Geometry, v: torch.Tensor, dv: torch.Tensor, *, ws=None, out=None,
         stream=None) -> torch.Tensor:
    """fwi_born: Born traces J dv [ns, nt, nrec], the derivative of the
    traces along the velocity change dv (Eq. 4)."""
    _dev(v, "v", grid.shape)
    _dev(dv, "dv", grid.shape)
    d = out if out is not None else torch.empty((geom.nshots, grid.nt, geom.nrec), dtype=torch.float32,
                                                device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, None, "born"))
    g, ge = grid.c(), geom.c()
    L.check(L.load().fwi_born(ctypes.byref(g), ctypes.byref(ge), None, _ptr(v), _ptr(dv), _ptr(d), _ptr(buf),
                              nb, _stream(stream)), "fwi_born")
    return d


def gauss_newton_hvp(grid: Grid, geom: Geometry, v: torch.Tensor, dv: torch.Tensor, opts: Options | None = None,
                     *, ws=None, out=None, stream=None) -> torch.Tensor:
    """fwi_gauss_newton_hvp: J^T W^T W J dv [nz, nx], the Gauss-Newton
    Hessian of the misfit applied to dv (Born modelling, then adjoint imaging
    of the weighted Born traces; W = I for the OLS misfit, the time integral
    for misfit="integral")."""
    _dev(v, "v", grid.shape)
    _dev(dv, "dv", grid.shape)
    hv = out if out is not None else torch.empty(grid.shape, dtype=torch.float32, device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "gn_hvp"))
    g, ge = grid.c(), geom.c()
    o = opts.c() if opts is not None else None
    L.check(L.load().fwi_gauss_newton_hvp(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(o) if o is not None else None,
                                          _ptr(v), _ptr(dv), _ptr(hv), _ptr(buf), nb, _stream(stream)),
            "fwi_gauss_newton_hvp")
    return hv


def offset_hessian_diag(grid: Grid, geom: Geometry, v: torch.Tensor, opts: Options, *, ws=None,
                        stream=None) -> torch.Tensor:
    """fwi_offset_hessian_diag: [hmax+1, nz, nx] (3-D: [hmax+1, nz, ny, nx]) source-side
    offset-Hessian diagonal, offsets along x."""
    _dev(v, "v", grid.shape)
    out = torch.empty((opts.hmax + 1,) + grid.shape, dtype=torch.float32, device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "offset_hessian"))
    g, ge, oc = grid.c(), geom.c(), opts.c()
    L.check(L.load().fwi_offset_hessian_diag(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(oc),
                                             _ptr(v), _ptr(out), _ptr(buf), nb, _stream(stream)),
            "fwi_offset_hessian_diag")
    return out


def precondition(grid: Grid, grad: torch.Tensor, scale: torch.Tensor, kind: str, eps=1e-3, *,
                 ws=None, stream=None) -> torch.Tensor:
    """fwi_precondition: grad / (P + eps max P), kind 'illum' or 'offset'."""
    _dev(grad, "grad", grid.shape)
    k = {"illum": L.FWI_PRECOND_ILLUM, "offset": L.FWI_PRECOND_OFFSET}[kind]
    hmax = scale.shape[0] - 1 if kind == "offset" else 0
    _dev(scale, "scale", grid.shape if kind == "illum" else (hmax + 1,) + grid.shape)
    out = torch.empty_like(grad)
    g = grid.c()
    nbytes = ctypes.c_size_t(0)
    L.check(L.load().fwi_workspace_bytes(ctypes.byref(g), None, None, L.FWI_OP_PRECONDITION,
                                         ctypes.byref(nbytes)), "fwi_workspace_bytes")
    buf, nb = _ws(ws, int(nbytes.value))
    L.check(L.load().fwi_precondition(ctypes.byref(g), _ptr(grad), _ptr(scale), k, hmax, float(eps),
                                      _ptr(out), _ptr(buf), nb, _stream(stream)), "fwi_precondition")
    return out


def receiver_factor(grid: Grid, geom: Geometry, kind: str = "pm", v: torch.Tensor | None = None,
                    opts: Options | None = None, *, ws=None, stream=None) -> torch.Tensor:
    """fwi_receiver_factor for a fixed receiver spread: kind "pm" (Plessix
    and Mulder's asinh factor, [nz, nx]) or "green" (receiver Green's-function
    correlations in v, [max(hmax, 0) + 1, nz, nx] with hmax = opts.hmax)."""
    g, ge = grid.c(), geom.c()
    o = opts.c() if opts is not None else None
    lib = L.load()
    if kind == "pm":
        out = torch.empty(grid.shape, dtype=torch.float32, device=geom.wavelet.device)
        L.check(lib.fwi_receiver_factor(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(o) if o is not None else None,
                                        L.FWI_RECV_PLESSIX_MULDER, None, _ptr(out), None, 0, _stream(stream)),
                "fwi_receiver_factor")
        return out
    if kind != "green":
        raise ValueError(kind)
    _dev(v, "v", grid.shape)
    h = max(opts.hmax, 0) if opts is not None else 0
    out = torch.empty((h + 1,) + grid.shape, dtype=torch.float32, device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "receiver_factor"))
    L.check(lib.fwi_receiver_factor(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(o) if o is not None else None,
                                    L.FWI_RECV_GREEN, _ptr(v), _ptr(out), _ptr(buf), nb, _stream(stream)),
            "fwi_receiver_factor")
    return out


def plessix_mulder_hessian(grid: Grid, geom: Geometry, v: torch.Tensor, opts: Options | None = None, *,
                           ws=None, stream=None) -> torch.Tensor:
    """fwi_plessix_mulder_hessian: sum_s W_s(x) I_s(x) [nz, nx], each shot's
    illumination weighted by the asinh factor of its own receiver spread
    (any acquisition; runs of shots with one spread share a pass)."""
    _dev(v, "v", grid.shape)
    out = torch.empty(grid.shape, dtype=torch.float32, device=v.device)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "pm_hessian"))
    g, ge = grid.c(), geom.c()
    o = opts.c() if opts is not None else None
    L.check(L.load().fwi_plessix_mulder_hessian(ctypes.byref(g), ctypes.byref(ge),
                                                ctypes.byref(o) if o is not None else None, _ptr(v), _ptr(out),
                                                _ptr(buf), nb, _stream(stream)), "fwi_plessix_mulder_hessian")
    return out


def precondition_receiver(grid: Grid, grad: torch.Tensor, scale: torch.Tensor, kind: str, recv: torch.Tensor,
                          eps=1e-3, *, ws=None, stream=None) -> torch.Tensor:
    """fwi_precondition_receiver: grad / (P + eps max P) with P = scale x recv
    (kind 'illum': [nz, nx] scale; 'offset': [hmax+1, nz, nx], summed over
    offsets as fwi_precondition does). recv: [nz, nx] (one factor for every
    offset) or [k, nz, nx], k = 1 or >= hmax + 1."""
    _dev(grad, "grad", grid.shape)
    k = {"illum": L.FWI_PRECOND_ILLUM, "offset": L.FWI_PRECOND_OFFSET}[kind]
    hmax = scale.shape[0] - 1 if kind == "offset" else 0
    _dev(scale, "scale", grid.shape if kind == "illum" else (hmax + 1,) + grid.shape)
    rp = 1 if recv.dim() == 2 else recv.shape[0]
    _dev(recv, "recv", grid.shape if recv.dim() == 2 else (rp,) + grid.shape)
    out = torch.empty_like(grad)
    g = grid.c()
    nbytes = ctypes.c_size_t(0)
    L.check(L.load().fwi_workspace_bytes(ctypes.byref(g), None, None, L.FWI_OP_PRECONDITION_RECEIVER,
                                         ctypes.byref(nbytes)), "fwi_workspace_bytes")
    buf, nb = _ws(ws, int(nbytes.value))
    L.check(L.load().fwi_precondition_receiver(ctypes.byref(g), _ptr(grad), _ptr(scale), k, hmax, _ptr(recv), rp,
                                               float(eps), _ptr(out), _ptr(buf), nb, _stream(stream)),
            "fwi_precondition_receiver")
    return out


def autotune(grid: Grid, geom: Geometry, v: torch.Tensor, opts: Options | None = None, *, ws=None,
             stream=None) -> dict:
    """fwi_autotune: time the compiled tile variants and chunk sizes of this
    problem's forward and backward steps and keep the fastest for later calls
    of the same shape. Returns the choice."""
    opts = opts or Options()
    _dev(v, "v", grid.shape)
    buf, nb = _ws(ws, workspace_bytes(grid, geom, opts, "gradient"))
    g, ge, oc = grid.c(), geom.c(), opts.c()
    ch = (ctypes.c_int * 4)()
    L.check(L.load().fwi_autotune(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(oc), _ptr(v), _ptr(buf), nb,
                                  _stream(stream), ch), "fwi_autotune")
    return {"forward_variant": ch[0], "forward_chunk": ch[1], "backward_variant": ch[2], "backward_chunk": ch[3]}


def autotune_set(grid: Grid, geom: Geometry, opts: Options | None, choice: dict):
    """fwi_autotune_set: keep this choice (as returned by autotune) for the shape."""
    opts = opts or Options()
    g, ge, oc = grid.c(), geom.c(), opts.c()
    ch = (ctypes.c_int * 4)(choice["forward_variant"], choice["forward_chunk"], choice["backward_variant"],
                            choice["backward_chunk"])
    L.check(L.load().fwi_autotune_set(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(oc), ch),
            "fwi_autotune_set")


def autotune_reset():
    L.check(L.load().fwi_autotune_reset(), "fwi_autotune_reset")


def profile(on: bool = True):
    L.check(L.load().fwi_profile_enable(int(on)), "fwi_profile_enable")


def last_phase_times() -> dict:
    t = L.FwiPhaseTimes()
    L.check(L.load().fwi_profile_last(ctypes.byref(t)), "fwi_profile_last")
    return {k: getattr(t, k) for k, _ in L.FwiPhaseTimes._fields_}


# ------------------------------------------------------------------ conveniences

def from_problem(prob, device="cuda"):
    """(Grid, Geometry) of a workloads.Problem, the wavelet uploaded to the GPU."""
    grid = Grid(prob.nz, prob.nx, float(prob.dx), float(prob.dt), int(prob.nt), int(prob.sponge),
                float(prob.vref), float(prob.refl), ny=int(prob.ny), ndim=int(prob.ndim))
    wav = torch.as_tensor(np.ascontiguousarray(prob.wavelet, dtype=np.float32), device=device)
    return grid, Geometry(prob.src, prob.rec, wav)
