"""Outer inversion loops on top of the preconditioned gradient.

The paper inverts with L-BFGS (its first example, 200 iterations) and with
Polak-Ribiere conjugate gradients (PRCG, its second example, 270 iterations),
each steered by a diagonal preconditioner: the illumination of Eq. 1 or the
offset-Hessian diagonal of Sec. 3. This module implements both loops over an
objective that supplies the misfit, its gradient and the preconditioner:

* PRCG (preconditioned nonlinear CG): d_k = -M^-1 g_k + beta_k d_{k-1},
  beta_k = max(0, <g_k - g_{k-1}, M^-1 g_k> / <g_{k-1}, M^-1 g_{k-1}>)
  (Polak-Ribiere with restart), reset to -M^-1 g_k when d_k is not a descent
  direction or its line search fails (both methods stop when the line search
  along -M^-1 g_k fails too).
* L-BFGS: the two-loop recursion over the last m pairs s = x_{k+1} - x_k,
  y = g_{k+1} - g_k (pairs with <s, y> <= 0 are skipped), with the diagonal
  preconditioner as the initial inverse Hessian, H_0 = gamma M^-1,
  gamma = <s, y> / <y, M^-1 y> of the newest pair.
* Truncated Gauss-Newton: each outer step solves H dv = -g approximately,
  H the Gauss-Newton Hessian J^T W^T W J (fwi_gauss_newton_hvp), by CG
  preconditioned with M (at most cg_iters products, until the residual is
  cg_tol of the gradient, stopping at non-positive curvature), then searches
  along dv from the unit step.
* Line search: projected backtracking on the Armijo condition
  f(x + a d) <= f(x) + c1 a <g, d>, with parabolic steps (the minimum of the
  parabola through f(x), its slope and the last trial, kept within [0.1, 0.5]
  of the last step) and one parabolic extrapolation when the first trial is
  accepted. The first trial step of the first iteration moves the model by
  at most `max_update` (m/s); later L-BFGS iterations try the unit step (the
  curvature pairs scale the direction) unless it moves the model by more than
  10 max_update, later PRCG iterations the previous
  step times <g_{k-1}, d_{k-1}> / <g_k, d_k> (the same first-order change),
  kept within [0.1, 10] times the max_update step. Models are projected onto
  [vmin, vmax] after every step.

FwiObjective binds the library's gradient (fwi_adjoint_gradient, with the
misfit, illumination and offset Hessian of the same call), its misfit-only
forward pass (fwi_misfit) for the trial steps, and fwi_precondition as M^-1.
An optional mute (a 0/1 diagonal, applied on both sides of the diagonal
preconditioner, so M^-1 stays symmetric positive semi-definite) keeps rows
near the sources and receivers fixed, where the gradient carries the
acquisition footprint. Every vector operation is a torch operation on the
model's device.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np
import torch


@dataclass
class Evaluation:
    """The objective at one model: misfit f, gradient g and the inverse
    preconditioner minv (a function applying M^-1 to a model-shaped tensor)."""
    f: float
    g: torch.Tensor
    minv: Callable[[torch.Tensor], torch.Tensor]


@dataclass
class History:
    """Per iteration: misfit (before the first and after every step), step
    length, misfit evaluations of the line search, model error (when the
    true model is known); totals: restarts, Hessian-vector products (Gauss-
    Newton), gradient and misfit calls of the objective."""
    misfit: list = field(default_factory=list)
    step: list = field(default_factory=list)
    evals: list = field(default_factory=list)
    model_error: list = field(default_factory=list)
    restarts: int = 0
    hvps: int = 0
    n_gradients: int = 0
    n_misfits: int = 0
    n_hvps: int = 0


def _dot(a, b) -> float:
    return float(torch.sum(a.double() * b.double()))


def armijo_parabolic(value, x, f0, g, d, alpha0, project, c1=1e-4, max_trials=10, extrapolate=True,
                     max_expand=4):
    """Projected backtracking line search on the Armijo condition with
    parabolic steps. value(x) -> f. When the first trial is accepted, the step
    is extended while the misfit keeps falling (at most max_expand times): to
    the parabola's minimum (at most 4x) where the line is convex, to twice the
    step where it is not (a decrease beyond the linear prediction). Returns
    (alpha, x_new, f_new, trials); alpha = 0 when no trial decreased the
    misfit enough."""
    slope = _dot(g, d)
    alpha, trials = alpha0, 0
    best = None
    while trials < max_trials:
        xt = project(x + alpha * d)
        ft = value(xt)
        trials += 1
        if ft <= f0 + c1 * alpha * slope:
            best = (alpha, xt, ft)
            break
        # minimiser of the parabola through (0, f0) with slope `slope` and (alpha, ft)
        den = 2.0 * (ft - f0 - slope * alpha)
        a_new = -slope * alpha * alpha / den if den > 0 else 0.5 * alpha
        alpha = min(max(a_new, 0.1 * alpha), 0.5 * alpha)
    if best is None:
        return 0.0, x, f0, trials
    alpha, xt, ft = best
    if extrapolate and trials == 1:
        for _ in range(max_expand):
            if trials >= max_trials:
                break
            den = 2.0 * (ft - f0 - slope * alpha)
            if den > 0:
                a_p = min(-slope * alpha * alpha / den, 4.0 * alpha)
                if a_p <= 1.2 * alpha:
                    break
            else:
                a_p = 2.0 * alpha
            xp = project(x + a_p * d)
            fp = value(xp)
            trials += 1
            if fp >= ft:
                break
            alpha, xt, ft = a_p, xp, fp
    return alpha, xt, ft, trials


class _Base:
    def __init__(self, value_grad, value, *, max_update, project=None, line_search=None, callback=None):
        self.value_grad = value_grad
        self.value = value
        self.max_update = float(max_update)
        self.project = project or (lambda x: x)
        self.line_search = line_search
        self.callback = callback

    def _first_alpha(self, d):
        m = float(d.abs().max())
        return self.max_update / m if m > 0 else 0.0

    def _search(self, x, ev, d, alpha0):
        if self.line_search is not None:
            return self.line_search(self.value, x, ev.f, ev.g, d, alpha0, self.project)
        return armijo_parabolic(self.value, x, ev.f, ev.g, d, alpha0, self.project)


class PRCG(_Base):
    """Preconditioned Polak-Ribiere conjugate gradients (PR+, restarted when
    the direction is not a descent direction)."""

    def run(self, x, iters, hist: History | None = None):
        hist = hist or History()
        ev = self.value_grad(x)
        hist.misfit.append(ev.f)
        pg = ev.minv(ev.g)
        d = -pg
        gpg_prev = _dot(ev.g, pg)
        g_prev = ev.g
        alpha, gd_prev = 0.0, 0.0
        for k in range(iters):
            gd = _dot(ev.g, d)
            if gd >= 0:
                d = -pg
                gd = -_dot(ev.g, pg)
                hist.restarts += 1
            a_cap = self._first_alpha(d)
            alpha0 = a_cap if alpha == 0.0 else min(max(alpha * gd_prev / gd, 0.1 * a_cap), 10.0 * a_cap)
            gd_prev = gd
            alpha, x_new, f_new, trials = self._search(x, ev, d, alpha0)
            if alpha == 0.0 and not torch.equal(d, -pg):
                # restart along the preconditioned steepest-descent direction
                d = -pg
                gd_prev = -_dot(ev.g, pg)
                hist.restarts += 1
                alpha, x_new, f_new, t2 = self._search(x, ev, d, self._first_alpha(d))
                trials += t2
            hist.step.append(alpha)
            hist.evals.append(trials)
            if alpha == 0.0:
                break
            x = x_new
            ev = self.value_grad(x)
            hist.misfit.append(ev.f)
            if self.callback:
                self.callback(k, x, ev, hist)
            pg = ev.minv(ev.g)
            gpg = _dot(ev.g, pg)
            beta = max(0.0, (gpg - _dot(g_prev, pg)) / gpg_prev) if gpg_prev > 0 else 0.0
            d = -pg + beta * d
            g_prev, gpg_prev = ev.g, gpg
        return x, hist


class LBFGS(_Base):
    """Limited-memory BFGS with the diagonal preconditioner as H_0."""

    def __init__(self, value_grad, value, *, max_update, memory=5, scale_h0=True, **kw):
        super().__init__(value_grad, value, max_update=max_update, **kw)
        self.memory = int(memory)
        self.scale_h0 = scale_h0

    def direction(self, g, minv, pairs):
        q = g.clone()
        alphas = []
        for s, y, rho in reversed(pairs):
            a = rho * _dot(s, q)
            alphas.append(a)
            q = q - a * y
        r = minv(q)
        if pairs and self.scale_h0:
            s, y, _ = pairs[-1]
            yMy = _dot(y, minv(y))
            if yMy > 0:
                r = r * (_dot(s, y) / yMy)
        for (s, y, rho), a in zip(pairs, reversed(alphas)):
            b = rho * _dot(y, r)
            r = r + (a - b) * s
        return -r

    def run(self, x, iters, hist: History | None = None):
        hist = hist or History()
        ev = self.value_grad(x)
        hist.misfit.append(ev.f)
        pairs = []
        for k in range(iters):
            d = self.direction(ev.g, ev.minv, pairs)
            if _dot(ev.g, d) >= 0:
                d = -ev.minv(ev.g)
                pairs = []
                hist.restarts += 1
            alpha0 = self._first_alpha(d) if not pairs else min(1.0, 10.0 * self._first_alpha(d))
            alpha, x_new, f_new, trials = self._search(x, ev, d, alpha0)
            if alpha == 0.0 and pairs:
                # drop the memory and search along -M^-1 g
                d = -ev.minv(ev.g)
                pairs = []
                hist.restarts += 1
                alpha, x_new, f_new, t2 = self._search(x, ev, d, self._first_alpha(d))
                trials += t2
            hist.step.append(alpha)
            hist.evals.append(trials)
            if alpha == 0.0:
                break
            ev_new = self.value_grad(x_new)
            s, y = x_new - x, ev_new.g - ev.g
            sy = _dot(s, y)
            if sy > 0:
                pairs.append((s, y, 1.0 / sy))
                pairs = pairs[-self.memory:]
            x, ev = x_new, ev_new
            hist.misfit.append(ev.f)
            if self.callback:
                self.callback(k, x, ev, hist)
        return x, hist


class GaussNewton(_Base):
    """Truncated Gauss-Newton with a preconditioned CG inner solve. hvp(x, p)
    applies the Gauss-Newton Hessian at x to p."""

    def __init__(self, value_grad, value, hvp, *, max_update, cg_iters=5, cg_tol=0.1, **kw):
        super().__init__(value_grad, value, max_update=max_update, **kw)
        self.hvp = hvp
        self.cg_iters = int(cg_iters)
        self.cg_tol = float(cg_tol)

    def solve(self, x, g, minv):
        """Preconditioned CG on H d = -g from d = 0. Returns (d, products)."""
        d = torch.zeros_like(g)
        r = -g
        z = minv(r)
        p = z
        rz = _dot(r, z)
        gnorm = float(torch.linalg.vector_norm(g.double()))
        n = 0
        for _ in range(self.cg_iters):
            Hp = self.hvp(x, p)
            n += 1
            pHp = _dot(p, Hp)
            if pHp <= 0:
                break
            a = rz / pHp
            d = d + a * p
            r = r - a * Hp
            if float(torch.linalg.vector_norm(r.double())) <= self.cg_tol * gnorm:
                break
            z = minv(r)
            rz_new = _dot(r, z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        if not bool(d.any()):
            d = minv(-g)
        return d, n

    def run(self, x, iters, hist: History | None = None):
        hist = hist or History()
        ev = self.value_grad(x)
        hist.misfit.append(ev.f)
        for k in range(iters):
            d, n = self.solve(x, ev.g, ev.minv)
            hist.hvps += n
            if _dot(ev.g, d) >= 0:
                d = -ev.minv(ev.g)
                hist.restarts += 1
            alpha, x_new, f_new, trials = self._search(x, ev, d, min(1.0, 10.0 * self._first_alpha(d)))
            if alpha == 0.0:
                d = -ev.minv(ev.g)
                hist.restarts += 1
                alpha, x_new, f_new, t2 = self._search(x, ev, d, self._first_alpha(d))
                trials += t2
            hist.step.append(alpha)
            hist.evals.append(trials)
            if alpha == 0.0:
                break
            x = x_new
            ev = self.value_grad(x)
            hist.misfit.append(ev.f)
            if self.callback:
                self.callback(k, x, ev, hist)
        return x, hist


class FwiObjective:
    """The FWI misfit of the library: value_grad(v) runs fwi_adjoint_gradient
    (misfit, gradient and the chosen preconditioner's scale in one call),
    value(v) runs fwi_misfit. The inverse preconditioner divides by the
    call's scale as fwi_precondition does (precond "illum": the illumination
    of Eq. 1; "offset": the offset-Hessian diagonal of Sec. 3; "none").
    receiver = "pm" or "green" multiplies the scale by the receiver side of
    the diagonal Hessian (fwi_receiver_factor): Plessix and Mulder's factor
    (computed once for a fixed spread; for a spread that moves with the shots
    the scale is fwi_plessix_mulder_hessian's per-shot sum instead, with
    precond "illum"), or the receiver Green's-function correlations of a
    fixed spread in the current model. Model-dependent receiver terms are
    recomputed every receiver_every gradients."""

    def __init__(self, grid, geom, d_obs, opts, ws=None, mute_top=0, receiver=None, receiver_every=1):
        from . import fwi
        self.fwi = fwi
        self.grid, self.geom, self.d_obs, self.opts = grid, geom, d_obs, opts
        self.ws = ws if ws is not None else fwi.Workspace()
        if receiver not in (None, "pm", "green"):
            raise ValueError(receiver)
        if receiver is not None and opts.precond == "none":
            raise ValueError("a receiver factor needs precond 'illum' or 'offset'")
        self.receiver, self.receiver_every = receiver, max(1, int(receiver_every))
        self.n_hvps = 0
        self.fixed_spread = bool((geom.rec == geom.rec[:1]).all())
        if receiver == "pm" and not self.fixed_spread and opts.precond != "illum":
            raise ValueError("Plessix-Mulder with a moving spread needs precond 'illum'")
        self.recv = fwi.receiver_factor(grid, geom, "pm") if receiver == "pm" and self.fixed_spread else None
        self.pm_scale = None
        self.mask = None
        if mute_top > 0:
            self.mask = torch.ones(grid.shape, dtype=torch.float32, device=d_obs.device)
            self.mask[:mute_top] = 0.0
        self.n_gradients = 0
        self.n_misfits = 0

    def hvp(self, v, p):
        """The Gauss-Newton Hessian of the misfit at v applied to p
        (fwi_gauss_newton_hvp), restricted to the unmuted rows."""
        self.n_hvps += 1
        fwi = self.fwi
        q = p * self.mask if self.mask is not None else p
        hv = fwi.gauss_newton_hvp(self.grid, self.geom, v.contiguous(), q.contiguous(),
                                  fwi.Options(misfit=self.opts.misfit), ws=self.ws)
        return hv * self.mask if self.mask is not None else hv

    def value(self, v):
        self.n_misfits += 1
        return float(self.fwi.misfit(self.grid, self.geom, v.contiguous(), self.d_obs, self.opts, ws=self.ws))

    def value_grad(self, v):
        fwi = self.fwi
        self.n_gradients += 1
        o = self.opts
        r = fwi.adjoint_gradient(self.grid, self.geom, v.contiguous(), self.d_obs, o, want_pre=False,
                                 want_illum=o.precond == "illum", want_offh=o.precond == "offset", ws=self.ws)
        grid, mask = self.grid, self.mask
        if o.precond == "illum":
            scale, kind = r["illum"], "illum"
        elif o.precond == "offset":
            scale, kind = r["offh"], "offset"
        else:
            scale, kind = None, None

        refresh = (self.n_gradients - 1) % self.receiver_every == 0
        if self.receiver == "green" and (self.recv is None or refresh):
            self.recv = fwi.receiver_factor(grid, self.geom, "green", v.contiguous(), o, ws=self.ws)
        if self.receiver == "pm" and not self.fixed_spread:
            if self.pm_scale is None or refresh:
                self.pm_scale = fwi.plessix_mulder_hessian(grid, self.geom, v.contiguous(), o, ws=self.ws)
            scale = self.pm_scale
        recv = self.recv

        def minv(q):
            if mask is not None:
                q = q * mask
            if kind is not None and recv is not None:
                q = fwi.precondition_receiver(grid, q.contiguous(), scale, kind, recv, eps=o.eps, ws=self.ws)
            elif kind is not None:
                q = fwi.precondition(grid, q.contiguous(), scale, kind, eps=o.eps, ws=self.ws)
            return q * mask if mask is not None else q
        return Evaluation(float(r["misfit"]), r["grad"], minv)


def velocity_bounds(grid, v0, vmin=None, vmax=None, cfl_margin=0.98):
    """[vmin, vmax] for the projection: by default half the smallest and 1.5x
    the largest starting velocity, vmax capped below the stability limit
    v dt / dx <= FWI_CFL_LIMIT_2D (or _3D) and below the grid's vref (the
    sponge is designed for velocities up to vref)."""
    from . import _lib as L
    lim = L.FWI_CFL_LIMIT_3D if getattr(grid, "ndim", 2) == 3 else L.FWI_CFL_LIMIT_2D
    cap = min(cfl_margin * lim * grid.dx / grid.dt, float(grid.vref))
    lo = 0.5 * float(v0.min()) if vmin is None else float(vmin)
    hi = min(1.5 * float(v0.max()), cap) if vmax is None else min(float(vmax), cap)
    # float32 values inside [lo, hi]: a float32 clamp to them stays within
    lo32, hi32 = np.float32(lo), np.float32(hi)
    if float(lo32) < lo:
        lo32 = np.nextafter(lo32, np.float32(np.inf))
    if float(hi32) > hi:
        hi32 = np.nextafter(hi32, np.float32(0))
    return float(lo32), float(hi32)


def default_mute(geom):
    """Rows kept fixed by default: down to two cells below the deepest
    source or receiver."""
    z = [int(geom.src[:, 0].max())]
    if geom.nrec > 0:
        z.append(int(geom.rec[..., 0].max()))
    return max(z) + 3


def invert(grid, geom, d_obs, v0, opts, *, method="lbfgs", iters=10, max_update=50.0, memory=5, vmin=None,
           vmax=None, v_true=None, mute_top=None, receiver=None, receiver_every=1, cg_iters=5, cg_tol=0.1,
           ws=None):
    """Run `iters` iterations of L-BFGS, PRCG or truncated Gauss-Newton
    (method "lbfgs", "prcg", "gauss_newton") from v0 with the library's
    gradient and preconditioner (opts.precond), the rows above mute_top fixed
    (None: default_mute(geom); 0: none). Returns (v, History); with v_true,
    History.model_error holds ||v_k - v_true|| / ||v_0 - v_true||."""
    mute = default_mute(geom) if mute_top is None else int(mute_top)
    obj = FwiObjective(grid, geom, d_obs, opts, ws=ws, mute_top=mute, receiver=receiver,
                       receiver_every=receiver_every)
    lo, hi = velocity_bounds(grid, v0, vmin, vmax)
    hist = History()
    e0 = float(torch.linalg.vector_norm((v0 - v_true).double())) if v_true is not None else None
    if v_true is not None:
        hist.model_error.append(1.0)

    def cb(k, x, ev, h):
        if v_true is not None:
            h.model_error.append(float(torch.linalg.vector_norm((x - v_true).double())) / e0)

    kw = dict(max_update=max_update, project=lambda x: x.clamp(lo, hi), callback=cb)
    if method == "lbfgs":
        opt = LBFGS(obj.value_grad, obj.value, memory=memory, **kw)
    elif method == "prcg":
        opt = PRCG(obj.value_grad, obj.value, **kw)
    elif method == "gauss_newton":
        opt = GaussNewton(obj.value_grad, obj.value, obj.hvp, cg_iters=cg_iters, cg_tol=cg_tol, **kw)
    else:
        raise ValueError(method)
    v, hist = opt.run(v0.clone(), iters, hist)
    hist.n_gradients, hist.n_misfits, hist.n_hvps = obj.n_gradients, obj.n_misfits, obj.n_hvps
    return v, hist
