"""Forward modelling as a differentiable PyTorch operation.

`traces(v, grid, geom, opts)` returns the traces d[s, n, r] of every shot
(fwi_forward with save = 1) and registers, for autograd, the vector-Jacobian
product v_bar = J^T d_bar, which is the adjoint-state gradient of Sec. 2:
fwi_adjoint_apply back-propagates d_bar from the receivers and images it
against the forward wavefield. Any misfit written in torch on top of the
traces -- the OLS misfit, the time-integral misfit of Eq. 2 through
torch.cumsum, or another -- then yields its gradient with respect to v through
loss.backward(), with every wave-equation step in the library's kernels.

Each call owns its workspace (the forward checkpoints live there until the
backward pass has run), so several calls may be in flight in one graph.
opts.ckpt / opts.snap choose the checkpoints: the exact sponge-band mode (2-D),
or about sqrt(nt) whole-field snapshots in F32, bfloat16 or scaled float16
(2-D and 3-D).
"""
from __future__ import annotations

import torch

from . import fwi


class _Traces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, grid, geom, opts):
        v = v.detach().contiguous()
        ws = fwi.Workspace(v.device)
        seis = fwi.forward(grid, geom, v, save=True, ws=ws, opts=opts)
        ctx.save_for_backward(v)
        ctx.grid, ctx.geom, ctx.opts, ctx.ws = grid, geom, opts, ws
        return seis

    @staticmethod
    def backward(ctx, d_bar):
        (v,) = ctx.saved_tensors
        if ctx.ws is None:
            raise RuntimeError("the forward checkpoints of this call were already consumed")
        g = fwi.adjoint_apply(ctx.grid, ctx.geom, v, d_bar.contiguous(), ctx.ws, opts=ctx.opts)
        ctx.ws = None  # free the checkpoints
        return g, None, None, None


def traces(v: torch.Tensor, grid: fwi.Grid, geom: fwi.Geometry,
           opts: fwi.Options | None = None) -> torch.Tensor:
    """Traces [nshots, nt, nrec] of velocity v (grid.shape: [nz, nx], or
    [nz, ny, nx] on a 3-D grid, where opts needs ckpt="snapshot" and all shots
    in one group); differentiable in v."""
    return _Traces.apply(v, grid, geom, opts)


class Propagator(torch.nn.Module):
    """Module form of `traces` for one acquisition: forward(v) -> traces."""

    def __init__(self, grid: fwi.Grid, geom: fwi.Geometry, opts: fwi.Options | None = None):
        super().__init__()
        self.grid, self.geom, self.opts = grid, geom, opts

    def forward(self, v: torch.Tensor) -> torch.Tensor:
        return traces(v, self.grid, self.geom, self.opts)
