"""Shot-parallel FWI gradient over several GPUs, one process per GPU.

Shots are independent: the gradient of Sec. 2, the illumination of Eq. 1 and
the offset-Hessian diagonal of Sec. 3 are all sums over shots. Each rank
therefore models a contiguous range of the shots with the library on its own
GPU, and one sum over ranks (torch.distributed all-reduce: NCCL between GPUs,
gloo between CPU processes) combines the raw gradient, illumination, offset
Hessian and misfit. Preconditioning divides by the summed scale and its
global maximum, so it runs after the sum, on every rank. There is no other
exchange: no halo, no per-time-step communication.

`sharded_gradient` takes the per-rank compute and the preconditioner as
arguments that default to the library (fwi.adjoint_gradient without the
preconditioned output, fwi.precondition); the CPU tests pass their own
stand-ins to check the sharding and the reduction on gloo ranks.
"""
from __future__ import annotations

from typing import Callable

import torch

# summed over ranks, in this order on every rank
REDUCED = ("grad", "illum", "offh", "misfit")


def shot_range(nshots: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous shots [s0, s1) of `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    base, extra = divmod(nshots, world)
    s0 = rank * base + min(rank, extra)
    return s0, s0 + base + (1 if rank < extra else 0)


def reduce_partials(parts: dict, group=None) -> dict:
    """Sum the per-rank partial sums over all ranks, in place."""
    import torch.distributed as dist
    for k in REDUCED:
        if k in parts and parts[k] is not None:
            dist.all_reduce(parts[k], op=dist.ReduceOp.SUM, group=group)
    return parts


def _library_compute(grid, geom, v, d_obs, opts):
    from . import fwi
    return fwi.adjoint_gradient(grid, geom, v, d_obs, opts, want_pre=False, want_illum=True)


def _library_precondition(grid, grad, scale, kind, eps):
    from . import fwi
    return fwi.precondition(grid, grad, scale, kind, eps)


def zero_partials(grid, opts, device, field_dtype=torch.float32) -> dict:
    """What a rank without shots contributes to the sum."""
    out = {"grad": torch.zeros(grid.shape, dtype=field_dtype, device=device),
           "illum": torch.zeros(grid.shape, dtype=field_dtype, device=device),
           "misfit": torch.zeros((), dtype=torch.float64, device=device)}
    if opts.hmax >= 0:
        out["offh"] = torch.zeros((opts.hmax + 1,) + tuple(grid.shape), dtype=field_dtype, device=device)
    return out


def sharded_gradient(grid, geom, v, d_obs, opts, *, rank: int, world: int, group=None,
                     compute: Callable | None = None, precondition: Callable | None = None,
                     field_dtype=torch.float32) -> dict:
    """Preconditioned gradient of all shots of `geom`, this rank modelling
    shots shot_range(nshots, rank, world). `d_obs` holds this rank's shots
    only ([s1 - s0, nt, nrec]). Returns the summed grad, illum, offh
    (hmax >= 0), misfit and grad_pre (opts.precond), identical on every rank.
    field_dtype is the dtype of the compute's fields (what a rank without
    shots contributes).
    """
    compute = compute or _library_compute
    precondition = precondition or _library_precondition
    s0, s1 = shot_range(geom.nshots, rank, world)
    if d_obs.shape[0] != s1 - s0:
        raise ValueError(f"d_obs has {d_obs.shape[0]} shots, rank {rank} owns {s1 - s0}")
    if s1 > s0:
        part = compute(grid, geom.subset(s0, s1), v, d_obs, opts)
        part = {k: part[k] for k in REDUCED if k in part}
    else:
        part = zero_partials(grid, opts, v.device, field_dtype)
    if world > 1:
        reduce_partials(part, group)
    if opts.precond == "illum":
        part["grad_pre"] = precondition(grid, part["grad"], part["illum"], "illum", opts.eps)
    elif opts.precond == "offset":
        part["grad_pre"] = precondition(grid, part["grad"], part["offh"], "offset", opts.eps)
    else:
        part["grad_pre"] = part["grad"].clone()
    return part
