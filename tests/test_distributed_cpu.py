"""Shot-parallel gradient on gloo ranks (CPU processes).

paper_1406_1864_gb300.distributed.sharded_gradient splits the shots over the
ranks, sums the partial gradient / illumination / offset Hessian / misfit
with one all-reduce and preconditions after the sum. Here each rank's
partial sums come from the FP64 oracle for its own shots (no GPU in these
tests), and the result on every rank must equal the oracle's gradient of all
shots at once -- the sums over shots of Sec. 2, Eq. 1 and Sec. 3 -- up to the
order of the FP64 additions. Worlds of 2 ranks with 3 shots (uneven split)
and of 3 ranks with 2 shots (one rank without shots), and a 3-D model over
3 ranks with 2 shots and the offset preconditioner ([hmax+1, nz, ny, nx]
offset Hessians; the rank without shots contributes zeros of that shape).
"""
import socket

import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class HostGeometry:
    """The part of fwi.Geometry the sharding uses, with host arrays."""

    def __init__(self, src, rec, wav):
        self.src, self.rec, self.wav = src, rec, wav

    @property
    def nshots(self):
        return self.src.shape[0]

    def subset(self, s0, s1):
        return HostGeometry(self.src[s0:s1], self.rec[s0:s1], self.wav[s0:s1])


def problem(ns, ndim=2):
    if ndim == 3:
        return W.dipping3d(nz=8, ny=7, nx=9, dx=10.0, dt=5e-4, nt=70, ns=ns, rec_step=3, f0=20.0, seed=2,
                           sponge=4)
    return W.dipping(nz=18, nx=26, dx=10.0, dt=1e-3, nt=90, ns=ns, nrec=13, rec_step=2, f0=20.0,
                     seed=4, sponge=5)


def flat(a, ndim, lead=0):
    """The oracle's [.., nz, ny, nx] arrays as the library's shapes (2-D: ny dropped)."""
    return a if ndim == 3 else np.take(a, 0, axis=lead + 1)


def worker(rank, world, port, ns, hmax, precond, ndim, queue):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1406_1864_gb300 import distributed as D
    from paper_1406_1864_gb300 import fwi

    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}")
    try:
        p = problem(ns, ndim)
        g = oracle.Grid.of(p)
        w64 = p.wavelet.astype(np.float64)
        d_all = oracle.forward(g, p.v_true, p.src, p.rec, w64)["seis"]
        s0, s1 = D.shot_range(ns, rank, world)
        geom = HostGeometry(p.src, p.rec, w64)
        opts = fwi.Options(misfit="ols", hmax=hmax, precond=precond)

        def compute(grid, sub, v, d_obs, o):
            r = oracle.fwi_gradient(g, v, sub.src, sub.rec, sub.wav, d_obs.numpy(),
                                    hmax=None if o.hmax < 0 else o.hmax)
            out = {"grad": torch.from_numpy(flat(r["grad"], ndim).copy()),
                   "illum": torch.from_numpy(flat(r["illum"], ndim).copy()),
                   "misfit": torch.tensor(r["J"], dtype=torch.float64)}
            if o.hmax >= 0:
                out["offh"] = torch.from_numpy(flat(r["offh"], ndim, lead=1).copy())
            return out

        def precondition(grid, grad, scale, kind, eps):
            P = scale.numpy() if kind == "illum" else oracle.offset_scale(scale.numpy())
            return torch.from_numpy(oracle.precondition(grad.numpy(), P, eps))

        class G:  # grid stand-in: shape only
            shape = (p.nz, p.ny, p.nx) if ndim == 3 else (p.nz, p.nx)

        v = torch.from_numpy(np.ascontiguousarray(p.v_init, dtype=np.float64))
        res = D.sharded_gradient(G(), geom, v, torch.from_numpy(d_all[s0:s1].copy()), opts, rank=rank,
                                 world=world, compute=compute, precondition=precondition,
                                 field_dtype=torch.float64)
        queue.put((rank, s1 - s0, {k: t.numpy() for k, t in res.items()}))
    finally:
        dist.destroy_process_group()


def run_world(world, ns, hmax, precond, ndim=2):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, ns, hmax, precond, ndim, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = {}
    try:
        for _ in range(world):
            rank, n, res = q.get(timeout=240)
            out[rank] = (n, res)
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
    assert all(pr.exitcode == 0 for pr in procs), [pr.exitcode for pr in procs]
    return out


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_shot_range_partitions():
    from paper_1406_1864_gb300.distributed import shot_range
    for ns in (1, 2, 3, 7, 96):
        for world in (1, 2, 3, 8):
            ranges = [shot_range(ns, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == ns
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shot_range(4, 2, 2)


@pytest.mark.parametrize("world,ns,hmax,precond,ndim", [(2, 3, 2, "offset", 2), (3, 2, -1, "illum", 2),
                                                     (3, 2, 3, "offset", 3)])
def test_sharded_gradient_equals_all_shots(oracle_mod, world, ns, hmax, precond, ndim):
    from paper_1406_1864_gb300.distributed import shot_range
    out = run_world(world, ns, hmax, precond, ndim)
    for rank, (n, _) in out.items():
        s0, s1 = shot_range(ns, rank, world)
        assert n == s1 - s0
    p = problem(ns, ndim)
    g = oracle_mod.Grid.of(p)
    w64 = p.wavelet.astype(np.float64)
    d_all = oracle_mod.forward(g, p.v_true, p.src, p.rec, w64)["seis"]
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, w64, d_all,
                                  hmax=None if hmax < 0 else hmax)
    for rank, (_, res) in out.items():
        assert rel(res["grad"], flat(ref["grad"], ndim)) <= 1e-12, rank
        assert rel(res["illum"], flat(ref["illum"], ndim)) <= 1e-12, rank
        assert abs(float(res["misfit"]) - ref["J"]) <= 1e-12 * ref["J"], rank
        key = "grad_pre_illum" if precond == "illum" else "grad_pre_offset"
        assert rel(res["grad_pre"], flat(ref[key], ndim)) <= 1e-12, rank
        if hmax >= 0:
            assert res["offh"].shape == (hmax + 1,) + flat(ref["grad"], ndim).shape
            assert rel(res["offh"], flat(ref["offh"], ndim, lead=1)) <= 1e-12, rank
