"""The 3-D workload at full size, in the launch configuration it is timed in.

200 x 400 x 400 cells, dx 12.5 m, dt 1 ms, nt 3000, 8 shots, 400 x 400
receivers: the oracle would need hours in 3-D at this size (its parity is at
small sizes in test_gpu_3d.py), so the checks are properties that hold at any
size: the gradient against central finite differences of the misfit, and
bfloat16 snapshots within 1e-2 of F32.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_c5_3d_full_size():
    """200 x 400 x 400, dx 12.5 m, dt 1 ms, nt 3000, 8 shots, 400 x 400
    receivers, F32 snapshots in shot groups of 2 (an 80 GB workspace): the
    gradient against central finite differences of the misfit along a smooth
    direction, and bfloat16 snapshots within 1e-2 of F32."""
    import torch
    from paper_1406_1864_gb300 import fwi
    torch.cuda.empty_cache()  # the workspaces of earlier modules
    p = W.workload("dipping3d_200x400x400_8shots")
    grid, geom = fwi.from_problem(p)
    ws = fwi.Workspace()
    grp = fwi.Options(shot_group=2)
    d_obs = fwi.forward(grid, geom, torch.as_tensor(p.v_true, device="cuda"), ws=ws, opts=grp)
    v = torch.as_tensor(p.v_init, device="cuda")
    r = fwi.adjoint_gradient(grid, geom, v, d_obs, fwi.Options(ckpt="snapshot", snap="f32", shot_group=2), ws=ws)
    g = r["grad"].cpu().numpy().astype(np.float64)
    J0 = float(r["misfit"])

    def misfit(vv):
        d = fwi.forward(grid, geom, torch.as_tensor(vv.astype(np.float32), device="cuda"), ws=ws, opts=grp)
        return 0.5 * float(((d.double() - d_obs.double()) ** 2).sum())

    v0 = p.v_init.astype(np.float64)
    assert abs(misfit(v0) - J0) <= 1e-6 * J0
    dv = W.smooth_perturbation(v0.shape, 0, sigma_cells=15.0)
    eps = 2.0
    fd = (misfit(v0 + eps * dv) - misfit(v0 - eps * dv)) / (2 * eps)
    an = float(np.sum(g * dv))
    assert abs(fd - an) <= 5e-3 * max(abs(an), 0.05 * np.linalg.norm(g) * np.linalg.norm(dv)), (fd, an)
    bf = fwi.adjoint_gradient(grid, geom, v, d_obs, fwi.Options(ckpt="snapshot", snap="bf16", shot_group=2), ws=ws)
    assert rel(bf["grad"].cpu(), g) <= 1e-2
