"""Edge cases of the operators beyond the gradient, against the FP64 oracle:
nt = 2 and 3 (one and two time steps), geometries without receivers, one
shot, and a one-receiver spread. Tolerances as in the main tests (traces
1e-5, images and Hessian products 1e-4); where the exact result is zero, the
result must be exactly zero.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    torch.cuda.set_device(0)
    return torch


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / n) if n > 0 else float(np.linalg.norm(a))


def problem(nt, ns=2, nrec=10):
    p = W.dipping(nz=21, nx=45, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=max(nrec, 1), rec_step=4, f0=25.0, seed=6,
                  sponge=5)
    if nrec == 0:
        p.rec = np.zeros((ns, 0, 3), np.int32)
    # a source below the receivers close to them, so one step reaches them
    src = p.src.copy()
    src[:, 0] = 1
    p.src = src
    return p


@pytest.mark.parametrize("nt", [2, 3, 12])
def test_born_hvp_and_extended_few_steps(torch_cuda, oracle_mod, nt):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = problem(nt)
    g = oracle_mod.Grid.of(p)
    grid, geom = fwi.from_problem(p)
    w64 = p.wavelet.astype(np.float64)
    rng = np.random.default_rng(nt)
    dv = (rng.standard_normal((p.nz, p.nx)) * 30).astype(np.float32)
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    tdv = torch.as_tensor(dv, device="cuda")
    jdv = oracle_mod.born(g, p.v_init, dv, p.src, p.rec, w64)
    got = fwi.born(grid, geom, v, tdv).cpu().numpy()
    assert rel(got, jdv) <= 1e-5, rel(got, jdv)
    hv = oracle_mod.gradient_for_adjoint_source(g, p.v_init, p.src, p.rec, w64, jdv)["grad"][:, 0, :]
    assert rel(fwi.gauss_newton_hvp(grid, geom, v, tdv).cpu(), hv) <= 1e-4
    he = 2
    dve = (rng.standard_normal((2 * he + 1, p.nz, p.nx)) * 30).astype(np.float32)
    ref = oracle_mod.extended_born(g, p.v_init, dve[:, :, None, :], p.src, p.rec, w64, he)
    got = fwi.extended_born(grid, geom, v, torch.as_tensor(dve, device="cuda")).cpu().numpy()
    assert rel(got, ref) <= 1e-5
    adj = rng.standard_normal((p.nshots, p.nt, p.nrec)).astype(np.float32)
    ref = oracle_mod.extended_migration(g, p.v_init, p.src, p.rec, w64, adj, he)[:, :, 0, :]
    got = fwi.extended_migration(grid, geom, v, torch.as_tensor(adj, device="cuda"), he).cpu().numpy()
    assert rel(got, ref) <= 1e-4


def test_no_receivers(torch_cuda):
    """Without receivers the traces are empty and every adjoint quantity is
    exactly zero; fwi_misfit is zero."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = problem(40, nrec=0)
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    dv = torch.ones_like(v)
    assert fwi.born(grid, geom, v, dv).numel() == 0
    assert not fwi.gauss_newton_hvp(grid, geom, v, dv).any()
    empty = torch.zeros((p.nshots, p.nt, 0), device="cuda")
    assert not fwi.extended_migration(grid, geom, v, empty, 2).any()
    assert float(fwi.misfit(grid, geom, v, empty)) == 0.0
    with pytest.raises(fwi.FwiError):  # a receiver factor needs receivers
        fwi.receiver_factor(grid, geom, "pm")


def test_one_shot_one_receiver_spread(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = problem(60, ns=1, nrec=1)
    p.rec = np.array([[[0, 0, 30]]], np.int32)
    g = oracle_mod.Grid.of(p)
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    pm = fwi.receiver_factor(grid, geom, "pm").cpu().numpy()
    ref = oracle_mod.plessix_mulder_factor(p.nz, p.nx, p.dx, p.rec[0])
    # a one-point spread: x_min = x_max, the factor is zero everywhere
    assert not np.any(ref) and not np.any(pm)
    rg = fwi.receiver_factor(grid, geom, "green", v, fwi.Options(hmax=1)).cpu().numpy()
    rref = oracle_mod.receiver_green_factor(g, p.v_init, p.rec[0], p.wavelet[0].astype(np.float64), hmax=1)
    assert rel(rg, rref[:, :, 0, :]) <= 1e-4
