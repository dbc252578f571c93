"""Extended Born modelling (Eq. 5) and extended migration (Eq. 6) on the GPU
against the FP64 oracle, on the ragged grid (padded 51 x 97) with sources
and receivers on edges and corners.

* Extended Born traces for hext = 1, 2, 4, 6 (each compiled offset count)
  against the oracle (relative L2 <= 1e-5 per shot, as Born traces).
* Extended migration images for hext = 2, 5 against the oracle (1e-4, the
  gradient bound), and at hext = 0 against fwi_adjoint_apply's gradient of
  the same adjoint source (1e-6).
* hext = 0 extended Born against fwi_born (1e-6).
* The GPU pair's dot test <B dv, dd> = <dv, M dd> (1e-5: FP32).
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ragged_problem(nt=280, ns=3):
    p = W.dipping(nz=37, nx=83, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=20, rec_step=4, f0=15.0, seed=2, sponge=7)
    src = p.src.copy()
    src[0] = [0, 0, 0]
    src[1] = [36, 0, 82]
    rec = p.rec.copy()
    rec[:, 0] = [0, 0, 0]
    rec[:, 1] = [36, 0, 82]
    rec[:, 2] = [36, 0, 0]
    rec[:, 3] = [0, 0, 82]
    p.src, p.rec = src, rec
    return p


@pytest.fixture(scope="module")
def case(torch_cuda, oracle_mod):
    from paper_1406_1864_gb300 import fwi
    p = ragged_problem()
    grid, geom = fwi.from_problem(p)
    v = torch_cuda.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    return p, oracle_mod.Grid.of(p), grid, geom, v


def ext_pert(p, hext, seed=5):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((2 * hext + 1, p.nz, p.nx)) * 20.0).astype(np.float32)


@pytest.mark.parametrize("hext", [1, 2, 4, 6])
def test_extended_born_against_oracle(torch_cuda, oracle_mod, case, hext):
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = case
    dv = ext_pert(p, hext)
    ref = oracle_mod.extended_born(g, p.v_init, dv[:, :, None, :], p.src, p.rec, p.wavelet.astype(np.float64),
                                   hext)
    got = fwi.extended_born(grid, geom, v, torch_cuda.as_tensor(dv, device="cuda")).cpu().numpy()
    for s in range(p.nshots):
        assert rel(got[s], ref[s]) <= 1e-5, (hext, s, rel(got[s], ref[s]))


@pytest.mark.parametrize("hext", [2, 5])
def test_extended_migration_against_oracle(torch_cuda, oracle_mod, case, hext):
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = case
    adj = np.random.default_rng(8).standard_normal((p.nshots, p.nt, p.nrec)).astype(np.float32)
    ref = oracle_mod.extended_migration(g, p.v_init, p.src, p.rec, p.wavelet.astype(np.float64), adj, hext)
    got = fwi.extended_migration(grid, geom, v, torch_cuda.as_tensor(adj, device="cuda"), hext).cpu().numpy()
    assert got.shape == (2 * hext + 1, p.nz, p.nx)
    assert rel(got, ref[:, :, 0, :]) <= 1e-4, rel(got, ref[:, :, 0, :])
    for k in range(2 * hext + 1):
        assert rel(got[k], ref[k, :, 0, :]) <= 1e-4, (k - hext, rel(got[k], ref[k, :, 0, :]))


def test_zero_offset_matches_plain_operators(torch_cuda, case):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = case
    dv = ext_pert(p, 0)
    eb = fwi.extended_born(grid, geom, v, torch.as_tensor(dv, device="cuda"))
    b = fwi.born(grid, geom, v, torch.as_tensor(dv[0], device="cuda"))
    assert rel(eb.cpu(), b.cpu()) <= 1e-6
    adj = torch.as_tensor(np.random.default_rng(9).standard_normal((p.nshots, p.nt, p.nrec)).astype(np.float32),
                          device="cuda")
    img = fwi.extended_migration(grid, geom, v, adj, 0)
    ws = fwi.Workspace()
    fwi.forward(grid, geom, v, save=True, ws=ws)
    gr = fwi.adjoint_apply(grid, geom, v, adj, ws)
    assert rel(img[0].cpu(), gr.cpu()) <= 1e-6


def test_gpu_dot_test(torch_cuda, case):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = case
    hext = 4
    dv = torch.as_tensor(ext_pert(p, hext, seed=11), device="cuda")
    dd = torch.as_tensor(np.random.default_rng(12).standard_normal((p.nshots, p.nt, p.nrec)).astype(np.float32),
                         device="cuda")
    lhs = float((fwi.extended_born(grid, geom, v, dv).double() * dd.double()).sum())
    rhs = float((dv.double() * fwi.extended_migration(grid, geom, v, dd, hext).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs)), (lhs, rhs)
