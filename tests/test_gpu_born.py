"""Born modelling (fwi_born, Eq. 4) and Gauss-Newton Hessian-vector products
(fwi_gauss_newton_hvp) against the FP64 oracle.

* Born traces J dv against the oracle's Born modelling of the same discrete
  scheme (relative L2 <= 1e-5 per shot), for the reflectivity perturbation
  v_true - v_init and for white noise that reaches the model edges (edge
  replication into the sponge).
* J^T J dv against the oracle's adjoint imaging of the oracle's Born traces
  (<= 1e-4), J^T C^T C J dv (time-integral misfit, Eq. 2) likewise, and
  against the library's own adjoint_apply of its Born traces
  after forward(save=True): the Born pass must leave the same sponge
  checkpoint as the forward pass.
* Properties that hold at any size: linearity (J (2 dv) = 2 J dv to FP32
  rounding: every operation scales exactly with dv except in the subnormal
  range ahead of the wavefront, where rounding is absolute, and one flipped
  rounding there spreads through later roundings at the ulp level),
  dv = 0 gives zeros, the symmetry <dv1, H dv2> = <dv2, H dv1> and
  positivity <dv, H dv> = |J dv|^2.
* Full size (300 x 1000, 96 shots, nt 4000): Born traces of sampled shots
  against the oracle at the derivative bound 1e-4 (J dv is the derivative of
  the traces; it carries the FP32 rounding of u through dc2 q(u) on top of its
  own, about 1.1e-5 after 4000 levels), and <dv, H dv> = |J dv|^2.
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


def ragged_problem(nt=300, ns=3):
    """Padded 51 x 97 (not multiples of the 64 x 16 tiles), sources and
    receivers on edges and corners, two receivers on one cell."""
    p = W.dipping(nz=37, nx=83, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=20, rec_step=4, f0=15.0,
                  seed=2, sponge=7)
    src = p.src.copy()
    src[0] = [0, 0, 0]
    src[1] = [36, 0, 82]
    rec = p.rec.copy()
    rec[:, 0] = [0, 0, 0]
    rec[:, 1] = [36, 0, 82]
    rec[:, 2] = [36, 0, 0]
    rec[:, 3] = [0, 0, 82]
    rec[:, 4] = rec[:, 5]
    p.src, p.rec = src, rec
    return p


def perturbations(p):
    refl = (p.v_true - p.v_init).astype(np.float32)
    noise = np.random.default_rng(17).standard_normal(p.v_init.shape).astype(np.float32) * 20.0
    return {"reflectivity": refl, "noise": noise}


@pytest.fixture(scope="module")
def small(torch_cuda, oracle_mod):
    from paper_1406_1864_gb300 import fwi
    p = ragged_problem()
    g = oracle_mod.Grid.of(p)
    grid, geom = fwi.from_problem(p)
    v = torch_cuda.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    return p, g, grid, geom, v


@pytest.mark.parametrize("kind", ["reflectivity", "noise"])
def test_born_traces_against_oracle(torch_cuda, oracle_mod, small, kind):
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = small
    dv = perturbations(p)[kind]
    ref = oracle_mod.born(g, p.v_init, dv, p.src, p.rec, p.wavelet.astype(np.float64))
    got = fwi.born(grid, geom, v, torch_cuda.as_tensor(dv, device="cuda")).cpu().numpy()
    for s in range(p.nshots):
        assert rel(got[s], ref[s]) <= 1e-5, (kind, s, rel(got[s], ref[s]))


@pytest.mark.parametrize("kind", ["reflectivity", "noise"])
def test_gauss_newton_hvp_against_oracle(torch_cuda, oracle_mod, small, kind):
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = small
    dv = perturbations(p)[kind]
    w64 = p.wavelet.astype(np.float64)
    jdv = oracle_mod.born(g, p.v_init, dv, p.src, p.rec, w64)
    ref = oracle_mod.gradient_for_adjoint_source(g, p.v_init, p.src, p.rec, w64, jdv)["grad"][:, 0, :]
    got = fwi.gauss_newton_hvp(grid, geom, v, torch_cuda.as_tensor(dv, device="cuda")).cpu().numpy()
    assert rel(got, ref) <= 1e-4, (kind, rel(got, ref))


def test_gauss_newton_hvp_time_integral_misfit(torch_cuda, oracle_mod, small):
    """H dv of the Eq. 2 misfit: J^T C^T C J dv."""
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = small
    dv = perturbations(p)["reflectivity"]
    w64 = p.wavelet.astype(np.float64)
    jdv = oracle_mod.born(g, p.v_init, dv, p.src, p.rec, w64)
    adj = oracle_mod.time_integral_adjoint(oracle_mod.time_integral(jdv, p.dt), p.dt)
    ref = oracle_mod.gradient_for_adjoint_source(g, p.v_init, p.src, p.rec, w64, adj)["grad"][:, 0, :]
    got = fwi.gauss_newton_hvp(grid, geom, v, torch_cuda.as_tensor(dv, device="cuda"),
                               fwi.Options(misfit="integral")).cpu().numpy()
    assert rel(got, ref) <= 1e-4, rel(got, ref)


def test_hvp_equals_adjoint_apply_of_born_traces(torch_cuda, small):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = small
    dv = torch.as_tensor(perturbations(p)["noise"], device="cuda")
    ws = fwi.Workspace()
    jdv = fwi.born(grid, geom, v, dv, ws=ws)
    hv = fwi.gauss_newton_hvp(grid, geom, v, dv, ws=ws)
    fwi.forward(grid, geom, v, save=True, ws=ws)
    ref = fwi.adjoint_apply(grid, geom, v, jdv, ws)
    assert rel(hv.cpu(), ref.cpu()) <= 1e-6


def test_born_linearity_zero_and_hvp_symmetry(torch_cuda, small):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = small
    pert = perturbations(p)
    d1 = torch.as_tensor(pert["reflectivity"], device="cuda")
    d2 = torch.as_tensor(pert["noise"], device="cuda")
    b1 = fwi.born(grid, geom, v, d1)
    b2 = fwi.born(grid, geom, v, 2 * d1)
    assert rel(b2.cpu(), 2 * b1.cpu()) <= 1e-5
    zero = torch.zeros_like(d1)
    assert not fwi.born(grid, geom, v, zero).any()
    assert not fwi.gauss_newton_hvp(grid, geom, v, zero).any()
    h1 = fwi.gauss_newton_hvp(grid, geom, v, d1).double()
    h2 = fwi.gauss_newton_hvp(grid, geom, v, d2).double()
    a, b = float((d2.double() * h1).sum()), float((d1.double() * h2).sum())
    assert abs(a - b) <= 1e-5 * max(abs(a), abs(b)), (a, b)
    # <dv, J^T J dv> = |J dv|^2
    q = float((d1.double() * h1).sum())
    n2 = float((b1.double() ** 2).sum())
    assert q > 0 and abs(q - n2) <= 1e-5 * n2, (q, n2)


def test_born_errors_and_options(torch_cuda, small):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi, _lib
    p, g, grid, geom, v = small
    dv = torch.as_tensor(perturbations(p)["noise"], device="cuda")
    o = fwi.Options(ckpt="snapshot")
    with pytest.raises(_lib.FwiError):  # Born passes keep sponge checkpoints
        fwi.workspace_bytes(grid, geom, o, "gn_hvp")
    fast = v.clone()
    fast[3, 4] = 40000.0
    with pytest.raises(_lib.FwiError) as e:
        fwi.born(grid, geom, fast, dv)
    assert e.value.status == _lib.FWI_ERR_CFL
    again = fwi.gauss_newton_hvp(grid, geom, v, dv)
    assert torch.isfinite(again).all()


@pytest.fixture(scope="module")
def full(torch_cuda):
    from paper_1406_1864_gb300 import fwi
    p = W.workload("dipping_300x1000_96shots")
    grid, geom = fwi.from_problem(p)
    v = torch_cuda.as_tensor(p.v_init, device="cuda")
    dv = torch_cuda.as_tensor((p.v_true - p.v_init).astype(np.float32), device="cuda")
    return p, grid, geom, v, dv, fwi.Workspace()


def test_full_size_born_sampled_shots(torch_cuda, oracle_mod, full):
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, dv, ws = full
    got = fwi.born(grid, geom, v, dv, ws=ws).cpu().numpy()
    shots = [0, 95]
    g = oracle_mod.Grid.of(p)
    ref = oracle_mod.born(g, p.v_init, dv.cpu().numpy(), p.src[shots], p.rec[shots],
                          p.wavelet[shots].astype(np.float64), nthreads=len(shots))
    for i, s in enumerate(shots):
        assert rel(got[s], ref[i]) <= 1e-4, (s, rel(got[s], ref[i]))


def test_full_size_hvp_quadratic_form(torch_cuda, full):
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, dv, ws = full
    jdv = fwi.born(grid, geom, v, dv, ws=ws).double()
    hv = fwi.gauss_newton_hvp(grid, geom, v, dv, ws=ws).double()
    q = float((dv.double() * hv).sum())
    n2 = float((jdv ** 2).sum())
    assert abs(q - n2) <= 1e-4 * n2, (q, n2)
