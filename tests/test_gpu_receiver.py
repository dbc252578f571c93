"""Receiver side of the diagonal Hessian for a fixed spread (Sec. 1) against
the FP64 oracle.

* Plessix and Mulder's asinh factor (relative L2 <= 1e-5: one asinh pair per
  cell in FP32) for a partial spread (cells inside and outside it) on a
  ragged grid.
* Receiver Green's-function correlations R(x, h), h = 0..3, in the initial
  model (<= 1e-4, the Hessian bound), receivers on model edges and corners.
* fwi_precondition_receiver: grad / (P + eps max P) with P = scale x recv for
  the illumination and the offset kinds, one factor for every offset and one
  per offset (<= 1e-5 on the same float32 inputs), and the combination the
  paper's H_a calls for: the source-side offset Hessian times R (<= 1e-4).
* A geometry whose shots record at different cells is refused.
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


def fixed_spread(nt=300, ns=3):
    p = W.dipping(nz=37, nx=83, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=18, rec_step=4, f0=15.0, seed=2, sponge=7)
    rec = p.rec[0].copy()
    rec[0] = [0, 0, 0]
    rec[1] = [36, 0, 82]
    rec[2] = [0, 0, 82]
    rec[3:, 2] = np.arange(15, 15 + 4 * (rec.shape[0] - 3), 4)[: rec.shape[0] - 3] % 83
    p.rec = np.repeat(rec[None], ns, axis=0)
    return p


@pytest.fixture(scope="module")
def case(torch_cuda, oracle_mod):
    from paper_1406_1864_gb300 import fwi
    p = fixed_spread()
    grid, geom = fwi.from_problem(p)
    v = torch_cuda.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    return p, oracle_mod.Grid.of(p), grid, geom, v


def test_plessix_mulder_factor(torch_cuda, oracle_mod, case):
    from paper_1406_1864_gb300 import fwi
    p = W.dipping(nz=40, nx=97, dx=12.5, dt=1e-3, nt=50, ns=2, nrec=20, rec_step=3, f0=10.0, sponge=5)
    grid, geom = fwi.from_problem(p)
    got = fwi.receiver_factor(grid, geom, "pm").cpu().numpy()
    ref = oracle_mod.plessix_mulder_factor(p.nz, p.nx, p.dx, p.rec[0])
    assert rel(got, ref) <= 1e-5, rel(got, ref)


def test_receiver_green_factor(torch_cuda, oracle_mod, case):
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = case
    got = fwi.receiver_factor(grid, geom, "green", v, fwi.Options(hmax=3)).cpu().numpy()
    ref = oracle_mod.receiver_green_factor(g, p.v_init, p.rec[0], p.wavelet[0].astype(np.float64), hmax=3)
    assert got.shape == (4, p.nz, p.nx)
    for h in range(4):
        assert rel(got[h], ref[h, :, 0, :]) <= 1e-4, (h, rel(got[h], ref[h, :, 0, :]))
    h0 = fwi.receiver_factor(grid, geom, "green", v).cpu().numpy()  # no options: h = 0 only
    assert h0.shape == (1, p.nz, p.nx) and rel(h0[0], got[0]) <= 1e-6


@pytest.mark.parametrize("kind,planes", [("illum", 1), ("offset", 1), ("offset", 5)])
def test_precondition_receiver_kernel(torch_cuda, oracle_mod, kind, planes):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = fixed_spread(nt=10, ns=1)
    grid, _ = fwi.from_problem(p)
    rng = np.random.default_rng(3)
    hmax = 4
    grad = rng.standard_normal((p.nz, p.nx)).astype(np.float32)
    scale = (rng.uniform(0.0, 2.0, (p.nz, p.nx)) if kind == "illum"
             else rng.standard_normal((hmax + 1, p.nz, p.nx))).astype(np.float32)
    if kind == "offset":
        scale[0] = np.abs(scale[0]) + 1.0
    recv = rng.uniform(0.1, 3.0, (planes, p.nz, p.nx)).astype(np.float32)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")  # noqa: E731
    got = fwi.precondition_receiver(grid, t(grad), t(scale), kind, t(recv[0] if planes == 1 else recv), eps=1e-3)
    prod = scale.astype(np.float64) * (recv[0] if planes == 1 else recv).astype(np.float64)
    P = prod if kind == "illum" else oracle_mod.offset_scale(prod)
    ref = oracle_mod.precondition(grad, P, 1e-3)
    assert rel(got.cpu(), ref) <= 1e-5, rel(got.cpu(), ref)


def test_receiver_inclusive_offset_preconditioned_gradient(torch_cuda, oracle_mod, case):
    """The preconditioned gradient of H_a's diagonal with both Green's
    function sums: g / offset_scale(H_src(x, h) R(x, h))."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = case
    w64 = p.wavelet.astype(np.float64)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, w64)["seis"]
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, w64, d_obs.astype(np.float32).astype(np.float64),
                                  hmax=3)
    R = oracle_mod.receiver_green_factor(g, p.v_init, p.rec[0], w64[0], hmax=3)
    P = oracle_mod.offset_scale(ref["offh"] * R)[:, 0, :]
    ref_pre = oracle_mod.precondition(ref["grad"][:, 0, :], P, 1e-3)
    opts = fwi.Options(hmax=3, precond="offset")
    r = fwi.adjoint_gradient(grid, geom, v, torch.as_tensor(d_obs.astype(np.float32), device="cuda"), opts)
    Rg = fwi.receiver_factor(grid, geom, "green", v, opts)
    got = fwi.precondition_receiver(grid, r["grad"], r["offh"], "offset", Rg, eps=1e-3)
    assert rel(got.cpu(), ref_pre) <= 1e-4, rel(got.cpu(), ref_pre)


def test_moving_spread_refused(torch_cuda, case):
    from paper_1406_1864_gb300 import fwi, _lib
    p, g, grid, geom, v = case
    rec = p.rec.copy()
    rec[1, 0, 2] += 1
    grid2, geom2 = fwi.from_problem(p)
    geom2.rec = np.ascontiguousarray(rec, dtype=np.int32)
    for kind in ("pm", "green"):
        with pytest.raises(_lib.FwiError):
            fwi.receiver_factor(grid2, geom2, kind, v)


def moving_spread(nt=300, ns=4):
    """An end-on spread that moves with the shot: receivers on the 12 cells
    behind each source, two shots per spread position (runs of two)."""
    p = W.dipping(nz=37, nx=83, dx=10.0, dt=1e-3, nt=nt, ns=ns, nrec=12, rec_step=1, f0=15.0, seed=2, sponge=7)
    src = p.src.copy()
    rec = np.zeros((ns, 12, 3), np.int32)
    for s in range(ns):
        x0 = 14 + 20 * (s // 2)
        src[s] = [2, 0, x0 + 1 + (s % 2)]
        rec[s, :, 0] = 1
        rec[s, :, 2] = np.arange(x0 - 12, x0)
    p.src, p.rec = src, rec
    return p


@pytest.mark.parametrize("utt", [False, True])
def test_plessix_mulder_hessian_moving_spread(torch_cuda, oracle_mod, utt):
    from paper_1406_1864_gb300 import fwi
    p = moving_spread()
    g = oracle_mod.Grid.of(p)
    grid, geom = fwi.from_problem(p)
    v = torch_cuda.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    got = fwi.plessix_mulder_hessian(grid, geom, v, fwi.Options(illum="utt2" if utt else "u2")).cpu().numpy()
    ref = oracle_mod.plessix_mulder_hessian(g, p.v_init, p.src, p.rec, p.wavelet.astype(np.float64),
                                            illum_utt=utt)[:, 0, :]
    assert rel(got, ref) <= 1e-4, rel(got, ref)


def test_plessix_mulder_hessian_fixed_spread(torch_cuda, case):
    """One spread: the factor of fwi_receiver_factor times the illumination."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v = case
    H = fwi.plessix_mulder_hessian(grid, geom, v)
    ref = fwi.receiver_factor(grid, geom, "pm") * fwi.illumination(grid, geom, v, fwi.Options())
    assert rel(H.cpu(), ref.cpu()) <= 1e-5

