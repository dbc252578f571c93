"""3-D modelling and gradients (25-point 8th-order stencil) against the FP64
oracle, which runs the same scheme in 3-D.

Small ragged grid (padded 30 x 33 x 38: not a multiple of the 64 x 8
columns), receivers on the surface grid plus some at depth, on edges and in
corners. Tolerances as in 2-D: traces 1e-5, gradient / illumination /
preconditioned gradient 1e-4 with F32 snapshots, 1e-2 with bfloat16 ones;
shot groups (opts.shot_group) give the all-at-once result. The offset-Hessian
diagonal (Sec. 3, offsets along x) and the offset-preconditioned gradient
1e-4, on grids whose sponge width makes the sums' copies 16-byte (sponge 8)
or 4-byte (sponge 6).
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


def problem3(nt=150, ns=3):
    p = W.dipping3d(nz=18, ny=21, nx=26, dx=10.0, dt=8e-4, nt=nt, ns=ns, rec_step=3, f0=15.0, seed=3, sponge=6)
    rec = p.rec.copy()
    extra = np.array([[5, 4, 7], [17, 20, 25], [17, 0, 0], [0, 20, 25], [9, 10, 0], [12, 0, 13]], np.int32)
    rec[:, :len(extra)] = extra[None]
    p.rec = rec
    src = p.src.copy()
    src[-1] = [17, 20, 25]  # a source in the bottom corner
    p.src = src
    return p


@pytest.fixture(scope="module")
def case(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = problem3()
    g = oracle_mod.Grid.of(p)
    w64 = p.wavelet.astype(np.float64)
    d_true = oracle_mod.forward(g, p.v_true, p.src, p.rec, w64)["seis"]
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, w64, d_true.astype(np.float32).astype(np.float64))
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    d = torch.as_tensor(d_true.astype(np.float32), device="cuda")
    return p, g, grid, geom, v, d, d_true, ref


def test_3d_forward_traces(torch_cuda, case):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v, d, d_true, ref = case
    seis = fwi.forward(grid, geom, torch.as_tensor(np.ascontiguousarray(p.v_true), device="cuda")).cpu().numpy()
    for s in range(p.nshots):
        assert rel(seis[s], d_true[s]) <= 1e-5, (s, rel(seis[s], d_true[s]))


def test_3d_gradient_f32_snapshots(torch_cuda, case):
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v, d, d_true, ref = case
    r = fwi.adjoint_gradient(grid, geom, v, d, fwi.Options(ckpt="snapshot", snap="f32"))
    assert rel(r["grad"].cpu(), ref["grad"]) <= 1e-4
    assert rel(r["illum"].cpu(), ref["illum"]) <= 1e-4
    assert rel(r["grad_pre"].cpu(), ref["grad_pre_illum"]) <= 1e-4
    assert abs(float(r["misfit"]) - ref["J"]) <= 1e-5 * ref["J"]


def test_3d_gradient_16bit_snapshots_and_groups(torch_cuda, case):
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v, d, d_true, ref = case
    bf = fwi.adjoint_gradient(grid, geom, v, d, fwi.Options(ckpt="snapshot", snap="bf16"))
    assert rel(bf["grad"].cpu(), ref["grad"]) <= 1e-2
    whole = fwi.adjoint_gradient(grid, geom, v, d, fwi.Options(ckpt="snapshot", snap="f32", snap_interval=7))
    for grp in (1, 2):
        part = fwi.adjoint_gradient(grid, geom, v, d, fwi.Options(ckpt="snapshot", snap="f32", snap_interval=7,
                                                                  shot_group=grp))
        assert rel(part["grad"].cpu(), whole["grad"].cpu()) <= 1e-6, grp
        assert rel(part["illum"].cpu(), whole["illum"].cpu()) <= 1e-6, grp
        assert abs(float(part["misfit"]) - float(whole["misfit"])) <= 1e-12 * float(whole["misfit"])
    assert rel(whole["grad"].cpu(), ref["grad"]) <= 1e-4


def test_3d_illumination_entry_point(torch_cuda, case):
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v, d, d_true, ref = case
    il = fwi.illumination(grid, geom, v, fwi.Options(shot_group=2))
    assert rel(il.cpu(), ref["illum"]) <= 1e-4


def test_3d_errors(torch_cuda, case):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi, _lib
    p, g, grid, geom, v, d, d_true, ref = case
    with pytest.raises(_lib.FwiError):  # sponge checkpoints are 2-D only
        fwi.adjoint_gradient(grid, geom, v, d, fwi.Options())
    with pytest.raises(_lib.FwiError):  # offsets 0..12 only
        fwi.adjoint_gradient(grid, geom, v, d, fwi.Options(ckpt="snapshot", hmax=13, precond="illum"))
    with pytest.raises(_lib.FwiError):  # the offset-Hessian diagonal needs hmax >= 0
        fwi.offset_hessian_diag(grid, geom, v, fwi.Options(hmax=-1))
    fast = v.clone()
    fast[3, 4, 5] = 9000.0
    with pytest.raises(_lib.FwiError) as e:
        fwi.adjoint_gradient(grid, geom, fast, d, fwi.Options(ckpt="snapshot"))
    assert e.value.status == _lib.FWI_ERR_CFL
    again = fwi.adjoint_gradient(grid, geom, v, d, fwi.Options(ckpt="snapshot"))
    assert np.isfinite(again["grad"].cpu().numpy()).all()


def problem3h(sponge, nx):
    """The ragged grid with another sponge width and nx: sponge 8 and nx 24
    put every offset-Hessian window on a 16-byte boundary and every row of
    sums on one (the vector paths), sponge 6 and nx 26 neither."""
    p = W.dipping3d(nz=18, ny=21, nx=nx, dx=10.0, dt=8e-4, nt=150, ns=3, rec_step=3, f0=15.0, seed=3,
                    sponge=sponge)
    src = p.src.copy()
    src[-1] = [17, 20, nx - 1]  # a source in the bottom corner
    p.src = src
    return p


@pytest.fixture(scope="module", params=[(6, 26), (8, 24)], ids=["unaligned", "aligned"])
def case_h(request, torch_cuda, oracle_mod):
    """Oracle gradient with the offset Hessian at hmax 12 and both
    preconditioners, on the grid of problem3h."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p = problem3h(*request.param)
    g = oracle_mod.Grid.of(p)
    w64 = p.wavelet.astype(np.float64)
    d_true = oracle_mod.forward(g, p.v_true, p.src, p.rec, w64)["seis"]
    ref = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, w64, d_true.astype(np.float32).astype(np.float64),
                                  hmax=12)
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    d = torch.as_tensor(d_true.astype(np.float32), device="cuda")
    return p, grid, geom, v, d, ref


@pytest.mark.parametrize("hmax", [0, 3, 7, 12])
def test_3d_offset_hessian_entry_point(torch_cuda, case_h, hmax):
    """fwi_offset_hessian_diag on 3-D grids (Sec. 3, offsets along x): every
    offset against the oracle (1e-4) for each compiled offset count (4, 11,
    13), H(x, 0) against the oracle's illumination, in shot groups of 2."""
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, d, ref = case_h
    H = fwi.offset_hessian_diag(grid, geom, v, fwi.Options(hmax=hmax, shot_group=2)).cpu().numpy()
    assert H.shape == (hmax + 1, p.nz, p.ny, p.nx)
    for h in range(hmax + 1):
        assert rel(H[h], ref["offh"][h]) <= 1e-4, h
    assert rel(H[0], ref["illum"]) <= 1e-4


def test_3d_gradient_offset_preconditioned(torch_cuda, case_h):
    """fwi_adjoint_gradient on a 3-D grid with the offset Hessian (hmax 12)
    and the offset preconditioner (Sec. 3.1): gradient, every offset of H
    and the preconditioned gradient against the oracle (1e-4), F32
    snapshots; without the offh output (the sums finished in place) the
    preconditioned gradient is the same; hess_v6 scales H by 4 / v^6."""
    import torch
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, d, ref = case_h
    o = fwi.Options(ckpt="snapshot", snap="f32", hmax=12, precond="offset", shot_group=2)
    r = fwi.adjoint_gradient(grid, geom, v, d, o)
    assert rel(r["grad"].cpu(), ref["grad"]) <= 1e-4
    for h in range(13):
        assert rel(r["offh"][h].cpu(), ref["offh"][h]) <= 1e-4, h
    assert rel(r["grad_pre"].cpu(), ref["grad_pre_offset"]) <= 1e-4
    r2 = fwi.adjoint_gradient(grid, geom, v, d, o, want_offh=False)
    assert "offh" not in r2
    assert rel(r2["grad_pre"].cpu(), r["grad_pre"].cpu()) <= 1e-6
    pre = fwi.precondition(grid, r["grad"], r["offh"], "offset")  # the entry point on a 3-D grid
    assert rel(pre.cpu(), r["grad_pre"].cpu()) <= 1e-6
    o6 = fwi.Options(hmax=3, shot_group=2, hess_v6=True)
    H6 = fwi.offset_hessian_diag(grid, geom, v, o6)
    w6 = 4.0 / v.double() ** 6
    H1 = fwi.offset_hessian_diag(grid, geom, v, fwi.Options(hmax=3, shot_group=2))
    assert rel(H6.cpu().double(), (H1.double() * w6).cpu()) <= 1e-5
    assert torch.isfinite(H6).all()


N3_FWD, N3_BWD = 3, 4  # compiled 3-D step variants


def test_3d_every_variant_matches_the_oracle(torch_cuda, case):
    """Each 3-D step variant (ring depth, CTAs per SM), pinned with
    fwi_autotune_set, gives the oracle's gradient (1e-4) and the default
    variant's (the same arithmetic: 1e-6); fwi_autotune's choice is in range
    and used by the next call."""
    import itertools
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v, d, d_true, ref = case
    opts = fwi.Options(ckpt="snapshot", snap="f32", shot_group=2)
    fwi.autotune_reset()
    default = fwi.adjoint_gradient(grid, geom, v, d, opts)
    try:
        for fv, bv in itertools.product(range(N3_FWD), range(N3_BWD)):
            fwi.autotune_set(grid, geom, opts, {"forward_variant": fv, "forward_chunk": 1,
                                                 "backward_variant": bv, "backward_chunk": 1})
            r = fwi.adjoint_gradient(grid, geom, v, d, opts)
            assert rel(r["grad"].cpu(), ref["grad"]) <= 1e-4, (fv, bv)
            assert rel(r["grad"].cpu(), default["grad"].cpu()) <= 1e-6, (fv, bv)
            assert rel(r["illum"].cpu(), ref["illum"]) <= 1e-4, (fv, bv)
            assert abs(float(r["misfit"]) - float(default["misfit"])) <= 1e-12 * float(default["misfit"])
        choice = fwi.autotune(grid, geom, v, opts)
        assert 0 <= choice["forward_variant"] < N3_FWD and 0 <= choice["backward_variant"] < N3_BWD
        r = fwi.adjoint_gradient(grid, geom, v, d, opts)
        assert rel(r["grad"].cpu(), ref["grad"]) <= 1e-4
    finally:
        fwi.autotune_reset()


def test_3d_z_segments_match_the_oracle(torch_cuda, case):
    """Columns cut into z-segments (items of segment x column x shot; a
    segment's first window planes loaded straight from global memory),
    pinned with the 3-D chunks of fwi_autotune_set: 2 to 30 segments of the
    30 padded planes (down to one plane per item), so that the receivers at
    depth and the source in the bottom corner fall in later segments. Traces
    are the oracle's (1e-5), gradient and illumination too (1e-4), and the
    gradient is the one-segment gradient up to summation order (1e-6)."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    p, g, grid, geom, v, d, d_true, ref = case
    opts = fwi.Options(ckpt="snapshot", snap="f32")
    vt = torch.as_tensor(np.ascontiguousarray(p.v_true), device="cuda")
    try:
        fwi.autotune_set(grid, geom, opts, {"forward_variant": 0, "forward_chunk": 1,
                                             "backward_variant": 0, "backward_chunk": 1})
        one = fwi.adjoint_gradient(grid, geom, v, d, opts)
        for fs, bs in ((2, 2), (3, 7), (7, 3), (30, 5)):
            fwi.autotune_set(grid, geom, opts, {"forward_variant": 0, "forward_chunk": fs,
                                                 "backward_variant": 1, "backward_chunk": bs})
            seis = fwi.forward(grid, geom, vt, opts=opts).cpu().numpy()
            for s in range(p.nshots):
                assert rel(seis[s], d_true[s]) <= 1e-5, (fs, s)
            r = fwi.adjoint_gradient(grid, geom, v, d, opts)
            assert rel(r["grad"].cpu(), ref["grad"]) <= 1e-4, (fs, bs)
            assert rel(r["illum"].cpu(), ref["illum"]) <= 1e-4, (fs, bs)
            assert rel(r["grad"].cpu(), one["grad"].cpu()) <= 1e-6, (fs, bs)
            assert abs(float(r["misfit"]) - float(one["misfit"])) <= 1e-12 * float(one["misfit"])
    finally:
        fwi.autotune_reset()


def test_3d_autograd_with_snapshots(torch_cuda, case):
    """autograd.traces on a 3-D grid: fwi_forward(save = 1) keeps F32 (or
    bfloat16) snapshots, fwi_adjoint_apply is the backward. The OLS loss
    gives the oracle's gradient (1e-4; 1e-2 with bfloat16 snapshots) and its
    traces are the oracle's (1e-5); a shot group smaller than the shots is
    refused for the forward that keeps checkpoints."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import autograd, fwi, _lib
    p, g, grid, geom, v, d, d_true, ref = case
    for snap, tol in (("f32", 1e-4), ("bf16", 1e-2)):
        vv = v.clone().requires_grad_(True)
        seis = autograd.traces(vv, grid, geom, fwi.Options(ckpt="snapshot", snap=snap))
        assert rel(seis.detach().cpu(), ref["seis"]) <= 1e-5
        (0.5 * ((seis.double() - d.double()) ** 2).sum()).backward()
        assert rel(vv.grad.cpu(), ref["grad"]) <= tol, snap
    with pytest.raises(_lib.FwiError):
        autograd.traces(v.clone().requires_grad_(True), grid, geom,
                        fwi.Options(ckpt="snapshot", shot_group=1))
