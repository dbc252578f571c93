"""Tile autotuning: every compiled tile variant and chunk size gives the
oracle's gradient, and fwi_autotune's choice is used by later calls.

The variants differ only in tile height, ring depth and register cap; each is
pinned with fwi_autotune_set and checked against the FP64 oracle (1e-4) and
against the default variant (the same arithmetic; 1e-6).
"""
import itertools

import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_FWD, N_FWDH, N_BWD = 4, 5, 2  # compiled variants of each kind (offset Hessian: 3 fused, 2 split)


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


@pytest.fixture(scope="module")
def case(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi
    # padded 57 x 107: ragged against tile heights 8, 16, 32
    p = W.dipping(nz=41, nx=91, dx=10.0, dt=1e-3, nt=240, ns=5, nrec=30, rec_step=3, f0=15.0, seed=9, sponge=8)
    g = oracle_mod.Grid.of(p)
    w64 = p.wavelet.astype(np.float64)
    d = oracle_mod.forward(g, p.v_true, p.src, p.rec, w64)["seis"].astype(np.float32)
    refs = {h: oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, w64, d.astype(np.float64),
                                       hmax=None if h < 0 else h) for h in (-1, 3)}
    grid, geom = fwi.from_problem(p)
    return p, grid, geom, torch.as_tensor(p.v_init, device="cuda"), torch.as_tensor(d, device="cuda"), refs


@pytest.mark.parametrize("hmax", [-1, 3])
def test_every_variant_matches_the_oracle(torch_cuda, case, hmax):
    from paper_1406_1864_gb300 import fwi
    p, grid, geom, v, d, refs = case
    ref = refs[hmax]
    opts = fwi.Options(hmax=hmax, precond="offset" if hmax >= 0 else "illum")
    nf = N_FWDH if hmax >= 0 else N_FWD
    fwi.autotune_reset()
    default = fwi.adjoint_gradient(grid, geom, v, d, opts)["grad"].cpu().numpy()
    try:
        for fv, bv, chunk in itertools.product(range(nf), range(N_BWD), (3, 16)):
            fwi.autotune_set(grid, geom, opts, {"forward_variant": fv, "forward_chunk": chunk,
                                                 "backward_variant": bv, "backward_chunk": chunk})
            r = fwi.adjoint_gradient(grid, geom, v, d, opts)
            case_id = (fv, bv, chunk)
            assert rel(r["grad"].cpu(), ref["grad"][:, 0, :]) <= 1e-4, case_id
            assert rel(r["grad"].cpu(), default) <= 1e-6, case_id
            assert rel(r["illum"].cpu(), ref["illum"][:, 0, :]) <= 1e-4, case_id
            if hmax >= 0:
                assert rel(r["offh"].cpu(), ref["offh"][:, :, 0, :]) <= 1e-4, case_id
    finally:
        fwi.autotune_reset()


def test_autotune_choice_is_used(torch_cuda, case):
    from paper_1406_1864_gb300 import fwi, _lib
    p, grid, geom, v, d, refs = case
    opts = fwi.Options()
    try:
        choice = fwi.autotune(grid, geom, v, opts)
        assert 0 <= choice["forward_variant"] < N_FWD and 0 <= choice["backward_variant"] < N_BWD
        assert choice["forward_chunk"] in (8, 16) and choice["backward_chunk"] in (8, 16)
        r = fwi.adjoint_gradient(grid, geom, v, d, opts)  # runs with the tuned tiles
        assert rel(r["grad"].cpu(), refs[-1]["grad"][:, 0, :]) <= 1e-4
        with pytest.raises(_lib.FwiError):
            fwi.autotune_set(grid, geom, opts, {"forward_variant": N_FWD, "forward_chunk": 8,
                                                 "backward_variant": 0, "backward_chunk": 8})
    finally:
        fwi.autotune_reset()
