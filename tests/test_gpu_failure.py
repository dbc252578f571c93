"""Failure detection on the GPU without a fault: every wait of the step
kernels is bounded (%globaltimer) and a wait that runs out raises a status
bit that the host turns into FWI_ERR_TIMEOUT, leaving the context usable.
fwi_selftest_wait makes one such wait run out (an mbarrier that nothing
arrives at) with the same wait helper; after it, modelling runs normally.
"""
import time

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


@pytest.mark.parametrize("limit_us", [1000, 20000])
def test_bounded_wait_runs_out_and_the_context_survives(torch_cuda, oracle_mod, limit_us):
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi, _lib as L
    t0 = time.perf_counter()
    st = fwi.selftest_wait(limit_us)
    dt = time.perf_counter() - t0
    assert st == L.FWI_ERR_TIMEOUT, (st, L.load().fwi_last_error())
    assert b"as designed" in L.load().fwi_last_error()
    assert limit_us * 1e-6 <= dt < 5.0, dt
    # the context is usable: modelling afterwards matches the oracle
    p = W.dipping(nz=20, nx=40, dx=10.0, dt=1e-3, nt=120, ns=1, nrec=10, rec_step=4, f0=15.0, sponge=5)
    grid, geom = fwi.from_problem(p)
    seis = fwi.forward(grid, geom, torch.as_tensor(np.ascontiguousarray(p.v_true), device="cuda")).cpu().numpy()
    ref = oracle_mod.forward(oracle_mod.Grid.of(p), p.v_true, p.src, p.rec, p.wavelet.astype(np.float64))["seis"]
    assert np.linalg.norm(seis - ref) <= 1e-5 * np.linalg.norm(ref)


def test_non_finite_wavefield_is_reported(torch_cuda, oracle_mod):
    """A non-finite source sample (a blow-up injected on the host, no GPU
    fault) makes the wavefield non-finite; the finite check at the end of the
    time loop turns it into FWI_ERR_UNSTABLE, and the next call with a finite
    wavelet models normally."""
    torch = torch_cuda
    from paper_1406_1864_gb300 import fwi, _lib as L
    p = W.dipping(nz=20, nx=40, dx=10.0, dt=1e-3, nt=60, ns=2, nrec=10, rec_step=4, f0=15.0, sponge=5)
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(np.ascontiguousarray(p.v_true), device="cuda")
    bad_w = geom.wavelet.clone()
    bad_w[1, 5] = float("nan")
    with pytest.raises(L.FwiError) as e:
        fwi.forward(grid, fwi.Geometry(p.src, p.rec, bad_w), v)
    assert e.value.status == L.FWI_ERR_UNSTABLE
    seis = fwi.forward(grid, geom, v).cpu().numpy()
    ref = oracle_mod.forward(oracle_mod.Grid.of(p), p.v_true, p.src, p.rec, p.wavelet.astype(np.float64))["seis"]
    assert np.linalg.norm(seis - ref) <= 1e-5 * np.linalg.norm(ref)
