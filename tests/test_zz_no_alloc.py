"""fwi_forward_noalloc: forward modelling for callers that cannot allocate
device memory.

Code that may not call cudaMalloc (a host framework that owns all device
memory, a plugin given only its input and output buffers) uses this entry
point: it runs the same forward modelling as fwi_forward(save=0) in a scratch
array the library holds itself. Checked here through the C ABI against
fwi_forward with a caller workspace, on two calls in a row on different
problems (the second call reuses the scratch the first one left behind), and
for its size limit.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_SEIS = 1e-5  # relative L2, as for every trace comparison in the suite


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def call_noalloc(lib, grid, geom, v, out, torch):
    g, ge = grid.c(), geom.c()
    return lib.fwi_forward_noalloc(ctypes.byref(g), ctypes.byref(ge), ctypes.c_void_p(v.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_forward_noalloc_matches_forward_twice():
    """Two calls in a row on different problems: the second has another
    model, more shots and other receiver positions, so scratch contents left
    by the first (c2, receiver tables, wavefields) would show up in its
    traces if set-up failed to replace or clear them."""
    import torch
    from paper_1406_1864_gb300 import _lib, fwi
    assert torch.cuda.is_available()
    lib = _lib.load()
    problems = [W.dipping(nz=70, nx=150, nt=500, ns=3, nrec=75, f0=12.0, seed=3, sponge=12),
                W.dipping(nz=64, nx=170, nt=420, ns=5, nrec=41, rec_step=4, f0=10.0, seed=8, sponge=10)]
    assert problems[1].nshots > problems[0].nshots
    for call, p in enumerate(problems):
        grid, geom = fwi.from_problem(p)
        v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
        ref = fwi.forward(grid, geom, v).cpu().numpy()
        out = torch.full((p.nshots, p.nt, p.nrec), float("nan"), device="cuda")
        _lib.check(call_noalloc(lib, grid, geom, v, out, torch), "fwi_forward_noalloc")
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), call
        assert rel(got, ref) <= TOL_SEIS, (call, rel(got, ref))


def test_forward_noalloc_rejects_oversized_problem():
    import torch
    from paper_1406_1864_gb300 import _lib, fwi
    lib = _lib.load()
    p = W.two_layer(nz=1500, nx=1500, nt=10, ns=4, nrec=10, sponge=20)
    grid, geom = fwi.from_problem(p)
    v = torch.as_tensor(np.ascontiguousarray(p.v_init), device="cuda")
    out = torch.empty((p.nshots, p.nt, p.nrec), device="cuda")
    st = call_noalloc(lib, grid, geom, v, out, torch)
    assert st == _lib.FWI_ERR_NOMEM
    assert b"scratch" in lib.fwi_last_error()
