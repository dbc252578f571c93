"""Stored expected values (tests/golden/two_layer_40x70.json).

The paper prints no worked numerical example; the stored values were written
by tests/golden/make_golden.py from the FP64 oracle alone (traces, OLS
gradient, Eq. 1 illumination, Sec. 3 offset Hessian at 64 seeded positions,
and the misfit). The CPU test recomputes them with the oracle (any change of
the oracle's arithmetic shows here); the GPU test compares the CUDA path at
the same positions, relative to the norm of each sampled vector: traces
1e-5, gradient / illumination / offset Hessian 1e-4, and the misfit 1e-4
(the GPU residual subtracts two FP32-modelled trace sets, the stored one two
FP64 sets).
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "two_layer_40x70.json")


def load():
    with open(GOLD) as f:
        return json.load(f)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_oracle_reproduces_stored_values(oracle_mod):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    now, gold = mg.compute(), load()
    assert now["positions"] == gold["positions"]
    for k in ("d_obs", "seis_init", "grad", "illum", "offh"):
        assert rel(now[k], gold[k]) <= 1e-12, k
    assert abs(now["misfit"] - gold["misfit"]) <= 1e-12 * gold["misfit"]


@pytest.mark.gpu
def test_cuda_path_at_stored_positions():
    import torch
    from paper_1406_1864_gb300 import fwi, workloads as W
    gold = load()
    p = W.two_layer(nz=40, nx=70, nt=300, ns=2, nrec=70, sponge=10)
    grid, geom = fwi.from_problem(p)
    d_obs = fwi.forward(grid, geom, torch.as_tensor(p.v_true, device="cuda"))
    v = torch.as_tensor(p.v_init, device="cuda")
    seis = fwi.forward(grid, geom, v).cpu().numpy()
    res = fwi.adjoint_gradient(grid, geom, v, d_obs, fwi.Options(hmax=3))
    si = tuple(np.array(gold["positions"]["seis"]).T)
    fz, fx = np.array(gold["positions"]["field"]).T
    assert rel(d_obs.cpu().numpy()[si], gold["d_obs"]) <= 1e-5
    assert rel(seis[si], gold["seis_init"]) <= 1e-5
    # the GPU misfit uses its own d_obs (FP32 modelling of v_true)
    assert abs(float(res["misfit"]) - gold["misfit"]) <= 1e-4 * gold["misfit"]
    assert rel(res["grad"].cpu().numpy()[fz, fx], gold["grad"]) <= 1e-4
    assert rel(res["illum"].cpu().numpy()[fz, fx], gold["illum"]) <= 1e-4
    offh = res["offh"].cpu().numpy()
    for h in range(4):
        assert rel(offh[h][fz, fx], gold["offh"][h]) <= 1e-4, h
