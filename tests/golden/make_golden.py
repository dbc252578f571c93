"""Writes the stored expected values of tests/test_golden.py.

The paper prints no worked numerical example, so the stored values are
outputs of the FP64 oracle (oracle/, nothing else) on a small seeded
problem: 40 x 70 two-layer model (Sec. 2 set-up: 2000 / 3000 m/s, starting
model a linear gradient), 2 shots, nt 300, 10-cell sponge.
Stored: traces d_s^n(r) (Sec. 2), the gradient of the OLS misfit (Sec. 2),
the illumination of Eq. 1 and the offset-Hessian diagonal of Sec. 3 for
hmax 3, each at 64 seeded sample positions, plus the misfit.

Run from the repository root: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1406_1864_gb300 import workloads as W  # noqa: E402

FILE = os.path.join(HERE, "two_layer_40x70.json")


def problem():
    return W.two_layer(nz=40, nx=70, nt=300, ns=2, nrec=70, sponge=10)


def sample_positions(p, n=64, seed=11):
    rng = np.random.default_rng(seed)
    return {"seis": np.stack([rng.integers(0, p.nshots, n), rng.integers(0, p.nt, n),
                              rng.integers(0, p.nrec, n)], 1).tolist(),
            "field": np.stack([rng.integers(0, p.nz, n), rng.integers(0, p.nx, n)], 1).tolist()}


def compute():
    oracle.build()
    p = problem()
    g = oracle.Grid.of(p)
    w64 = p.wavelet.astype(np.float64)
    d_obs = oracle.forward(g, p.v_true, p.src, p.rec, w64)["seis"]
    r = oracle.fwi_gradient(g, p.v_init, p.src, p.rec, w64, d_obs, hmax=3)
    pos = sample_positions(p)
    si = tuple(np.array(pos["seis"]).T)
    fz, fx = np.array(pos["field"]).T
    return {
        "what": "FP64 oracle outputs (see make_golden.py)",
        "problem": "two_layer nz=40 nx=70 nt=300 ns=2 nrec=70 sponge=10; d_obs modelled on v_true",
        "positions": pos,
        "d_obs": d_obs[si].tolist(),
        "seis_init": r["seis"][si].tolist(),
        "grad": r["grad"][fz, 0, fx].tolist(),
        "illum": r["illum"][fz, 0, fx].tolist(),
        "offh": [r["offh"][h, fz, 0, fx].tolist() for h in range(4)],
        "misfit": r["J"],
    }


if __name__ == "__main__":
    d = compute()
    with open(FILE, "w") as f:  # one key per line, compact values
        f.write("{\n" + ",\n".join(f"{json.dumps(k)}: {json.dumps(v)}" for k, v in d.items()) + "\n}\n")
    print("wrote", FILE)
