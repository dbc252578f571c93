"""The synthetic inputs match their stated recipe (the stand-ins for the
paper's Marmousi experiments): sizes, velocity ranges, acquisition geometry,
stability, and seeded reproducibility."""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W


def test_two_layer_recipe():
    p = W.workload("two_layer_100x200")
    assert (p.nz, p.nx, p.dx, p.dt, p.nt, p.nshots, p.nrec) == (100, 200, 10.0, 1e-3, 1000, 4, 200)
    assert set(np.unique(p.v_true)) == {2000.0, 3000.0}
    assert np.all(p.v_true[:50] == 2000.0) and np.all(p.v_true[50:] == 3000.0)
    assert np.allclose(p.v_init[:, 0], np.linspace(2000.0, 3000.0, 100), atol=1e-3)
    assert np.all(p.src[:, 0] * p.dx == 20.0) and np.all(p.rec[:, :, 0] == 0)


def test_dipping_recipe_and_seed():
    p = W.workload("dipping_300x1000_96shots")
    assert (p.nz, p.nx, p.dx, p.dt, p.nt, p.nshots, p.nrec, p.sponge) == (300, 1000, 10.0, 8e-4, 4000, 96, 500, 20)
    assert 1500.0 <= p.v_true.min() and p.v_true.max() <= 4500.0 + 600.0 + 1e-3
    layers = np.unique(np.round(p.v_true[p.v_true < 1500.0 + 1e-3]))  # the top layer outside the body
    assert layers.tolist() == [1500.0]
    # the Gaussian body: +600 m/s at its centre, in the middle third, sigma 200 m
    body = p.v_true - W.dipping_layers_model(p.nz, p.nx, p.dx, seed=0, body_dv=0.0)
    iz, ix = np.unravel_index(np.argmax(body), body.shape)
    assert body.max() == pytest.approx(600.0, abs=1.0)
    assert p.nz / 3 <= iz <= 2 * p.nz / 3 and p.nx / 3 <= ix <= 2 * p.nx / 3
    assert body[iz, ix + 20] == pytest.approx(600.0 * np.exp(-0.5), rel=0.05)  # 200 m = 20 cells away
    assert set(np.unique(W.dipping_layers_model(p.nz, p.nx, p.dx, seed=0, body_dv=0.0))) == \
        {1500.0, 2100.0, 2700.0, 3300.0, 3900.0, 4500.0}
    assert np.all(p.src[:, 0] * p.dx == 20.0) and np.all(p.rec[:, :, 0] * p.dx == 10.0)
    assert np.all(np.diff(p.rec[0, :, 2]) == 2) and np.all(p.rec == p.rec[:1])
    assert np.all(np.diff(p.src[:, 2]) > 0)
    assert p.courant() == pytest.approx(p.v_true.max() * p.dt / p.dx)
    assert p.courant() <= 0.41
    q = W.dipping(nz=60, nx=200, nt=10, ns=4, nrec=50)
    r = W.dipping(nz=60, nx=200, nt=10, ns=4, nrec=50)
    assert np.array_equal(q.v_true, r.v_true) and np.array_equal(q.v_init, r.v_init)
    assert not np.array_equal(W.dipping(nz=60, nx=200, nt=10, ns=4, nrec=50, seed=1).v_true, q.v_true)
    # the starting model is the true model smoothed with sigma 300 m (30 cells):
    # its largest step per cell is a few per cent of the true model's jumps
    assert np.allclose(p.v_init, W.smooth(p.v_true, 30.0), atol=1e-2)
    jump = np.abs(np.diff(p.v_true, axis=0)).max()
    assert jump >= 600.0 - 1e-3 and np.abs(np.diff(p.v_init, axis=0)).max() < 0.05 * jump


def test_ricker_peak_and_delay():
    dt, f0 = 1e-4, 10.0
    w = W.ricker(4000, dt, f0)
    assert np.argmax(w) == round(1.5 / f0 / dt) and w.max() == pytest.approx(1.0)
    spec = np.abs(np.fft.rfft(w))
    f = np.fft.rfftfreq(w.size, dt)
    assert f[np.argmax(spec)] == pytest.approx(f0, abs=0.5)


def test_3d_and_uneven_recipes():
    p = W.dipping3d(nz=20, ny=40, nx=40, nt=10, ns=8)
    assert p.ndim == 3 and p.nrec == 40 * 40 and p.nshots == 8
    assert np.all(p.src[:, 0] == 2) and len({tuple(s) for s in p.src.tolist()}) == 8
    assert p.courant() <= 0.4528
    b = W.uneven_batch(nt=10, ns=4)
    assert [(m.nz, m.nx) for m in b] == [(200, 400), (350, 900), (500, 1500)]
    assert [m.nrec for m in b] == [200, 450, 750] and all(m.nt == 10 for m in b)
