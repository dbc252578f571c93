"""Pins of the oracle's preconditioning (Sec. 3, Sec. 3.1).

* The per-point scale of the offset-Hessian preconditioner (reading A7) is
  the sum over the offsets -hmax..hmax of |H(x, h)|, H(x, h) = sum_s sum_n
  u_s^n(x + h) u_s^n(x - h) dt (Sec. 3: the diagonal of the localized
  subsurface-offset Hessian, horizontal offsets). ``oracle.offset_scale``
  computes it from the accumulated h >= 0 slices as |H(x,0)| + 2 sum_{h>=1}
  |H(x,h)|. Here the sum is built instead from the dumped wavefields of each
  shot with explicit shifts for every negative and positive offset (zero
  outside the padded grid), with no use of the symmetry in h, and summed
  over shots. Two plausible mistakes are planted in the oracle's formula and
  fail: the factor 2 dropped, and signed instead of absolute values of H
  (the wavefield products of h >= 1 change sign, which the test checks).
* The stabilised division g / (P + eps max P) (reading A8) is checked on a
  hand case whose quotients follow by exact arithmetic; a water level taken
  from the mean of P instead of its maximum fails.
* The whole offset-preconditioned gradient of ``oracle.fwi_gradient`` equals
  the gradient divided by the brute-force scale.
"""
import numpy as np
import pytest

from paper_1406_1864_gb300 import workloads as W

HMAX = 5


def _problem():
    # two shots, so the shot sum is part of what is pinned
    return W.dipping(nz=24, nx=34, dx=10.0, dt=1e-3, nt=200, ns=2, nrec=10, rec_step=3, f0=15.0,
                     sponge=6, seed=7)


def _shift(u, d):
    """u(x + d) along the last axis, zero where x + d leaves the padded grid."""
    out = np.zeros_like(u)
    n = u.shape[-1]
    if d >= 0:
        out[..., :n - d] = u[..., d:]
    else:
        out[..., -d:] = u[..., :n + d]
    return out


def _brute_force(oracle_mod, p, hmax):
    """H(x, h) for h = -hmax..hmax (index h + hmax) on the physical grid, from
    each shot's dumped padded wavefield, summed over shots."""
    g = oracle_mod.Grid.of(p)
    P = p.sponge
    H = np.zeros((2 * hmax + 1, p.nz, p.nx))
    for s in range(p.nshots):
        one = p.subset([s])
        u = oracle_mod.forward(g, one.v_init, one.src, one.rec, one.wavelet, dump_shot=0)["dump"][:, :, 0, :]
        for h in range(-hmax, hmax + 1):
            prod = np.sum(_shift(u, h) * _shift(u, -h), axis=0) * p.dt
            H[h + hmax] += prod[P:P + p.nz, P:P + p.nx]
    return H


@pytest.fixture(scope="module")
def pinned(oracle_mod):
    p = _problem()
    g = oracle_mod.Grid.of(p)
    offh = oracle_mod.forward(g, p.v_init, p.src, p.rec, p.wavelet, hmax=HMAX)["offh"][:, :, 0, :]
    return p, offh, _brute_force(oracle_mod, p, HMAX)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_offset_scale_sums_every_signed_offset(oracle_mod, pinned):
    p, offh, H = pinned
    ref = np.sum(np.abs(H), axis=0)
    assert _rel(oracle_mod.offset_scale(offh), ref) <= 1e-12
    # the accumulated slices are the brute-force ones for h >= 0 ...
    assert _rel(offh, H[HMAX:]) <= 1e-12
    # ... and the negative offsets, computed on their own, mirror them
    assert _rel(H[:HMAX][::-1], H[HMAX + 1:]) <= 1e-12


def test_offset_scale_planted_mistakes_fail(oracle_mod, pinned):
    p, offh, H = pinned
    ref = np.sum(np.abs(H), axis=0)
    # the products of h >= 1 take both signs, so |H| and H differ
    assert np.any(H[HMAX + 1:] < 0) and np.any(H[HMAX + 1:] > 0)

    def dropped_two(o):
        return np.abs(o[0]) + np.sum(np.abs(o[1:]), axis=0)

    def signed(o):
        return np.abs(o[0]) + 2.0 * np.sum(o[1:], axis=0)

    for planted in (dropped_two, signed):
        assert _rel(planted(offh), ref) > 1e-2, planted.__name__


def test_precondition_hand_case(oracle_mod):
    # P = (0, 1, 4, 1000) with eps = 1e-3: water level eps max P = 1 (exact
    # in binary64), denominators 1, 2, 5, 1001
    P = np.array([[0.0, 1.0], [4.0, 1000.0]])
    g = np.array([[3.0, 4.0], [-10.0, 2002.0]])
    expected = np.array([[3.0, 2.0], [-2.0, 2.0]])
    assert np.array_equal(oracle_mod.precondition(g, P, eps=1e-3), expected)
    # eps = 0.5: water level 500, denominators 500, 501, 504, 1500
    out = oracle_mod.precondition(np.array([500.0, 1002.0, 252.0, 3000.0]),
                                  np.array([0.0, 1.0, 4.0, 1000.0]), eps=0.5)
    assert np.array_equal(out, np.array([1.0, 2.0, 0.5, 2.0]))

    # planted: the water level from the mean of P (251.25) instead of its maximum
    def mean_level(grad, PP, eps=1e-3):
        return grad / (PP + eps * PP.mean())

    assert not np.allclose(mean_level(g, P), expected, rtol=1e-6, atol=0)


def test_offset_preconditioned_gradient(oracle_mod, pinned):
    p, _, H = pinned
    g = oracle_mod.Grid.of(p)
    w = p.wavelet.astype(np.float64)
    d_obs = oracle_mod.forward(g, p.v_true, p.src, p.rec, w)["seis"]
    res = oracle_mod.fwi_gradient(g, p.v_init, p.src, p.rec, w, d_obs, misfit="integral", hmax=HMAX)
    scale = np.sum(np.abs(H), axis=0)
    grad = res["grad"][:, 0, :]
    ref = grad / (scale + 1e-3 * scale.max())
    assert _rel(res["grad_pre_offset"][:, 0, :], ref) <= 1e-12
    # and the illumination preconditioner is the h = 0 slice of the same sum
    il = H[HMAX]
    assert _rel(res["grad_pre_illum"][:, 0, :], grad / (il + 1e-3 * il.max())) <= 1e-12
