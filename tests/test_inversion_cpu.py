"""The outer inversion loops (inversion.py) on functions whose minimisers and
iterates mathematics fixes (CPU, float64):

* preconditioned CG with exact line searches minimises an n-dimensional
  strictly convex quadratic in at most n iterations (finite termination);
* BFGS with a fixed initial inverse Hessian M^-1 and exact line searches
  produces, on a quadratic, the iterates of CG preconditioned with M (so
  L-BFGS with memory >= iterations and an unscaled H_0 must reproduce PRCG
  iterate by iterate);
* with the exact inverse of a diagonal Hessian as the preconditioner, both
  methods reach the minimiser of a diagonal quadratic in one step;
* on the Rosenbrock function, the Armijo/parabolic line search drives both to
  the minimiser (1, 1);
* the projection keeps every iterate within the bounds, and the bounds'
  default respects the stability limit.
A planted mistake (PR beta with the wrong sign) must break finite termination.
"""
import numpy as np
import pytest
import torch

from paper_1406_1864_gb300 import inversion as I


def quadratic(n=12, cond=100.0, seed=0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    A = torch.tensor(Q @ np.diag(lam) @ Q.T)
    b = torch.tensor(rng.standard_normal(n))
    xstar = torch.linalg.solve(A, b)
    return A, b, xstar


def objective(A, b, minv=lambda q: q):
    def value(x):
        return float(0.5 * x @ A @ x - b @ x)

    def value_grad(x):
        return I.Evaluation(value(x), A @ x - b, minv)
    return value, value_grad


def exact_search(A):
    def ls(value, x, f0, g, d, alpha0, project):
        a = -float(g @ d) / float(d @ A @ d)
        xn = project(x + a * d)
        return a, xn, value(xn), 1
    return ls


def test_prcg_finite_termination():
    A, b, xs = quadratic()
    value, vg = objective(A, b)
    opt = I.PRCG(vg, value, max_update=1.0, line_search=exact_search(A))
    x, h = opt.run(torch.zeros(12, dtype=torch.float64), 12)
    assert float(torch.linalg.vector_norm(x - xs)) <= 1e-8 * float(torch.linalg.vector_norm(xs))


def test_lbfgs_reproduces_preconditioned_cg():
    A, b, xs = quadratic(n=10, seed=3)
    dg = torch.tensor(np.random.default_rng(4).uniform(0.5, 2.0, 10))
    minv = lambda q: q / dg  # noqa: E731  M = diag(dg)
    value, vg = objective(A, b, minv)
    iters_cg, iters_bfgs = [], []
    cg = I.PRCG(vg, value, max_update=1.0, line_search=exact_search(A),
                callback=lambda k, x, ev, h: iters_cg.append(x.clone()))
    bf = I.LBFGS(vg, value, max_update=1.0, memory=10, scale_h0=False, line_search=exact_search(A),
                 callback=lambda k, x, ev, h: iters_bfgs.append(x.clone()))
    x0 = torch.zeros(10, dtype=torch.float64)
    cg.run(x0, 6)
    bf.run(x0, 6)
    for k, (a, c) in enumerate(zip(iters_cg, iters_bfgs)):
        assert float(torch.linalg.vector_norm(a - c)) <= 1e-9 * float(torch.linalg.vector_norm(a)), k


def test_exact_diagonal_preconditioner_one_step():
    a = torch.tensor([1.0, 10.0, 100.0, 1000.0], dtype=torch.float64)
    A, b = torch.diag(a), torch.tensor([1.0, -2.0, 3.0, -4.0], dtype=torch.float64)
    value, vg = objective(A, b, lambda q: q / a)
    for opt in (I.PRCG(vg, value, max_update=1.0, line_search=exact_search(A)),
                I.LBFGS(vg, value, max_update=1.0, line_search=exact_search(A))):
        x, h = opt.run(torch.zeros(4, dtype=torch.float64), 1)
        assert torch.allclose(x, b / a, rtol=0, atol=1e-12)


def rosenbrock():
    def value(x):
        return float((1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2)

    def value_grad(x):
        g = torch.stack([-2 * (1 - x[0]) - 400 * x[0] * (x[1] - x[0] ** 2), 200 * (x[1] - x[0] ** 2)])
        return I.Evaluation(value(x), g, lambda q: q)
    return value, value_grad


@pytest.mark.parametrize("method,iters", [("lbfgs", 200), ("prcg", 2000)])
def test_armijo_line_search_on_rosenbrock(method, iters):
    value, vg = rosenbrock()
    cls = I.LBFGS if method == "lbfgs" else I.PRCG
    opt = cls(vg, value, max_update=0.5)
    x, h = opt.run(torch.tensor([-1.2, 1.0], dtype=torch.float64), iters)
    assert float(torch.linalg.vector_norm(x - torch.ones(2, dtype=torch.float64))) <= 1e-4, (method, x)
    m = np.array(h.misfit)
    assert (np.diff(m) <= 1e-15).all()  # monotone decrease


def test_projection_and_bounds():
    A, b, xs = quadratic(n=6, seed=5)
    value, vg = objective(A, b)
    lo, hi = -0.1, 0.1
    seen = []
    opt = I.LBFGS(vg, value, max_update=1.0, project=lambda x: x.clamp(lo, hi),
                  callback=lambda k, x, ev, h: seen.append(x.clone()))
    opt.run(torch.zeros(6, dtype=torch.float64), 20)
    assert seen and all(float(x.min()) >= lo and float(x.max()) <= hi for x in seen)
    from paper_1406_1864_gb300 import _lib as L

    class G:
        dx, dt, vref, ndim = 10.0, 1e-3, 9000.0, 2
    v0 = torch.full((3, 3), 2000.0)
    lo2, hi2 = I.velocity_bounds(G, v0)
    assert lo2 == 1000.0 and hi2 == 3000.0
    v0[0, 0] = 5000.0
    lo2, hi2 = I.velocity_bounds(G, v0)
    assert hi2 <= L.FWI_CFL_LIMIT_2D * G.dx / G.dt


def test_planted_wrong_beta_sign_breaks_termination(monkeypatch):
    """PR beta with its sign flipped (planted on the CPU): CG loses finite
    termination on the same quadratic."""
    A, b, xs = quadratic()
    value, vg = objective(A, b)
    real_max = max

    def bad_max(a, b):
        return real_max(a, -b) if a == 0.0 else real_max(a, b)
    monkeypatch.setattr(I, "max", bad_max, raising=False)
    opt = I.PRCG(vg, value, max_update=1.0, line_search=exact_search(A))
    x, h = opt.run(torch.zeros(12, dtype=torch.float64), 12)
    assert float(torch.linalg.vector_norm(x - xs)) > 1e-6 * float(torch.linalg.vector_norm(xs))


def test_default_mute_depth():
    """The default mute keeps the rows down to two cells below the deepest
    source or receiver fixed."""
    class Geo:
        src = np.array([[2, 0, 5], [3, 0, 1]])
        rec = np.array([[[1, 0, 0], [1, 0, 7]], [[1, 0, 0], [4, 0, 7]]])
        nrec = 2
    assert I.default_mute(Geo) == 7
    Geo.nrec = 0
    assert I.default_mute(Geo) == 6


@pytest.mark.parametrize("cls", [I.PRCG, I.LBFGS])
def test_failed_line_search_restarts_along_steepest_descent(cls):
    """A line search that fails along every direction but -M^-1 g: both
    methods restart along -M^-1 g instead of stopping, and still converge."""
    A, b, xs = quadratic(n=8, seed=6)
    value, vg = objective(A, b)
    exact = exact_search(A)

    def picky(value, x, f0, g, d, alpha0, project):
        cos = float(-(g @ d) / (torch.linalg.vector_norm(g) * torch.linalg.vector_norm(d)))
        if cos < 1 - 1e-12:
            return 0.0, x, f0, 1
        return exact(value, x, f0, g, d, alpha0, project)
    x, h = cls(vg, value, max_update=1.0, line_search=picky).run(torch.zeros(8, dtype=torch.float64), 300)
    assert h.restarts > 0 and len(h.misfit) > 10
    assert float(torch.linalg.vector_norm(x - xs)) <= 1e-3 * float(torch.linalg.vector_norm(xs))


def test_gauss_newton_solves_linear_least_squares_in_one_step():
    """f = 1/2 |A x - b|^2 has the exact Gauss-Newton Hessian A^T A: with CG
    run to convergence the first step (unit step) lands on the minimiser."""
    rng = np.random.default_rng(4)
    A = torch.tensor(rng.standard_normal((20, 8)))
    b = torch.tensor(rng.standard_normal(20))
    xs = torch.linalg.lstsq(A, b).solution
    value = lambda x: float(0.5 * torch.sum((A @ x - b) ** 2))  # noqa: E731
    vg = lambda x: I.Evaluation(value(x), A.T @ (A @ x - b), lambda q: q)  # noqa: E731
    hvp = lambda x, p: A.T @ (A @ p)  # noqa: E731
    gn = I.GaussNewton(vg, value, hvp, max_update=10.0, cg_iters=8, cg_tol=0.0)
    x, h = gn.run(torch.zeros(8, dtype=torch.float64), 1)
    assert float(torch.linalg.vector_norm(x - xs)) <= 1e-8 * float(torch.linalg.vector_norm(xs))
    assert h.step == [1.0] and h.hvps == 8


def test_gauss_newton_on_rosenbrock_residuals():
    """Rosenbrock as the least-squares problem r = (10 (x2 - x1^2), 1 - x1):
    Gauss-Newton with J^T J products converges to (1, 1)."""
    def res(x):
        return torch.stack([10 * (x[1] - x[0] ** 2), 1 - x[0]])

    def jac(x):
        return torch.tensor([[-20 * float(x[0]), 10.0], [-1.0, 0.0]], dtype=torch.float64)
    value = lambda x: float(0.5 * torch.sum(res(x) ** 2))  # noqa: E731
    vg = lambda x: I.Evaluation(value(x), jac(x).T @ res(x), lambda q: q)  # noqa: E731
    hvp = lambda x, p: jac(x).T @ (jac(x) @ p)  # noqa: E731
    x, h = I.GaussNewton(vg, value, hvp, max_update=0.5, cg_iters=2, cg_tol=1e-12).run(
        torch.tensor([-1.2, 1.0], dtype=torch.float64), 50)
    assert float(torch.linalg.vector_norm(x - torch.ones(2, dtype=torch.float64))) <= 1e-6, x

