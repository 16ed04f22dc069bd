"""Pins of the TV ∩ box projection of Sec. 3.1 (oracle/tv.py).

  - div is the negative adjoint of grad (exact identity, random arrays);
  - TV of images with closed-form total variation (step edge, ramp,
    diagonal plane, constant);
  - the TV prox against the exact solution of the one-row problem, whose dual
    is a box-constrained least-squares problem (scipy's bounded solver), and in
    2D against the duality gap of the ROF problem, a certificate that is zero
    exactly at the optimum;
  - the TV-ball projection: identity inside the ball, TV on the sphere within
    tol_tv outside it, and the obtuse-angle property against the constant
    images (TV 0, inside the ball);
  - Dykstra's result against a brute-force QP of the one-row projection onto
    {TV <= tau, x >= 0}.
"""
import numpy as np
import pytest
from scipy.optimize import lsq_linear, minimize, LinearConstraint

from oracle import tv as T


def _rng(s):
    return np.random.default_rng(s)


@pytest.mark.parametrize("shape", [(7, 9), (1, 12), (10, 1), (5, 5)])
def test_div_is_negative_adjoint_of_grad(shape):
    r = _rng(1)
    x = r.normal(size=shape)
    px, py = r.normal(size=shape), r.normal(size=shape)
    gx, gy = T.grad(x)
    lhs = float((gx * px).sum() + (gy * py).sum())
    rhs = -float((x * T.div(px, py)).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


def test_tv_closed_forms():
    ny, nx = 6, 9
    step = np.zeros((ny, nx))
    step[:, 4:] = 2.5
    assert T.tv(step) == pytest.approx(ny * 2.5, rel=1e-14)
    ramp = np.tile(0.3 * np.arange(nx), (ny, 1))
    assert T.tv(ramp) == pytest.approx(0.3 * (nx - 1) * ny, rel=1e-14)
    ii, jj = np.mgrid[0:ny, 0:nx]
    plane = (ii + jj).astype(float)
    ref = (nx - 1) * (ny - 1) * np.sqrt(2.0) + (nx - 1) + (ny - 1)
    assert T.tv(plane) == pytest.approx(ref, rel=1e-14)
    assert T.tv(np.full((ny, nx), 3.0)) == 0.0


def _grad_matrix_1d(n):
    D = np.zeros((n, n))  # rows: forward difference at j (last row zero)
    for j in range(n - 1):
        D[j, j], D[j, j + 1] = -1.0, 1.0
    return D


@pytest.mark.parametrize("lam", [0.3, 1.0, 4.0])
def test_prox_matches_exact_one_row_solution(lam):
    n = 12
    z = _rng(2).uniform(0, 1, n) + np.where(np.arange(n) >= 6, 1.0, 0.0)
    theta = lam / 2
    D = _grad_matrix_1d(n)
    # dual: min_{|p| <= 1} 1/2 || z - theta D^T p ||^2 over the n - 1 active components
    res = lsq_linear(theta * D.T[:, : n - 1], z, bounds=(-1.0, 1.0), tol=1e-14, method="bvls")
    x_exact = z - theta * D.T[:, : n - 1] @ res.x
    x, _, _ = T.prox_tv(z[None, :], lam, 4000)
    np.testing.assert_allclose(x[0], x_exact, atol=1e-7)


def test_prox_duality_gap_vanishes_2d():
    z = _rng(3).uniform(0, 1, (12, 10))
    lam = 0.8
    theta = lam / 2
    x, px, py = T.prox_tv(z, lam, 3000)
    primal = 0.5 * float(((x - z) ** 2).sum()) + theta * T.tv(x)
    assert np.sqrt(px ** 2 + py ** 2).max() <= 1.0 + 1e-12
    dual = 0.5 * float((z ** 2).sum()) - 0.5 * float(((z + theta * T.div(px, py)) ** 2).sum())
    assert primal >= dual - 1e-12
    assert primal - dual <= 1e-6 * primal


def test_prox_special_cases():
    c = np.full((5, 7), 0.7)
    x, _, _ = T.prox_tv(c, 2.0, 50)
    np.testing.assert_array_equal(x, c)
    z = _rng(4).uniform(0, 1, (6, 6))
    a, _, _ = T.prox_tv(z, 0.5, 200)
    b, _, _ = T.prox_tv(z + 3.0, 0.5, 200)
    np.testing.assert_allclose(b, a + 3.0, atol=1e-12)


def test_tv_ball_projection():
    opts = T.TvOptions(fgp_iters=200, tol_tv=1e-6, max_bisect=80)
    z = _rng(5).uniform(0, 1, (10, 12))
    tau_in = T.tv(z) * 1.01
    y, lam, _, _, solves = T.project_tv_ball(z, tau_in, opts, 0.0, np.zeros_like(z), np.zeros_like(z))
    assert solves == 0 and np.array_equal(y, z)
    tau = 0.4 * T.tv(z)
    y, lam, _, _, _ = T.project_tv_ball(z, tau, opts, 0.0, np.zeros_like(z), np.zeros_like(z))
    assert abs(T.tv(y) - tau) <= 1e-6
    for c in (0.0, 0.5, 2.0):
        w = np.full_like(z, c)
        assert float(((z - y) * (w - y)).sum()) <= 1e-4 * float(((z - y) ** 2).sum())


@pytest.mark.parametrize("z,tau", [
    ([0.2, -0.3, 0.9, 1.4, 0.1, -0.5, 0.8, 0.3], 1.0),
    # here plain alternating projections stop at a different point of X
    ([1.2, 0.39, -0.44, -0.62, -0.16, 0.52, -0.71, 0.09], 0.8),
    # and here Dykstra without the correction of the box step does
    ([-0.93, -0.38, 0.23, -0.64, 0.2, 0.4, 0.34, -0.21], 1.5),
])
def test_dykstra_matches_brute_force_qp_one_row(z, tau):
    n = 8
    z = np.array(z)
    opts = T.TvOptions(fgp_iters=400, tol_tv=1e-8, max_bisect=100, max_dykstra=400, tol_dykstra=1e-10)
    res = T.project_tv_box(z[None, :], tau, 0.0, np.inf, opts)
    # brute force: variables (x, s) with s_j >= |x_{j+1} - x_j|, sum s <= tau, x >= 0
    m = n - 1
    A = np.zeros((2 * m + 1, n + m))
    for j in range(m):
        A[j, j + 1], A[j, j], A[j, n + j] = 1.0, -1.0, -1.0        # x_{j+1} - x_j - s_j <= 0
        A[m + j, j + 1], A[m + j, j], A[m + j, n + j] = -1.0, 1.0, -1.0  # -(x_{j+1} - x_j) - s_j <= 0
    A[2 * m, n:] = 1.0
    ub = np.concatenate([np.zeros(2 * m), [tau]])
    cons = LinearConstraint(A, -np.inf, ub)
    fun = lambda v: 0.5 * float(((v[:n] - z) ** 2).sum())
    jac = lambda v: np.concatenate([v[:n] - z, np.zeros(m)])
    v0 = np.concatenate([np.clip(z, 0, None) * 0 + z.clip(0).mean(), np.zeros(m)])
    bounds = [(0, None)] * n + [(0, None)] * m
    hess = lambda v: np.diag(np.concatenate([np.ones(n), np.zeros(m)]))
    sol = minimize(fun, v0, jac=jac, hess=hess, constraints=[cons], bounds=bounds, method="trust-constr",
                   options={"gtol": 1e-12, "xtol": 1e-14, "maxiter": 20000})
    x_ref = sol.x[:n]
    assert T.tv(res.x) <= tau + 1e-5 and res.x.min() >= 0.0
    np.testing.assert_allclose(res.x[0], x_ref, atol=2e-4)


def _small_problem():
    import math
    import oracle
    from tests.cases import problem
    geom = dict(beam=0, nx=16, ny=14, n_views=20, n_bins=23, angle_range=math.pi)
    p = problem(geom, K=5, W=2, I0=1e4, seed=12)
    nA, _ = oracle.norm_estimate(p["g_or"], 300, 1e-12)
    eta = 1.0 / (4.0 * oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))
    return oracle, p, eta


def test_solve_tv_with_a_loose_ball_is_the_box_solve():
    # a TV radius no iterate reaches: every projection is the box clamp
    oracle, p, eta = _small_problem()
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 15)
    res = T.solve_tv(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 15, tau=1e9)
    np.testing.assert_allclose(res.x, ref.x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(res.rel_res, ref.rel_res, rtol=1e-10)


def test_solve_prox_tv_with_a_vanishing_lambda_is_the_unconstrained_solve():
    # x = w + theta div p with |p| <= 1: the step moves x by at most 4 theta
    oracle, p, eta = _small_problem()
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 10, lo=-np.inf, hi=np.inf)
    x = T.solve_prox_tv(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 10, lam=1e-10, fgp_iters=5,
                        lo=-np.inf, hi=np.inf)
    np.testing.assert_allclose(x, ref.x, rtol=0, atol=1e-8)
