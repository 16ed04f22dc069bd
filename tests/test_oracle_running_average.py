"""Pins of the running-average stopping rule of Sec. 3.1 (oracle side).

The paper reports, at each iteration t, the average of the previous t/2
iterates and stops at the first t with ||xbar_t - xbar_{t-1}|| <= 1e-5.  The
window reading (m_t = max(1, floor(t/2)) iterates ending at x_t) is pinned
here by closed forms of the running average of sequences whose window sums
are known exactly (arithmetic and geometric), independently of the oracle's
own averaging code; the solver is pinned against the matrix-free C solve
(same iterates) and against a brute-force scan of its change history.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.cases import problem


def test_window_sizes():
    assert [oracle.window_size(t) for t in range(1, 10)] == [1, 1, 1, 2, 2, 3, 3, 4, 4]


def test_running_average_of_arithmetic_sequence():
    # x_t = t: the mean of t-m+1 .. t is t - (m - 1)/2
    T = 41
    avgs = oracle.running_averages([np.array([float(t)]) for t in range(1, T + 1)])
    for t in range(1, T + 1):
        m = max(1, t // 2)
        assert avgs[t - 1][0] == pytest.approx(t - (m - 1) / 2.0, abs=1e-12)
    # the change is 1/2 when the window grows (t even, t >= 4) and 1 when it slides
    for t in range(2, T + 1):
        grow = max(1, t // 2) > max(1, (t - 1) // 2)
        assert avgs[t - 1][0] - avgs[t - 2][0] == pytest.approx(0.5 if grow else 1.0, abs=1e-12)


@pytest.mark.parametrize("rho", [0.5, 0.9, 1.1])
def test_running_average_of_geometric_sequence(rho):
    # x_t = rho^t: sum_{s=t-m+1}^{t} rho^s = rho^(t-m+1) (1 - rho^m) / (1 - rho)
    T = 30
    avgs = oracle.running_averages([np.array([rho ** t, 2.0 * rho ** t]) for t in range(1, T + 1)])
    for t in range(1, T + 1):
        m = max(1, t // 2)
        ref = rho ** (t - m + 1) * (1.0 - rho ** m) / ((1.0 - rho) * m)
        assert avgs[t - 1] == pytest.approx([ref, 2.0 * ref], rel=1e-12)


def _small_case():
    geom = dict(beam=0, nx=24, ny=20, n_views=30, n_bins=33, angle_range=math.pi)
    p = problem(geom, K=6, W=2, I0=1e4, seed=4)
    nA, _ = oracle.norm_estimate(p["g_or"], 200, 1e-10)
    eta = 0.5 / oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays)
    return p, eta


def test_running_average_solve_iterates_match_the_c_solve():
    p, eta = _small_case()
    T = 12
    res = oracle.solve_running_average(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, T, tol=0.0)
    assert res.iters == T and len(res.changes) == T - 1
    # brute force: the iterates x_t from independent C solves of t iterations
    xs = [oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, t).x for t in range(1, T + 1)]
    np.testing.assert_allclose(res.x_last, xs[-1], rtol=0, atol=1e-12)
    m = max(1, T // 2)
    np.testing.assert_allclose(res.x_avg, sum(xs[T - m:]) / m, rtol=0, atol=1e-12)
    avgs = oracle.running_averages(xs)
    ref_changes = [np.linalg.norm(avgs[t] - avgs[t - 1]) for t in range(1, T)]
    np.testing.assert_allclose(res.changes, ref_changes, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("check_every", [1, 3])
def test_running_average_stop_is_the_first_iteration_below_tol(check_every):
    p, eta = _small_case()
    full = oracle.solve_running_average(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 40, tol=0.0)
    ch = full.changes  # ch[k] belongs to t = k + 2
    tol = math.sqrt(ch[14] * ch[15])  # strictly between two consecutive changes
    expect = next(t for t in range(2, 41) if t % check_every == 0 and ch[t - 2] <= tol)
    res = oracle.solve_running_average(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 40, tol=tol,
                                       check_every=check_every)
    assert res.iters == expect
    np.testing.assert_allclose(res.changes, ch[:expect - 1], rtol=1e-12)


def test_running_average_converges_to_the_noiseless_solution():
    # noiseless identifiable case (Theorem 1 with Err = 0): the iterates
    # converge linearly to x*, and so does their running average
    g = oracle.Geometry(beam=0, nx=8, ny=8, n_views=40, n_bins=25, angle_range=math.pi, bin_pitch=0.5)
    e = synth.energy_grid(3)
    S = synth.window_partition(3, 1) * synth.smooth_spectrum(e, 5)[None, :]
    mu = synth.power_law_mu(e, 2.0 / 8)
    xs = synth.rasterize_ellipses(synth.random_ellipses(8, 3, 5), 8, 8, supersample=4)
    I0 = 1e3
    y = oracle.expected_counts(oracle.forward(g, xs), S, mu, I0)
    nA, _ = oracle.norm_estimate(g, 500, 1e-12)
    eta = 1.0 / (4.0 * oracle.lipschitz(nA, S, mu, I0, g.n_rays))
    res = oracle.solve_running_average(g, S, mu, I0, y, eta, 6000, tol=1e-10)
    assert res.iters < 6000
    assert np.linalg.norm(res.x_avg - xs) <= 1e-6 * np.linalg.norm(xs)
