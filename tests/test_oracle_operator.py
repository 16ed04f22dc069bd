"""Pins for the oracle's link, residual, operator F, extragradient solver and
step-size rule.

Pins used: the link's closed-form values (h(0) = sum_k S_k, flat for t < 0,
derivative -sum_k S_k mu_k at 0+, exact logarithmic inversion in the
monochromatic case, Sec. 1.1); F(x*) = 0 for noiseless data (Sec. 1.2,
observation (a)); the monotonicity identity of Eq. (9) computed from the
projections alone, and its sign on random pairs; the Lipschitz bound of
Sec. 4.2; linear convergence of the extragradient iteration in the noiseless
identifiable case (Theorem 1 with Err = 0); the dense-matrix operator on the
same tiny problem; the Gaussian experiment of Sec. 3.2.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import Geometry, dense
from tests.geom_cases import tiny_geometries
from tests.test_oracle_projector import dense_A

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _spectrum(K, W, seed, n_pix):
    e = synth.energy_grid(K)
    phi = synth.smooth_spectrum(e, seed)
    S = synth.window_partition(K, W) * phi[None, :]
    mu = synth.power_law_mu(e, 2.0 / n_pix)
    return S, mu


def test_link_closed_forms():
    S, mu = _spectrum(10, 1, 3, 64)
    s_w, m = S[0], mu
    assert oracle.h(0.0, s_w, m) == pytest.approx(s_w.sum(), rel=1e-15)
    # ReLU: flat for negative projections (Eq. (4))
    for t in (-1e-9, -0.5, -30.0):
        assert oracle.h(t, s_w, m) == pytest.approx(s_w.sum(), rel=1e-15)
    # one-sided derivative at 0+ is -sum_k s_k mu_k (Sec. 4.2, |h'| bound attained at 0)
    eps = 1e-7
    d = (oracle.h(eps, s_w, m) - oracle.h(0.0, s_w, m)) / eps
    assert d == pytest.approx(-(s_w * m).sum(), rel=1e-5)
    # nonincreasing
    ts = np.linspace(0, 200, 400)
    hs = [oracle.h(t, s_w, m) for t in ts]
    assert all(a >= b for a, b in zip(hs, hs[1:]))


def test_monochromatic_log_inversion():
    """W = K = 1: counts I0 s exp(-mu z) invert exactly to z by a logarithm (Sec. 1.1)."""
    z = np.linspace(0.0, 40.0, 101)
    S = np.array([[0.7]])
    mu = np.array([0.23])
    lam = oracle.expected_counts(z, S, mu, 1e4)[0]
    zr = -np.log(lam / (1e4 * 0.7)) / 0.23
    np.testing.assert_allclose(zr, z, rtol=1e-12, atol=1e-12)
    # residual of the exact counts is zero, of scaled counts is the difference
    assert np.abs(oracle.residual(z, S, mu, 1e4, lam[None])).max() < 1e-9
    np.testing.assert_allclose(oracle.residual(z, S, mu, 1e4, 2 * lam[None]), lam, rtol=1e-12)


def test_residual_sums_windows():
    z = np.array([0.0, 1.5, 7.0])
    S, mu = _spectrum(8, 3, 1, 16)
    lam = oracle.expected_counts(z, S, mu, 50.0)
    y = lam + np.arange(9, dtype=float).reshape(3, 3)
    np.testing.assert_allclose(oracle.residual(z, S, mu, 50.0, y), np.arange(9).reshape(3, 3).sum(0),
                               rtol=0, atol=1e-12)
    # at z = 0 every window sees its full intensity I0 * sum_k S[w][k]
    np.testing.assert_allclose(lam[:, 0], 50.0 * S.sum(axis=1), rtol=1e-14)


def _problem(g, W=3, K=12, I0=1e3, seed=0):
    S, mu = _spectrum(K, W, seed, max(g.nx, g.ny))
    xs = synth.ellipse_phantom(max(g.nx, g.ny), 4, seed)[: g.ny, : g.nx]
    lam = oracle.expected_counts(oracle.forward(g, xs), S, mu, I0)
    return S, mu, xs, lam


@pytest.mark.parametrize("gi", [0, 1, 3, 4])
def test_operator_zero_at_truth_noiseless(gi):
    g = tiny_geometries()[gi]
    S, mu, xs, lam = _problem(g)
    F = oracle.operator(g, xs, S, mu, 1e3, lam)
    scale = np.abs(oracle.operator(g, np.zeros_like(xs), S, mu, 1e3, lam)).max()
    assert np.abs(F).max() <= 1e-13 * scale


@pytest.mark.parametrize("gi", [1, 4])
def test_operator_matches_dense(gi):
    g = tiny_geometries()[gi]
    S, mu, xs, lam = _problem(g)
    y = synth.poisson_counts(lam, seed=7)
    x = synth.random_image(g.nx, g.ny, seed=3)
    F = oracle.operator(g, x, S, mu, 1e3, y)
    Fd = dense.operator(dense_A(g), x.ravel(), S, mu, 1e3, y.reshape(S.shape[0], -1))
    np.testing.assert_allclose(F.ravel(), Fd, rtol=1e-10, atol=1e-12 * np.abs(Fd).max())


@pytest.mark.parametrize("gi", [0, 2, 4, 5])
def test_monotonicity_identity_and_sign(gi):
    """<F(x)-F(x'), x-x'> = (I0/m) sum_{w,i} [h_w(z'_i) - h_w(z_i)] (z_i - z'_i) >= 0, Eq. (9)."""
    g = tiny_geometries()[gi]
    S, mu, xs, lam = _problem(g, I0=1e4)
    y = synth.poisson_counts(lam, seed=11)
    rng = np.random.default_rng(gi)
    W = S.shape[0]
    m = W * g.n_rays
    for _ in range(100):
        x = rng.uniform(0, 2, (g.ny, g.nx))
        xp = rng.uniform(0, 2, (g.ny, g.nx))
        lhs = float(((oracle.operator(g, x, S, mu, 1e4, y) - oracle.operator(g, xp, S, mu, 1e4, y))
                     * (x - xp)).sum())
        z, zp = oracle.forward(g, x).ravel(), oracle.forward(g, xp).ravel()
        hz = oracle.expected_counts(z, S, mu, 1e4).sum(0)
        hzp = oracle.expected_counts(zp, S, mu, 1e4).sum(0)
        rhs = float(((hzp - hz) * (z - zp)).sum()) / m
        assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-14)
        assert lhs >= -1e-14


@pytest.mark.parametrize("gi", [1, 3])
def test_lipschitz_bound(gi):
    """||F(x)-F(x')|| <= L ||x-x'|| with L = I0 (||A||^2/m) sum_k C_k mu_k (Sec. 4.2)."""
    g = tiny_geometries()[gi]
    S, mu, xs, lam = _problem(g, I0=1e4)
    y = synth.poisson_counts(lam, seed=1)
    nA, _ = oracle.norm_estimate(g, 3000, 1e-14)
    L = oracle.lipschitz(nA, S, mu, 1e4, S.shape[0] * g.n_rays)
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(50):
        x = rng.uniform(0, 1, (g.ny, g.nx))
        xp = x + rng.uniform(0, 1e-3, x.shape)
        ratio = np.linalg.norm(oracle.operator(g, x, S, mu, 1e4, y) - oracle.operator(g, xp, S, mu, 1e4, y)) \
            / np.linalg.norm(x - xp)
        worst = max(worst, ratio)
    assert worst <= L * (1 + 1e-9)
    assert worst >= 0.01 * L  # the bound is not vacuous


def test_extragradient_linear_convergence_noiseless():
    """Theorem 1 with Err = 0: with eta = 1/(4L) the iterates converge
    linearly to x* when A has full column rank (many views and half-pixel
    bins on a small image give cond(A^T A) ~ 40)."""
    g = Geometry(beam=0, nx=8, ny=8, n_views=40, n_bins=25, angle_range=np.pi, bin_pitch=0.5)
    S, mu = _spectrum(8, 2, 2, 8)
    xs = synth.ellipse_phantom(8, 4, 2, supersample=4)
    lam = oracle.expected_counts(oracle.forward(g, xs), S, mu, 1e4)
    nA, _ = oracle.norm_estimate(g, 3000, 1e-12)
    L = oracle.lipschitz(nA, S, mu, 1e4, S.shape[0] * g.n_rays)
    res = oracle.solve(g, S, mu, 1e4, lam, eta=1.0 / (4 * L), iters=4000)
    assert np.linalg.norm(res.x - xs) <= 1e-6 * np.linalg.norm(xs)
    # geometric decay: equal iteration counts buy equal factors
    h = res.rel_res
    assert h[1999] < 0.1 * h[999] and h[3999] < 0.1 * h[1999]


def test_extragradient_solve_matches_dense_loop():
    g = tiny_geometries()[4]
    S, mu, xs, lam = _problem(g, I0=1e3, seed=4)
    y = synth.poisson_counts(lam, seed=9)
    nA, _ = oracle.norm_estimate(g, 2000, 1e-12)
    eta = 1.0 / (4 * oracle.lipschitz(nA, S, mu, 1e3, S.shape[0] * g.n_rays))
    res = oracle.solve(g, S, mu, 1e3, y, eta, 60)
    xd, _ = dense.solve(dense_A(g), S, mu, 1e3, y.reshape(S.shape[0], -1), eta, 60, lo=0.0, hi=np.inf)
    np.testing.assert_allclose(res.x.ravel(), xd, rtol=1e-9, atol=1e-12)
    assert (res.x >= 0).all()
    # box projection: an upper bound binds
    res2 = oracle.solve(g, S, mu, 1e3, y, eta, 60, hi=0.05)
    assert res2.x.max() <= 0.05 and res2.x.min() >= 0.0


def test_tolerance_stopping_and_average():
    g = tiny_geometries()[0]
    S, mu, xs, lam = _problem(g, W=1, K=6, I0=1e4, seed=3)
    nA, _ = oracle.norm_estimate(g, 2000, 1e-12)
    eta = 1.0 / (4 * oracle.lipschitz(nA, S, mu, 1e4, g.n_rays))
    full = oracle.solve(g, S, mu, 1e4, lam, eta, 300)
    tol = full.rel_res[100] * 1.0001
    stop = oracle.solve(g, S, mu, 1e4, lam, eta, 300, tol=tol, check_every=5)
    first = next(t for t in range(4, 300, 5) if full.rel_res[t] <= tol)
    assert stop.iters == first + 1
    np.testing.assert_allclose(stop.rel_res, full.rel_res[: stop.iters], rtol=1e-15)
    avg = oracle.solve(g, S, mu, 1e4, lam, eta, 10, average_tail=True)
    iterates = [oracle.solve(g, S, mu, 1e4, lam, eta, t).x for t in range(6, 11)]
    np.testing.assert_allclose(avg.x_avg, np.mean(iterates, axis=0), rtol=1e-12, atol=1e-15)


def test_gaussian_experiment_reaches_machine_precision():
    """Sec. 3.2 / Fig. 6: Gaussian a_i, noiseless, W = 1, I0 = 1, mu = 1,
    d = 100, ||x*|| = 3, step 0.25, no projection.  The error reaches machine
    precision, and more samples need fewer iterations."""
    with open(os.path.join(GOLDEN, "gaussian_sec3_2.json")) as f:
        cfg = json.load(f)
    d, norm, step = cfg["d"], cfg["norm_x"], cfg["step"]
    iters_to = {}
    for mult, iters in ((5, 15000), (20, 8000)):
        A, xs = synth.gaussian_case(mult * d, d, norm, seed=mult)
        y = np.exp(-np.maximum(A @ xs, 0.0))  # noiseless counts, I0 = 1, one energy, mu = 1
        _, errs = dense.solve(A, [[1.0]], [1.0], 1.0, y[None], step, iters, x_true=xs)
        assert (errs < 1e-8).any()
        iters_to[mult] = int(np.argmax(errs < 1e-8))
        if mult == 20:
            assert errs.min() < 1e-12 * norm
    assert iters_to[20] < iters_to[5] / 2
