"""Pins for the known-background link (Appendix A.1: single-material recovery
when the other materials are known).

(i) The paper's reparametrisation: with known projections P_i and the same
attenuation spectrum, the counts equal I'_i sum_j s'_ij exp(-mu_j z_i) with
I'_i = I sum_j s_j exp(-mu_j P_i) and s'_ij = s_j exp(-mu_j P_i) / sum_j (...);
(ii) a background with the unknown material's own spectrum is a shift of the
projection: h(z; p) = h(z + p) for z >= 0; (iii) F stays monotone (Eq. (9))."""
import numpy as np
import pytest

import oracle
import synth
from tests.geom_cases import tiny_geometries


def _spec(K, W, seed):
    e = synth.energy_grid(K)
    S = synth.window_partition(K, W) * synth.smooth_spectrum(e, seed)[None, :]
    return S, synth.power_law_mu(e, 0.05), e


def test_appendix_reparametrisation():
    S, mu, _ = _spec(12, 1, 1)
    rng = np.random.default_rng(0)
    z = rng.uniform(0, 20, 50)
    P1, P2 = rng.uniform(0, 10, 50), rng.uniform(0, 5, 50)
    I0 = 3e3
    lam = oracle.expected_counts(z, S, mu, I0, bg=(np.stack([mu, mu]), np.stack([P1, P2])))[0]
    s = S[0] / S[0].sum()
    Ibar = I0 * S[0].sum()
    att = np.exp(-np.outer(P1 + P2, mu))               # [i][j]
    I_prime = Ibar * (att * s).sum(axis=1)
    s_prime = (att * s) / (att * s).sum(axis=1, keepdims=True)
    ref = I_prime * (s_prime * np.exp(-np.outer(z, mu))).sum(axis=1)
    np.testing.assert_allclose(lam, ref, rtol=1e-12)


def test_background_with_own_spectrum_is_a_shift():
    S, mu, _ = _spec(10, 3, 2)
    rng = np.random.default_rng(1)
    z = rng.uniform(0, 30, 40)
    p = rng.uniform(0, 10, 40)
    y = rng.uniform(0, 500, (3, 40))
    np.testing.assert_allclose(oracle.residual(z, S, mu, 1e3, y, bg=(mu[None], p[None])),
                               oracle.residual(z + p, S, mu, 1e3, y), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("gi", [1, 4])
def test_background_operator_monotone(gi):
    g = tiny_geometries()[gi]
    S, mu, e = _spec(10, 2, 3)
    mu_bone = synth.power_law_mu(e, 0.12) + 0.01
    xb = synth.random_image(g.nx, g.ny, seed=9, hi=0.5)
    p = oracle.forward(g, xb)[None]
    xs = synth.ellipse_phantom(max(g.nx, g.ny), 3, gi)[: g.ny, : g.nx]
    lam = oracle.expected_counts(oracle.forward(g, xs), S, mu, 1e4, bg=(mu_bone[None], p))
    # noiseless: F vanishes at the truth with the background in the model
    F = oracle.operator(g, xs, S, mu, 1e4, lam, bg=(mu_bone[None], p))
    F0 = oracle.operator(g, np.zeros_like(xs), S, mu, 1e4, lam, bg=(mu_bone[None], p))
    assert np.abs(F).max() <= 1e-12 * np.abs(F0).max()
    rng = np.random.default_rng(gi)
    for _ in range(30):
        x, xp = rng.uniform(0, 1, xs.shape), rng.uniform(0, 1, xs.shape)
        d = (oracle.operator(g, x, S, mu, 1e4, lam, bg=(mu_bone[None], p))
             - oracle.operator(g, xp, S, mu, 1e4, lam, bg=(mu_bone[None], p)))
        assert float((d * (x - xp)).sum()) >= -1e-14
