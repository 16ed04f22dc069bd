"""GPU parity of dense-measurement EXACT (Sec. 2.2 Gaussian model, Sec. 3.2)
against oracle/dense.py, both in FP64.  The operator and whole solves agree
to 1e-10 relative (the sums differ only in order); the experiment of Fig. 6
reaches the error threshold at the same iteration as the oracle."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import dense
import paper_2503_19925_gb300 as ex
from tests.cases import rel_l2

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def test_dense_operator_parity_polychromatic():
    n, d, W, K = 700, 37, 2, 5
    rng = np.random.default_rng(1)
    A = rng.standard_normal((n, d))
    S = rng.uniform(0.1, 1.0, (W, K))
    mu = rng.uniform(0.2, 1.5, K)
    xs = rng.standard_normal(d)
    y = synth.poisson_counts(50.0 * np.stack([dense.h(A @ xs, S[w], mu) for w in range(W)]), 3)
    D = ex.Dense(_t(A), mu, S)
    for x in (np.zeros(d), rng.standard_normal(d), xs):
        F = D.operator(_t(x), _t(y), 50.0).cpu().numpy()
        ref = dense.operator(A, x, S, mu, 50.0, y)
        assert rel_l2(F, ref) <= 1e-12
    D.close()


def test_dense_solve_parity_with_box():
    n, d = 500, 40
    A, xs = synth.gaussian_case(n, d, 3.0, seed=4)
    y = np.exp(-np.maximum(A @ xs, 0.0))
    D = ex.Dense(_t(A), [1.0], [[1.0]])
    x, _ = D.solve(_t(y[None]), 1.0, 0.25, 200, lo=-0.5, hi=0.5)
    ref, _ = dense.solve(A, [[1.0]], [1.0], 1.0, y[None], 0.25, 200, lo=-0.5, hi=0.5)
    assert rel_l2(x.cpu().numpy(), ref) <= 1e-10
    D.close()


def test_gaussian_experiment_fig6_matches_oracle():
    """Fig. 6 setting at n = 20 d: the GPU error trajectory follows the
    oracle's over the first 2000 iterations and goes on to machine precision."""
    with open(os.path.join(GOLDEN, "gaussian_sec3_2.json")) as f:
        cfg = json.load(f)
    d, norm, step = cfg["d"], cfg["norm_x"], cfg["step"]
    mult = 20
    A, xs = synth.gaussian_case(mult * d, d, norm, seed=mult)
    y = np.exp(-np.maximum(A @ xs, 0.0))
    D = ex.Dense(_t(A), [1.0], [[1.0]])
    _, err = D.solve(_t(y[None]), 1.0, step, 10000, x_true=_t(xs))
    err = err.cpu().numpy()
    _, ref = dense.solve(A, [[1.0]], [1.0], 1.0, y[None], step, 2000, x_true=xs)
    np.testing.assert_allclose(err[:2000], ref, rtol=1e-7)
    assert err.min() < 1e-12 * norm
    D.close()
