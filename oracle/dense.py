"""Dense-matrix form of the EXACT operator and solver -- TEST INFRASTRUCTURE.

Plain numpy, FP64.  Used for the Gaussian measurement model of Sec. 2.2 and
Sec. 3.2 (a_i ~ N(0, I_d), no projector) and for brute-force checks of the
matrix-free oracle on tiny images.
"""
from __future__ import annotations

import numpy as np


def h(t, S_w, mu):
    """Link of Eq. (7) for one window: sum_k S_w[k] exp(-mu_k max(t, 0))."""
    tp = np.maximum(np.asarray(t, dtype=np.float64), 0.0)
    return np.exp(-np.multiply.outer(tp, np.asarray(mu, dtype=np.float64))) @ np.asarray(S_w, dtype=np.float64)


def operator(A, x, S, mu, I0, y):
    """F(x) = (1/(W n)) sum_{w,i} (y[w][i] - I0 h_w(<a_i, x>)) a_i  (Eq. (8))."""
    A = np.asarray(A, dtype=np.float64)
    S = np.atleast_2d(np.asarray(S, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64).reshape(S.shape[0], A.shape[0])
    z = A @ x
    r = np.zeros(A.shape[0])
    for w in range(S.shape[0]):
        r += y[w] - I0 * h(z, S[w], mu)
    return A.T @ r / (S.shape[0] * A.shape[0])


def solve(A, S, mu, I0, y, eta, iters, x1=None, lo=-np.inf, hi=np.inf, x_true=None):
    """Projected extragradient, Eq. (11), on the box [lo, hi].

    Returns (x, errors) where errors[t] = ||x_{t+1} - x_true|| when ``x_true``
    is given."""
    x = np.zeros(A.shape[1]) if x1 is None else np.array(x1, dtype=np.float64)
    errs = []
    for _ in range(iters):
        xh = np.clip(x - eta * operator(A, x, S, mu, I0, y), lo, hi)
        x = np.clip(x - eta * operator(A, xh, S, mu, I0, y), lo, hi)
        if x_true is not None:
            errs.append(float(np.linalg.norm(x - x_true)))
    return x, np.array(errs)
