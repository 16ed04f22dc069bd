"""Projection onto the TV ball intersected with a box -- TEST INFRASTRUCTURE.

Plain numpy, FP64.  Sec. 3.1 (implementation of projections) constrains the
reconstruction to X = X1 ∩ X2 with X1 = {x : ||x||_TV <= tau} and X2 the
nonnegative orthant (here any box [lo, hi], the orthant being lo = 0,
hi = +inf), and computes P_X by Dykstra's alternating projections between
P_X1 and P_X2.  P_X1(z) is approximated by the TV-regularised problem
    argmin_x ||x - z||^2 + lam ||x||_TV
with lam found by bisection until | ||x||_TV - tau | <= tol_tv.

Readings of what the paper leaves open (each mirrored by the CUDA path):
  - ||x||_TV is the isotropic total variation with forward differences and
    zero difference past the last row / column (Neumann boundary);
  - the TV-regularised problem is solved by the fast gradient projection
    method of Beck and Teboulle (FISTA on the dual of the Chambolle
    formulation) with a fixed number of iterations; the dual variable is
    carried from one solve to the next within a projection (warm start);
  - the bisection starts at lam0 (1 if lam0 <= 0), doubles lam while the TV
    is too large and no upper end is known, then halves the bracket; at most
    max_bisect solves per P_X1;
  - Dykstra stops when ||z_{k+1} - z_k|| <= tol_dykstra or after max_dykstra
    rounds; when ||z + p||_TV <= tau already, P_X1 is the identity.
The steps follow the paper's order and notation (z_k, p_k, q_k, y_k).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def grad(x):
    """Forward differences (gx along columns j, gy along rows i); zero at the
    last column / row."""
    x = np.asarray(x, dtype=np.float64)
    gx = np.zeros_like(x)
    gy = np.zeros_like(x)
    gx[:, :-1] = x[:, 1:] - x[:, :-1]
    gy[:-1, :] = x[1:, :] - x[:-1, :]
    return gx, gy


def div(px, py):
    """Discrete divergence, the negative adjoint of grad: <grad x, p> = -<x, div p>."""
    px = np.asarray(px, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    d = np.zeros_like(px)
    d[:, :-1] += px[:, :-1]
    d[:, 1:] -= px[:, :-1]
    d[:-1, :] += py[:-1, :]
    d[1:, :] -= py[:-1, :]
    return d


def tv(x) -> float:
    """Isotropic total variation sum_ij sqrt(gx^2 + gy^2)."""
    gx, gy = grad(x)
    return float(np.sqrt(gx * gx + gy * gy).sum())


def prox_tv(z, lam: float, iters: int, px=None, py=None):
    """argmin_x ||x - z||^2 + lam ||x||_TV, i.e. the ROF problem
    1/2 ||x - z||^2 + theta ||x||_TV with theta = lam / 2, by `iters` steps of
    the fast gradient projection method on its dual
        min_{|p_ij| <= 1} 1/2 ||z + theta div p||^2,
    whose gradient is -theta grad(z + theta div p) with Lipschitz constant
    8 theta^2.  (px, py) is the starting dual (zeros if None).  Returns
    (x, px, py) with x = z + theta div p."""
    z = np.asarray(z, dtype=np.float64)
    theta = 0.5 * lam
    px = np.zeros_like(z) if px is None else np.array(px, dtype=np.float64)
    py = np.zeros_like(z) if py is None else np.array(py, dtype=np.float64)
    rx, ry = px.copy(), py.copy()
    t = 1.0
    step = 1.0 / (8.0 * theta)
    for _ in range(iters):
        gx, gy = grad(z + theta * div(rx, ry))
        qx = rx + step * gx
        qy = ry + step * gy
        nrm = np.maximum(1.0, np.sqrt(qx * qx + qy * qy))
        nx_, ny_ = qx / nrm, qy / nrm
        t_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        beta = (t - 1.0) / t_next
        rx = nx_ + beta * (nx_ - px)
        ry = ny_ + beta * (ny_ - py)
        px, py, t = nx_, ny_, t_next
    return z + theta * div(px, py), px, py


@dataclass
class TvOptions:
    fgp_iters: int = 40
    max_bisect: int = 40
    max_dykstra: int = 50
    tol_tv: float = 0.01
    tol_dykstra: float = 1e-4
    lam0: float = 0.0


def project_tv_ball(w, tau: float, opts: TvOptions, lam: float, px, py):
    """Approximate P_X1(w) by bisection on lam.  Returns (y, lam, px, py,
    solves); lam, px, py carry over to the next call of the same projection."""
    w = np.asarray(w, dtype=np.float64)
    if tv(w) <= tau:
        return w.copy(), lam, px, py, 0
    lam = lam if lam > 0.0 else 1.0
    lo, hi = 0.0, np.inf
    x = w
    solves = 0
    for _ in range(opts.max_bisect):
        x, px, py = prox_tv(w, lam, opts.fgp_iters, px, py)
        solves += 1
        T = tv(x)
        if abs(T - tau) <= opts.tol_tv:
            break
        if T > tau:
            lo = lam
        else:
            hi = lam
        lam = 2.0 * lam if hi == np.inf else 0.5 * (lo + hi)
    return x, lam, px, py, solves


@dataclass
class TvResult:
    x: np.ndarray
    lam: float
    rounds: int
    solves: int


def project_tv_box(z, tau: float, lo: float = 0.0, hi: float = np.inf, opts: TvOptions | None = None) -> TvResult:
    """Dykstra's algorithm for P_X(z), X = {||x||_TV <= tau} ∩ [lo, hi]^d:
        y_k = P_X1(z_k + p_k),  p_{k+1} = z_k + p_k - y_k,
        z_{k+1} = P_X2(y_k + q_k),  q_{k+1} = y_k + q_k - z_{k+1},
    from z_0 = z, p_0 = q_0 = 0, until ||z_{k+1} - z_k|| <= tol_dykstra."""
    opts = opts or TvOptions()
    zk = np.array(z, dtype=np.float64)
    p = np.zeros_like(zk)
    q = np.zeros_like(zk)
    px = np.zeros_like(zk)
    py = np.zeros_like(zk)
    lam = opts.lam0
    solves = 0
    k = 0
    for k in range(1, opts.max_dykstra + 1):
        w = zk + p
        y, lam, px, py, s = project_tv_ball(w, tau, opts, lam, px, py)
        solves += s
        p = w - y
        zn = np.clip(y + q, lo, hi)
        q = y + q - zn
        change = float(np.linalg.norm(zn - zk))
        zk = zn
        if change <= opts.tol_dykstra:
            break
    return TvResult(zk, lam, k, solves)


@dataclass
class TvSolveResult:
    x: np.ndarray            # x_T, or xbar_T with the running-average rule
    rel_res: np.ndarray
    lam_half: float
    lam_full: float
    iters: int = 0
    changes: np.ndarray | None = None  # running-average rule: ||xbar_t - xbar_{t-1}||, t = 2 .. T


def solve_tv(g, S, mu, I0: float, y, eta: float, iters: int, tau: float, lo: float = 0.0, hi: float = np.inf,
             opts: TvOptions | None = None, x1=None, bg=None, running_average: bool = False, tol: float = 0.0,
             check_every: int = 1) -> TvSolveResult:
    """Projected extragradient (Eq. (11)) on X = {||x||_TV <= tau} ∩ [lo, hi]^d:
        x_{t+1/2} = P_X(x_t - eta F(x_t)),  x_{t+1} = P_X(x_t - eta F(x_{t+1/2})),
    P_X by project_tv_box.  Each of the two projections of an iteration starts
    its bisection from its own lam of the previous iteration (opts.lam0 at the
    first).  x1 (default 0) is clamped to the box only (0 lies in X).  With
    running_average the stopping rule and output of Sec. 3.1 apply (see
    oracle.solve_running_average), else the relative-change rule with tol."""
    import oracle
    opts = opts or TvOptions()
    x = np.zeros((g.ny, g.nx)) if x1 is None else np.array(x1, dtype=np.float64).reshape(g.ny, g.nx)
    x = np.clip(x, lo, hi)
    lam_h = lam_f = opts.lam0
    rel, window, changes = [], [], []
    prev = None
    t = 0
    for t in range(1, iters + 1):
        w = x - eta * oracle.operator(g, x, S, mu, I0, y, bg)
        r1 = project_tv_box(w, tau, lo, hi, TvOptions(**{**opts.__dict__, "lam0": lam_h}))
        lam_h = r1.lam
        w2 = x - eta * oracle.operator(g, r1.x, S, mu, I0, y, bg)
        r2 = project_tv_box(w2, tau, lo, hi, TvOptions(**{**opts.__dict__, "lam0": lam_f}))
        lam_f = r2.lam
        rel.append(float(np.linalg.norm(r2.x - x) / max(np.linalg.norm(x), 1e-30)))
        x = r2.x
        stop = False
        if running_average:
            window.append(x.copy())
            m = oracle.window_size(t)
            del window[:-m]
            xbar = sum(window) / m
            if prev is not None:
                changes.append(float(np.linalg.norm(xbar - prev)))
                stop = tol > 0.0 and check_every > 0 and t % check_every == 0 and changes[-1] <= tol
            prev = xbar
        else:
            stop = tol > 0.0 and check_every > 0 and t % check_every == 0 and rel[-1] <= tol
        if stop:
            break
    out = (sum(window) / len(window)) if running_average and window else x
    return TvSolveResult(out, np.array(rel), lam_h, lam_f, t, np.array(changes) if running_average else None)


def solve_prox_tv(g, S, mu, I0: float, y, eta: float, iters: int, lam: float, fgp_iters: int = 40, x1=None,
                  lo: float = 0.0, hi: float = np.inf, bg=None) -> np.ndarray:
    """The proximal variant of the extragradient iteration proposed in the
    Discussion (Sec. 5), with l_X = ||.||_TV and a constant lam:
        x_{t+1/2} = argmin_x ||x - (x_t - eta F(x_t))||^2 + lam ||x||_TV,
        x_{t+1}   = argmin_x ||x - (x_t - eta F(x_{t+1/2}))||^2 + lam ||x||_TV,
    each solved by prox_tv with fgp_iters steps from a zero dual.  There is no
    constraint; x1 (default 0) is clamped to [lo, hi] once."""
    import oracle
    x = np.zeros((g.ny, g.nx)) if x1 is None else np.array(x1, dtype=np.float64).reshape(g.ny, g.nx)
    x = np.clip(x, lo, hi)
    for _ in range(iters):
        xh, _, _ = prox_tv(x - eta * oracle.operator(g, x, S, mu, I0, y, bg), lam, fgp_iters)
        x, _, _ = prox_tv(x - eta * oracle.operator(g, xh, S, mu, I0, y, bg), lam, fgp_iters)
    return x
