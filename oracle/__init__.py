"""FP64 CPU oracle for the EXACT hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The CUDA path never does, and it shares no
code with it (geometry conventions are restated, not imported).

``exact_oracle.c`` holds the arithmetic (Joseph projector, scatter adjoint,
per-window link, operator F, projected extragradient, power iteration); this
module compiles it with gcc on first use (or via :func:`build`) and wraps it
with ctypes.  ``dense.py`` holds the dense-matrix (Gaussian measurement) form
of the same operator and solver.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, exact identities and brute force (see the test
docstrings); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# EXACT_ORACLE_SRC points the oracle at another copy of its C source; the
# mutation tests use it to check that the pins catch planted mistakes.
_SRC = os.environ.get("EXACT_ORACLE_SRC") or os.path.join(_HERE, "exact_oracle.c")
_OUT_DIR = os.path.join(os.path.dirname(os.path.abspath(_SRC)), "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("pixel", ctypes.c_double), ("n_views", ctypes.c_int),
                ("angle0", ctypes.c_double), ("angle_range", ctypes.c_double),
                ("n_bins", ctypes.c_int), ("bin_pitch", ctypes.c_double),
                ("det_offset", ctypes.c_double), ("src_to_center", ctypes.c_double),
                ("src_to_det", ctypes.c_double)]


@dataclass(frozen=True)
class Geometry:
    """Scan geometry (same meaning as ``exact_geometry`` of the C ABI)."""
    beam: int  # 0 parallel, 1 fan
    nx: int
    ny: int
    n_views: int
    n_bins: int
    pixel: float = 1.0
    angle0: float = 0.0
    angle_range: float = np.pi
    bin_pitch: float = 1.0
    det_offset: float = 0.0
    src_to_center: float = 0.0
    src_to_det: float = 0.0

    @property
    def n_rays(self) -> int:
        return self.n_views * self.n_bins

    @property
    def d(self) -> int:
        return self.nx * self.ny

    def _c(self) -> _Geom:
        return _Geom(self.beam, self.nx, self.ny, self.pixel, self.n_views, self.angle0,
                     self.angle_range, self.n_bins, self.bin_pitch, self.det_offset,
                     self.src_to_center, self.src_to_det)


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            G = ctypes.POINTER(_Geom)
            lib.ora_rays.argtypes = [G, _I, _D, _D, _D]
            lib.ora_forward.argtypes = [G, _D, _D]
            lib.ora_adjoint.argtypes = [G, _D, _D]
            lib.ora_h.argtypes = [ctypes.c_double, ctypes.c_int, _D, _D]
            lib.ora_h.restype = ctypes.c_double
            lib.ora_expected_counts.argtypes = [ctypes.c_long, _D, ctypes.c_int, ctypes.c_int, _D, _D,
                                                ctypes.c_double, _D]
            lib.ora_expected_counts_bg.argtypes = [ctypes.c_long, _D, ctypes.c_int, ctypes.c_int, _D, _D,
                                                   ctypes.c_double, ctypes.c_int, _D, _D, _D]
            lib.ora_residual_bg.argtypes = [ctypes.c_long, _D, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double,
                                            ctypes.c_int, _D, _D, _D, _D]
            lib.ora_operator_bg.argtypes = [G, _D, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double,
                                            ctypes.c_int, _D, _D, _D, _D, _D, _D]
            lib.ora_solve_bg.argtypes = [G, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_int, _D,
                                         _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, _D, _D, _D]
            lib.ora_solve_bg.restype = ctypes.c_int
            lib.ora_residual.argtypes = [ctypes.c_long, _D, ctypes.c_int, ctypes.c_int, _D, _D,
                                         ctypes.c_double, _D, _D]
            lib.ora_operator.argtypes = [G, _D, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double,
                                         _D, _D, _D, _D]
            lib.ora_solve.argtypes = [G, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, _D,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, _D, _D, _D]
            lib.ora_solve.restype = ctypes.c_int
            lib.ora_norm_estimate.argtypes = [G, ctypes.c_int, ctypes.c_double, _I]
            lib.ora_norm_estimate.restype = ctypes.c_double
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _bg(bg, n: int, K: int):
    """Known-background arguments: bg = (mu_bg [M][K], p [M][n...]) or None."""
    if bg is None:
        return 0, None, None, ()
    mu_bg = np.ascontiguousarray(bg[0], dtype=np.float64).reshape(-1, K)
    p = np.ascontiguousarray(bg[1], dtype=np.float64).reshape(mu_bg.shape[0], n)
    return mu_bg.shape[0], _p(mu_bg), _p(p), (mu_bg, p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def rays(g: Geometry):
    """Per-ray Joseph parameters (axis, alpha, beta, delta), each of length n_rays."""
    lib = _load()
    n = g.n_rays
    axis = np.zeros(n, dtype=np.int32)
    alpha, beta, delta = (np.zeros(n) for _ in range(3))
    gc = g._c()
    lib.ora_rays(ctypes.byref(gc), axis.ctypes.data_as(_I), _p(alpha), _p(beta), _p(delta))
    return axis, alpha, beta, delta


def forward(g: Geometry, x) -> np.ndarray:
    """z = A x for an image ``x`` of shape [ny][nx]; returns [n_views][n_bins]."""
    lib = _load()
    x = _f64(x).reshape(g.ny, g.nx)
    z = np.zeros((g.n_views, g.n_bins))
    gc = g._c()
    lib.ora_forward(ctypes.byref(gc), _p(x), _p(z))
    return z


def adjoint(g: Geometry, r) -> np.ndarray:
    """A^T r for a sinogram ``r`` [n_views][n_bins]; returns [ny][nx]."""
    lib = _load()
    r = _f64(r).reshape(g.n_views, g.n_bins)
    out = np.zeros((g.ny, g.nx))
    gc = g._c()
    lib.ora_adjoint(ctypes.byref(gc), _p(r), _p(out))
    return out


def h(t: float, S_w, mu) -> float:
    """Link of one window, sum_k S_w[k] exp(-mu_k max(t, 0))."""
    S_w, mu = _f64(S_w), _f64(mu)
    return _load().ora_h(float(t), len(mu), _p(S_w), _p(mu))


def expected_counts(z, S, mu, I0: float, bg=None) -> np.ndarray:
    """Mean counts lam[w][...] = I0 h_w(z) for projections ``z`` (any shape);
    bg = (mu_bg [M][K], p [M][...]) adds known background materials."""
    lib = _load()
    z = _f64(z)
    S, mu = _f64(S), _f64(mu)
    W, K = S.shape
    lam = np.zeros((W,) + z.shape)
    M, pm, pp, keep = _bg(bg, z.size, K)
    lib.ora_expected_counts_bg(z.size, _p(z), W, K, _p(S), _p(mu), float(I0), M, pm, pp, _p(lam))
    return lam


def residual(z, S, mu, I0: float, y, bg=None) -> np.ndarray:
    """r = sum_w (y[w] - I0 h_w(z)); ``y`` has shape [W] + z.shape."""
    lib = _load()
    z = _f64(z)
    S, mu, y = _f64(S), _f64(mu), _f64(y)
    W, K = S.shape
    assert y.shape == (W,) + z.shape
    r = np.zeros(z.shape)
    M, pm, pp, keep = _bg(bg, z.size, K)
    lib.ora_residual_bg(z.size, _p(z), W, K, _p(S), _p(mu), float(I0), M, pm, pp, _p(y), _p(r))
    return r


def operator(g: Geometry, x, S, mu, I0: float, y, bg=None) -> np.ndarray:
    """F(x) = (1/(W n)) A^T sum_w (y_w - I0 h_w(A x)); returns [ny][nx]."""
    lib = _load()
    x = _f64(x).reshape(g.ny, g.nx)
    S, mu, y = _f64(S), _f64(mu), _f64(y)
    W, K = S.shape
    assert y.size == W * g.n_rays
    F = np.zeros((g.ny, g.nx))
    z = np.zeros(g.n_rays)
    r = np.zeros(g.n_rays)
    gc = g._c()
    M, pm, pp, keep = _bg(bg, g.n_rays, K)
    lib.ora_operator_bg(ctypes.byref(gc), _p(x), W, K, _p(S), _p(mu), float(I0), M, pm, pp, _p(y), _p(F), _p(z),
                        _p(r))
    return F


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    rel_res: np.ndarray
    x_avg: np.ndarray | None = None


def solve(g: Geometry, S, mu, I0: float, y, eta: float, iters: int, x1=None,
          lo: float = 0.0, hi: float = np.inf, tol: float = 0.0, check_every: int = 1,
          average_tail: bool = False, bg=None) -> SolveResult:
    """Projected extragradient (Eq. (11)) on the box [lo, hi]; x1 defaults to 0."""
    lib = _load()
    S, mu, y = _f64(S), _f64(mu), _f64(y)
    W, K = S.shape
    x = np.zeros((g.ny, g.nx)) if x1 is None else _f64(x1).reshape(g.ny, g.nx).copy()
    hist = np.zeros(max(iters, 1))
    avg = np.zeros((g.ny, g.nx)) if average_tail else None
    gc = g._c()
    M, pm, pp, keep = _bg(bg, g.n_rays, K)
    done = lib.ora_solve_bg(ctypes.byref(gc), W, K, _p(S), _p(mu), float(I0), M, pm, pp, _p(y), float(eta),
                            int(iters), float(lo), float(hi), float(tol), int(check_every), _p(x), _p(hist),
                            _p(avg) if avg is not None else None)
    return SolveResult(x, done, hist[:done], avg)


def window_size(t: int) -> int:
    """Iterates in the running average at iteration t >= 1.  Sec. 3.1
    averages "the previous t/2 iterates"; read as floor(t/2), and at least
    one so that the average exists from the first iteration."""
    return max(1, t // 2)


def running_averages(iterates):
    """xbar_t for t = 1 .. T of the iterate sequence [x_1, ..., x_T]: the plain
    mean of x_{t-m+1} .. x_t with m = window_size(t) (brute force, FP64)."""
    xs = [np.asarray(v, dtype=np.float64) for v in iterates]
    out = []
    for t in range(1, len(xs) + 1):
        m = window_size(t)
        out.append(sum(xs[t - m:t]) / m)
    return out


@dataclass
class WindowSolveResult:
    x_avg: np.ndarray        # xbar_T
    iters: int               # T
    changes: np.ndarray      # ||xbar_t - xbar_{t-1}|| for t = 2 .. T
    x_last: np.ndarray       # x_T


def solve_running_average(g: Geometry, S, mu, I0: float, y, eta: float, iters: int, tol: float,
                          check_every: int = 1, x1=None, lo: float = 0.0, hi: float = np.inf,
                          bg=None) -> WindowSolveResult:
    """Projected extragradient (Eq. (11)) with the stopping rule of Sec. 3.1:
    stop after the first iteration t >= 2 (a multiple of check_every) with
    ||xbar_t - xbar_{t-1}||_2 <= tol, where xbar_t is the running average of
    window_size(t) iterates; return xbar_T.  x1 (default 0) is projected onto
    the box first.  Each step calls the C operator; the window is kept as a
    list of the FP64 iterates and averaged directly."""
    S, mu, y = _f64(S), _f64(mu), _f64(y)
    x = np.zeros((g.ny, g.nx)) if x1 is None else _f64(x1).reshape(g.ny, g.nx).copy()
    x = np.clip(x, lo, hi)
    window, changes = [], []
    prev = None
    xbar = x.copy()
    t = 0
    for t in range(1, iters + 1):
        xh = np.clip(x - eta * operator(g, x, S, mu, I0, y, bg), lo, hi)
        x = np.clip(x - eta * operator(g, xh, S, mu, I0, y, bg), lo, hi)
        window.append(x.copy())
        m = window_size(t)
        del window[:-m]
        xbar = sum(window) / m
        if prev is not None:
            changes.append(float(np.linalg.norm(xbar - prev)))
            if tol > 0.0 and check_every > 0 and t % check_every == 0 and changes[-1] <= tol:
                break
        prev = xbar
    return WindowSolveResult(xbar, t, np.array(changes), x)


def norm_estimate(g: Geometry, max_iters: int = 500, rtol: float = 1e-9):
    """Power-iteration estimate of ||A||_op^2; returns (lam, iterations)."""
    lib = _load()
    it = ctypes.c_int(0)
    gc = g._c()
    lam = lib.ora_norm_estimate(ctypes.byref(gc), int(max_iters), float(rtol), ctypes.byref(it))
    return lam, it.value


def lipschitz(normA_sq: float, S, mu, I0: float, n_meas: int) -> float:
    """L = I0 (||A||^2 / m) sum_k (sum_w S[w][k]) mu_k with m = W * n rays:
    the bound of Sec. 4.2 (proof of Theorem 2) with the 1/n of Sigma = A^T A / n,
    summed over windows."""
    S, mu = _f64(S), _f64(mu)
    return float(I0) * normA_sq / float(n_meas) * float((S.sum(axis=0) * mu).sum())


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
