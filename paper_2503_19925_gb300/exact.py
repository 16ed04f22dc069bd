"""Thin Python binding of ``libexact.so`` (include/exact.h).

Argument marshalling only: tensors are checked (device, dtype, shape,
contiguity) and passed as raw pointers with the current torch stream; every
step of the computation runs in the library's CUDA kernels.  Loading fails
loudly when the library cannot be built or loaded; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import torch

from . import _build

EXACT_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory", 4: "timeout",
          5: "non-finite residual", 6: "unsupported", 7: "no workspace bound"}
F32, BF16 = 0, 1
MAX_ENERGY = 256


class ExactError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)} (status {status})")
        self.status = status


class _Geometry(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("pixel", ctypes.c_double), ("n_views", ctypes.c_int),
                ("angle0", ctypes.c_double), ("angle_range", ctypes.c_double),
                ("n_bins", ctypes.c_int), ("bin_pitch", ctypes.c_double),
                ("det_offset", ctypes.c_double), ("src_to_center", ctypes.c_double),
                ("src_to_det", ctypes.c_double)]


class _Spectrum(ctypes.Structure):
    _fields_ = [("n_energy", ctypes.c_int), ("mu", ctypes.POINTER(ctypes.c_double))]


class _Windows(ctypes.Structure):
    _fields_ = [("n_windows", ctypes.c_int), ("S", ctypes.POINTER(ctypes.c_double))]


class _TvOpts(ctypes.Structure):
    _fields_ = [("fgp_iters", ctypes.c_int), ("max_bisect", ctypes.c_int), ("max_dykstra", ctypes.c_int),
                ("pad", ctypes.c_int), ("tol_tv", ctypes.c_double), ("tol_dykstra", ctypes.c_double),
                ("lam0", ctypes.c_double)]


class _TvInfo(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("solves", ctypes.c_int), ("lam", ctypes.c_double),
                ("status", ctypes.c_int)]


class _Tuning(ctypes.Structure):
    _fields_ = [("adj_split", ctypes.c_int), ("reserved", ctypes.c_int * 7)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double), ("hi", ctypes.c_double), ("tol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("average_tail", ctypes.c_int), ("stop_rule", ctypes.c_int),
                ("history_cap", ctypes.c_int), ("history", ctypes.c_void_p), ("tv_bound", ctypes.c_double),
                ("tv", _TvOpts), ("prox_lambda", ctypes.c_double), ("t0", ctypes.c_int),
                ("total_iters", ctypes.c_int), ("resume", ctypes.c_void_p), ("x_last", ctypes.c_void_p),
                ("launch", ctypes.c_int), ("pad", ctypes.c_int)]


class _SolveInfo(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int), ("rel_res", ctypes.c_double), ("status", ctypes.c_int),
                ("avg_change", ctypes.c_double)]


STOP_RULES = {"residual": 0, "average": 1}


class _Job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("y", ctypes.c_void_p), ("y_dtype", ctypes.c_int),
                ("I0", ctypes.c_double), ("eta", ctypes.c_double), ("iters", ctypes.c_int),
                ("opts", _SolveOpts), ("x", ctypes.c_void_p), ("info", ctypes.POINTER(_SolveInfo))]


_lib = None

# every function declared in include/exact.h: (name, restype, argtypes)
_VP, _CP = ctypes.c_void_p, ctypes.c_char_p
_SIGS = [
    ("exact_plan_create", ctypes.c_int, [ctypes.POINTER(_Geometry), ctypes.POINTER(_Spectrum),
                                         ctypes.POINTER(_Windows), ctypes.POINTER(_VP)]),
    ("exact_plan_destroy", ctypes.c_int, [_VP]),
    ("exact_plan_dims", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    ("exact_plan_workspace_bytes", ctypes.c_size_t, [_VP]),
    ("exact_plan_bind_workspace", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("exact_forward", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("exact_adjoint", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("exact_operator", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double, _VP, _VP]),
    ("exact_operator_static", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double, _VP, _VP]),
    ("exact_solve_opts_default", _SolveOpts, []),
    ("exact_solve_resume_bytes", ctypes.c_size_t, [_VP]),
    ("exact_solve", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(_SolveOpts), _VP, ctypes.POINTER(_SolveInfo), _VP]),
    ("exact_solve_host", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(_SolveOpts), _VP, ctypes.POINTER(_SolveInfo), _VP]),
    ("exact_norm_estimate", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int), _VP]),
    ("exact_norm_estimate_f32", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_int), _VP]),
    ("exact_recommended_eta", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_double)]),
    ("exact_plan_nnz", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    ("exact_plan_get_tuning", ctypes.c_int, [_VP, ctypes.POINTER(_Tuning)]),
    ("exact_plan_set_tuning", ctypes.c_int, [_VP, ctypes.POINTER(_Tuning)]),
    ("exact_plan_autotune", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_Tuning), _VP]),
    ("exact_dense_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, ctypes.POINTER(_Spectrum),
                                          ctypes.POINTER(_Windows), ctypes.POINTER(_VP)]),
    ("exact_dense_destroy", ctypes.c_int, [_VP]),
    ("exact_dense_operator", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, _VP, _VP]),
    ("exact_dense_solve", ctypes.c_int, [_VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, _VP, _VP, _VP, _VP]),
    ("exact_tv_opts_default", _TvOpts, []),
    ("exact_tv_workspace_bytes", ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    ("exact_tv_prox", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, ctypes.c_double, ctypes.c_int, _VP, _VP,
                                     ctypes.c_size_t, _VP]),
    ("exact_tv_project", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(_TvOpts), _VP, _VP, ctypes.c_size_t,
                                        ctypes.POINTER(_TvInfo), _VP]),
    ("exact_plan_set_background", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _VP]),
    ("exact_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_VP)]),
    ("exact_batch_destroy", ctypes.c_int, [_VP]),
    ("exact_batch_solve", ctypes.c_int, [_VP, ctypes.POINTER(_Job), ctypes.c_int, _VP]),
    ("exact_batch_set_policy", ctypes.c_int, [_VP, ctypes.c_int]),
    ("exact_batch_get_policy", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    ("exact_batch_autotune", ctypes.c_int, [_VP, ctypes.POINTER(_Job), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            _VP]),
    ("exact_profile_enable", ctypes.c_int, [_VP, ctypes.c_int]),
    ("exact_profile_read", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    ("exact_probe_gather_ceiling", ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                                  _VP]),
    ("exact_debug_inject", ctypes.c_int, [ctypes.c_int, ctypes.c_longlong]),
    ("exact_status_string", _CP, [ctypes.c_int]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libexact.so (building it first if missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_needed else _build.LIB
        lib = ctypes.CDLL(path)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(fn: str, status: int):
    if status != EXACT_OK:
        raise ExactError(fn, status)


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


@dataclass(frozen=True)
class Geometry:
    """Scan geometry, same fields and meaning as ``exact_geometry``."""
    beam: int
    nx: int
    ny: int
    n_views: int
    n_bins: int
    pixel: float = 1.0
    angle0: float = 0.0
    angle_range: float = math.pi
    bin_pitch: float = 1.0
    det_offset: float = 0.0
    src_to_center: float = 0.0
    src_to_det: float = 0.0

    @property
    def n_rays(self) -> int:
        return self.n_views * self.n_bins

    def _c(self) -> _Geometry:
        return _Geometry(self.beam, self.nx, self.ny, self.pixel, self.n_views, self.angle0,
                         self.angle_range, self.n_bins, self.bin_pitch, self.det_offset,
                         self.src_to_center, self.src_to_det)


@dataclass
class SolveInfo:
    iters_done: int
    rel_res: float
    status: int
    avg_change: float = 0.0


def tv_options(changes: dict | None = None) -> _TvOpts:
    """exact_tv_opts_default() with the given fields replaced."""
    o = load().exact_tv_opts_default()
    for k, v in (changes or {}).items():
        if k not in dict(_TvOpts._fields_) or k == "pad":
            raise KeyError(f"unknown TV option {k!r}")
        setattr(o, k, v)
    return o


@dataclass
class TvInfo:
    rounds: int
    solves: int
    lam: float
    status: int


def tv_project(z: torch.Tensor, tau: float, lo: float = 0.0, hi: float = math.inf, opts: dict | None = None,
               out: torch.Tensor | None = None):
    """Projection of the device image z [ny][nx] FP32 onto
    {||x||_TV <= tau} ∩ [lo, hi]^d (exact_tv_project; the workspace is
    allocated here).  Returns (x, TvInfo)."""
    lib = load()
    if z.dtype != torch.float32 or z.dim() != 2 or not z.is_cuda or not z.is_contiguous():
        raise ValueError("z must be a contiguous CUDA float32 [ny][nx] tensor")
    ny, nx = z.shape
    nb = lib.exact_tv_workspace_bytes(nx, ny)
    if nb == 0:
        raise RuntimeError("exact_tv_workspace_bytes returned 0")
    ws = torch.empty(nb, dtype=torch.uint8, device=z.device)
    x = out if out is not None else torch.empty_like(z)
    o = tv_options(opts)
    info = _TvInfo()
    _check("exact_tv_project", lib.exact_tv_project(nx, ny, _ptr(z), float(tau), float(lo), float(hi),
                                                    ctypes.byref(o), _ptr(x), _ptr(ws), nb, ctypes.byref(info),
                                                    _stream()))
    return x, TvInfo(info.rounds, info.solves, info.lam, info.status)


def gather_ceiling() -> tuple[float, int]:
    """Measured shared-memory gather rate of the current device (words/s) and
    its SM count (exact_probe_gather_ceiling; synchronises)."""
    w = ctypes.c_double()
    n = ctypes.c_int()
    _check("exact_probe_gather_ceiling", load().exact_probe_gather_ceiling(ctypes.byref(w), ctypes.byref(n),
                                                                           _stream()))
    return w.value, n.value


class Dense:
    """EXACT with an explicit FP64 measurement matrix A [n][d] on the device
    (the Gaussian model of Sec. 2.2 / the experiment of Sec. 3.2); A must stay
    alive and unchanged while the context is used."""

    def __init__(self, A: torch.Tensor, mu, S):
        lib = load()
        if A.dtype != torch.float64 or A.dim() != 2 or not A.is_cuda or not A.is_contiguous():
            raise ValueError("A must be a contiguous CUDA float64 [n][d] tensor")
        self.A = A
        self.n, self.d = A.shape
        mu = [float(v) for v in mu]
        rows = [[float(v) for v in r] for r in S]
        self.W, self.K = len(rows), len(mu)
        mu_arr = (ctypes.c_double * self.K)(*mu)
        s_arr = (ctypes.c_double * (self.W * self.K))(*[v for r in rows for v in r])
        h = ctypes.c_void_p()
        _check("exact_dense_create", lib.exact_dense_create(self.n, self.d, _ptr(A), ctypes.byref(_Spectrum(self.K, mu_arr)),
                                                            ctypes.byref(_Windows(self.W, s_arr)), ctypes.byref(h)))
        self._h = h

    def _v(self, t, size, name):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != size:
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {size} values")

    def operator(self, x: torch.Tensor, y: torch.Tensor, I0: float) -> torch.Tensor:
        self._v(x, self.d, "x")
        self._v(y, self.W * self.n, "y")
        F = torch.empty(self.d, dtype=torch.float64, device=self.A.device)
        _check("exact_dense_operator", load().exact_dense_operator(self._h, _ptr(x), _ptr(y), float(I0), _ptr(F),
                                                                   _stream()))
        return F

    def solve(self, y: torch.Tensor, I0: float, eta: float, iters: int, x: torch.Tensor | None = None,
              lo: float = -math.inf, hi: float = math.inf, x_true: torch.Tensor | None = None):
        """Returns (x, err) with err[t] = ||x_t - x_true|| (None without x_true)."""
        self._v(y, self.W * self.n, "y")
        if x is None:
            x = torch.zeros(self.d, dtype=torch.float64, device=self.A.device)
        self._v(x, self.d, "x")
        err = None
        if x_true is not None:
            self._v(x_true, self.d, "x_true")
            err = torch.empty(max(int(iters), 1), dtype=torch.float64, device=self.A.device)
        _check("exact_dense_solve", load().exact_dense_solve(self._h, _ptr(y), float(I0), float(eta), int(iters),
                                                             float(lo), float(hi), _ptr(x),
                                                             None if x_true is None else _ptr(x_true),
                                                             None if err is None else _ptr(err), _stream()))
        return x, (err[: int(iters)] if err is not None else None)

    def close(self):
        if getattr(self, "_h", None):
            load().exact_dense_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tv_prox(z: torch.Tensor, lam: float, fgp_iters: int = 40, out: torch.Tensor | None = None) -> torch.Tensor:
    """argmin_x ||x - z||^2 + lam ||x||_TV of the device image z (exact_tv_prox)."""
    lib = load()
    if z.dtype != torch.float32 or z.dim() != 2 or not z.is_cuda or not z.is_contiguous():
        raise ValueError("z must be a contiguous CUDA float32 [ny][nx] tensor")
    ny, nx = z.shape
    nb = lib.exact_tv_workspace_bytes(nx, ny)
    ws = torch.empty(nb, dtype=torch.uint8, device=z.device)
    x = out if out is not None else torch.empty_like(z)
    _check("exact_tv_prox", lib.exact_tv_prox(nx, ny, _ptr(z), float(lam), int(fgp_iters), _ptr(x), _ptr(ws), nb,
                                              _stream()))
    return x


class Plan:
    """An EXACT plan on the current CUDA device, with its workspace.

    ``mu``: attenuation per energy bin (K values > 0); ``S``: window weights
    [W][K] >= 0 (fraction of I0 recorded by window w from energy k)."""

    def __init__(self, geometry: Geometry, mu, S, device=None):
        lib = load()
        self.geometry = geometry
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        mu_l = [float(v) for v in mu]
        S_rows = [[float(v) for v in row] for row in S]
        self.K, self.W = len(mu_l), len(S_rows)
        if any(len(r) != self.K for r in S_rows):
            raise ValueError("S must be [n_windows][n_energy]")
        self._mu = (ctypes.c_double * self.K)(*mu_l)
        self._S = (ctypes.c_double * (self.K * self.W))(*[v for r in S_rows for v in r])
        g = geometry._c()
        sp = _Spectrum(self.K, ctypes.cast(self._mu, ctypes.POINTER(ctypes.c_double)))
        wn = _Windows(self.W, ctypes.cast(self._S, ctypes.POINTER(ctypes.c_double)))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check("exact_plan_create", lib.exact_plan_create(ctypes.byref(g), ctypes.byref(sp),
                                                              ctypes.byref(wn), ctypes.byref(h)))
            self._h = h
            nbytes = int(lib.exact_plan_workspace_bytes(h))
            # over-allocate so the start can be rounded up to 256 bytes
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            off = (-self._ws.data_ptr()) % 256
            _check("exact_plan_bind_workspace",
                   lib.exact_plan_bind_workspace(h, ctypes.c_void_p(self._ws.data_ptr() + off), nbytes))
        self.n_rays = geometry.n_views * geometry.n_bins
        self.shape_img = (geometry.ny, geometry.nx)
        self.shape_sino = (geometry.n_views, geometry.n_bins)

    def close(self):
        if getattr(self, "_h", None):
            with torch.cuda.device(self.device):
                torch.cuda.synchronize(self.device)
                load().exact_plan_destroy(self._h)
            self._h = None
            self._pending = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- argument checks ----------------------------------------------------
    def _t(self, t: torch.Tensor, shape, dtypes=(torch.float32,), name="tensor") -> torch.Tensor:
        if not isinstance(t, torch.Tensor) or t.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} must have dtype in {dtypes}, got {t.dtype}")
        if tuple(t.shape) != tuple(shape) and t.numel() != math.prod(shape):
            raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _y(self, y: torch.Tensor):
        self._t(y, (self.W,) + self.shape_sino, (torch.float32, torch.bfloat16), "y")
        return F32 if y.dtype == torch.float32 else BF16

    # ---- entry points -------------------------------------------------------
    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._t(x, self.shape_img, name="x")
        z = out if out is not None else torch.empty(self.shape_sino, dtype=torch.float32, device=self.device)
        self._t(z, self.shape_sino, name="z")
        _check("exact_forward", load().exact_forward(self._h, _ptr(x), _ptr(z), _stream()))
        return z

    def adjoint(self, r: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._t(r, self.shape_sino, name="r")
        g = out if out is not None else torch.empty(self.shape_img, dtype=torch.float32, device=self.device)
        self._t(g, self.shape_img, name="g")
        _check("exact_adjoint", load().exact_adjoint(self._h, _ptr(r), _ptr(g), _stream()))
        return g

    def operator(self, x: torch.Tensor, y: torch.Tensor, I0: float, out: torch.Tensor | None = None):
        self._t(x, self.shape_img, name="x")
        dt = self._y(y)
        F = out if out is not None else torch.empty(self.shape_img, dtype=torch.float32, device=self.device)
        self._t(F, self.shape_img, name="F")
        _check("exact_operator", load().exact_operator(self._h, _ptr(x), _ptr(y), dt, float(I0), _ptr(F),
                                                       _stream()))
        return F

    def resume_state(self) -> torch.Tensor:
        """A device buffer for the ``resume`` option of :meth:`solve`
        (exact_solve_resume_bytes; FP64 averaging sums and the TV lam pair)."""
        nb = int(load().exact_solve_resume_bytes(self._h))
        return torch.zeros(nb // 8, dtype=torch.float64, device=self.device)

    def solve(self, y: torch.Tensor, I0: float, eta: float, iters: int, x: torch.Tensor | None = None,
              lo: float = 0.0, hi: float = math.inf, tol: float = 0.0, check_every: int = 1,
              average_tail: bool = False, stop_rule: str = "residual", tv_bound: float = 0.0,
              tv_opts: dict | None = None, prox_lambda: float = 0.0, sync: bool = True, t0: int = 0,
              total_iters: int = 0, resume: torch.Tensor | None = None, x_last: torch.Tensor | None = None,
              history: torch.Tensor | None = None, launch: str = "auto"):
        """Run up to ``iters`` extragradient iterations in place on ``x``
        (zeros if None).  stop_rule "residual" tests the relative change of the
        iterate, "average" the change of the running average of the last half
        of the iterates (and returns that average; its window ring is
        allocated here unless ``history`` is given).  tv_bound > 0 intersects
        the box with the TV ball of that radius (tv_opts: fields of
        exact_tv_opts to change).  t0 / total_iters / resume / x_last continue
        an earlier call of the same solve (see exact_solve_opts); launch
        "auto" loops on the device in a CUDA graph where possible, "stream"
        launches every kernel from the host.  Returns (x, SolveInfo); with
        sync=False the info is filled once the current stream reaches the end
        of the solve."""
        dt = self._y(y)
        if x is None:
            x = torch.zeros(self.shape_img, dtype=torch.float32, device=self.device)
        self._t(x, self.shape_img, name="x")
        if stop_rule not in STOP_RULES:
            raise ValueError(f"stop_rule must be one of {sorted(STOP_RULES)}")
        if launch not in ("auto", "stream"):
            raise ValueError("launch must be 'auto' or 'stream'")
        hist = None
        if stop_rule == "average":
            if history is not None:
                hist = history
                if hist.dtype != torch.float32 or hist.device != self.device or not hist.is_contiguous() or \
                        tuple(hist.shape[1:]) != tuple(self.shape_img):
                    raise ValueError("history must be a contiguous float32 [cap][ny][nx] tensor on the plan's device")
            else:
                cap = max(1, (int(t0) + int(iters)) // 2)
                hist = torch.empty((cap,) + tuple(self.shape_img), dtype=torch.float32, device=self.device)
        if resume is not None and (resume.dtype != torch.float64 or resume.device != self.device
                                   or not resume.is_contiguous()
                                   or resume.numel() * 8 < load().exact_solve_resume_bytes(self._h)):
            raise ValueError("resume must come from resume_state()")
        if x_last is not None:
            self._t(x_last, self.shape_img, name="x_last")
        opts = _SolveOpts(float(lo), float(hi), float(tol), int(check_every), int(bool(average_tail)),
                          STOP_RULES[stop_rule], 0 if hist is None else hist.shape[0],
                          None if hist is None else hist.data_ptr(), float(tv_bound), tv_options(tv_opts),
                          float(prox_lambda), int(t0), int(total_iters),
                          None if resume is None else resume.data_ptr(),
                          None if x_last is None else x_last.data_ptr(), 0 if launch == "auto" else 1, 0)
        info = _SolveInfo()
        _check("exact_solve", load().exact_solve(self._h, _ptr(y), dt, float(I0), float(eta), int(iters),
                                                 ctypes.byref(opts), _ptr(x), ctypes.byref(info), _stream()))
        # the library writes `info` from a stream callback: keep it alive until
        # the stream has passed the end of this solve
        done = torch.cuda.Event()
        done.record()
        self._pending = [(e, i) for e, i in getattr(self, "_pending", []) if not e.query()]
        self._pending.append((done, (info, hist)))
        if sync:
            done.synchronize()
        return x, info

    def norm_estimate(self, max_iters: int = 500, rtol: float = 1e-9):
        """FP64 power-iteration estimate of ||A||^2 (synchronises); returns (lam, iterations)."""
        lam = ctypes.c_double()
        it = ctypes.c_int()
        _check("exact_norm_estimate", load().exact_norm_estimate(self._h, int(max_iters), float(rtol),
                                                                 ctypes.byref(lam), ctypes.byref(it), _stream()))
        return lam.value, it.value

    def norm_estimate_f32(self, max_iters: int = 100, rtol: float = 1e-6):
        """Power iteration with the FP32 projector (FP64 norms); returns (lam, iterations)."""
        lam = ctypes.c_double()
        it = ctypes.c_int()
        _check("exact_norm_estimate_f32", load().exact_norm_estimate_f32(
            self._h, int(max_iters), float(rtol), ctypes.byref(lam), ctypes.byref(it), _stream()))
        return lam.value, it.value

    def set_background(self, mu_bg=None, p: torch.Tensor | None = None):
        """Known background materials (Appendix A.1): mu_bg [M][K] attenuations,
        p [M][n_views][n_bins] device FP32 projections (kept referenced)."""
        if p is None:
            _check("exact_plan_set_background", load().exact_plan_set_background(self._h, 0, None, None))
            self._bg = None
            return
        rows = [[float(v) for v in r] for r in mu_bg]
        M = len(rows)
        self._t(p, (M,) + self.shape_sino, name="p")
        arr = (ctypes.c_double * (M * self.K))(*[v for r in rows for v in r])
        _check("exact_plan_set_background", load().exact_plan_set_background(self._h, M, arr, _ptr(p)))
        self._bg = p

    @property
    def tuning(self) -> dict:
        """Kernel tuning of this plan (exact_plan_get_tuning)."""
        t = _Tuning()
        _check("exact_plan_get_tuning", load().exact_plan_get_tuning(self._h, ctypes.byref(t)))
        return {"adj_split": t.adj_split}

    def set_tuning(self, adj_split: int):
        t = _Tuning()
        t.adj_split = int(adj_split)
        _check("exact_plan_set_tuning", load().exact_plan_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, force: bool = False) -> dict:
        """Time the kernel variants on this geometry and keep the fastest
        (exact_plan_autotune; cached per geometry shape in this process)."""
        t = _Tuning()
        _check("exact_plan_autotune", load().exact_plan_autotune(self._h, int(bool(force)), ctypes.byref(t),
                                                                 _stream()))
        return {"adj_split": t.adj_split}

    def nnz(self) -> int:
        """Nonzero entries of A (counted on the host, cached)."""
        v = ctypes.c_longlong()
        _check("exact_plan_nnz", load().exact_plan_nnz(self._h, ctypes.byref(v)))
        return v.value

    def profile_enable(self, sample_every: int):
        _check("exact_profile_enable", load().exact_profile_enable(self._h, int(sample_every)))

    def profile_read(self):
        """{kind: (total ms, launches)} for kinds forward_link, adjoint_half,
        adjoint_full, reduce, since the last read."""
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_longlong * 4)()
        _check("exact_profile_read", load().exact_profile_read(self._h, ms, cnt))
        names = ("forward_link", "adjoint_half", "adjoint_full", "reduce")
        return {n: (ms[i], cnt[i]) for i, n in enumerate(names)}

    def solve_host(self, y_host: torch.Tensor, I0: float, eta: float, iters: int, x_host: torch.Tensor,
                   lo: float = 0.0, hi: float = math.inf, tol: float = 0.0, check_every: int = 1):
        """Solve from host buffers (exact_solve_host): the library copies y and
        x_1 from (pinned) host memory into the plan's workspace, solves, and
        copies the result back into ``x_host``, on the current stream, and
        synchronises.  Returns (x_host, SolveInfo)."""
        for t, name in ((y_host, "y_host"), (x_host, "x_host")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous host tensor")
        if y_host.dtype not in (torch.float32, torch.bfloat16) or y_host.numel() != self.W * self.n_rays:
            raise ValueError("y_host must hold [n_windows][n_views][n_bins] float32 or bfloat16 counts")
        if x_host.dtype != torch.float32 or x_host.numel() != self.shape_img[0] * self.shape_img[1]:
            raise ValueError("x_host must be a float32 [ny][nx] tensor")
        dt = F32 if y_host.dtype == torch.float32 else BF16
        opts = load().exact_solve_opts_default()
        opts.lo, opts.hi, opts.tol, opts.check_every = float(lo), float(hi), float(tol), int(check_every)
        info = _SolveInfo()
        _check("exact_solve_host", load().exact_solve_host(self._h, _ptr(y_host), dt, float(I0), float(eta),
                                                           int(iters), ctypes.byref(opts), _ptr(x_host),
                                                           ctypes.byref(info), _stream()))
        return x_host, info

    def recommended_eta(self, I0: float, normA_sq: float) -> float:
        eta = ctypes.c_double()
        _check("exact_recommended_eta", load().exact_recommended_eta(self._h, float(I0), float(normA_sq),
                                                                     ctypes.byref(eta)))
        return eta.value


@dataclass
class Job:
    """One reconstruction of a batch (see exact_job)."""
    plan: Plan
    y: torch.Tensor
    I0: float
    eta: float
    iters: int
    x: torch.Tensor | None = None
    lo: float = 0.0
    hi: float = math.inf
    tol: float = 0.0
    check_every: int = 1


class Batch:
    """Multi-job solver context (exact_batch_*): policy 0 or 1 runs all jobs in
    one persistent kernel launch, policy 2 each job's own solve on one of the
    context's streams (see `autotune`, `set_policy`)."""

    def __init__(self, max_jobs: int = 64):
        lib = load()
        h = ctypes.c_void_p()
        _check("exact_batch_create", lib.exact_batch_create(int(max_jobs), ctypes.byref(h)))
        self._h = h
        self.max_jobs = max_jobs
        self._pending = []

    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.synchronize()
            load().exact_batch_destroy(self._h)
            self._h = None
            self._pending = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _jobs(self, jobs: list[Job]):
        n = len(jobs)
        arr = (_Job * n)()
        infos = [_SolveInfo() for _ in range(n)]
        xs = []
        for k, jb in enumerate(jobs):
            p = jb.plan
            dt = p._y(jb.y)
            x = jb.x if jb.x is not None else torch.zeros(p.shape_img, dtype=torch.float32, device=p.device)
            p._t(x, p.shape_img, name="x")
            xs.append(x)
            arr[k] = _Job(p._h.value, jb.y.data_ptr(), dt, float(jb.I0), float(jb.eta), int(jb.iters),
                          _SolveOpts(float(jb.lo), float(jb.hi), float(jb.tol), int(jb.check_every), 0, 0, 0, None,
                                     0.0, tv_options(None), 0.0, 0, 0, None, None, 0, 0),
                          x.data_ptr(), ctypes.pointer(infos[k]))
        return arr, infos, xs

    @property
    def policy(self) -> int:
        v = ctypes.c_int(0)
        _check("exact_batch_get_policy", load().exact_batch_get_policy(self._h, ctypes.byref(v)))
        return v.value

    def set_policy(self, policy: int):
        """0: persistent kernel, one CTA per adjoint tile; 1: persistent kernel,
        each plan's adj_split; 2: each job's exact_solve on the context's
        streams (exact_batch_set_policy)."""
        _check("exact_batch_set_policy", load().exact_batch_set_policy(self._h, int(policy)))

    def autotune(self, jobs: list[Job]) -> int:
        """Pick this context's policy (0, 1 or 2) by timing these jobs
        (exact_batch_autotune; the jobs' images are left as they were)."""
        arr, _, _ = self._jobs(jobs)
        policy = ctypes.c_int(0)
        _check("exact_batch_autotune", load().exact_batch_autotune(self._h, arr, len(jobs), ctypes.byref(policy),
                                                                   _stream()))
        return policy.value

    def solve(self, jobs: list[Job], sync: bool = True):
        """Run all jobs (one persistent launch, or one solve per job on the
        context's streams under policy 2); returns the images and the list of
        SolveInfo (filled once the stream passes the end of the batch)."""
        n = len(jobs)
        arr, infos, xs = self._jobs(jobs)
        _check("exact_batch_solve", load().exact_batch_solve(self._h, arr, n, _stream()))
        if torch.cuda.is_current_stream_capturing():
            # a captured graph writes `infos` on every replay: keep them alive
            self._captured = getattr(self, "_captured", []) + [(arr, infos)]
            return xs, infos
        done = torch.cuda.Event()
        done.record()
        self._pending = [(e, i) for e, i in self._pending if not e.query()]
        self._pending.append((done, (arr, infos)))
        if sync:
            done.synchronize()
        return xs, infos
