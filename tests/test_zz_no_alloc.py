"""exact_operator_static -- the operator for callers that cannot allocate
device memory when they need F (allocator-free real-time loops, processes whose
device memory belongs to another framework's pool) -- against exact_operator,
through the C ABI.

It runs last (file name) so that a failure here cannot hide other results; it
also passes alone in a fresh process.  Two calls in a row check that the shared
static scratch, which keeps the previous call's contents, gives the same
answer again."""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2503_19925_gb300 as ex
from paper_2503_19925_gb300 import exact as binding
from tests.cases import problem, rel_l2

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

CASES = [
    (dict(beam=1, nx=96, ny=80, n_views=61, n_bins=137, angle0=0.05, angle_range=2 * math.pi, bin_pitch=1.5,
          src_to_center=300.0, src_to_det=450.0), 3, 16, torch.bfloat16),
    (dict(beam=0, nx=77, ny=45, n_views=33, n_bins=101, angle0=0.2, angle_range=math.pi, bin_pitch=0.9,
          det_offset=0.31), 2, 12, torch.float32),
]


def _static(lib, plan, x, y, I0, F):
    dt = binding.F32 if y.dtype == torch.float32 else binding.BF16
    return lib.exact_operator_static(plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), dt,
                                     ctypes.c_double(I0), ctypes.c_void_p(F.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_scratch_operator_matches_operator():
    lib = ex.load()
    for geom, W, K, ydt in CASES:
        p = problem(geom, K=K, W=W, I0=1e4, seed=11, bf16=ydt == torch.bfloat16)
        plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
        y = torch.as_tensor(p["y"], dtype=ydt, device="cuda:0").contiguous()
        rng = np.random.default_rng(3)
        for _ in range(2):  # two calls in a row share (and reuse) the static scratch
            x = torch.as_tensor(rng.uniform(0, 1, (geom["ny"], geom["nx"])), dtype=torch.float32,
                                device="cuda:0")
            F_ref = plan.operator(x, y, p["I0"])
            F = torch.full_like(F_ref, float("nan"))
            assert _static(lib, plan, x, y, p["I0"], F) == 0
            torch.cuda.synchronize()
            assert torch.isfinite(F).all()
            assert rel_l2(F.double().cpu().numpy(), F_ref.double().cpu().numpy()) <= 1e-5
        plan.close()


def test_static_scratch_rejects_too_large_plans():
    lib = ex.load()
    geom = dict(beam=0, nx=1024, ny=1024, n_views=2000, n_bins=1449, angle_range=math.pi)
    plan = ex.Plan(ex.Geometry(**geom), [1.0], [[1.0]])
    x = torch.zeros((1024, 1024), device="cuda:0")
    y = torch.zeros((1, 2000, 1449), device="cuda:0")
    F = torch.zeros_like(x)
    assert _static(lib, plan, x, y, 1.0, F) == 6  # EXACT_ERR_UNSUPPORTED
    plan.close()


def _raw_plan(lib, geom, mu, S):
    """A plan created through the C ABI with no workspace bound (the situation
    of a caller that cannot allocate one)."""
    g = binding.Geometry(**geom)._c()
    mu_a = (ctypes.c_double * len(mu))(*[float(v) for v in mu])
    rows = [[float(v) for v in r] for r in S]
    s_a = (ctypes.c_double * (len(rows) * len(mu)))(*[v for r in rows for v in r])
    sp = binding._Spectrum(len(mu), ctypes.cast(mu_a, ctypes.POINTER(ctypes.c_double)))
    wn = binding._Windows(len(rows), ctypes.cast(s_a, ctypes.POINTER(ctypes.c_double)))
    h = ctypes.c_void_p()
    assert lib.exact_plan_create(ctypes.byref(g), ctypes.byref(sp), ctypes.byref(wn), ctypes.byref(h)) == 0
    return h, (mu_a, s_a)


def test_static_scratch_without_workspace_and_with_a_view_split():
    """A plan with no bound workspace: exact_operator refuses it
    (EXACT_ERR_NO_WORKSPACE), exact_operator_static runs and matches the
    workspace path of a plan whose adjoint splits each tile's views over 4
    CTAs (the static path always runs one CTA per tile), twice in a row."""
    lib = ex.load()
    geom, W, K, ydt = CASES[0]
    p = problem(geom, K=K, W=W, I0=1e4, seed=12, bf16=True)
    ref_plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
    ref_plan.set_tuning(4)
    h, keep = _raw_plan(lib, geom, p["mu"], p["S"])
    y = torch.as_tensor(p["y"], dtype=torch.bfloat16, device="cuda:0").contiguous()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(5)
    try:
        for _ in range(2):
            x = torch.as_tensor(rng.uniform(0, 1, (geom["ny"], geom["nx"])), dtype=torch.float32, device="cuda:0")
            F_ref = ref_plan.operator(x, y, p["I0"])
            F = torch.full_like(F_ref, float("nan"))
            args = (ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), binding.BF16,
                    ctypes.c_double(p["I0"]), ctypes.c_void_p(F.data_ptr()), stream)
            assert lib.exact_operator(h, *args) == 7  # EXACT_ERR_NO_WORKSPACE
            assert lib.exact_operator_static(h, *args) == 0
            torch.cuda.synchronize()
            assert torch.isfinite(F).all()
            assert rel_l2(F.double().cpu().numpy(), F_ref.double().cpu().numpy()) <= 1e-5
    finally:
        torch.cuda.synchronize()
        lib.exact_plan_destroy(h)
        ref_plan.close()
