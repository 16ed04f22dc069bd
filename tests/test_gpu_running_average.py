"""GPU parity of the running-average stopping rule of Sec. 3.1
(stop_rule EXACT_STOP_AVERAGE) against the FP64 oracle.

The tolerance is taken strictly between two consecutive changes of the
oracle's history, so the stopping iteration is unique unless FP32 rounding
moves a change across it (the gap between neighbours is many orders above
that rounding); the returned average is compared like a whole solve
(relative L2 <= 1e-3, PSNR within 0.05 dB)."""
import math

import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2503_19925_gb300 as ex
from synth import configs
from tests.cases import problem, rel_l2, psnr

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

DEV = "cuda:0"


def _eta(p):
    nA, _ = oracle.norm_estimate(p["g_or"], 300, 1e-10)
    return 1.0 / (4.0 * oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))


@pytest.mark.parametrize("case,check_every", [("C1", 1), ("fan", 4)])
def test_running_average_stop_and_output(case, check_every):
    if case == "C1":
        c = configs.C1
        geom, K, W, I0, seed = c["geometry"], c["K"], c["W"], c["I0"], 1
    else:
        geom = dict(beam=1, nx=96, ny=80, n_views=61, n_bins=137, angle0=0.05, angle_range=2 * math.pi,
                    bin_pitch=1.5, src_to_center=300.0, src_to_det=450.0)
        K, W, I0, seed = 12, 2, 1e4, 5
    p = problem(geom, K=K, W=W, I0=I0, seed=seed)
    eta = _eta(p)
    T = 120
    full = oracle.solve_running_average(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, T, tol=0.0)
    ch = full.changes  # ch[k] belongs to iteration k + 2
    k = 60
    tol = math.sqrt(ch[k] * ch[k + 1])
    expect = next(t for t in range(2, T + 1) if t % check_every == 0 and ch[t - 2] <= tol)
    ref = oracle.solve_running_average(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, T, tol=tol,
                                       check_every=check_every)
    assert ref.iters == expect

    plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
    y = torch.as_tensor(p["y"], dtype=torch.float32, device=DEV)
    x, info = plan.solve(y, p["I0"], eta, T, tol=tol, check_every=check_every, stop_rule="average")
    assert info.status == 0
    assert info.iters_done == expect
    assert info.avg_change == pytest.approx(ch[expect - 2], rel=1e-2)
    xg = x.double().cpu().numpy()
    assert rel_l2(xg, ref.x_avg) <= 1e-3
    assert abs(psnr(xg, p["xs"]) - psnr(ref.x_avg, p["xs"])) <= 0.05
    # without a tolerance it runs all iterations and returns xbar_T
    x2, info2 = plan.solve(y, p["I0"], eta, 30, stop_rule="average")
    ref2 = oracle.solve_running_average(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 30, tol=0.0)
    assert info2.iters_done == 30
    assert rel_l2(x2.double().cpu().numpy(), ref2.x_avg) <= 1e-4
    assert info2.avg_change == pytest.approx(ref2.changes[-1], rel=1e-2)


def test_running_average_rejects_bad_options():
    geom = dict(beam=0, nx=16, ny=16, n_views=10, n_bins=23, angle_range=math.pi)
    plan = ex.Plan(ex.Geometry(**geom), [1.0], [[1.0]])
    y = torch.ones((1, 10, 23), device=DEV)
    lib = ex.load()
    x = torch.zeros((16, 16), device=DEV)
    hist = torch.zeros((2, 16, 16), device=DEV)
    from paper_2503_19925_gb300 import exact as b
    info = b._SolveInfo()

    def run(iters, cap, ptr, tail=0):
        o = b._SolveOpts(0.0, math.inf, 0.0, 1, tail, 1, cap, ptr)
        return lib.exact_solve(plan._h, y.data_ptr(), b.F32, 1.0, 0.1, iters, b.ctypes.byref(o), x.data_ptr(),
                               b.ctypes.byref(info), torch.cuda.current_stream().cuda_stream)

    assert run(6, 2, None) == 1              # no ring
    assert run(6, 2, hist.data_ptr()) == 1   # ring of 2 < floor(6/2)
    assert run(4, 2, hist.data_ptr(), tail=1) == 1  # tail average and the window rule together
    assert run(4, 2, hist.data_ptr()) == 0
    torch.cuda.synchronize()
    assert info.iters_done == 4
