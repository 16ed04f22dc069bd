"""Checkpoint/resume and the device-side solve loop.

- A solve of 300 iterations split into two calls of 150 (the second with
  t0 = 150, the first call's last iterate and the resume state) gives bitwise
  the same image and info as one call of 300, for the plain iteration, the
  tail average (average_tail) and the running-average rule of Sec. 3.1, in
  both launch modes.
- The CUDA-graph loop (launch "auto") and one stream launch per kernel
  ("stream") give bitwise the same results, including where a tolerance stop
  ends the solve early, and the graph loop runs no iterations after the stop.
All against each other and, for the plain case, against the FP64 oracle."""
import math
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2503_19925_gb300 as ex
from tests.cases import problem, rel_l2

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

GEOM = dict(beam=1, nx=96, ny=80, n_views=61, n_bins=137, angle0=0.05, angle_range=2 * math.pi, bin_pitch=1.5,
            src_to_center=300.0, src_to_det=450.0)


@pytest.fixture(scope="module")
def case():
    p = problem(GEOM, K=16, W=2, I0=1e4, seed=21)
    plan = ex.Plan(ex.Geometry(**GEOM), p["mu"], p["S"])
    plan.set_tuning(3)  # a view split: the combine order is part of what must repeat
    lam, _ = oracle.norm_estimate(p["g_or"], 50, 0.0)
    eta = 1.0 / (4.0 * oracle.lipschitz(lam, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))
    y = torch.as_tensor(p["y"], dtype=torch.float32, device="cuda:0").contiguous()
    return p, plan, y, eta


def _same(a, b):
    return torch.equal(a, b)


@pytest.mark.parametrize("launch", ["auto", "stream"])
@pytest.mark.parametrize("mode", ["plain", "tail", "running"])
def test_two_resumed_calls_equal_one_call(case, launch, mode):
    p, plan, y, eta = case
    kw = {}
    if mode == "tail":
        kw["average_tail"] = True
    elif mode == "running":
        kw["stop_rule"] = "average"
    hist = None
    if mode == "running":
        hist = torch.zeros((150,) + plan.shape_img, dtype=torch.float32, device="cuda:0")
        kw["history"] = hist
    x_one, info_one = plan.solve(y, p["I0"], eta, 300, launch=launch, **kw)
    x_one = x_one.clone()
    if hist is not None:
        hist.zero_()
    resume = plan.resume_state()
    last = torch.empty(plan.shape_img, dtype=torch.float32, device="cuda:0")
    x1, info1 = plan.solve(y, p["I0"], eta, 150, total_iters=300, resume=resume, x_last=last, launch=launch, **kw)
    assert info1.iters_done == 150
    x2 = last.clone()
    x2, info2 = plan.solve(y, p["I0"], eta, 150, x=x2, t0=150, total_iters=300, resume=resume, launch=launch, **kw)
    assert info2.iters_done == 300 == info_one.iters_done
    assert _same(x2, x_one), (mode, launch, (x2 - x_one).abs().max().item())
    assert info2.rel_res == info_one.rel_res and info2.avg_change == info_one.avg_change
    if mode == "plain":
        ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 300)
        assert rel_l2(x_one.double().cpu().numpy(), ref.x) <= 1e-3


@pytest.mark.parametrize("mode", ["plain", "tail", "running"])
def test_graph_loop_equals_stream_launches(case, mode):
    p, plan, y, eta = case
    kw = {"average_tail": True} if mode == "tail" else ({"stop_rule": "average"} if mode == "running" else {})
    xa, ia = plan.solve(y, p["I0"], eta, 120, launch="auto", **kw)
    xb, ib = plan.solve(y, p["I0"], eta, 120, launch="stream", **kw)
    assert _same(xa, xb) and ia.iters_done == ib.iters_done == 120 and ia.rel_res == ib.rel_res


def test_tolerance_stop_in_the_graph_loop(case):
    """A tolerance stop ends the device loop: the same iterate and count as
    the stream launches, and a cap of 20000 iterations costs about what the
    iterations actually run cost (no launches after the stop)."""
    p, plan, y, eta = case
    tol = 2e-4
    xa, ia = plan.solve(y, p["I0"], eta, 20000, tol=tol, launch="auto")
    xb, ib = plan.solve(y, p["I0"], eta, 20000, tol=tol, launch="stream")
    assert 1 < ia.iters_done < 20000 and ia.iters_done == ib.iters_done
    assert ia.rel_res <= tol and ia.rel_res == ib.rel_res
    assert _same(xa, xb)
    k = ia.iters_done

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t

    t_cap = timed(lambda: plan.solve(y, p["I0"], eta, 20000, tol=tol, launch="auto", sync=False))
    t_k = timed(lambda: plan.solve(y, p["I0"], eta, k, launch="auto", sync=False))
    assert t_cap < 2.0 * t_k + 5e-3, (t_cap, t_k, k)


def test_resume_argument_checks(case):
    p, plan, y, eta = case
    with pytest.raises(ex.ExactError):
        plan.solve(y, p["I0"], eta, 10, t0=-1)
    with pytest.raises(ex.ExactError):
        plan.solve(y, p["I0"], eta, 10, t0=5, total_iters=12)  # total below t0 + iters
    # a batch job cannot resume
    job = ex.Job(plan=plan, y=y, I0=p["I0"], eta=eta, iters=5)
    xs, infos = ex.Batch(2).solve([job])
    assert infos[0].iters_done == 5
