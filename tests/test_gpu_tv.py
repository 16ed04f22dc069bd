"""GPU parity of the TV-ball ∩ box projection of Sec. 3.1 (exact_tv_project)
and of extragradient solves on that feasible set, against oracle/tv.py.

Both sides run the same algorithm with the same control flow (Dykstra rounds,
bisection on lam, fixed dual-step counts, lam carried between calls); the
CUDA path computes the pixel arrays in FP32 and the decisions on FP64 sums.
Projections are compared to relative L2 <= 1e-3 (the bisection tolerance
used here is 1e-4 of tau), with the TV of the GPU result within the
tolerance of tau and the box respected; an input already in X comes back
unchanged, bit for bit."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import tv as T
import paper_2503_19925_gb300 as ex
import synth
from tests.cases import problem, rel_l2, psnr

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

DEV = "cuda:0"


def _noisy_phantom(nx, ny, seed):
    n = max(nx, ny)
    x = synth.rasterize_ellipses(synth.random_ellipses(n, 5, seed), nx, ny, supersample=2)
    return x + 0.15 * np.random.default_rng(seed).normal(size=x.shape)


@pytest.mark.parametrize("nx,ny,frac,seed", [(64, 64, 0.5, 1), (96, 80, 0.3, 2), (37, 53, 0.7, 3)])
def test_tv_projection_parity(nx, ny, frac, seed):
    z = _noisy_phantom(nx, ny, seed)
    tau = frac * T.tv(z)
    o = dict(fgp_iters=40, max_bisect=40, max_dykstra=30, tol_tv=1e-4 * tau, tol_dykstra=1e-3)
    ref = T.project_tv_box(z, tau, 0.0, np.inf, T.TvOptions(**o))
    x, info = ex.tv_project(torch.as_tensor(z, dtype=torch.float32, device=DEV), tau, 0.0, math.inf, o)
    xg = x.double().cpu().numpy()
    assert info.status == 0
    assert rel_l2(xg, ref.x) <= 1e-3
    assert xg.min() >= 0.0
    assert T.tv(xg) <= tau * (1 + 1e-3)
    assert info.rounds == ref.rounds
    assert abs(info.solves - ref.solves) <= 2


def test_tv_projection_identity_inside_the_set():
    z = np.abs(_noisy_phantom(40, 30, 4))
    zt = torch.as_tensor(z, dtype=torch.float32, device=DEV)
    x, info = ex.tv_project(zt, 1.5 * T.tv(z), 0.0, math.inf)
    assert torch.equal(x, zt)
    assert info.rounds == 1 and info.solves == 0


def test_tv_projection_box_only_when_tv_is_loose():
    z = _noisy_phantom(40, 30, 5)
    zt = torch.as_tensor(z, dtype=torch.float32, device=DEV)
    x, info = ex.tv_project(zt, 10.0 * T.tv(z), 0.1, 0.9)
    np.testing.assert_array_equal(x.cpu().numpy(), np.clip(z.astype(np.float32), 0.1, 0.9))


def test_solve_on_tv_ball_parity():
    geom = dict(beam=0, nx=48, ny=48, n_views=40, n_bins=69, angle_range=math.pi)
    p = problem(geom, K=8, W=2, I0=1e4, seed=6)
    nA, _ = oracle.norm_estimate(p["g_or"], 300, 1e-10)
    eta = 1.0 / (4.0 * oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))
    tau = T.tv(p["xs"])
    o = dict(fgp_iters=30, max_bisect=40, max_dykstra=20, tol_tv=1e-4 * tau, tol_dykstra=1e-3)
    iters = 6
    ref = T.solve_tv(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, iters, tau, opts=T.TvOptions(**o))
    plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
    y = torch.as_tensor(p["y"], dtype=torch.float32, device=DEV)
    x, info = plan.solve(y, p["I0"], eta, iters, tv_bound=tau, tv_opts=o)
    xg = x.double().cpu().numpy()
    assert info.status == 0 and info.iters_done == iters
    assert rel_l2(xg, ref.x) <= 1e-3
    assert abs(psnr(xg, p["xs"]) - psnr(ref.x, p["xs"])) <= 0.05
    assert info.rel_res == pytest.approx(ref.rel_res[-1], rel=1e-2)
    assert T.tv(xg) <= tau * (1 + 1e-3) and xg.min() >= 0.0


def test_tv_options_rejected():
    z = torch.zeros((8, 8), device=DEV)
    with pytest.raises(RuntimeError):
        ex.tv_project(z, -1.0)
    with pytest.raises(RuntimeError):
        ex.tv_project(z, 1.0, opts=dict(fgp_iters=0))


def test_solve_on_tv_ball_with_the_running_average_rule():
    geom = dict(beam=1, nx=40, ny=36, n_views=30, n_bins=61, angle_range=2 * math.pi, bin_pitch=1.5,
                src_to_center=150.0, src_to_det=240.0)
    p = problem(geom, K=6, W=2, I0=1e4, seed=8)
    nA, _ = oracle.norm_estimate(p["g_or"], 300, 1e-10)
    eta = 1.0 / (4.0 * oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))
    tau = T.tv(p["xs"])
    o = dict(fgp_iters=20, max_bisect=30, max_dykstra=10, tol_tv=1e-4 * tau, tol_dykstra=1e-3)
    iters = 24
    full = T.solve_tv(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, iters, tau, opts=T.TvOptions(**o),
                      running_average=True)
    ch = full.changes
    tol = math.sqrt(ch[12] * ch[13])
    expect = next(t for t in range(2, iters + 1) if ch[t - 2] <= tol)
    ref = T.solve_tv(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, iters, tau, opts=T.TvOptions(**o),
                     running_average=True, tol=tol)
    assert ref.iters == expect
    plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
    y = torch.as_tensor(p["y"], dtype=torch.float32, device=DEV)
    x, info = plan.solve(y, p["I0"], eta, iters, tv_bound=tau, tv_opts=o, stop_rule="average", tol=tol)
    assert info.status == 0 and info.iters_done == expect
    xg = x.double().cpu().numpy()
    assert rel_l2(xg, ref.x) <= 1e-3
    assert info.avg_change == pytest.approx(ch[expect - 2], rel=1e-2)


@pytest.mark.parametrize("nx,ny,lam", [(64, 64, 0.3), (37, 53, 1.5)])
def test_tv_prox_parity(nx, ny, lam):
    z = _noisy_phantom(nx, ny, 9)
    ref, _, _ = T.prox_tv(z, lam, 60)
    x = ex.tv_prox(torch.as_tensor(z, dtype=torch.float32, device=DEV), lam, 60)
    assert rel_l2(x.double().cpu().numpy(), ref) <= 1e-5


def test_proximal_variant_solve_parity():
    geom = dict(beam=0, nx=40, ny=40, n_views=36, n_bins=59, angle_range=math.pi)
    p = problem(geom, K=6, W=2, I0=1e4, seed=11)
    nA, _ = oracle.norm_estimate(p["g_or"], 300, 1e-10)
    eta = 1.0 / (4.0 * oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))
    lam, iters = 0.05, 8
    ref = T.solve_prox_tv(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, iters, lam, fgp_iters=30)
    plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
    y = torch.as_tensor(p["y"], dtype=torch.float32, device=DEV)
    x, info = plan.solve(y, p["I0"], eta, iters, prox_lambda=lam, tv_opts={"fgp_iters": 30})
    assert info.status == 0 and info.iters_done == iters
    assert rel_l2(x.double().cpu().numpy(), ref) <= 1e-4
    with pytest.raises(RuntimeError):
        plan.solve(y, p["I0"], eta, 2, prox_lambda=lam, tv_bound=10.0)
