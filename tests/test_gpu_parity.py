"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: A x, A^T r and F(x) to relative L2 error <= 1e-5 (FP32
arithmetic against FP64); final images of whole solves to relative L2 error
<= 1e-3 and PSNR within 0.05 dB; the FP64 norm estimate to 1e-9 relative.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import synth
from synth import configs
import paper_2503_19925_gb300 as ex
from tests.cases import problem, rel_l2, psnr
from tests.geom_cases import tiny_geometries

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

DEV = "cuda:0"

# small geometries spanning several tiles and ragged tails, both beams
GEOMS = [
    dict(beam=0, nx=64, ny=64, n_views=90, n_bins=91, angle_range=math.pi),
    dict(beam=0, nx=77, ny=45, n_views=33, n_bins=101, angle0=0.2, angle_range=math.pi, bin_pitch=0.9,
         det_offset=0.31),
    dict(beam=1, nx=96, ny=80, n_views=61, n_bins=137, angle0=0.05, angle_range=2 * math.pi, bin_pitch=1.5,
         src_to_center=300.0, src_to_det=450.0),
    dict(beam=1, nx=33, ny=130, n_views=40, n_bins=150, angle0=1.0, angle_range=2 * math.pi, bin_pitch=1.1,
         det_offset=-2.0, src_to_center=120.0, src_to_det=200.0),
    dict(beam=0, nx=1, ny=1, n_views=3, n_bins=2, angle_range=math.pi),
]


def _gpu(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _plan(geom, S, mu):
    return ex.Plan(ex.Geometry(**geom), mu, S)


def _geom_dict(g):
    return {k: getattr(g, k) for k in ("beam", "nx", "ny", "n_views", "n_bins", "pixel", "angle0", "angle_range",
                                       "bin_pitch", "det_offset", "src_to_center", "src_to_det")}


ALL_GEOMS = GEOMS + [_geom_dict(g) for g in tiny_geometries()]


@pytest.mark.parametrize("gi", range(len(ALL_GEOMS)))
def test_forward_parity(gi):
    geom = ALL_GEOMS[gi]
    S, mu = np.ones((1, 1)), np.ones(1)
    plan = _plan(geom, S, mu)
    x = synth.random_image(geom["nx"], geom["ny"], seed=gi)
    z = plan.forward(_gpu(x)).double().cpu().numpy()
    ref = oracle.forward(oracle.Geometry(**geom), x)
    assert rel_l2(z, ref) <= 1e-5
    assert np.abs(z - ref).max() <= 1e-5 * max(np.abs(ref).max(), 1e-30)


@pytest.mark.parametrize("gi", range(len(ALL_GEOMS)))
def test_adjoint_parity(gi):
    geom = ALL_GEOMS[gi]
    S, mu = np.ones((1, 1)), np.ones(1)
    plan = _plan(geom, S, mu)
    r = synth.random_sinogram(geom["n_views"], geom["n_bins"], seed=gi, lo=-1, hi=1)
    g = plan.adjoint(_gpu(r)).double().cpu().numpy()
    ref = oracle.adjoint(oracle.Geometry(**geom), r)
    assert rel_l2(g, ref) <= 1e-5
    # ones: every entry is a sum of nonnegative terms, so compare entrywise
    g1 = plan.adjoint(_gpu(np.ones_like(r))).double().cpu().numpy()
    ref1 = oracle.adjoint(oracle.Geometry(**geom), np.ones_like(r))
    np.testing.assert_allclose(g1, ref1, rtol=2e-6, atol=1e-6 * ref1.max())


@pytest.mark.parametrize("gi", [0, 2, 3])
def test_adjoint_identity_fp32(gi):
    geom = GEOMS[gi]
    plan = _plan(geom, np.ones((1, 1)), np.ones(1))
    x = synth.random_image(geom["nx"], geom["ny"], seed=10 + gi)
    r = synth.random_sinogram(geom["n_views"], geom["n_bins"], seed=20 + gi, lo=0, hi=1)
    z = plan.forward(_gpu(x)).double().cpu().numpy()
    g = plan.adjoint(_gpu(r)).double().cpu().numpy()
    lhs, rhs = float((z * r).sum()), float((x * g).sum())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


@pytest.mark.parametrize("gi,W,K,bf16", [(0, 1, 10, False), (1, 3, 32, False), (2, 4, 64, True), (3, 2, 7, True)])
def test_operator_parity(gi, W, K, bf16):
    geom = GEOMS[gi]
    p = problem(geom, K=K, W=W, I0=1e4, seed=gi, bf16=bf16)
    plan = _plan(geom, p["S"], p["mu"])
    rng = np.random.default_rng(gi)
    for x in (np.zeros((geom["ny"], geom["nx"])), rng.uniform(0, 1, (geom["ny"], geom["nx"])), 0.5 * p["xs"]):
        y = _gpu(p["y"], torch.bfloat16 if bf16 else torch.float32)
        F = plan.operator(_gpu(x), y, p["I0"]).double().cpu().numpy()
        ref = oracle.operator(p["g_or"], x, p["S"], p["mu"], p["I0"], p["y"])
        assert rel_l2(F, ref) <= 1e-5


def test_norm_estimate_parity():
    for gi in (0, 2):
        geom = GEOMS[gi]
        plan = _plan(geom, np.ones((1, 1)), np.ones(1))
        lam, it = plan.norm_estimate(max_iters=40, rtol=0.0)
        ref, it_ref = oracle.norm_estimate(oracle.Geometry(**geom), max_iters=40, rtol=0.0)
        assert it == it_ref == 40
        assert lam == pytest.approx(ref, rel=1e-9)
        lam2, it2 = plan.norm_estimate(max_iters=2000, rtol=1e-10)
        ref2, it2_ref = oracle.norm_estimate(oracle.Geometry(**geom), max_iters=2000, rtol=1e-10)
        assert lam2 == pytest.approx(ref2, rel=1e-9)
        assert abs(it2 - it2_ref) <= 2


def _eta(p):
    nA, _ = oracle.norm_estimate(p["g_or"], 1000, 1e-10)
    return 1.0 / (4.0 * oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))


def test_solve_parity_c1():
    c = configs.C1
    p = problem(c["geometry"], K=c["K"], W=c["W"], I0=c["I0"], n_ellipses=c["n_ellipses"], seed=1)
    eta = _eta(p)
    plan = _plan(c["geometry"], p["S"], p["mu"])
    x, info = plan.solve(_gpu(p["y"]), p["I0"], eta, c["iters"])
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, c["iters"])
    xg = x.double().cpu().numpy()
    assert info.iters_done == c["iters"] and info.status == 0
    assert rel_l2(xg, ref.x) <= 1e-3
    assert abs(psnr(xg, p["xs"]) - psnr(ref.x, p["xs"])) <= 0.05
    assert info.rel_res == pytest.approx(ref.rel_res[-1], rel=1e-2)
    assert (xg >= 0).all()


@pytest.mark.parametrize("I0", [1e3, 1e5])
def test_solve_parity_c2_short(I0):
    c = configs.C2
    p = problem(c["geometry"], K=c["K"], W=c["W"], I0=I0, n_ellipses=c["n_ellipses"], seed=2)
    eta = _eta(p)
    plan = _plan(c["geometry"], p["S"], p["mu"])
    x, info = plan.solve(_gpu(p["y"]), I0, eta, 20)
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], I0, p["y"], eta, 20)
    xg = x.double().cpu().numpy()
    assert rel_l2(xg, ref.x) <= 1e-3
    assert abs(psnr(xg, p["xs"]) - psnr(ref.x, p["xs"])) <= 0.05


def test_solve_parity_c2_full():
    c = configs.C2
    p = problem(c["geometry"], K=c["K"], W=c["W"], I0=c["I0"], n_ellipses=c["n_ellipses"], seed=3)
    eta = _eta(p)
    plan = _plan(c["geometry"], p["S"], p["mu"])
    x, info = plan.solve(_gpu(p["y"]), p["I0"], eta, c["iters"])
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, c["iters"])
    xg = x.double().cpu().numpy()
    assert info.iters_done == c["iters"]
    assert rel_l2(xg, ref.x) <= 1e-3
    assert abs(psnr(xg, p["xs"]) - psnr(ref.x, p["xs"])) <= 0.05


def test_solve_options_box_tolerance_average():
    geom = GEOMS[2]
    p = problem(geom, K=12, W=2, I0=1e4, seed=5)
    eta = _eta(p)
    plan = _plan(geom, p["S"], p["mu"])
    y = _gpu(p["y"])
    # upper bound binds
    x, _ = plan.solve(y, p["I0"], eta, 15, hi=0.2)
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 15, hi=0.2)
    xg = x.double().cpu().numpy()
    assert xg.max() <= 0.2 and rel_l2(xg, ref.x) <= 1e-3
    # tail average
    x, _ = plan.solve(y, p["I0"], eta, 15, average_tail=True)
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 15, average_tail=True)
    assert rel_l2(x.double().cpu().numpy(), ref.x_avg) <= 1e-3
    # tolerance stop: same stopping iteration up to one check interval
    full = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 200)
    tol = float(full.rel_res[60])
    x, info = plan.solve(y, p["I0"], eta, 200, tol=tol, check_every=3)
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 200, tol=tol, check_every=3)
    assert abs(info.iters_done - ref.iters) <= 3
    assert info.rel_res <= tol
    # warm start: x_1 given, projected onto the box
    x1 = _gpu(np.full((geom["ny"], geom["nx"]), -1.0))
    x, _ = plan.solve(y, p["I0"], eta, 0, x=x1)
    assert float(x.min()) == 0.0


def test_solve_deterministic():
    geom = GEOMS[3]
    p = problem(geom, K=8, W=2, I0=1e4, seed=6)
    plan = _plan(geom, p["S"], p["mu"])
    y = _gpu(p["y"])
    a, _ = plan.solve(y, p["I0"], _eta(p), 25)
    b, _ = plan.solve(y, p["I0"], _eta(p), 25)
    assert torch.equal(a, b)


def test_invalid_arguments():
    geom = dict(GEOMS[0])
    with pytest.raises(ex.ExactError):
        ex.Plan(ex.Geometry(**dict(geom, nx=0)), [1.0], [[1.0]])
    with pytest.raises(ex.ExactError):
        ex.Plan(ex.Geometry(**geom), [-1.0], [[1.0]])
    with pytest.raises(ex.ExactError):
        ex.Plan(ex.Geometry(**geom), [1.0], [[0.0]])
    with pytest.raises(ex.ExactError):  # fan source inside the image
        ex.Plan(ex.Geometry(**dict(geom, beam=1, src_to_center=10.0, src_to_det=20.0)), [1.0], [[1.0]])
    plan = _plan(geom, np.ones((1, 1)), np.ones(1))
    y = torch.zeros((1, geom["n_views"], geom["n_bins"]), device=DEV)
    with pytest.raises(ex.ExactError):
        plan.solve(y, -1.0, 1.0, 3)
    with pytest.raises(ex.ExactError):
        plan.solve(y, 1.0, 1.0, 3, lo=1.0, hi=0.0)


def test_nonfinite_counts_stop_with_status():
    geom = GEOMS[0]
    plan = _plan(geom, np.ones((1, 1)), np.ones(1) * 0.05)
    y = torch.full((1, geom["n_views"], geom["n_bins"]), float("nan"), device=DEV)
    x, info = plan.solve(y, 100.0, 1e-3, 10)
    assert info.status == 5 and info.iters_done == 1


# ---- full-size workload (512^2 fan beam, 720 views x 736 bins, 4 windows over
# 64 energies, BF16 counts) in the launch configuration the benchmark times ----

@pytest.fixture(scope="module")
def c3():
    c = configs.C3
    p = problem(c["geometry"], K=c["K"], W=c["W"], I0=c["I0"], n_ellipses=c["n_ellipses"], seed=3, bf16=True)
    plan = _plan(c["geometry"], p["S"], p["mu"])
    plan.autotune()  # as the benchmark does
    return c, p, plan


def test_c3_forward_adjoint_operator(c3):
    c, p, plan = c3
    x = p["xs"]
    z = plan.forward(_gpu(x)).double().cpu().numpy()
    assert rel_l2(z, oracle.forward(p["g_or"], x)) <= 1e-5
    r = synth.random_sinogram(c["geometry"]["n_views"], c["geometry"]["n_bins"], seed=4, lo=-1, hi=1)
    ref = oracle.adjoint(p["g_or"], r)
    tuned = plan.tuning["adj_split"]
    for s in (tuned, 1, 8):  # the autotuned split, and the extremes
        plan.set_tuning(s)
        g = plan.adjoint(_gpu(r)).double().cpu().numpy()
        assert rel_l2(g, ref) <= 1e-5
    plan.set_tuning(tuned)
    F = plan.operator(_gpu(0.5 * x), _gpu(p["y"], torch.bfloat16), p["I0"]).double().cpu().numpy()
    assert rel_l2(F, oracle.operator(p["g_or"], 0.5 * x, p["S"], p["mu"], p["I0"], p["y"])) <= 1e-5


def test_c3_solve_first_iterations_and_norm(c3):
    c, p, plan = c3
    lam, it = plan.norm_estimate(max_iters=5, rtol=0.0)
    ref, _ = oracle.norm_estimate(p["g_or"], 5, 0.0)
    assert lam == pytest.approx(ref, rel=1e-9)
    eta = plan.recommended_eta(p["I0"], lam)
    x, info = plan.solve(_gpu(p["y"], torch.bfloat16), p["I0"], eta, 3)
    refx = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 3)
    assert rel_l2(x.double().cpu().numpy(), refx.x) <= 1e-4


# ---- the largest request of the serving stream: 1024^2 image, 1440 views ----

def test_max_size_forward_adjoint_operator():
    """1024^2 fan beam, 1440 views x 1449 bins (the top of the serving mix):
    A x, A^T r (autotuned split and no split) and F(x) against the oracle."""
    geom = dict(beam=1, nx=1024, ny=1024, n_views=1440, n_bins=1449, angle_range=2 * math.pi, bin_pitch=1.5,
                src_to_center=2000.0, src_to_det=3000.0)
    p = problem(geom, K=16, W=2, I0=1e4, seed=11, bf16=True)
    plan = _plan(geom, p["S"], p["mu"])
    plan.autotune()
    x = p["xs"]
    z = plan.forward(_gpu(x)).double().cpu().numpy()
    assert rel_l2(z, oracle.forward(p["g_or"], x)) <= 1e-5
    r = synth.random_sinogram(geom["n_views"], geom["n_bins"], seed=12, lo=-1, hi=1)
    ref = oracle.adjoint(p["g_or"], r)
    tuned = plan.tuning["adj_split"]
    for s in sorted({tuned, 1}):
        plan.set_tuning(s)
        g = plan.adjoint(_gpu(r)).double().cpu().numpy()
        assert rel_l2(g, ref) <= 1e-5
    plan.set_tuning(tuned)
    F = plan.operator(_gpu(0.5 * x), _gpu(p["y"], torch.bfloat16), p["I0"]).double().cpu().numpy()
    assert rel_l2(F, oracle.operator(p["g_or"], 0.5 * x, p["S"], p["mu"], p["I0"], p["y"])) <= 1e-5


@pytest.mark.parametrize("gi", [0, 2])
def test_known_background_operator_and_solve(gi):
    """Appendix A.1: known materials enter through their projections."""
    geom = GEOMS[gi]
    p = problem(geom, K=16, W=2, I0=1e4, seed=60 + gi)
    e = synth.energy_grid(16)
    mu_bg = np.stack([synth.power_law_mu(e, 0.03) + 0.002, synth.power_law_mu(e, 0.08)])
    g_or = p["g_or"]
    xb = [synth.random_image(geom["nx"], geom["ny"], seed=5 + m, hi=0.3) for m in range(2)]
    pb = np.stack([oracle.forward(g_or, x) for x in xb])
    lam = oracle.expected_counts(oracle.forward(g_or, p["xs"]), p["S"], p["mu"], p["I0"], bg=(mu_bg, pb))
    y = synth.poisson_counts(lam, 3)
    plan = _plan(geom, p["S"], p["mu"])
    pg = _gpu(pb)
    plan.set_background(mu_bg, pg)
    x = 0.5 * p["xs"]
    F = plan.operator(_gpu(x), _gpu(y), p["I0"]).double().cpu().numpy()
    ref = oracle.operator(g_or, x, p["S"], p["mu"], p["I0"], y, bg=(mu_bg, pb))
    assert rel_l2(F, ref) <= 1e-5
    eta = _eta(p)
    xg, info = plan.solve(_gpu(y), p["I0"], eta, 30)
    xr = oracle.solve(g_or, p["S"], p["mu"], p["I0"], y, eta, 30, bg=(mu_bg, pb))
    assert rel_l2(xg.double().cpu().numpy(), xr.x) <= 1e-3
    # and the batch path uses the same background
    xs, infos = ex.Batch(2).solve([ex.Job(plan=plan, y=_gpu(y), I0=p["I0"], eta=eta, iters=30)])
    assert rel_l2(xs[0].double().cpu().numpy(), xr.x) <= 1e-3
    plan.set_background()
    F0 = plan.operator(_gpu(x), _gpu(y), p["I0"]).double().cpu().numpy()
    assert rel_l2(F0, oracle.operator(g_or, x, p["S"], p["mu"], p["I0"], y)) <= 1e-5
