"""The adjoint's view split (exact_tuning.adj_split) and the autotuner.

Every split value must give the same A^T r up to FP32 rounding (checked
against the FP64 oracle at the parity tolerance and against split 1), be
bit-for-bit reproducible, and keep solves and batches at parity; the
autotuner must pick a listed value and reuse it for a plan of the same shape.
"""
import math

import pytest

torch = pytest.importorskip("torch")

import oracle
import synth
import paper_2503_19925_gb300 as ex
from synth import configs
from tests.cases import problem, rel_l2, psnr

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

DEV = "cuda:0"
GEOMS = [
    dict(beam=0, nx=64, ny=64, n_views=90, n_bins=91, angle_range=math.pi),
    dict(beam=1, nx=96, ny=80, n_views=61, n_bins=137, angle0=0.05, angle_range=2 * math.pi, bin_pitch=1.5,
         src_to_center=300.0, src_to_det=450.0),
    dict(beam=0, nx=37, ny=29, n_views=7, n_bins=51, angle0=0.3, angle_range=math.pi),
]


@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_split_adjoint_parity_and_determinism(gi):
    geom = GEOMS[gi]
    plan = ex.Plan(ex.Geometry(**geom), [1.0], [[1.0]])
    r = synth.random_sinogram(geom["n_views"], geom["n_bins"], seed=40 + gi)
    ref = oracle.adjoint(oracle.Geometry(**geom), r)
    rg = torch.as_tensor(r, dtype=torch.float32, device=DEV)
    base = None
    for s in (1, 2, 3, 8):
        plan.set_tuning(s)
        assert plan.tuning["adj_split"] == s
        g1 = plan.adjoint(rg).clone()
        g2 = plan.adjoint(rg)
        assert torch.equal(g1, g2)
        gd = g1.double().cpu().numpy()
        assert rel_l2(gd, ref) <= 1e-5
        if base is None:
            base = gd
        else:
            assert rel_l2(gd, base) <= 2e-6
    plan.close()


def test_split_solve_parity():
    c = configs.C1
    p = problem(c["geometry"], K=c["K"], W=c["W"], I0=c["I0"], n_ellipses=c["n_ellipses"], seed=1)
    nA, _ = oracle.norm_estimate(p["g_or"], 300, 1e-10)
    eta = 1.0 / (4.0 * oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))
    plan = ex.Plan(ex.Geometry(**c["geometry"]), p["mu"], p["S"])
    plan.set_tuning(4)
    y = torch.as_tensor(p["y"], dtype=torch.float32, device=DEV)
    x1, _ = plan.solve(y, p["I0"], eta, 100)
    x2, _ = plan.solve(y, p["I0"], eta, 100)
    assert torch.equal(x1, x2)
    ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 100)
    xg = x1.double().cpu().numpy()
    assert rel_l2(xg, ref.x) <= 1e-3
    assert abs(psnr(xg, p["xs"]) - psnr(ref.x, p["xs"])) <= 0.05


def test_split_batch_matches_single_solves():
    """Plans with splits 3, 1 and 8 in one batch."""
    jobs_in = []
    for k, (n, v, s) in enumerate([(64, 40, 3), (48, 30, 1), (80, 50, 8)]):
        geom = dict(beam=0, nx=n, ny=n, n_views=v, n_bins=int(math.ceil(n * math.sqrt(2))) | 1,
                    angle_range=math.pi)
        p = problem(geom, K=6, W=1 + k % 2, I0=1e4, seed=60 + k)
        plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
        plan.set_tuning(s)
        nA, _ = plan.norm_estimate(100, 1e-6)
        jobs_in.append((plan, torch.as_tensor(p["y"], dtype=torch.float32, device=DEV),
                        plan.recommended_eta(1e4, nA)))
    singles = [pl.solve(y, 1e4, eta, 25)[0].clone() for pl, y, eta in jobs_in]
    batch = ex.Batch(4)
    xs, infos = batch.solve([ex.Job(plan=pl, y=y, I0=1e4, eta=eta, iters=25) for pl, y, eta in jobs_in])
    # the persistent kernel splits each tile's views over its own warp count,
    # so it agrees with the single solves to FP32 rounding, not bit for bit
    for xb, xsg in zip(xs, singles):
        assert rel_l2(xb.double().cpu().numpy(), xsg.double().cpu().numpy()) <= 1e-5
    xs2, _ = batch.solve([ex.Job(plan=pl, y=y, I0=1e4, eta=eta, iters=25) for pl, y, eta in jobs_in])
    for a, b in zip(xs, xs2):
        assert torch.equal(a, b)
    batch.close()


def test_autotune_picks_a_listed_split_and_caches_it():
    geom = dict(beam=0, nx=96, ny=96, n_views=60, n_bins=137, angle_range=math.pi)
    p1 = ex.Plan(ex.Geometry(**geom), [1.0], [[1.0]])
    t1 = p1.autotune()
    assert t1["adj_split"] in (1, 2, 3, 4, 6, 8, 12, 16)
    p2 = ex.Plan(ex.Geometry(**geom), [2.0], [[0.5]])
    assert p2.autotune() == t1  # cached shape
    t3 = p2.autotune(force=True)
    assert t3["adj_split"] in (1, 2, 3, 4, 6, 8, 12, 16)
    with pytest.raises(RuntimeError):
        p1.set_tuning(17)
    # a large image's limit is below 16 (about 64 CTAs per SM in all)
    big = ex.Plan(ex.Geometry(beam=0, nx=2048, ny=2048, n_views=8, n_bins=2897, angle_range=math.pi),
                  [1.0], [[1.0]])
    with pytest.raises(RuntimeError):
        big.set_tuning(16)
    big.set_tuning(2)
    big.close()


def test_batch_autotune_leaves_the_jobs_unchanged():
    jobs_in = []
    for k, (n, v) in enumerate([(64, 40), (48, 30)]):
        geom = dict(beam=0, nx=n, ny=n, n_views=v, n_bins=int(math.ceil(n * math.sqrt(2))) | 1,
                    angle_range=math.pi)
        p = problem(geom, K=6, W=1, I0=1e4, seed=70 + k)
        plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
        plan.set_tuning(4)
        nA, _ = plan.norm_estimate(100, 1e-6)
        x = torch.rand((n, n), device=DEV)
        jobs_in.append(ex.Job(plan=plan, y=torch.as_tensor(p["y"], dtype=torch.float32, device=DEV), I0=1e4,
                              eta=plan.recommended_eta(1e4, nA), iters=10, x=x))
    before = [j.x.clone() for j in jobs_in]
    batch = ex.Batch(4)
    policy = batch.autotune(jobs_in)
    assert policy in (0, 1, 2)
    assert batch.policy == policy
    for j, b in zip(jobs_in, before):
        assert torch.equal(j.x, b)
    batch.close()
