"""Batched solves against single solves and the oracle, under policies 0 and 1
(one persistent launch for all jobs, one CTA per adjoint tile or each plan's
view split) and policy 2 (each job's own solve on one of the batch context's
streams): a job's result is bitwise the same alone and in
any mix, matches the single-job path (bit for bit under policy 2) and the FP64
oracle within the solve tolerances, and replays from a captured CUDA graph."""
import math

import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2503_19925_gb300 as ex
from tests.cases import problem, rel_l2, psnr

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

DEV = "cuda:0"

MIX = [
    (dict(beam=0, nx=64, ny=64, n_views=90, n_bins=91, angle_range=math.pi), 1, 10, False),
    (dict(beam=1, nx=96, ny=80, n_views=61, n_bins=137, angle0=0.05, angle_range=2 * math.pi, bin_pitch=1.5,
          src_to_center=300.0, src_to_det=450.0), 3, 16, True),
    (dict(beam=0, nx=77, ny=45, n_views=33, n_bins=101, angle0=0.2, angle_range=math.pi, bin_pitch=0.9,
          det_offset=0.31), 2, 12, False),
    (dict(beam=1, nx=33, ny=130, n_views=40, n_bins=150, angle0=1.0, angle_range=2 * math.pi, bin_pitch=1.1,
          det_offset=-2.0, src_to_center=120.0, src_to_det=200.0), 4, 8, True),
    (dict(beam=0, nx=128, ny=128, n_views=120, n_bins=183, angle_range=math.pi), 2, 32, False),
]


def _eta(p):
    nA, _ = oracle.norm_estimate(p["g_or"], 1000, 1e-10)
    return 1.0 / (4.0 * oracle.lipschitz(nA, p["S"], p["mu"], p["I0"], p["S"].shape[0] * p["g_or"].n_rays))


@pytest.fixture(scope="module")
def mix():
    out = []
    for k, (geom, W, K, bf16) in enumerate(MIX):
        p = problem(geom, K=K, W=W, I0=10 ** (3 + k % 3), seed=40 + k, bf16=bf16)
        plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
        y = torch.as_tensor(p["y"], dtype=torch.bfloat16 if bf16 else torch.float32, device=DEV).contiguous()
        out.append((p, plan, y, _eta(p)))
    return out


def _jobs(mix, iters, idx=None, **kw):
    idx = range(len(mix)) if idx is None else idx
    return [ex.Job(plan=mix[k][1], y=mix[k][2], I0=mix[k][0]["I0"], eta=mix[k][3],
                   iters=iters[k] if isinstance(iters, (list, tuple)) else iters, **kw) for k in idx]


POLICIES = [0, 1, 2]


def _batch(n, policy):
    b = ex.Batch(n)
    b.set_policy(policy)
    assert b.policy == policy
    return b


@pytest.mark.parametrize("policy", POLICIES)
def test_batch_matches_single_solve_and_oracle(mix, policy):
    batch = _batch(8, policy)
    xs, infos = batch.solve(_jobs(mix, 12))
    for k, (p, plan, y, eta) in enumerate(mix):
        single, _ = plan.solve(y, p["I0"], eta, 12)
        assert rel_l2(xs[k].double().cpu().numpy(), single.double().cpu().numpy()) <= 1e-5
        if policy == 2:
            assert torch.equal(xs[k], single)
        ref = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 12)
        xb = xs[k].double().cpu().numpy()
        assert rel_l2(xb, ref.x) <= 1e-3
        assert abs(psnr(xb, p["xs"]) - psnr(ref.x, p["xs"])) <= 0.05
        assert infos[k].iters_done == 12 and infos[k].status == 0
    batch.close()


@pytest.mark.parametrize("policy", POLICIES)
def test_result_independent_of_mix(mix, policy):
    batch = _batch(8, policy)
    iters = [9, 14, 5, 11, 7]
    xs_all, infos_all = batch.solve(_jobs(mix, iters))
    for k in range(len(mix)):
        xs_one, infos_one = batch.solve(_jobs(mix, iters, idx=[k]))
        assert torch.equal(xs_all[k], xs_one[0]), k
        assert infos_all[k].iters_done == iters[k] == infos_one[0].iters_done
    # reversed order, another subset
    xs_rev, _ = batch.solve(_jobs(mix, iters, idx=[4, 2, 0]))
    assert torch.equal(xs_rev[0], xs_all[4]) and torch.equal(xs_rev[2], xs_all[0])
    batch.close()


@pytest.mark.parametrize("policy", POLICIES)
def test_batch_tolerance_stop_and_box(mix, policy):
    batch = _batch(8, policy)
    p, plan, y, eta = mix[0]
    full = oracle.solve(p["g_or"], p["S"], p["mu"], p["I0"], p["y"], eta, 150)
    tol = float(full.rel_res[40])
    xs, infos = batch.solve(_jobs(mix, 150, idx=[0, 1], tol=tol, check_every=2, hi=0.5))
    single, sinfo = plan.solve(y, p["I0"], eta, 150, tol=tol, check_every=2, hi=0.5)
    assert infos[0].iters_done == sinfo.iters_done
    assert float(xs[0].max()) <= 0.5
    assert rel_l2(xs[0].double().cpu().numpy(), single.double().cpu().numpy()) <= 1e-5
    batch.close()


@pytest.mark.parametrize("policy", POLICIES)
def test_batch_in_cuda_graph(mix, policy):
    batch = _batch(8, policy)
    jobs = _jobs(mix, 6)
    xs_ref, _ = batch.solve(jobs)
    ref = [x.clone() for x in xs_ref]
    xs = [torch.zeros_like(x) for x in ref]
    for jb, x in zip(jobs, xs):
        jb.x = x
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.solve(jobs, sync=False)
    for _ in range(2):
        for x in xs:
            x.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(xs, ref):
            assert torch.equal(a, b)
    batch.close()


def test_batch_policy_argument():
    batch = ex.Batch(2)
    assert batch.policy == 0  # a new context runs the persistent kernel
    for bad in (-1, 3):
        with pytest.raises(ex.ExactError):
            batch.set_policy(bad)
    assert batch.policy == 0
    batch.close()


@pytest.mark.parametrize("policy", POLICIES)
def test_batch_invalid_arguments(mix, policy):
    batch = _batch(2, policy)
    with pytest.raises(ex.ExactError):  # more jobs than the context holds
        batch.solve(_jobs(mix, 3))
    with pytest.raises(ex.ExactError):  # the same plan twice
        batch.solve(_jobs(mix, 3, idx=[0, 0]))
    batch.close()
