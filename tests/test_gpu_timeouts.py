"""Bounded device waits run out into EXACT_ERR_TIMEOUT, and the device stays
usable: a batch job whose dependency can never be met (the persistent
kernel's phase wait) and a TV projection whose grid barrier can never complete
(exact_debug_inject), each with a short poll limit.  Neither faults, traps or
hangs the GPU: the wait gives up, every thread block leaves, the call returns
the status, and the next call on the same context is correct."""
import math
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2503_19925_gb300 as ex
from tests.cases import problem, rel_l2

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

TIMEOUT = 4
WAIT_POLLS, BLOCK_BATCH_JOB, BLOCK_TV_BARRIER = 1, 2, 3


@pytest.fixture
def inject():
    lib = ex.load()
    yield lib
    # leave nothing armed for later tests
    assert lib.exact_debug_inject(WAIT_POLLS, 0) == 0
    assert lib.exact_debug_inject(BLOCK_BATCH_JOB, -1) == 0
    assert lib.exact_debug_inject(BLOCK_TV_BARRIER, 0) == 0


def _jobs():
    geoms = [dict(beam=0, nx=48, ny=48, n_views=40, n_bins=69, angle_range=math.pi),
             dict(beam=1, nx=40, ny=56, n_views=36, n_bins=91, angle_range=2 * math.pi, bin_pitch=1.5,
                  src_to_center=120.0, src_to_det=180.0)]
    out = []
    for k, geom in enumerate(geoms):
        p = problem(geom, K=8, W=1 + k, I0=1e4, seed=90 + k)
        plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
        y = torch.as_tensor(p["y"], dtype=torch.float32, device="cuda:0").contiguous()
        out.append((plan, y, p["I0"]))
    return out


def test_batch_dependency_wait_runs_out(inject):
    lib = inject
    jobs_in = _jobs()
    batch = ex.Batch(4)

    def run():
        xs = [torch.zeros(p.shape_img, dtype=torch.float32, device="cuda:0") for p, _, _ in jobs_in]
        jobs = [ex.Job(plan=p, y=y, I0=I0, eta=1e-3, iters=12, x=x) for (p, y, I0), x in zip(jobs_in, xs)]
        return batch.solve(jobs)

    ref_xs, ref_infos = run()
    assert all(i.status == 0 and i.iters_done == 12 for i in ref_infos)
    assert lib.exact_debug_inject(WAIT_POLLS, 4096) == 0
    assert lib.exact_debug_inject(BLOCK_BATCH_JOB, 1) == 0
    t = time.perf_counter()
    _, infos = run()
    assert time.perf_counter() - t < 30.0
    assert infos[1].status == TIMEOUT
    assert infos[1].iters_done < 12
    # the block was one-shot: the same context computes the same results again
    assert lib.exact_debug_inject(WAIT_POLLS, 0) == 0
    xs, infos = run()
    assert all(i.status == 0 and i.iters_done == 12 for i in infos)
    for a, b in zip(xs, ref_xs):
        assert torch.equal(a, b)
    batch.close()
    for p, _, _ in jobs_in:
        p.close()


def test_tv_grid_barrier_runs_out(inject):
    lib = inject
    rng = np.random.default_rng(3)
    z = torch.as_tensor(rng.uniform(0, 1, (64, 80)), dtype=torch.float32, device="cuda:0")
    x_ref, info_ref = ex.tv_project(z, 20.0)
    assert info_ref.status == 0
    assert lib.exact_debug_inject(WAIT_POLLS, 4096) == 0
    assert lib.exact_debug_inject(BLOCK_TV_BARRIER, 1) == 0
    with pytest.raises(ex.ExactError) as err:
        ex.tv_project(z, 20.0)
    assert err.value.status == TIMEOUT
    assert lib.exact_debug_inject(WAIT_POLLS, 0) == 0
    x, info = ex.tv_project(z, 20.0)
    assert info.status == 0 and torch.equal(x, x_ref)


def test_tv_solve_stops_with_timeout(inject):
    """A solve on the TV ball whose projection's barrier cannot complete stops
    with EXACT_ERR_TIMEOUT in its info; the next solve is correct."""
    lib = inject
    geom = dict(beam=0, nx=40, ny=40, n_views=30, n_bins=59, angle_range=math.pi)
    p = problem(geom, K=8, W=1, I0=1e4, seed=95)
    plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
    y = torch.as_tensor(p["y"], dtype=torch.float32, device="cuda:0").contiguous()
    opts = {"fgp_iters": 10, "max_bisect": 5, "max_dykstra": 3}
    x_ref, info_ref = plan.solve(y, p["I0"], 1e-3, 4, tv_bound=30.0, tv_opts=opts)
    assert info_ref.status == 0
    assert lib.exact_debug_inject(WAIT_POLLS, 4096) == 0
    assert lib.exact_debug_inject(BLOCK_TV_BARRIER, 1) == 0
    _, info = plan.solve(y, p["I0"], 1e-3, 4, tv_bound=30.0, tv_opts=opts)
    assert info.status == TIMEOUT and info.iters_done < 4
    assert lib.exact_debug_inject(WAIT_POLLS, 0) == 0
    x, info = plan.solve(y, p["I0"], 1e-3, 4, tv_bound=30.0, tv_opts=opts)
    assert info.status == 0 and torch.equal(x, x_ref)
    plan.close()


def test_inject_argument_checks():
    lib = ex.load()
    assert lib.exact_debug_inject(99, 0) == 1
    assert lib.exact_debug_inject(WAIT_POLLS, -5) == 1
    assert lib.exact_debug_inject(BLOCK_BATCH_JOB, 100000) == 1
