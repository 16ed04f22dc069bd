"""Serving: continuous batching returns, for every request, the image of the
request served alone and the image of a plain single solve, within 1e-4
relative L2 (a round with one resident job runs the plain solve, a shared
round the persistent kernel, so the FP32 rounding differs with the mix); new
arrivals join while earlier requests run.  Also the FP32 power iteration
against the FP64 one."""
import math

import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2503_19925_gb300 as ex
from paper_2503_19925_gb300.serve import Request, Server, serve_sequential
from tests.cases import problem, rel_l2

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

GEOMS = [
    (dict(beam=0, nx=64, ny=64, n_views=90, n_bins=91, angle_range=math.pi), 1, 10),
    (dict(beam=1, nx=96, ny=96, n_views=72, n_bins=181, angle_range=2 * math.pi, bin_pitch=1.5,
          src_to_center=192.0, src_to_det=288.0), 3, 16),
    (dict(beam=0, nx=80, ny=48, n_views=50, n_bins=97, angle_range=math.pi), 2, 12),
    (dict(beam=0, nx=128, ny=128, n_views=60, n_bins=183, angle_range=math.pi), 4, 24),
]


@pytest.fixture(scope="module")
def requests():
    out = []
    for k, (geom, W, K) in enumerate(GEOMS):
        p = problem(geom, K=K, W=W, I0=10 ** (3 + k % 3), seed=70 + k)
        out.append(Request(ex.Geometry(**geom), list(p["mu"]), p["S"].tolist(),
                           torch.tensor(p["y"], dtype=torch.float32), p["I0"], tol=2e-3, max_iters=400,
                           arrival=0.02 * k, tag=k))
    return out


@pytest.mark.parametrize("mode", ["streams", "rounds"])
def test_served_equals_alone_and_plain(requests, mode):
    """Streams mode: all requests resident at once, their solves overlapping
    on the device, each bitwise its plain solve.  Rounds mode: arrivals join
    running rounds, results within 1e-4 of the plain solve."""
    server = Server(budget_bytes=4e9, max_slots=8, round_iters=10, mode=mode)
    mixed = {r.tag: r for r in server.run(requests, realtime=mode == "rounds")}
    server.close()
    assert sorted(mixed) == list(range(len(requests)))
    if mode == "rounds":
        assert server.rounds > 1
    else:
        assert server.peak_resident >= 2  # solves overlapped on the device
    plain = {r.tag: r for r in serve_sequential(requests, realtime=False)}
    for req in requests:
        alone_server = Server(budget_bytes=4e9, max_slots=8, round_iters=10, mode=mode)
        alone = alone_server.run([req], realtime=False)[0]
        alone_server.close()
        m = mixed[req.tag]
        assert rel_l2(m.x.double().numpy(), alone.x.double().numpy()) <= 1e-4, req.tag
        assert abs(alone.iters - m.iters) <= 1 and m.status == 0
        assert rel_l2(m.x.double().numpy(), plain[req.tag].x.double().numpy()) <= 1e-4
        assert abs(m.iters - plain[req.tag].iters) <= 1
        assert m.rel_res <= req.tol or m.iters == req.max_iters
        if mode == "streams":
            assert torch.equal(m.x, plain[req.tag].x) and m.iters == plain[req.tag].iters


def test_budget_limits_residency(requests):
    from paper_2503_19925_gb300.serve import footprint_bytes
    big = max(footprint_bytes(r.geometry, len(r.S), 4) for r in requests)
    server = Server(budget_bytes=big * 1.5, max_slots=8, round_iters=10)
    res = server.run(requests, realtime=False)
    server.close()
    assert len(res) == len(requests)
    assert server.peak_used <= big * 1.5


def test_norm_estimate_f32_matches_fp64():
    geom = GEOMS[1][0]
    p = problem(geom, K=8, W=1, seed=1)
    plan = ex.Plan(ex.Geometry(**geom), p["mu"], p["S"])
    l64, _ = plan.norm_estimate(200, 1e-10)
    l32, it = plan.norm_estimate_f32(200, 1e-7)
    ref, _ = oracle.norm_estimate(p["g_or"], 200, 1e-10)
    assert l64 == pytest.approx(ref, rel=1e-9)
    assert l32 == pytest.approx(ref, rel=1e-5)
    assert it < 200
