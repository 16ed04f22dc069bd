"""Host logic of the serving loop with the GPU parts replaced by fakes:
admission by memory budget and slots, round scheduling, retirement on the
tolerance, iteration caps, failing jobs, arrivals that join mid-run."""
import math
import sys
import types

import pytest

torch = pytest.importorskip("torch")

import paper_2503_19925_gb300.serve as serve


class FakeInfo:
    def __init__(self, iters, rel, status=0):
        self.iters_done, self.rel_res, self.status = iters, rel, status


class FakePlan:
    live = 0

    def __init__(self, geometry, mu, S):
        self.geometry = geometry
        self.shape_img = (geometry.ny, geometry.nx)
        self.device = torch.device("cpu")
        self.closed = False
        FakePlan.live += 1

    def autotune(self, force=False):
        self.tuned = True
        return {"adj_split": 1}

    def norm_estimate_f32(self, iters, rtol):
        return 100.0, 5

    def recommended_eta(self, I0, lam):
        return 0.1

    def close(self):
        assert not self.closed
        self.closed = True
        FakePlan.live -= 1


class FakeBatch:
    """Each job's residual halves every iteration from 1.0; a job whose tag is
    'bad' reports a non-finite residual."""

    def __init__(self, max_slots):
        self.calls = []

    def solve(self, jobs, sync=True):
        import time
        self.calls.append(len(jobs))
        time.sleep(0.002)
        infos = []
        for jb in jobs:
            done = getattr(jb.plan, "progress", 0)
            if getattr(jb.plan, "bad", False):
                infos.append(FakeInfo(1, float("nan"), 5))
                continue
            k = 0
            rel = 0.5 ** done
            while k < jb.iters:
                k += 1
                rel = 0.5 ** (done + k)
                if jb.tol > 0 and rel <= jb.tol:
                    break
            jb.plan.progress = done + k
            infos.append(FakeInfo(k, rel))
        return [jb.x for jb in jobs], infos

    def close(self):
        pass


@pytest.fixture(autouse=True)
def fakes(monkeypatch):
    monkeypatch.setattr(serve, "Plan", FakePlan)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    FakePlan.live = 0
    yield


def _req(n, tol=1e-3, max_iters=100, tag=None, arrival=0.0):
    from paper_2503_19925_gb300.exact import Geometry
    g = Geometry(beam=0, nx=n, ny=n, n_views=10, n_bins=n)
    return serve.Request(g, [1.0], [[1.0]], torch.zeros(1, 10, n), 1e3, tol=tol, max_iters=max_iters,
                         arrival=arrival, tag=tag)


def test_all_requests_finish_and_memory_is_released():
    reqs = [_req(32 + 8 * k, tag=k) for k in range(10)]
    s = serve.Server(budget_bytes=1e12, max_slots=4, round_iters=3)
    res = s.run(reqs, realtime=False)
    assert sorted(r.tag for r in res) == list(range(10))
    assert all(r.iters == 10 and r.rel_res <= 1e-3 for r in res)  # 0.5^10 < 1e-3
    assert FakePlan.live == 0 and s.used == 0
    assert max(s.batch.calls) <= 4  # never more than max_slots resident


def test_budget_admits_one_at_a_time():
    reqs = [_req(64, tag=k) for k in range(3)]
    one = serve.footprint_bytes(reqs[0].geometry, 1, 4)
    s = serve.Server(budget_bytes=one * 1.5, max_slots=8, round_iters=4)
    res = s.run(reqs, realtime=False)
    assert len(res) == 3 and max(s.batch.calls) == 1
    assert s.peak_used <= one * 1.5


def test_iteration_cap_and_failure():
    reqs = [_req(32, tol=0.0, max_iters=7, tag="cap"), _req(32, tag="bad")]
    s = serve.Server(budget_bytes=1e12, max_slots=4, round_iters=3)
    orig = s._admit

    def admit():
        orig()
        for a in s.active:
            if a.req.tag == "bad":
                a.plan.bad = True
    s._admit = admit
    res = {r.tag: r for r in s.run(reqs, realtime=False)}
    assert res["cap"].iters == 7 and res["cap"].status == 0
    assert res["bad"].status == 5
    assert FakePlan.live == 0


def test_late_arrivals_join_running_batch():
    reqs = [_req(32, tol=0.0, max_iters=100, tag="early")] + [_req(32, tag=f"late{k}", arrival=0.05) for k in range(2)]
    s = serve.Server(budget_bytes=1e12, max_slots=4, round_iters=2)
    res = {r.tag: r for r in s.run(reqs, realtime=True)}
    assert set(res) == {"early", "late0", "late1"}
    assert max(s.batch.calls) == 3  # the late requests ran alongside the early one
