"""Host logic of the serving loop with the GPU parts replaced by fakes:
admission by memory budget and slots, round scheduling, retirement on the
tolerance, iteration caps, failing jobs, arrivals that join mid-run."""
import math

import pytest

torch = pytest.importorskip("torch")

import paper_2503_19925_gb300.serve as serve


class FakeInfo:
    def __init__(self, iters, rel, status=0):
        self.iters_done, self.rel_res, self.status = iters, rel, status


def _advance(plan, iters, tol):
    """A job's residual halves every iteration from 1.0; a plan marked bad
    reports a non-finite residual."""
    done = getattr(plan, "progress", 0)
    if getattr(plan, "bad", False):
        return FakeInfo(1, float("nan"), 5)
    k = 0
    rel = 0.5 ** done
    while k < iters:
        k += 1
        rel = 0.5 ** (done + k)
        if tol > 0 and rel <= tol:
            break
    plan.progress = done + k
    return FakeInfo(k, rel)


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

    solo_calls = 0

    def solve(self, y, I0, eta, iters, x=None, lo=0.0, hi=math.inf, tol=0.0, check_every=1, sync=True):
        import time
        FakePlan.solo_calls += 1
        time.sleep(0.002)
        return x, _advance(self, iters, tol)

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
        infos = [_advance(jb.plan, jb.iters, jb.tol) for jb in jobs]
        return [jb.x for jb in jobs], infos

    def close(self):
        pass


@pytest.fixture(autouse=True)
def fakes(monkeypatch):
    monkeypatch.setattr(serve, "Plan", FakePlan)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    FakePlan.live = 0
    FakePlan.solo_calls = 0
    yield


def _req(n, tol=1e-3, max_iters=100, tag=None, arrival=0.0):
    from paper_2503_19925_gb300.exact import Geometry
    g = Geometry(beam=0, nx=n, ny=n, n_views=10, n_bins=n)
    return serve.Request(g, [1.0], [[1.0]], torch.zeros(1, 10, n), 1e3, tol=tol, max_iters=max_iters,
                         arrival=arrival, tag=tag)


def test_all_requests_finish_and_memory_is_released():
    reqs = [_req(32 + 8 * k, tag=k) for k in range(10)]
    s = serve.Server(mode="rounds", budget_bytes=1e12, max_slots=4, round_iters=3)
    res = s.run(reqs, realtime=False)
    assert sorted(r.tag for r in res) == list(range(10))
    assert all(r.iters == 10 and r.rel_res <= 1e-3 for r in res)  # 0.5^10 < 1e-3
    assert FakePlan.live == 0 and s.used == 0
    assert max(s.batch.calls) <= 4  # never more than max_slots resident


def test_budget_admits_one_at_a_time():
    reqs = [_req(64, tag=k) for k in range(3)]
    one = serve.footprint_bytes(reqs[0].geometry, 1, 4)
    s = serve.Server(mode="rounds", budget_bytes=one * 1.5, max_slots=8, round_iters=4)
    res = s.run(reqs, realtime=False)
    assert len(res) == 3 and s.batch.calls == []  # one job resident at a time: plain solves
    assert FakePlan.solo_calls == s.rounds
    assert s.peak_used <= one * 1.5


def test_iteration_cap_and_failure():
    reqs = [_req(32, tol=0.0, max_iters=7, tag="cap"), _req(32, tag="bad")]
    s = serve.Server(mode="rounds", budget_bytes=1e12, max_slots=4, round_iters=3)
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
    s = serve.Server(mode="rounds", budget_bytes=1e12, max_slots=4, round_iters=2)
    res = {r.tag: r for r in s.run(reqs, realtime=True)}
    assert set(res) == {"early", "late0", "late1"}
    assert max(s.batch.calls) == 3  # the late requests ran alongside the early one


def test_saturating_jobs_run_one_after_another():
    """Jobs whose work alone reaches the admission limit are not interleaved:
    each runs its rounds alone, through the plain solve, in arrival order."""
    reqs = [_req(16, tol=1e-3, tag=k) for k in range(3)]
    work = serve.work_per_iter(reqs[0].geometry)
    srv = serve.Server(mode="rounds", budget_bytes=1e12, max_slots=8, round_iters=4, sat_work=work)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert sorted(r.tag for r in res) == [0, 1, 2]
    assert srv.batch.calls == []  # never more than one job resident
    assert FakePlan.solo_calls == srv.rounds
    assert [r.tag for r in sorted(res, key=lambda r: r.finished)] == [0, 1, 2]
    assert all(r.admitted >= prev.finished for prev, r in zip(sorted(res, key=lambda r: r.finished),
                                                               sorted(res, key=lambda r: r.finished)[1:]))


def test_small_jobs_share_rounds_below_the_limit():
    reqs = [_req(16, tol=1e-3, tag=k) for k in range(3)]
    work = serve.work_per_iter(reqs[0].geometry)
    srv = serve.Server(mode="rounds", budget_bytes=1e12, max_slots=8, round_iters=4, sat_work=3 * work)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert sorted(r.tag for r in res) == [0, 1, 2]
    assert max(srv.batch.calls) == 3  # all three in one persistent launch



def test_preparation_overlaps_running_rounds(monkeypatch):
    """A request whose preparation (plan build, uploads, step size) is slow is
    prepared on the worker thread while the resident job keeps running
    rounds; it joins once ready."""
    import threading
    import time
    marks = {}

    class SlowPlan(FakePlan):
        def __init__(self, geometry, mu, S):
            if geometry.nx == 48:
                marks["prep_start"] = time.perf_counter()
                marks["prep_thread"] = threading.current_thread() is not threading.main_thread()
                time.sleep(0.15)
                marks["prep_end"] = time.perf_counter()
            super().__init__(geometry, mu, S)

    calls = []

    def solo(self, y, I0, eta, iters, x=None, lo=0.0, hi=math.inf, tol=0.0, check_every=1, sync=True):
        calls.append(time.perf_counter())
        time.sleep(0.002)
        return x, _advance(self, iters, tol)

    monkeypatch.setattr(SlowPlan, "solve", solo)
    monkeypatch.setattr(serve, "Plan", SlowPlan)
    reqs = [_req(32, tol=0.0, max_iters=200, tag="running"), _req(48, tag="slow", arrival=0.01)]
    s = serve.Server(mode="rounds", budget_bytes=1e12, max_slots=4, round_iters=1)
    res = {r.tag: r for r in s.run(reqs, realtime=True)}
    s.close()
    assert set(res) == {"running", "slow"} and FakePlan.live == 0
    assert marks["prep_thread"]
    during = [t for t in calls if marks["prep_start"] < t < marks["prep_end"]]
    assert len(during) >= 5  # rounds went on while the slow request was prepared


# ---- streams mode: each resident job's whole solve on its own stream ----

def test_streams_mode_all_finish_within_slots_and_budget():
    reqs = [_req(32 + 8 * k, tag=k) for k in range(10)]
    s = serve.Server(budget_bytes=1e12, max_slots=4)
    res = s.run(reqs, realtime=False)
    s.close()
    assert sorted(r.tag for r in res) == list(range(10))
    assert all(r.iters == 10 and r.rel_res <= 1e-3 for r in res)
    assert FakePlan.live == 0 and s.used == 0
    assert 1 < s.peak_resident <= 4 and s.launches == 10


def test_streams_mode_cap_failure_and_saturation():
    reqs = [_req(32, tol=0.0, max_iters=7, tag="cap"), _req(32, tag="bad")]

    class BadPlan(FakePlan):
        def __init__(self, geometry, mu, S):
            super().__init__(geometry, mu, S)
            self.bad = geometry.n_views == 11

    import paper_2503_19925_gb300.exact as exm
    reqs[1] = serve.Request(exm.Geometry(beam=0, nx=32, ny=32, n_views=11, n_bins=32), [1.0], [[1.0]],
                            torch.zeros(1, 11, 32), 1e3, tag="bad")
    serve.Plan = BadPlan
    s = serve.Server(budget_bytes=1e12, max_slots=4)
    res = {r.tag: r for r in s.run(reqs, realtime=False)}
    s.close()
    assert res["cap"].iters == 7 and res["cap"].status == 0
    assert res["bad"].status == 5
    # jobs that each fill the GPU run one after another
    reqs = [_req(16, tol=1e-3, tag=k) for k in range(3)]
    s = serve.Server(budget_bytes=1e12, max_slots=8, sat_work=serve.work_per_iter(reqs[0].geometry))
    res = s.run(reqs, realtime=False)
    s.close()
    assert s.peak_resident == 1 and len(res) == 3
