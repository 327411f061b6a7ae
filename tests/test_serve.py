"""The serving loop's scheduling (admission by footprint, continuous
batching, chunking, cancellation, failures, latency accounting) on a fake
engine with a simulated clock: no GPU needed."""
import numpy as np
import pytest

from paper_2207_01173_gb300 import workloads
from paper_2207_01173_gb300.serve import EngineError, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, s):
        self.t += max(0.0, s)


class FakeEngine:
    """Each step of a batch costs 1 us per cell of all its problems."""

    def __init__(self, clock):
        self.clock = clock
        self.live = {}
        self.steps_log = []
        self.released = []

    def footprint(self, req):
        return int(np.prod(req["n"])) * 100

    def create(self, req):
        if req.get("fail_create"):
            raise EngineError("injected create failure")
        h = dict(id=req["id"], cells=int(np.prod(req["n"])), step=0, bad_at=req.get("bad_at"),
                 poison=req.get("poison", False))
        self.live[req["id"]] = h
        return req["id"]

    def step(self, handles, nsteps):
        if any(self.live[h].get("poison") for h in handles):
            raise EngineError("injected batch failure")
        self.steps_log.append((tuple(handles), nsteps))
        self.clock.t += nsteps * sum(self.live[h]["cells"] for h in handles) * 1e-6
        out = []
        for h in handles:
            p = self.live[h]
            for _ in range(nsteps):
                if p["bad_at"] is not None and p["step"] == p["bad_at"]:
                    break
                p["step"] += 1
            out.append(p["step"])
        return out

    def result(self, h, keep_state=False):
        return {"step": self.live[h]["step"]}, None

    def release(self, h):
        self.released.append(h)
        del self.live[h]


def req(i, t, n, steps, **kw):
    return dict(id=i, t=t, kind="tgv", n=(n, n, n), steps=steps, Ma=0.1, Re=1600.0, **kw)


def serve(reqs, budget=10 ** 9, max_chunk=8):
    clk = FakeClock()
    eng = FakeEngine(clk)
    srv = Server(eng, budget, max_chunk=max_chunk, clock=clk, sleep=clk.sleep)
    res, summ = srv.run(reqs)
    return res, summ, eng


def test_all_complete_with_continuous_batching():
    reqs = [req(0, 0.0, 40, 50), req(1, 0.5, 20, 10), req(2, 0.6, 30, 30), req(3, 100.0, 20, 5)]
    res, summ, eng = serve(reqs)
    assert summ["done"] == 4 and summ["requests"] == 4
    for r in reqs:
        out = res[r["id"]]
        assert out["status"] == "done" and out["stats"]["step"] == r["steps"] == out["steps_done"]
        assert out["latency"] == pytest.approx(out["t_done"] - r["t"])
        assert out["t_admit"] >= r["t"]
    # request 1 arrived while request 0 ran and joined it (no drain first)
    assert any(set(h) == {0, 1, 2} for h, _ in eng.steps_log)
    # chunks stay within max_chunk and never overshoot a completion
    assert max(n for _, n in eng.steps_log) <= 8
    assert sorted(eng.released) == [0, 1, 2, 3]
    assert summ["mean_concurrency"] > 1.0
    assert summ["cell_updates"] == sum(workloads.request_work(r) for r in reqs)


def test_admission_respects_the_footprint_budget_fifo():
    # budget for two 20^3 problems at a time (800 kB each)
    reqs = [req(i, 0.01 * i, 20, 12) for i in range(6)]
    res, summ, eng = serve(reqs, budget=2 * 20 ** 3 * 100)
    assert summ["done"] == 6
    assert summ["peak_bytes"] <= 2 * 20 ** 3 * 100
    assert all(len(h) <= 2 for h, _ in eng.steps_log)
    admits = [res[i]["t_admit"] for i in range(6)]
    assert admits == sorted(admits)  # first come, first served


def test_oversize_request_is_rejected_not_stuck():
    reqs = [req(0, 0.0, 20, 5), req(1, 0.0, 60, 5), req(2, 0.1, 20, 5)]
    res, summ, _ = serve(reqs, budget=30 ** 3 * 100)
    assert res[1]["status"] == "rejected" and "budget" in res[1]["error"]
    assert res[0]["status"] == res[2]["status"] == "done"


def test_create_failure_and_bad_state_stop_only_that_request():
    reqs = [req(0, 0.0, 20, 30), req(1, 0.0, 20, 30, fail_create=True), req(2, 0.0, 20, 30, bad_at=11),
            req(3, 0.2, 20, 30)]
    res, summ, eng = serve(reqs)
    assert res[1]["status"] == "failed" and "injected" in res[1]["error"]
    assert res[2]["status"] == "failed" and res[2]["steps_done"] == 11
    assert res[0]["status"] == res[3]["status"] == "done"
    assert 2 in eng.released and 1 not in eng.released
    assert summ["failed"] == 2 and summ["done"] == 2


def test_cancel_waiting_and_running():
    reqs = [req(0, 0.0, 40, 200, cancel_after=0.1), req(1, 0.0, 40, 20), req(2, 0.0, 40, 20, cancel_after=0.0)]
    res, summ, eng = serve(reqs, budget=2 * 40 ** 3 * 100)
    assert res[0]["status"] == "cancelled" and 0 < res[0]["steps_done"] < 200
    assert res[2]["status"] == "cancelled" and "t_admit" not in res[2]
    assert res[1]["status"] == "done"
    assert summ["cancelled"] == 2 and not eng.live


def test_serve_stream_is_seeded_and_mixed():
    a, b = workloads.serve_requests(), workloads.serve_requests()
    assert a == b and len(a) == 500
    tgv = [r for r in a if r["kind"] == "tgv"]
    assert 0.5 < len(tgv) / 500 < 0.7
    assert {r["n"][0] for r in tgv} <= {32, 48, 64, 96, 128, 160, 192}
    assert {r["n"][0] for r in a if r["kind"] == "channel"} <= {64, 96, 128}
    assert min(r["steps"] for r in a) >= 20 and max(r["steps"] for r in a) <= 200
    gaps = np.diff([0.0] + [r["arrival"] for r in a])
    assert (gaps > 0).all() and 0.85 < gaps.mean() < 1.15  # unit-rate Poisson arrivals


def test_srpt_lets_small_requests_pass_large_ones():
    # a large request runs; a small one arrives; under "srpt" with a fill
    # target below the large request's size, the small one runs alone first
    reqs = [req(0, 0.0, 60, 100), req(1, 1.0, 10, 10)]
    out = {}
    for policy in ("fair", "srpt"):
        clk = FakeClock()
        eng = FakeEngine(clk)
        srv = Server(eng, 10 ** 9, max_chunk=8, clock=clk, sleep=clk.sleep, policy=policy, fill_cells=1)
        res, summ = srv.run(reqs)
        assert summ["done"] == 2 and res[0]["steps_done"] == 100 and res[1]["steps_done"] == 10
        out[policy] = (res, eng)
    fair, srpt = out["fair"][0], out["srpt"][0]
    assert srpt[1]["latency"] < fair[1]["latency"]
    assert srpt[1]["t_done"] < srpt[0]["t_done"]
    # while the small request ran, the large one waited (working set of one)
    assert any(h == (1,) for h, _ in out["srpt"][1].steps_log)
    with pytest.raises(ValueError):
        Server(FakeEngine(FakeClock()), 1, policy="lifo")


def test_srpt_aging_lets_a_long_waiting_request_in():
    # a medium request waits behind a sustained stream of small ones (each
    # arrives a little before the previous one is done); with pure SRPT it
    # runs only after the stream, with aging it gets in once the ratio of its
    # age to theirs outweighs its 4.7x larger remaining work
    reqs = [req(0, 0.0, 12, 20), req(1, 0.001, 16, 40)] + [req(i, 0.03 * (i - 1), 12, 20) for i in range(2, 70)]
    done = {}
    for age in (0.0, 0.05):
        clk = FakeClock()
        srv = Server(FakeEngine(clk), 10 ** 9, max_chunk=4, clock=clk, sleep=clk.sleep, policy="srpt",
                     fill_cells=1, age_s=age)
        res, summ = srv.run(reqs)
        assert summ["done"] == 70
        last_small = max(r["t_done"] for i, r in res.items() if i != 1)
        done[age] = (res[1]["t_done"], last_small)
    assert done[0.0][0] > done[0.0][1]    # pure SRPT: after the whole stream
    assert done[0.05][0] < done[0.05][1]  # aging: before the stream ends


def test_failed_batch_step_fails_its_working_set_only():
    # request 1 makes every batch it is in fail; under "srpt" with a small
    # fill target the other requests run in working sets of their own
    reqs = [req(0, 0.0, 10, 6), req(1, 0.0, 20, 6, poison=True), req(2, 0.5, 10, 6)]
    clk = FakeClock()
    eng = FakeEngine(clk)
    srv = Server(eng, 10 ** 9, max_chunk=8, clock=clk, sleep=clk.sleep, policy="srpt", fill_cells=1)
    res, summ = srv.run(reqs)
    assert res[1]["status"] == "failed" and "injected batch failure" in res[1]["error"]
    assert res[0]["status"] == res[2]["status"] == "done"
    assert 1 in eng.released and not eng.live
