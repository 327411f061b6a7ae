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
        h = dict(id=req["id"], cells=int(np.prod(req["n"])), step=0, bad_at=req.get("bad_at"))
        self.live[req["id"]] = h
        return req["id"]

    def step(self, handles, nsteps):
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
