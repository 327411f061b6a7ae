"""Serving loop: continuous batching of HGKS solve requests on one GPU.

Requests arrive over time.  A request is admitted when its device footprint
(hgks_footprint_bytes of its grid and precision) fits in what the memory
budget has left; admission is first come, first served, so a large request
at the head of the queue is not starved by smaller ones behind it.  Every
admitted request gets its own solver with its state resident on the device,
and all running requests advance together as one batch (one persistent
kernel per pass over all of them, one CUDA graph per step).  The batch runs
in chunks of at most `max_chunk` steps, never past the nearest completion, so
that after every chunk finished requests leave (their statistics are read
back and their memory freed), waiting requests that now fit join, and the
batch is rebuilt for the new membership.  Because a batch reproduces its
problems stepped one by one bit for bit, each result is the same alone and
in the mix.

The scheduling here is host logic over an engine: `CudaEngine` runs the
solves through the C-ABI library; tests may plug in any object with the same
methods.
"""
import collections
import time

import numpy as np

from . import hgks, workloads


class EngineError(RuntimeError):
    pass


class CudaEngine:
    """Solves through the CUDA library: one Solver per request, one Batch
    over the running set (rebuilt when the set changes)."""

    def __init__(self, precision=hgks.MIXED, cfl=0.5):
        self.precision = precision
        self.cfl = cfl
        self.batch = None
        self.members = ()
        self.rebuilds = 0
        # host seconds spent rebuilding batches: creating them (work-lists on
        # the device) and, in the first step after each rebuild, capturing and
        # instantiating the step graph (that call's wall time minus its
        # device time)
        self.rebuild_create_s = 0.0
        self.rebuild_capture_s = 0.0

    def footprint(self, req):
        return hgks.footprint_bytes(req["n"], self.precision)

    def create(self, req):
        try:
            if req["kind"] == "tgv":
                s = hgks.Solver(req["n"], precision=self.precision,
                                **workloads.tgv_solver_kwargs(req["Ma"], req["Re"]))
                s.init_tgv(req["Ma"], 1.0, 1.0)
            elif req["kind"] == "channel":
                s = hgks.Solver(req["n"], precision=self.precision,
                                **workloads.channel_solver_kwargs(req["Ma"], req["Re"]))
                s.init_channel(req["Ma"], 0.1, req.get("seed", 2800))
            else:
                raise EngineError("unknown problem kind %r" % req["kind"])
        except hgks.HgksError as e:
            raise EngineError(str(e)) from e
        return s

    def _drop_batch(self):
        if self.batch is not None:
            self.batch.close()
        self.batch, self.members = None, ()

    def step(self, handles, nsteps):
        """Advance all handles nsteps; returns the step counters after."""
        try:
            rebuilt = tuple(handles) != self.members
            if rebuilt:
                self._drop_batch()
                t0 = time.perf_counter()
                self.batch = hgks.Batch(handles)
                self.rebuild_create_s += time.perf_counter() - t0
                self.members = tuple(handles)
                self.rebuilds += 1
            t1 = time.perf_counter()
            try:
                self.batch.step(nsteps, self.cfl)
            except hgks.HgksError as e:
                if e.status != hgks.HGKS_ERR_NONFINITE:
                    raise
            if rebuilt:
                wall = time.perf_counter() - t1
                self.rebuild_capture_s += max(0.0, wall - self.batch.info()["last_ms"] * 1e-3)
            return self.batch.steps()
        except hgks.HgksError as e:
            self._drop_batch()
            raise EngineError(str(e)) from e

    def result(self, h, keep_state=False):
        st = h.stats()
        return st, (h.get_state() if keep_state else None)

    def release(self, h):
        if h in self.members:
            self._drop_batch()
        h.close()

    def close(self):
        self._drop_batch()


class Server:
    """policy "fair": every running request advances in every chunk.
    policy "srpt": each chunk advances the running requests with the least
    remaining work (cells x steps left), smallest first, until they hold at
    least `fill_cells` cells; the others keep their memory and wait.  Small
    requests then finish without waiting behind large ones, and the batch
    still fills the GPU.  With age_s > 0 the remaining work of a request is
    discounted by (1 + age / age_s), age the time since its arrival, so a
    large request is not starved by a stream of small ones."""

    def __init__(self, engine, budget_bytes, max_chunk=8, keep_state=False, clock=time.perf_counter,
                 sleep=time.sleep, policy="fair", fill_cells=8 * 2 ** 20, age_s=0.0):
        if policy not in ("fair", "srpt"):
            raise ValueError("policy must be 'fair' or 'srpt'")
        self.engine = engine
        self.budget = int(budget_bytes)
        self.max_chunk = int(max_chunk)
        self.keep_state = keep_state
        self.clock = clock
        self.sleep = sleep
        self.policy = policy
        self.fill_cells = int(fill_cells)
        self.age_s = float(age_s)
        self._cancel = set()

    def cancel(self, rid):
        """Cancel a request (waiting or running) at the next chunk boundary."""
        self._cancel.add(rid)

    def run(self, requests):
        """Serve `requests` (dicts with id, t = arrival in seconds from the
        start, kind, n, steps, problem parameters; optional cancel_after in
        seconds after arrival).  Returns (results by id, summary)."""
        pending = collections.deque(sorted(requests, key=lambda r: r["t"]))
        waiting = collections.deque()
        running = {}  # id -> dict(req, h, bytes, done)
        results = {}
        used = peak = 0
        conc = []  # (chunk seconds, problems) for the mean concurrency
        chunks = 0
        t0 = self.clock()

        def rec(req, status, **kw):
            r = dict(id=req["id"], status=status, t_arrive=req["t"], steps=req["steps"], kind=req["kind"],
                     n=tuple(req["n"]), work=workloads.request_work(req))
            r.update(kw)
            results[req["id"]] = r

        def retire(rid, status, now, **kw):
            nonlocal used
            run = running.pop(rid)
            used -= run["bytes"]
            stats = state = None
            if status == "done":
                stats, state = self.engine.result(run["h"], self.keep_state)
            self.engine.release(run["h"])
            rec(run["req"], status, t_admit=run["t_admit"], t_done=now, latency=now - run["req"]["t"],
                steps_done=run["done"], stats=stats, state=state, **kw)

        while pending or waiting or running:
            now = self.clock() - t0
            while pending and pending[0]["t"] <= now:
                req = pending.popleft()
                fp = self.engine.footprint(req)
                if fp > self.budget:
                    rec(req, "rejected", error="footprint %d B exceeds the budget %d B" % (fp, self.budget))
                else:
                    req = dict(req, bytes=fp)
                    waiting.append(req)
            # cancellations
            for req in list(waiting):
                if req["id"] in self._cancel or ("cancel_after" in req and now >= req["t"] + req["cancel_after"]):
                    waiting.remove(req)
                    rec(req, "cancelled", t_done=now)
            for rid in list(running):
                req = running[rid]["req"]
                if rid in self._cancel or ("cancel_after" in req and now >= req["t"] + req["cancel_after"]):
                    retire(rid, "cancelled", now)
            # admission, first come first served
            while waiting and used + waiting[0]["bytes"] <= self.budget:
                req = waiting.popleft()
                try:
                    h = self.engine.create(req)
                except EngineError as e:
                    rec(req, "failed", error=str(e), t_done=now)
                    continue
                running[req["id"]] = dict(req=req, h=h, bytes=req["bytes"], done=0, t_admit=now)
                used += req["bytes"]
                peak = max(peak, used)
            if not running:
                if pending:
                    self.sleep(max(0.0, pending[0]["t"] - (self.clock() - t0)))
                continue
            ids = self._working_set(running, now)
            chunk = min(self.max_chunk, min(running[i]["req"]["steps"] - running[i]["done"] for i in ids))
            c0 = self.clock()
            try:
                counts = self.engine.step([running[i]["h"] for i in ids], chunk)
            except EngineError as e:
                # the batch step itself failed: its requests fail, the others go on
                now = self.clock() - t0
                for i in ids:
                    retire(i, "failed", now, error="batch step failed: %s" % e)
                continue
            conc.append((self.clock() - c0, len(ids)))
            chunks += 1
            now = self.clock() - t0
            for i, c in zip(ids, counts):
                run = running[i]
                if c < run["done"] + chunk:  # the problem stopped on a bad state
                    run["done"] = c
                    retire(i, "failed", now, error="non-finite or non-positive state after step %d" % c)
                    continue
                run["done"] = c
                if c >= run["req"]["steps"]:
                    retire(i, "done", now)
        return results, summarize(results, peak, self.budget, conc, chunks)

    def _working_set(self, running, now):
        if self.policy == "fair":
            return sorted(running)

        def left(i):
            r = running[i]
            work = int(np.prod(r["req"]["n"])) * (r["req"]["steps"] - r["done"])
            return work / (1.0 + max(0.0, now - r["req"]["t"]) / self.age_s) if self.age_s > 0 else work

        ids, cells = [], 0
        for i in sorted(running, key=lambda i: (left(i), i)):
            if ids and cells >= self.fill_cells:
                break
            ids.append(i)
            cells += int(np.prod(running[i]["req"]["n"]))
        return sorted(ids)


def summarize(results, peak_bytes, budget, conc, chunks):
    done = [r for r in results.values() if r["status"] == "done"]
    lat = np.array([r["latency"] for r in done]) if done else np.zeros(0)
    out = {s: sum(1 for r in results.values() if r["status"] == s)
           for s in ("done", "rejected", "failed", "cancelled")}
    out["requests"] = len(results)
    if done:
        t_first = min(r["t_arrive"] for r in done)
        t_last = max(r["t_done"] for r in done)
        work = sum(r["work"] for r in done)
        out.update(p50_ms=float(np.percentile(lat, 50)) * 1e3, p99_ms=float(np.percentile(lat, 99)) * 1e3,
                   mean_ms=float(lat.mean()) * 1e3, max_ms=float(lat.max()) * 1e3,
                   makespan_s=t_last - t_first, cell_updates=work,
                   cell_updates_per_s=work / max(t_last - t_first, 1e-12))
    busy = sum(dt for dt, _ in conc)
    out.update(peak_bytes=int(peak_bytes), budget_bytes=int(budget), chunks=chunks, busy_s=busy,
               mean_concurrency=(sum(dt * k for dt, k in conc) / busy) if busy > 0 else 0.0)
    return out
