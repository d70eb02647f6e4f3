"""Continuous batching of disk integrations on one GPU.

Requests (a disk of N moonlets, its expansion order p and a number of
steps) arrive over time.  The loop keeps every admitted disk resident in one
batch (ncorp_batch_*: disks of equal (p, theta, dt) side by side in one
forest, one launch per stage), and repeats ticks:

  1. admit, in arrival order, every request that has arrived and fits the
     batch's device-memory budget (the batch refuses a disk with
     NCORP_ENOMEM when it does not fit; the request then waits, and so do
     the ones behind it, until a disk leaves);
  2. advance all resident disks by k steps in one ncorp_batch_run, k = the
     tick length, shortened so that no disk runs past its request; if the
     run cannot lay out its disks in device memory (it then steps none of
     them), the requests admitted at this tick leave the batch again, newest
     first, until it fits, go back to the head of the queue, and admission
     pauses until a disk finishes;
  3. hand every finished disk's final state to the caller and remove it.

Requests that arrive while others are on the GPU join at the next tick, so
their work overlaps with the disks already running.  The batch is reached
through a small adapter (BatchBackend), so the loop itself can be tested
without a GPU against a fake batch with a simulated clock.

Reported latencies, all host wall times:
  * tick_ms: one ncorp_batch_run of k steps (every disk resident in it
    advances k steps);
  * step_ms: tick_ms / k, one sample per disk and step, i.e. the time a
    disk waits for each of its steps while it is resident;
  * request_s: from a request's arrival to its last step (admission wait
    included);
  * admission_wait_s: from arrival to admission.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


class BudgetFull(Exception):
    """The batch cannot take the disk now (device-memory budget)."""


@dataclasses.dataclass
class Request:
    arrival: float              # seconds after the start of the run
    n: int
    p: int
    steps: int
    disk: object = None         # whatever the backend's add() takes (the disk's arrays)
    # filled in by the loop
    admitted: float = None
    done: float = None
    steps_left: int = 0
    disk_id: int = None


class BatchBackend:
    """Adapter of the loop to ncorp_batch (the GPU batch): add / run / finish."""

    def __init__(self, ncorp, batch, theta, dt):
        self.ncorp, self.b, self.theta, self.dt = ncorp, batch, theta, dt

    def add(self, req: Request) -> int:
        d = req.disk
        try:
            return self.ncorp.ncorp_batch_add_disk(self.b, d["pos"], d["vel"], d["mass"], d["radius"], req.n, req.p,
                                                   self.theta, self.dt)
        except self.ncorp.NcorpError as e:
            if e.code == self.ncorp.NCORP_ENOMEM:
                raise BudgetFull(f"{e} (batch: {self.ncorp.ncorp_batch_info(self.b)})") from None
            raise

    def run(self, k: int) -> None:
        try:
            self.ncorp.ncorp_batch_run(self.b, k)
        except self.ncorp.NcorpError as e:
            if e.code == self.ncorp.NCORP_ENOMEM:   # no disk was stepped
                raise BudgetFull(str(e)) from None
            raise
        info = self.ncorp.ncorp_batch_info(self.b)
        self.peak_bytes = max(getattr(self, "peak_bytes", 0), info["bytes"])
        self.peak_moonlets = max(getattr(self, "peak_moonlets", 0), info["moonlets"])

    def evict(self, req: Request) -> None:
        """Removes a disk that has not been stepped (it goes back to the queue)."""
        self.ncorp.ncorp_batch_remove_disk(self.b, req.disk_id)

    def finish(self, req: Request, out=None) -> None:
        """Removes the disk; with out = (positions, velocities) its final state is copied there first."""
        if out is None:
            self.ncorp.ncorp_batch_remove_disk(self.b, req.disk_id)
        else:
            self.ncorp.ncorp_batch_remove_disk(self.b, req.disk_id, out[0], out[1])


def serve(backend, requests, tick_steps=10, clock=time.perf_counter, sleep=time.sleep, on_done=None,
          max_wall=None, progress=None):
    """Runs the requests (sorted by arrival) to completion; returns the statistics (see the module doc).

    on_done(req) -> None or (positions, velocities) arrays for the finished disk's final state.
    max_wall (seconds): stop admitting new requests after this time (the admitted ones finish).
    progress(dict) is called before every run and after every tick with the loop's state (elapsed s, event,
    ticks, steps k, resident disks and moonlets, waiting and served counts), so that a log written from
    it shows where a run that was cut off from outside stood."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    waiting = collections.deque(reqs)
    active: dict[int, Request] = {}
    ticks = []            # (start, end, k, moonlets resident, disks resident)
    step_ms = []          # (value, weight): per disk-step
    concurrent = []
    start = clock()
    hold = False          # admission paused after a run did not fit, until a disk finishes
    solo = False          # a run did not fit with only fresh disks: admit one at a time
    while waiting or active:
        now = clock() - start
        # 1. admission, in arrival order
        while not hold and waiting and waiting[0].arrival <= now and (max_wall is None or now <= max_wall):
            if solo and active:
                break
            r = waiting[0]
            try:
                r.disk_id = backend.add(r)
            except BudgetFull as e:
                if not active:
                    raise RuntimeError(f"a disk of {r.n} moonlets does not fit the batch's budget on its own: {e}")
                break
            waiting.popleft()
            r.admitted = clock() - start
            r.steps_left = r.steps
            active[r.disk_id] = r
        if max_wall is not None and now > max_wall:
            waiting.clear()
        if not active:
            if waiting:
                sleep(max(0.0, min(waiting[0].arrival - now, 0.01)))
            continue
        # 2. one tick
        k = min(tick_steps, min(r.steps_left for r in active.values()))
        t0 = clock()
        while True:
            if progress:
                progress(_state("run", t0 - start, ticks, k, active, waiting, reqs))
            try:
                backend.run(k)
                break
            except BudgetFull:
                fresh = [r for r in active.values() if r.steps_left == r.steps]   # admitted at this tick
                if not fresh:
                    raise
                if solo and len(active) == 1:
                    raise RuntimeError(f"a disk of {fresh[0].n} moonlets does not fit the device on its own")
                r = max(fresh, key=lambda q: (q.admitted, q.arrival))
                backend.evict(r)
                del active[r.disk_id]
                r.disk_id, r.admitted = None, None
                # back to the head of the queue, ahead of the later arrivals
                waiting.appendleft(r)
                hold = True
                if not active:   # nothing left to run: admit the evicted ones again, one at a time
                    hold, solo = False, True
                    break
        if not active:
            continue
        solo = False
        t1 = clock()
        moonlets = sum(r.n for r in active.values())
        ticks.append((t0 - start, t1 - start, k, moonlets, len(active)))
        step_ms.append((1e3 * (t1 - t0) / k, k * len(active)))
        concurrent.append(len(active))
        # 3. finished disks leave
        for did, r in list(active.items()):
            r.steps_left -= k
            if r.steps_left == 0:
                r.done = t1 - start
                out = on_done(r) if on_done else None
                backend.finish(r, out)
                del active[did]
                hold = False
        if progress:
            progress(_state("tick", t1 - start, ticks, k, active, waiting, reqs))
    wall = clock() - start
    return summarize(reqs, ticks, step_ms, concurrent, wall)


def _state(event, t, ticks, k, active, waiting, reqs):
    return {"t": round(t, 3), "event": event, "ticks": len(ticks), "k": k, "disks": len(active),
            "moonlets": sum(r.n for r in active.values()), "waiting": len(waiting),
            "served": sum(1 for r in reqs if r.done is not None)}


def _pct(values, q, weights=None):
    if len(values) == 0:
        return None
    v = np.asarray(values, dtype=float)
    if weights is None:
        return float(np.percentile(v, q))
    w = np.asarray(weights, dtype=float)
    order = np.argsort(v)
    cw = np.cumsum(w[order])
    i = int(np.searchsorted(cw, q / 100.0 * cw[-1], side="left"))
    return float(v[order][min(i, len(v) - 1)])


def summarize(reqs, ticks, step_ms, concurrent, wall):
    served = [r for r in reqs if r.done is not None]
    work = sum(r.n * r.steps for r in served)
    tick_ms = [1e3 * (t1 - t0) for t0, t1, _, _, _ in ticks]
    sv = [v for v, _ in step_ms]
    sw = [w for _, w in step_ms]
    busy = sum(t1 - t0 for t0, t1, _, _, _ in ticks)
    return {
        "requests": len(reqs), "served": len(served), "moonlet_steps": work, "wall_s": wall,
        "throughput": work / wall if wall > 0 else 0.0,
        "busy_throughput": work / busy if busy > 0 else 0.0,
        "ticks": len(ticks),
        "batch_steps": sum(k for _, _, k, _, _ in ticks),
        "tick_ms_p50": _pct(tick_ms, 50), "tick_ms_p99": _pct(tick_ms, 99),
        "step_ms_p50": _pct(sv, 50, sw), "step_ms_p99": _pct(sv, 99, sw),
        "request_s_p50": _pct([r.done - r.arrival for r in served], 50),
        "request_s_p99": _pct([r.done - r.arrival for r in served], 99),
        "admission_wait_s_p50": _pct([r.admitted - r.arrival for r in served], 50),
        "admission_wait_s_p99": _pct([r.admitted - r.arrival for r in served], 99),
        "concurrent_disks_mean": float(np.mean(concurrent)) if concurrent else 0.0,
        "concurrent_disks_max": int(max(concurrent)) if concurrent else 0,
    }


def poisson_requests(rate, seconds, n_lo, n_hi, ps, steps, seed):
    """Poisson arrivals at `rate` per second over `seconds`, N log-uniform in [n_lo, n_hi], p uniform in ps."""
    rng = np.random.default_rng(seed)
    t, out = rng.exponential(1.0 / rate), []
    while t < seconds:
        out.append(t)
        t += rng.exponential(1.0 / rate)
    u = rng.random(len(out))
    sizes = np.exp(np.log(n_lo) + u * (np.log(n_hi) - np.log(n_lo))).astype(np.int64)
    pp = rng.choice(list(ps), size=len(out))
    return [Request(arrival=a, n=int(n), p=int(p), steps=steps) for a, n, p in zip(out, sizes, pp)]
