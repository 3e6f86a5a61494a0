"""Continuous-batching server of GP solves over a ``Pool`` (include/gp.h, pools).

Requests (ground-state solves in imaginary time, quench dynamics in real time) are
admitted into the pool's device arena as they arrive and as room frees up: in arrival
order, except that while the oldest waiting request does not fit, later ones that do
fit are admitted past it (backfill) until the oldest has waited max_head_wait_s, after
which admission waits for it.  Every live solve stays resident on the device and all
of them advance together in quanta of steps (one batched launch per sweep direction
and mode per step); a solve that has done its steps retires between quanta, its
observables are read, and its arena range goes to the next waiting request.  A
request can be cancelled (Server.cancel, or its own cancel_at time) or time out (its
timeout_s): it then leaves the queue, or the pool between quanta, without a result.
A solve's arithmetic does not depend on which other solves share the pool, so its
result is the same alone and in the mix.

The GPU work is the library's; this module only schedules.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from typing import Callable, Optional

from .gp import GP_ERR_NOMEM, GPError, Pool


class Server:
    """One pool and an admission queue.

    arena_bytes: the pool's arena (default: half of the device's free memory at
    construction, as reported by cudaMemGetInfo through PyTorch); quantum: steps per
    pool call (a quantum is cut short so that no solve overshoots its step count);
    backfill: admit later requests that fit past an oldest one that does not, for at
    most max_head_wait_s of the oldest one's wait (backfill=False: strict FIFO).
    Requests may carry timeout_s (latency after which an unfinished request is
    dropped) and cancel_at (a time, from the start, at which the client cancels it).
    """

    def __init__(self, arena_bytes: Optional[int] = None, max_slots: int = 1024,
                 quantum: int = 100, tune: bool = False, backfill: bool = True,
                 max_head_wait_s: float = 1.0, graph: Optional[bool] = None):
        if arena_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            arena_bytes = int(free * 0.5)
        self.pool = Pool(arena_bytes, max_slots)
        if graph is not None:
            self.pool.set_graph(graph)
        self.quantum = int(quantum)
        self.tune = tune
        self.backfill = bool(backfill)
        self.max_head_wait_s = float(max_head_wait_s)
        self.stats = {"quanta": 0, "steps": 0, "admitted": 0, "max_live": 0, "backfilled": 0,
                      "cancelled": 0, "timed_out": 0,
                      "step_s": 0.0, "admit_s": 0.0, "retire_s": 0.0, "live_sum": 0}
        self.cancelled = []               # records of requests dropped without a result
        self._cancel_ids = set()
        self._cancel_lock = threading.Lock()

    def cancel(self, request_id) -> None:
        """Ask for request `request_id` to be dropped: it leaves the queue, or the pool
        at the next quantum boundary (its slot is freed), without a result.  May be
        called from another thread or from an on_done callback."""
        with self._cancel_lock:
            self._cancel_ids.add(request_id)

    def close(self):
        self.pool.close()

    def _admit(self, req, now):
        slot = self.pool.add(**req["params"])
        if req["kind"] == "quench":
            self.pool.set_real_time(slot)
        return dict(req, slot=slot, remaining=int(req["steps"]), admitted=now)

    def run(self, requests, realtime: bool = True, virtual_step_s: float = 1e-4,
            on_done: Optional[Callable] = None):
        """Serve `requests` (dicts with id, arrival [s from start], kind 'ground' or
        'quench', steps, params) and return one record per request: arrival, admitted
        and finished times [s], latency = finished - arrival, and the observables.

        realtime: arrivals follow the wall clock.  Otherwise time is virtual: a quantum
        of q steps takes q * virtual_step_s and an idle server jumps to the next arrival,
        which makes the admission order reproducible (tests)."""
        pending = deque(sorted(requests, key=lambda r: r["arrival"]))
        waiting: deque = deque()
        live = {}
        done = []
        t0 = time.perf_counter()
        vnow = 0.0

        def now():
            return time.perf_counter() - t0 if realtime else vnow

        tuned = not self.tune

        def drop(r, t, why, slot=None):
            if slot is not None:
                self.pool.remove(slot)
            self.cancelled.append({"id": r["id"], "kind": r["kind"], "status": why,
                                   "arrival": r["arrival"], "dropped": t,
                                   "steps_done": r["steps"] - r.get("remaining", r["steps"])})
            self.stats["cancelled" if why == "cancelled" else "timed_out"] += 1

        def reason(r, t):
            with self._cancel_lock:
                if r["id"] in self._cancel_ids:
                    return "cancelled"
            if r.get("cancel_at") is not None and t >= r["cancel_at"]:
                return "cancelled"
            if r.get("timeout_s") is not None and t - r["arrival"] > r["timeout_s"]:
                return "timeout"
            return None

        while pending or waiting or live:
            t = now()
            while pending and pending[0]["arrival"] <= t:
                waiting.append(pending.popleft())
            # cancellations and timeouts, between quanta
            for r in [r for r in waiting if reason(r, t)]:
                waiting.remove(r)
                drop(r, t, reason(r, t))
            for slot in [s for s, r in live.items() if reason(r, t)]:
                r = live.pop(slot)
                drop(r, t, reason(r, t), slot)
            ta = time.perf_counter()
            i = 0
            while i < len(waiting):
                r = waiting[i]
                try:
                    rec = self._admit(r, t)
                except GPError as e:
                    if e.code != GP_ERR_NOMEM:
                        raise
                    # no room for r: later requests may fit past it while the oldest
                    # waiting request has not waited too long
                    head_wait = t - waiting[0]["arrival"]
                    if not self.backfill or head_wait > self.max_head_wait_s:
                        break
                    i += 1
                    continue
                del waiting[i]
                live[rec["slot"]] = rec
                self.stats["admitted"] += 1
                if i > 0:
                    self.stats["backfilled"] += 1
            self.stats["admit_s"] += time.perf_counter() - ta
            if not live:
                if pending or (waiting and any(r.get("timeout_s") is not None or
                                               r.get("cancel_at") is not None for r in waiting)):
                    # idle until the next arrival (or the next deadline of a waiting request)
                    nxt = pending[0]["arrival"] if pending else float("inf")
                    for r in waiting:
                        for d in (r.get("cancel_at"), None if r.get("timeout_s") is None
                                  else r["arrival"] + r["timeout_s"]):
                            if d is not None:
                                nxt = min(nxt, d + 1e-9)
                    if waiting and not pending and nxt == float("inf"):
                        raise RuntimeError("a request does not fit the empty pool")
                    if realtime:
                        time.sleep(max(0.0, nxt - now()))
                    else:
                        vnow = max(vnow, nxt)
                    continue
                if not waiting:
                    break
                raise RuntimeError("a request does not fit the empty pool")
            if not tuned:
                self.pool.tune(3)
                tuned = True
            self.stats["max_live"] = max(self.stats["max_live"], len(live))
            q = min(self.quantum, min(r["remaining"] for r in live.values()))
            ts = time.perf_counter()
            self.pool.step(q)
            self.stats["step_s"] += time.perf_counter() - ts
            self.stats["quanta"] += 1
            self.stats["steps"] += q
            self.stats["live_sum"] += len(live)
            if not realtime:
                vnow += q * virtual_step_s
            t = now()
            tr = time.perf_counter()
            for slot in [s for s, r in live.items() if r["remaining"] == q]:
                r = live.pop(slot)
                obs = self.pool.observables(slot)
                self.pool.remove(slot)
                out = {"id": r["id"], "kind": r["kind"], "steps": r["steps"],
                       "arrival": r["arrival"], "admitted": r["admitted"], "finished": t,
                       "latency": t - r["arrival"], "obs": obs}
                done.append(out)
                if on_done:
                    on_done(out)
            for r in live.values():
                r["remaining"] -= q
            self.stats["retire_s"] += time.perf_counter() - tr
        return done


def serve_one_at_a_time(requests, prec: str = "f64", realtime: bool = True):
    """The comparison server: one request at a time, FIFO, each a single solver of the
    library (gp_create, gp_init_gaussian, gp_step_imag / gp_step_real) in `prec`.
    Returns records like Server.run."""
    from .gp import Solver
    done = []
    t0 = time.perf_counter()
    vnow = 0.0
    for r in sorted(requests, key=lambda r: r["arrival"]):
        if realtime:
            wait = r["arrival"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        p = r["params"]
        s = Solver(p["nx"], p["ny"], p["nz"], p["dx"], dt=p["dt"], gamma=p["gamma"], nu=p["nu"],
                   lam=p["lam"], g=p["g"], prec=prec)
        start = time.perf_counter() - t0
        s.init_gaussian()
        if r["kind"] == "quench":
            s.step_real(r["steps"])
        else:
            s.step_imag(r["steps"])
        obs = s.observables()
        s.close()
        t = time.perf_counter() - t0
        done.append({"id": r["id"], "kind": r["kind"], "steps": r["steps"], "arrival": r["arrival"],
                     "admitted": start, "finished": t, "latency": t - r["arrival"], "obs": obs})
    return done
