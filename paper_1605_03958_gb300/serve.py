"""Continuous-batching server of GP solves over a ``Pool`` (include/gp.h, pools).

Requests (ground-state solves in imaginary time, quench dynamics in real time) are
admitted into the pool's device arena as they arrive and as room frees up, FIFO;
every live solve stays resident on the device and all of them advance together in
quanta of steps (one batched launch per sweep direction and mode per step); a solve
that has done its steps retires between quanta, its observables are read, and its
arena range goes to the next waiting request.  A solve's arithmetic does not depend
on which other solves share the pool, so its result is the same alone and in the mix.

The GPU work is the library's; this module only schedules.
"""
from __future__ import annotations

import time
from collections import deque
from typing import Callable, Optional

from .gp import GP_ERR_NOMEM, GPError, Pool


class Server:
    """One pool and a FIFO admission queue.

    arena_bytes: the pool's arena (default: half of the device's free memory at
    construction, as reported by cudaMemGetInfo through PyTorch); quantum: steps per
    pool call (a quantum is cut short so that no solve overshoots its step count).
    """

    def __init__(self, arena_bytes: Optional[int] = None, max_slots: int = 1024,
                 quantum: int = 100, tune: bool = False):
        if arena_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            arena_bytes = int(free * 0.5)
        self.pool = Pool(arena_bytes, max_slots)
        self.quantum = int(quantum)
        self.tune = tune
        self.stats = {"quanta": 0, "steps": 0, "admitted": 0, "max_live": 0,
                      "step_s": 0.0, "admit_s": 0.0, "retire_s": 0.0, "live_sum": 0}

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
        while pending or waiting or live:
            t = now()
            while pending and pending[0]["arrival"] <= t:
                waiting.append(pending.popleft())
            ta = time.perf_counter()
            while waiting:
                try:
                    rec = self._admit(waiting[0], t)
                except GPError as e:
                    if e.code == GP_ERR_NOMEM:
                        break   # no room until a solve retires
                    raise
                waiting.popleft()
                live[rec["slot"]] = rec
                self.stats["admitted"] += 1
            self.stats["admit_s"] += time.perf_counter() - ta
            if not live:
                if pending:   # idle until the next arrival
                    nxt = pending[0]["arrival"]
                    if realtime:
                        time.sleep(max(0.0, nxt - now()))
                    else:
                        vnow = max(vnow, nxt)
                    continue
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
