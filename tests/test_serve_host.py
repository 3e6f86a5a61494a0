"""Host logic of the continuous-batching server (serve.Server) on the CPU, with the
pool replaced by a fake that keeps the pool's contract (slots, an arena that runs
out, steps applied to every live slot) and no GPU work.  Time is virtual, so the
admission order and every latency are reproducible."""
import pytest

from paper_1605_03958_gb300 import serve, workloads
from paper_1605_03958_gb300.gp import GP_ERR_NOMEM, GPError


class FakePool:
    """Slots of `bytes_of(params)` in an arena of `arena_bytes`; step(q) advances every
    live slot by q steps; observables report a slot's steps so far."""

    def __init__(self, arena_bytes, max_slots):
        self.arena, self.max_slots = int(arena_bytes), int(max_slots)
        self.live = {}            # slot -> dict(bytes, steps, real)
        self.next_id = 0
        self.calls = []

    @staticmethod
    def bytes_of(p):
        return p["nx"] * p["ny"] * p["nz"] * 4

    def used(self):
        return sum(s["bytes"] for s in self.live.values())

    def add(self, **p):
        b = self.bytes_of(p)
        if len(self.live) >= self.max_slots or self.used() + b > self.arena:
            raise GPError(GP_ERR_NOMEM, "arena full")
        sid = self.next_id
        self.next_id += 1
        self.live[sid] = dict(bytes=b, steps=0, real=False)
        self.calls.append(("add", sid))
        return sid

    def set_real_time(self, sid):
        self.live[sid]["real"] = True

    def tune(self, n):
        self.calls.append(("tune", n))
        return 1.0

    def step(self, q):
        assert q > 0
        for s in self.live.values():
            s["steps"] += q
        self.calls.append(("step", q, len(self.live)))

    def observables(self, sid):
        s = self.live[sid]
        return {"steps_done": s["steps"], "real": s["real"]}

    def remove(self, sid):
        del self.live[sid]
        self.calls.append(("remove", sid))

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(serve, "Pool", FakePool)


def req(i, arrival, steps, kind="ground", n=32):
    return dict(id=i, arrival=arrival, kind=kind, steps=steps,
                params=dict(nx=n, ny=n, nz=n, dx=0.2, dt=0.004, gamma=1.0, nu=1.0, lam=1.0, g=1.0))


def test_every_request_gets_exactly_its_steps_and_quanta_are_cut(fake):
    srv = serve.Server(arena_bytes=1 << 30, quantum=100)
    reqs = [req(0, 0.0, 250), req(1, 0.0, 120, "quench"), req(2, 0.0, 400)]
    done = srv.run(reqs, realtime=False, virtual_step_s=1e-3)
    by_id = {d["id"]: d for d in done}
    assert set(by_id) == {0, 1, 2}
    for r in reqs:
        assert by_id[r["id"]]["obs"]["steps_done"] == r["steps"]   # no overshoot
    assert by_id[1]["obs"]["real"] and not by_id[0]["obs"]["real"]
    steps = [c[1] for c in srv.pool.calls if c[0] == "step"]
    # quanta cut to the nearest completion: 100, 20 (120 done), 100, 30 (250 done), 100, 50
    assert steps == [100, 20, 100, 30, 100, 50]
    assert srv.stats["steps"] == 400 and srv.stats["admitted"] == 3
    # retirement order follows completion; latency = finish - arrival in virtual time
    assert [d["id"] for d in done] == [1, 0, 2]
    assert by_id[2]["latency"] == pytest.approx(0.4)


def test_fifo_admission_waits_for_room(fake):
    # the arena holds two 32^3 slots at a time
    srv = serve.Server(arena_bytes=2 * 32 ** 3 * 4, quantum=50)
    reqs = [req(i, 0.0, 100) for i in range(5)]
    done = srv.run(reqs, realtime=False, virtual_step_s=1e-3)
    assert srv.stats["max_live"] == 2
    adds = [c[1] for c in srv.pool.calls if c[0] == "add"]
    assert adds == sorted(adds)                          # FIFO
    admitted = sorted((d["admitted"], d["id"]) for d in done)
    assert [i for _, i in admitted] == [0, 1, 2, 3, 4]
    assert all(d["obs"]["steps_done"] == 100 for d in done)


def test_idle_server_jumps_to_the_next_arrival(fake):
    srv = serve.Server(arena_bytes=1 << 30, quantum=100)
    done = srv.run([req(0, 0.0, 100), req(1, 5.0, 100)], realtime=False, virtual_step_s=1e-3)
    by_id = {d["id"]: d for d in done}
    assert by_id[1]["admitted"] == pytest.approx(5.0)
    assert by_id[1]["latency"] == pytest.approx(0.1)


def test_request_larger_than_the_empty_pool_is_an_error(fake):
    srv = serve.Server(arena_bytes=1000, quantum=10)
    with pytest.raises(RuntimeError):
        srv.run([req(0, 0.0, 10)], realtime=False)


def test_synthetic_request_stream_matches_its_recipe():
    reqs = workloads.serve_requests(count=400)
    assert [r["id"] for r in reqs] == list(range(400))
    assert all(b["arrival"] > a["arrival"] for a, b in zip(reqs, reqs[1:]))
    ground = [r for r in reqs if r["kind"] == "ground"]
    quench = [r for r in reqs if r["kind"] == "quench"]
    assert 0.6 < len(ground) / len(reqs) < 0.8
    assert all(r["steps"] == 2000 for r in ground)
    assert all(500 <= r["steps"] <= 5000 for r in quench)
    for r in reqs:
        p = r["params"]
        assert p["nx"] % 16 == 0 and 32 <= p["nx"] <= 128
        assert p["ny"] % 16 == 0 and 32 <= p["ny"] <= 96
        assert p["nz"] % 16 == 0 and 32 <= p["nz"] <= 64
        assert 1.0 <= p["g"] <= 1000.0
    assert workloads.serve_requests(count=50) == workloads.serve_requests(count=50)   # seeded


def test_backfill_admits_smaller_requests_past_a_blocked_head(fake):
    # arena of one 48^3 slot: a 48^3 request waits behind a live 32^3 one, while a later
    # 32^3 request fits beside it and is admitted past the blocked one
    srv = serve.Server(arena_bytes=48 ** 3 * 4, quantum=50, max_head_wait_s=10.0)
    reqs = [req(0, 0.0, 200), req(1, 0.001, 100, n=48), req(2, 0.002, 100)]
    done = srv.run(reqs, realtime=False, virtual_step_s=1e-3)
    order = [i for _, i in sorted((d["admitted"], d["id"]) for d in done)]
    assert order == [0, 2, 1]
    assert srv.stats["backfilled"] == 1
    assert all(d["obs"]["steps_done"] == d["steps"] for d in done)


def test_head_wait_bound_stops_backfill(fake):
    # the same stream with no backfill allowed once the head has waited at all
    srv = serve.Server(arena_bytes=48 ** 3 * 4, quantum=50, max_head_wait_s=0.0)
    reqs = [req(0, 0.0, 200), req(1, 0.001, 100, n=48), req(2, 0.002, 100)]
    done = srv.run(reqs, realtime=False, virtual_step_s=1e-3)
    order = [i for _, i in sorted((d["admitted"], d["id"]) for d in done)]
    assert order == [0, 1, 2]
    assert srv.stats["backfilled"] == 0


def test_strict_fifo_when_backfill_is_off(fake):
    srv = serve.Server(arena_bytes=48 ** 3 * 4, quantum=50, backfill=False)
    reqs = [req(0, 0.0, 200), req(1, 0.001, 100, n=48), req(2, 0.002, 100)]
    done = srv.run(reqs, realtime=False, virtual_step_s=1e-3)
    assert [i for _, i in sorted((d["admitted"], d["id"]) for d in done)] == [0, 1, 2]


def test_cancelled_live_request_frees_its_slot(fake):
    # the arena holds one 32^3 slot: request 0 is cancelled while live (at t = 0.05 s of
    # virtual time, 50 of its 1000 steps done), its slot goes to request 1
    srv = serve.Server(arena_bytes=32 ** 3 * 4, quantum=50)
    r0 = dict(req(0, 0.0, 1000), cancel_at=0.05)
    done = srv.run([r0, req(1, 0.0, 100)], realtime=False, virtual_step_s=1e-3)
    assert [d["id"] for d in done] == [1]
    (c,) = srv.cancelled
    assert c["id"] == 0 and c["status"] == "cancelled" and c["steps_done"] == 50
    removes = [x for x in srv.pool.calls if x[0] == "remove"]
    assert removes[0] == ("remove", 0)            # freed before request 1 was admitted
    assert srv.pool.calls.index(removes[0]) < srv.pool.calls.index(("add", 1))
    assert srv.stats["cancelled"] == 1 and not srv.pool.live


def test_cancelled_waiting_request_is_never_admitted(fake):
    srv = serve.Server(arena_bytes=32 ** 3 * 4, quantum=50)
    done = srv.run([req(0, 0.0, 200), dict(req(1, 0.0, 100), cancel_at=0.1), req(2, 0.0, 100)],
                   realtime=False, virtual_step_s=1e-3)
    assert sorted(d["id"] for d in done) == [0, 2]
    assert [c["id"] for c in srv.cancelled] == [1] and srv.cancelled[0]["steps_done"] == 0
    assert len([x for x in srv.pool.calls if x[0] == "add"]) == 2   # requests 0 and 2 only


def test_request_timeout_drops_an_unfinished_solve(fake):
    srv = serve.Server(arena_bytes=1 << 30, quantum=100)
    done = srv.run([dict(req(0, 0.0, 5000), timeout_s=0.25), req(1, 0.0, 300)],
                   realtime=False, virtual_step_s=1e-3)
    assert [d["id"] for d in done] == [1]
    (c,) = srv.cancelled
    assert c["id"] == 0 and c["status"] == "timeout" and 0 < c["steps_done"] < 5000
    assert srv.stats["timed_out"] == 1 and not srv.pool.live


def test_cancel_from_a_callback(fake):
    # a client cancels request 2 when request 0 finishes
    srv = serve.Server(arena_bytes=1 << 30, quantum=100)
    done = srv.run([req(0, 0.0, 100), req(1, 0.0, 300), req(2, 0.0, 1000)], realtime=False,
                   virtual_step_s=1e-3, on_done=lambda d: d["id"] == 0 and srv.cancel(2))
    assert sorted(d["id"] for d in done) == [0, 1]
    assert [c["id"] for c in srv.cancelled] == [2] and srv.cancelled[0]["steps_done"] == 100
