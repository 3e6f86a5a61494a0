"""GPU tests of the continuous-batching server (paper_1605_03958_gb300/serve.py).

Each served result must be the same alone and in the mix: a request's observables
from the server (admitted into a pool shared with other grids, modes and step counts,
stepped in quanta, retired between quanta) equal, bit for bit, those of the same
request run by itself in its own pool.  Against the one-at-a-time FP64 solver the
FP32 results agree to the FP32 tolerance.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03958_gb300 as pkg
    return pkg


def small_stream(n=10, seed=7):
    rng = np.random.default_rng(seed)
    reqs, t = [], 0.0
    for i in range(n):
        t += float(rng.exponential(0.002))
        quench = bool(rng.uniform() < 0.4)
        reqs.append(dict(id=i, arrival=t, kind="quench" if quench else "ground",
                         steps=int(rng.integers(15, 60)),
                         params=dict(nx=int(rng.choice([32, 40, 48])), ny=int(rng.choice([24, 32])),
                                     nz=int(rng.choice([16, 24, 32])), dx=0.2, dt=0.004,
                                     gamma=float(rng.uniform(0.5, 3)), nu=float(rng.uniform(0.5, 3)),
                                     lam=float(rng.uniform(0.5, 3)), g=float(rng.uniform(1, 300)))))
    return reqs


def run_alone(P, req):
    pool = P.Pool(64 << 20, max_slots=1)
    s = pool.add(**req["params"])
    if req["kind"] == "quench":
        pool.set_real_time(s)
    pool.step(req["steps"])
    obs = pool.observables(s)
    pool.close()
    return obs


def test_served_results_equal_results_alone(P):
    from paper_1605_03958_gb300.serve import Server
    reqs = small_stream()
    srv = Server(arena_bytes=256 << 20, max_slots=16, quantum=7)
    done = srv.run(reqs, realtime=False, virtual_step_s=1e-4)
    assert sorted(d["id"] for d in done) == list(range(len(reqs)))
    assert srv.stats["max_live"] > 1          # the requests really shared the pool
    for d in done:
        want = run_alone(P, reqs[d["id"]])
        assert d["obs"] == want, (d["id"], d["obs"], want)
    srv.close()


def test_admission_waits_for_arena_room(P):
    from paper_1605_03958_gb300.serve import Server
    reqs = [dict(id=i, arrival=0.0, kind="ground", steps=10,
                 params=dict(nx=48, ny=48, nz=48, dx=0.2, dt=0.004, gamma=1.0, nu=1.0, lam=1.0,
                             g=10.0)) for i in range(5)]
    one = P.Pool.slot_bytes(**reqs[0]["params"])
    srv = Server(arena_bytes=2 * one + 4096, max_slots=8, quantum=4)
    done = srv.run(reqs, realtime=False)
    assert len(done) == 5
    assert srv.stats["max_live"] == 2
    first = [d for d in done if d["admitted"] == 0.0]
    assert len(first) == 2                  # the others waited for a retirement
    srv.close()


def test_served_fp32_agrees_with_one_at_a_time_fp64(P):
    from paper_1605_03958_gb300.serve import Server, serve_one_at_a_time
    reqs = small_stream(6, seed=11)
    srv = Server(arena_bytes=256 << 20, max_slots=16, quantum=10)
    got = {d["id"]: d for d in srv.run(reqs, realtime=False)}
    ref = {d["id"]: d for d in serve_one_at_a_time(reqs, prec="f64", realtime=False)}
    for i, r in got.items():
        o, w = r["obs"], ref[i]["obs"]
        key = "mu" if r["kind"] == "ground" else "energy"
        assert abs(o[key] - w[key]) <= 1e-5 * abs(w[key]), (i, key, o[key], w[key])
        assert abs(o["norm"] - w["norm"]) <= 1e-5
    srv.close()
