"""GPU tests of pools (batched uneven FP32 solves, the serving path) through the C ABI.

A slot of a pool runs the same SSCN step as an FP32 solver, so it is compared with
the FP64 oracle at the FP32 tolerance; and a slot's arithmetic may not depend on the
other live slots, so a slot stepped alone and the same slot stepped in a mix of other
grids, modes and admissions must agree bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

H, DT = 0.2, 0.004
# uneven grids, traps and nonlinearities (h and dt shared, as in the batched workload)
SLOTS = [
    dict(nx=48, ny=32, nz=40, gamma=1.0, nu=1.4, lam=2.2, g=30.0),
    dict(nx=37, ny=29, nz=23, gamma=0.7, nu=1.9, lam=1.2, g=400.0),
    dict(nx=64, ny=16, nz=24, gamma=2.5, nu=0.8, lam=1.6, g=5.0),
]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03958_gb300 as pkg
    return pkg


def kw(d):
    return dict(nx=d["nx"], ny=d["ny"], nz=d["nz"], dx=H, dt=DT, gamma=d["gamma"], nu=d["nu"],
                lam=d["lam"], g=d["g"])


def oracle_problem(orc, d):
    return orc.Problem(d["nx"], d["ny"], d["nz"], H, H, H, DT, gamma=d["gamma"], nu=d["nu"],
                       lam=d["lam"], g=d["g"])


def make_pool(P, slots, arena=256 << 20):
    pool = P.Pool(arena, max_slots=16)
    ids = [pool.add(**kw(d)) for d in slots]
    return pool, ids


def test_pool_imag_matches_oracle(P, orc):
    pool, ids = make_pool(P, SLOTS)
    pool.step(20)
    for d, s in zip(SLOTS, ids):
        p = oracle_problem(orc, d)
        ref = orc.step_imag(p, orc.init_gaussian(p), 20)
        tol = 3e-6 * np.max(np.abs(ref))
        assert np.max(np.abs(pool.get_psi(s) - ref)) <= tol, d
        got, want = pool.observables(s), orc.observables(p, ref)
        assert abs(got["mu"] - want["mu"]) / abs(want["mu"]) <= 1e-5
        assert abs(got["norm"] - 1.0) <= 1e-6
    pool.close()


def test_pool_slot_alone_equals_slot_in_mix(P):
    mix, ids = make_pool(P, SLOTS)
    mix.step(15)
    for d, s in zip(SLOTS, ids):
        alone, (a,) = make_pool(P, [d])
        alone.step(15)
        assert np.array_equal(alone.get_psi(a), mix.get_psi(s)), d
        alone.close()
    mix.close()


def test_pool_real_time_quench_matches_oracle_and_alone(P, orc):
    """10 imaginary steps, hand-off to real time, g doubled, 20 real steps; the other
    slots stay in imaginary time in the same pool."""
    mix, ids = make_pool(P, SLOTS)
    alone, (a,) = make_pool(P, [SLOTS[0]])
    for pool, s in ((mix, ids[0]), (alone, a)):
        pool.step(10)
        pool.set_real_time(s)
        pool.set_g(s, 2 * SLOTS[0]["g"])
        pool.step(20)
    p = oracle_problem(orc, SLOTS[0])
    psi = orc.step_imag(p, orc.init_gaussian(p), 10).astype(complex)
    p2 = oracle_problem(orc, dict(SLOTS[0], g=2 * SLOTS[0]["g"]))
    ref = orc.step_real(p2, psi, 20)
    got = mix.get_psi(ids[0], as_complex=True)
    assert np.max(np.abs(got - ref)) <= 3e-6 * np.max(np.abs(ref))
    assert np.array_equal(got, alone.get_psi(a, as_complex=True))
    assert abs(mix.observables(ids[0])["norm"] - 1.0) <= 1e-5
    mix.close()
    alone.close()


def test_pool_admission_and_retirement_leave_other_slots_unchanged(P):
    mix, ids = make_pool(P, SLOTS)
    mix.step(10)
    mix.remove(ids[1])
    extra = mix.add(**kw(dict(nx=40, ny=40, nz=40, gamma=1.0, nu=1.0, lam=1.0, g=50.0)))
    mix.set_real_time(extra)
    mix.step(10)
    for i in (0, 2):
        alone, (a,) = make_pool(P, [SLOTS[i]])
        alone.step(20)
        assert np.array_equal(alone.get_psi(a), mix.get_psi(ids[i]))
        alone.close()
    mix.close()


def test_pool_graph_replay_equals_direct_launches(P):
    a, ia = make_pool(P, SLOTS)
    b, ib = make_pool(P, SLOTS)
    b.set_graph(False)
    a.step(12)
    b.step(12)
    assert a.info()["graph"] == 1 and b.info()["graph"] == 0
    for s, t in zip(ia, ib):
        assert np.array_equal(a.get_psi(s), b.get_psi(t))
    a.close()
    b.close()


def test_pool_tune_advances_no_solve(P):
    pool, ids = make_pool(P, SLOTS)
    pool.step(5)
    before = [pool.get_psi(s) for s in ids]
    ms = pool.tune(3)
    assert ms > 0
    info = pool.info()
    assert info["x_stages"] in (2, 3, 4) and info["seg_turns"] in (1, 2, 3, 4)
    for s, b in zip(ids, before):
        assert np.array_equal(pool.get_psi(s), b)
    pool.step(5)   # still steps after tuning
    assert abs(pool.observables(ids[0])["norm"] - 1.0) <= 1e-6
    pool.close()


def test_pool_shape_changes_only_the_norm_rounding(P):
    """x stages and rows per warp do not touch the arithmetic; the y / z segment length
    changes only the summation order of the norm."""
    a, ia = make_pool(P, SLOTS)
    b, ib = make_pool(P, SLOTS)
    b.set_shape(4, 2)
    a.step(20)
    b.step(20)
    for s, t in zip(ia, ib):
        x, y = a.get_psi(s), b.get_psi(t)
        assert np.max(np.abs(x - y)) <= 1e-6 * np.max(np.abs(x))
    a.close()
    b.close()


def test_pool_rejects_and_reports(P):
    pool = P.Pool(32 << 20, max_slots=2)
    with pytest.raises(P.GPError) as e:
        pool.add(**kw(SLOTS[0]), prec="f64")
    assert e.value.code == P.gp.GP_ERR_ARG
    with pytest.raises(P.GPError) as e:
        pool.add(nx=6, ny=32, nz=32, dx=H, dt=DT)
    assert e.value.code == P.gp.GP_ERR_ARG
    big = dict(nx=160, ny=160, nz=160, gamma=1.0, nu=1.0, lam=1.0, g=1.0)
    assert P.Pool.slot_bytes(**kw(big)) > (32 << 20)
    with pytest.raises(P.GPError) as e:
        pool.add(**kw(big))
    assert e.value.code == P.gp.GP_ERR_NOMEM
    s0 = pool.add(**kw(SLOTS[2]))
    s1 = pool.add(**kw(SLOTS[2]))
    with pytest.raises(P.GPError) as e:
        pool.add(**kw(SLOTS[2]))   # both slots in use
    assert e.value.code == P.gp.GP_ERR_NOMEM
    free0, _ = pool.free_bytes()
    pool.remove(s0)
    free1, largest = pool.free_bytes()
    assert free1 > free0 and largest >= P.Pool.slot_bytes(**kw(SLOTS[2]))
    with pytest.raises(P.GPError):
        pool.step(-1)
    pool.remove(s1)
    assert pool.info()["live"] == 0
    pool.step(3)   # nothing live: a no-op
    pool.close()


def test_pool_register_row_x_gives_the_copy_fed_bits(P, monkeypatch):
    """A pool whose imaginary-time slots all have rows of 16 m points runs the x sweep with
    rows in registers (16 points per lane, several rows per warp); it gives the same bits
    as the copy-fed x sweep (same operations in the same order), which a mix with any
    other row length runs."""
    slots = [dict(nx=48, ny=32, nz=40, gamma=1.0, nu=1.4, lam=2.2, g=30.0),
             dict(nx=160, ny=20, nz=18, gamma=0.7, nu=1.9, lam=1.2, g=400.0),
             dict(nx=32, ny=16, nz=24, gamma=2.5, nu=0.8, lam=1.6, g=5.0)]
    outs = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("GP_X_REG", flag)
        pool, ids = make_pool(P, slots)
        pool.step(12)
        outs[flag] = ([pool.get_psi(s) for s in ids], pool.info()["x_reg"])
        pool.close()
    monkeypatch.delenv("GP_X_REG", raising=False)
    assert outs["1"][1] == 1 and outs["0"][1] == 0
    for a, b in zip(outs["1"][0], outs["0"][0]):
        assert np.array_equal(a, b)


# complex slots whose rows are 8 m <= 256 points (the register-row x sweep's condition)
CSLOTS = [
    dict(nx=48, ny=32, nz=24, gamma=1.0, nu=1.4, lam=2.2, g=30.0),
    dict(nx=128, ny=20, nz=18, gamma=0.7, nu=1.9, lam=1.2, g=400.0),
    dict(nx=32, ny=16, nz=24, gamma=2.5, nu=0.8, lam=1.6, g=5.0),
]


def quench_pool(P, slots, steps_imag=10, steps_real=20):
    """steps_imag imaginary steps, then every slot to real time at twice its g."""
    pool, ids = make_pool(P, slots)
    pool.step(steps_imag)
    for s, d in zip(ids, slots):
        pool.set_real_time(s)
        pool.set_g(s, 2 * d["g"])
    pool.step(steps_real)
    return pool, ids


def test_pool_complex_register_row_x_sweep(P, orc, monkeypatch):
    """Real-time slots with rows of 8 m complex points run the x sweep with rows in
    registers (8 complex points per lane, several rows per warp pass); it and the
    copy-fed x sweep both follow the oracle's quench at the FP32 tolerance."""
    outs = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("GP_X_REG", flag)
        pool, ids = quench_pool(P, CSLOTS)
        outs[flag] = ([pool.get_psi(s, as_complex=True) for s in ids], pool.info()["x_reg_complex"])
        pool.close()
    monkeypatch.delenv("GP_X_REG", raising=False)
    assert outs["1"][1] == 1 and outs["0"][1] == 0
    for k, d in enumerate(CSLOTS):
        p = oracle_problem(orc, d)
        psi = orc.step_imag(p, orc.init_gaussian(p), 10).astype(complex)
        ref = orc.step_real(oracle_problem(orc, dict(d, g=2 * d["g"])), psi, 20)
        tol = 3e-6 * np.max(np.abs(ref))
        for flag in ("1", "0"):
            assert np.max(np.abs(outs[flag][0][k] - ref)) <= tol, (d, flag)


def test_pool_complex_slot_alone_equals_slot_in_mix(P):
    """The register-row x sweep chooses the pointwise polynomial per row, so a complex
    slot gives the same bits alone and in a mix of other complex grids."""
    mix, ids = quench_pool(P, CSLOTS)
    assert mix.info()["x_reg_complex"] == 1
    for d, s in zip(CSLOTS, ids):
        alone, (a,) = quench_pool(P, [d])
        assert np.array_equal(alone.get_psi(a, as_complex=True), mix.get_psi(s, as_complex=True)), d
        alone.close()
    mix.close()
