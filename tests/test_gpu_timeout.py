"""Failure detection of the bounded device waits, made to run out on purpose.

Each sweep kernel waits on its own shared-memory copies (row copies of the x sweeps,
tile loads of the FP64 sweeps) with a bounded wait that, when it gives up, sets the
solver's timeout status, drains the copies still in flight (up to 2 s) and lets its
blocks exit.  gp_set_wait_limit(s, 0) makes the first wait on each copy give up at
once, so every warp or block takes that path.  Nothing faults: the host sees
GP_ERR_TIMEOUT from gp_sync, the status is cleared, and the next steps on the same
solver (limit restored) give the same bits as a solver that never timed out.
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


# x rows of 60 (one row per warp at a time) and 16 (grouped rows) 16-byte vectors in
# FP32 (the copy-fed banded x sweep); the tile kernels (bulk row tiles along x, TMA tiles along y
# and z), which FP64 solvers run when GP_SWEEP_KERNELS=tile (their default kernels
# stream lines through global memory and have no waits)
CASES = [("f32", (240, 40, 32)), ("f32", (64, 40, 32)), ("f64", (64, 48, 32))]


@pytest.mark.parametrize("prec,shape", CASES)
@pytest.mark.parametrize("mode", ["imag", "real"])
def test_wait_that_runs_out_is_reported_and_the_solver_recovers(P, prec, shape, mode, monkeypatch):
    if prec == "f64":
        monkeypatch.setenv("GP_SWEEP_KERNELS", "tile")
    else:   # the copy-fed banded x sweep (rows of 8 m <= 256 points run without copies)
        monkeypatch.setenv("GP_X_REG", "0")
    nx, ny, nz = shape
    args = (nx, ny, nz, 0.2, 0.2, 0.2, 0.004, 1.0, 1.41, 2.0)
    s = P.Solver(*args, g=50.0, prec=prec)
    step = s.step_imag if mode == "imag" else s.step_real
    s.init_gaussian()
    P.gp.gp_set_wait_limit(s.handle, 0)
    step(2)
    with pytest.raises(P.GPError) as e:
        s.sync()
    assert e.value.code == P.gp.GP_ERR_TIMEOUT
    s.sync()  # the status was cleared by the failed check

    # limit restored: the same solver gives the bits of one that never timed out
    P.gp.gp_set_wait_limit(s.handle, -1)
    ref = P.Solver(*args, g=50.0, prec=prec)
    for t in (s, ref):
        t.init_gaussian()
        if mode == "real":
            t.step_imag(3)
        (t.step_imag if mode == "imag" else t.step_real)(5)
        t.sync()
    cplx = mode == "real"
    assert np.array_equal(s.get_psi(as_complex=cplx), ref.get_psi(as_complex=cplx))
    s.close()
    ref.close()


def test_wait_limit_rejects_null_solver(P):
    with pytest.raises(P.GPError):
        P.gp.gp_set_wait_limit(None, 0)
