"""GPU tests of the single-step graph replay through the C ABI.

A call of gp_step_imag / gp_step_real with one step replays a CUDA graph of the
step's launches (captured once per mode); a longer call launches the sweeps
directly.  Both run the same kernels with the same parameters, so n single-step
calls and one n-step call must give the same bits — in imaginary and real time,
after a change of g (which drops the captured graphs), in 2D, in FP64, and with
the per-sweep timing on (which always launches directly).
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


def pair(P, nx=48, ny=40, nz=32, prec="f32", g=30.0):
    out = []
    for _ in range(2):
        s = P.Solver(nx, ny, nz, 0.2, dt=0.004, gamma=1.0, nu=1.4, lam=2.0, g=g, prec=prec)
        s.init_gaussian()
        out.append(s)
    return out


def singles(s, n, real=False):
    for _ in range(n):
        (s.step_real if real else s.step_imag)(1)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_single_step_calls_equal_one_call(P, prec):
    a, b = pair(P, prec=prec)
    singles(a, 12)
    b.step_imag(12)
    assert np.array_equal(a.get_psi(), b.get_psi())
    oa, ob = a.observables(), b.observables()
    assert oa["mu"] == ob["mu"] and oa["norm"] == ob["norm"]


def test_graph_follows_g_change_and_real_time(P):
    a, b = pair(P)
    singles(a, 5)
    b.step_imag(5)
    for s in (a, b):
        s.set_g(60.0)
    singles(a, 5)
    b.step_imag(5)
    assert np.array_equal(a.get_psi(), b.get_psi())
    singles(a, 6, real=True)
    b.step_real(6)
    assert np.array_equal(a.get_psi(as_complex=True), b.get_psi(as_complex=True))
    for s in (a, b):
        s.set_g(120.0)
    singles(a, 4, real=True)
    b.step_real(4)
    assert np.array_equal(a.get_psi(as_complex=True), b.get_psi(as_complex=True))


def test_graph_2d(P):
    a, b = pair(P, nx=64, ny=48, nz=1)
    singles(a, 10)
    b.step_imag(10)
    assert np.array_equal(a.get_psi(), b.get_psi())
    assert abs(a.observables()["norm"] - 1.0) <= 1e-6


def test_timing_mode_launches_directly_with_the_same_bits(P):
    a, b = pair(P)
    P.gp_set_timing(a.handle, True)
    singles(a, 6)
    ms, n = P.gp_get_timing(a.handle)
    P.gp_set_timing(a.handle, False)
    assert list(n) == [6, 6, 6]   # every sweep was launched (and timed) separately
    singles(b, 6)
    assert np.array_equal(a.get_psi(), b.get_psi())


def test_strang_single_steps(P):
    """Imaginary time: n single Strang steps (graph) equal one n-step call.  Real time:
    single steps by the graph equal single steps launched directly (timing on); an
    n-step call merges the inner half steps and is not the same arithmetic."""
    a, b = pair(P)
    for s in (a, b):
        s.set_splitting("strang")
    singles(a, 6)
    b.step_imag(6)
    assert np.array_equal(a.get_psi(), b.get_psi())
    P.gp_set_timing(b.handle, True)
    singles(a, 5, real=True)
    singles(b, 5, real=True)
    P.gp_set_timing(b.handle, False)
    assert np.array_equal(a.get_psi(as_complex=True), b.get_psi(as_complex=True))
