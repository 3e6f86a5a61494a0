"""GPU 2D solves (nz = 1) against the oracle's 2D problems."""
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


def p2(orc, nx, ny, g=50.0):
    return orc.Problem(nx, ny, 1, 0.15, 0.17, 0.5, 0.002, gamma=1.0, nu=1.6, lam=3.0, g=g)


def solver(P, p, prec):
    return P.Solver(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.dt, p.gamma, p.nu, p.lam, g=p.g, prec=prec)


@pytest.mark.parametrize("shape", [(96, 80), (37, 53), (300, 12)])
def test_2d_fp64_imag_and_real_match_oracle(P, orc, shape):
    p = p2(orc, *shape)
    ref = orc.step_imag(p, orc.init_gaussian(p), 60)
    s = solver(P, p, "f64")
    s.init_gaussian()
    s.step_imag(60)
    assert np.max(np.abs(s.get_psi() - ref)) <= 1e-10
    o, r = s.observables(), orc.observables(p, ref)
    for k in ("norm", "mu", "energy", "ekin", "epot", "eint", "rms_x", "rms_y"):
        assert abs(o[k] - r[k]) <= 1e-12 * abs(r[k]), k
    assert o["rms_z"] == 0.0
    d1 = s.density1d(0)
    assert np.max(np.abs(d1 - orc.density1d(p, ref, 0))) <= 1e-12 * np.max(d1)
    ref_c = orc.step_real(p, ref.astype(complex), 40)
    s.step_real(40)
    assert np.max(np.abs(s.get_psi(as_complex=True) - ref_c)) <= 1e-10
    s.close()


@pytest.mark.parametrize("kernels", ["auto", "stream", "tile"])
def test_2d_fp32_matches_oracle(P, orc, kernels, monkeypatch):
    if kernels == "auto":
        monkeypatch.delenv("GP_SWEEP_KERNELS", raising=False)
    else:
        monkeypatch.setenv("GP_SWEEP_KERNELS", kernels)
    p = p2(orc, 128, 96, g=200.0)
    ref = orc.step_imag(p, orc.init_gaussian(p), 50)
    s = solver(P, p, "f32")
    monkeypatch.delenv("GP_SWEEP_KERNELS", raising=False)
    s.init_gaussian()
    s.step_imag(50)
    assert np.max(np.abs(s.get_psi() - ref)) <= 3e-6 * np.max(np.abs(ref))
    assert abs(s.observables()["mu"] - orc.observables(p, ref)["mu"]) <= 1e-5 * orc.observables(p, ref)["mu"]
    s.close()


def test_2d_strang(P, orc):
    p = p2(orc, 64, 48)
    ref = orc.step_imag_strang(p, orc.init_gaussian(p), 30)
    s = solver(P, p, "f64")
    s.set_splitting("strang")
    s.init_gaussian()
    s.step_imag(30)
    assert np.max(np.abs(s.get_psi() - ref)) <= 1e-10
    s.close()
