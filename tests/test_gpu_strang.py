"""GPU Strang splitting (gp_set_splitting) against the oracle's Strang steps."""
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


def problem(orc, shape, g=60.0):
    return orc.Problem(*shape, 0.2, 0.22, 0.25, 0.004, gamma=1.0, nu=1.4, lam=1.9, g=g)


def solver(P, p, prec):
    return P.Solver(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.dt, p.gamma, p.nu, p.lam, g=p.g, prec=prec)


@pytest.mark.parametrize("shape", [(40, 32, 24), (17, 9, 30)])
def test_strang_fp64_matches_oracle(P, orc, shape):
    p = problem(orc, shape)
    ref_i = orc.step_imag_strang(p, orc.init_gaussian(p), 30)
    rng = np.random.default_rng(2)
    psi0 = ref_i.astype(complex) * np.exp(0.2j * rng.standard_normal(p.shape))
    ref_r = orc.step_real_strang(p, psi0, 25)
    s = solver(P, p, "f64")
    s.set_splitting("strang")
    s.init_gaussian()
    s.step_imag(30)
    assert np.max(np.abs(s.get_psi() - ref_i)) <= 1e-10
    o, r = s.observables(), orc.observables(p, ref_i)
    assert abs(o["mu"] - r["mu"]) <= 1e-12 * abs(r["mu"])
    s.set_psi(psi0)
    s.step_real(25)
    assert np.max(np.abs(s.get_psi(as_complex=True) - ref_r)) <= 1e-10
    s.close()


@pytest.mark.parametrize("kernels", ["auto", "stream", "tile"])
def test_strang_fp32_matches_oracle_on_every_kernel_family(P, orc, kernels, monkeypatch):
    if kernels == "auto":
        monkeypatch.delenv("GP_SWEEP_KERNELS", raising=False)
    else:
        monkeypatch.setenv("GP_SWEEP_KERNELS", kernels)
    p = problem(orc, (48, 40, 32))
    ref_i = orc.step_imag_strang(p, orc.init_gaussian(p), 40)
    ref_r = orc.step_real_strang(p, ref_i.astype(complex), 30)
    s = solver(P, p, "f32")
    monkeypatch.delenv("GP_SWEEP_KERNELS", raising=False)
    s.set_splitting("strang")
    s.init_gaussian()
    s.step_imag(40)
    assert np.max(np.abs(s.get_psi() - ref_i)) <= 3e-6 * np.max(np.abs(ref_i))
    s.step_real(30)
    assert np.max(np.abs(s.get_psi(as_complex=True) - ref_r)) <= 3e-6 * np.max(np.abs(ref_r))
    s.close()


def test_lie_stays_the_default_and_bad_scheme_is_rejected(P, orc):
    p = problem(orc, (20, 16, 12))
    s = solver(P, p, "f64")
    s.init_gaussian()
    s.step_imag(5)
    ref = orc.step_imag(p, orc.init_gaussian(p), 5)
    assert np.max(np.abs(s.get_psi() - ref)) <= 1e-10
    with pytest.raises(P.GPError):
        P.gp.gp_set_splitting(s.handle, 7)
    s.close()
