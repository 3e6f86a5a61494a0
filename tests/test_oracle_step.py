"""Brute-force pins of the oracle's SSCN step on tiny grids.

One split-step Crank-Nicolson step (Solution method; imag3d / real3d summaries) is,
with tau = dt (imaginary time) or i dt (real time):
  pointwise   psi <- psi exp(-tau (V + g |psi|^2)),
  kinetic     psi <- (M_z kron M_y kron M_x) psi,  M_a = (I - al_a L)^-1 (I + al_a L),
              al_a = tau / (4 h_a^2)  (one CN solve per line along every axis),
  imaginary   psi <- psi / sqrt(sum |psi|^2 dV).
Here the kinetic part is one dense Kronecker matrix applied to the flattened
field, so the test shares nothing with the oracle's line-by-line Thomas sweeps,
strides and axis loops.  Different spacings, trap ratios and sizes on each axis
make a transposed axis, a wrong stride or a dropped term fail.
"""
import numpy as np
import pytest


def lap(n):
    return np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)


def cn_matrix(n, alpha):
    I = np.eye(n)
    return np.linalg.solve(I - alpha * lap(n), I + alpha * lap(n))


def coords(n, h):
    return (np.arange(n) - (n - 1) / 2.0) * h


def potential(p):
    z, y, x = np.meshgrid(coords(p.nz, p.hz), coords(p.ny, p.hy), coords(p.nx, p.hx),
                          indexing="ij")
    return 0.5 * (p.gamma ** 2 * x ** 2 + p.nu ** 2 * y ** 2 + p.lam ** 2 * z ** 2)


def dense_step(p, psi, real_time):
    tau = 1j * p.dt if real_time else p.dt
    V = potential(p)
    phi = psi * np.exp(-tau * (V + p.g * np.abs(psi) ** 2))
    M = np.kron(cn_matrix(p.nz, tau / (4 * p.hz ** 2)),
                np.kron(cn_matrix(p.ny, tau / (4 * p.hy ** 2)), cn_matrix(p.nx, tau / (4 * p.hx ** 2))))
    out = (M @ phi.reshape(-1)).reshape(psi.shape)
    if not real_time:
        out = out / np.sqrt(np.sum(np.abs(out) ** 2) * p.hx * p.hy * p.hz)
    return out


GRIDS = [(3, 3, 3), (5, 4, 3), (6, 5, 4), (4, 7, 5), (1, 6, 3), (2, 1, 5)]


def make_problem(orc, shape, g, dt):
    nx, ny, nz = shape
    return orc.Problem(nx, ny, nz, 0.3, 0.25, 0.4, dt, gamma=1.1, nu=1.7, lam=0.6, g=g)


@pytest.mark.parametrize("shape", GRIDS)
@pytest.mark.parametrize("g", [0.0, 3.0, 40.0])
def test_imag_step_matches_dense(orc, shape, g):
    p = make_problem(orc, shape, g, 0.01)
    rng = np.random.default_rng(sum(shape) * 7 + int(g))
    psi = rng.uniform(0.1, 1.0, size=p.shape)
    want = psi.copy()
    for _ in range(3):
        want = dense_step(p, want, real_time=False)
    got = orc.step_imag(p, psi, 3)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("shape", GRIDS)
@pytest.mark.parametrize("g", [0.0, 3.0, 40.0])
def test_real_step_matches_dense(orc, shape, g):
    p = make_problem(orc, shape, g, 0.02)
    rng = np.random.default_rng(sum(shape) * 11 + int(g))
    psi = rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)
    want = psi.copy()
    for _ in range(3):
        want = dense_step(p, want, real_time=True)
    got = orc.step_real(p, psi, 3)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_large_step_imag_matches_dense(orc):
    """al well above 1 (dt = 4 h^2): the solve must not rely on diagonal dominance
    being strong."""
    p = orc.Problem(5, 6, 4, 0.1, 0.1, 0.1, 0.04, gamma=1.0, nu=1.3, lam=2.0, g=5.0)
    psi = np.random.default_rng(3).uniform(0.1, 1.0, p.shape)
    want = dense_step(p, psi, real_time=False)
    got = orc.step_imag(p, psi, 1)
    assert np.max(np.abs(got - want)) <= 1e-13


def test_mirror_symmetry_is_preserved(orc):
    """The box is centred on the origin (grid reading x_i = (i - (n-1)/2) h): a
    state even in x, y and z stays even under the step, on odd and even sizes."""
    for shape in [(9, 8, 7), (10, 11, 6)]:
        p = orc.Problem(*shape, 0.3, 0.35, 0.4, 0.01, gamma=1.0, nu=1.4, lam=2.0, g=25.0)
        psi = orc.init_gaussian(p, 0.7, 0.9, 1.3)
        out = orc.step_imag(p, psi, 20)
        for ax in range(3):
            assert np.max(np.abs(out - np.flip(out, axis=ax))) <= 1e-14


def test_g_physical_scaling(orc):
    """g = 4 pi N a_s / l_osc: linear in N and a_s, inverse in l_osc, independent of
    the common length unit, and 1 at N a_s / l_osc = 1 / (4 pi)."""
    base = orc.g_physical(2000.0, 0.0057, 1.2)
    assert orc.g_physical(4000.0, 0.0057, 1.2) == pytest.approx(2 * base, rel=1e-15)
    assert orc.g_physical(2000.0, 3 * 0.0057, 1.2) == pytest.approx(3 * base, rel=1e-15)
    assert orc.g_physical(2000.0, 0.0057, 2.4) == pytest.approx(base / 2, rel=1e-15)
    assert orc.g_physical(2000.0, 0.0057e-6, 1.2e-6) == pytest.approx(base, rel=1e-14)
    assert orc.g_physical(1.0, 1.0, 4 * np.pi) == pytest.approx(1.0, rel=1e-15)
