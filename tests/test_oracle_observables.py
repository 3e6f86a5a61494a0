"""Pins of the oracle's observables and integrated densities.

Outputs named by the paper ("Summary of revisions"): energy and chemical
potential, rms sizes, and the integrated densities of Eq. 1 and its 3D analogues
(1D: integrate out two coordinates; 2D: integrate out one).  The readings used:
  E_kin = <psi| -Lap_h / 2 |psi> dV with the same 3-point Laplacian and zero ghosts
          as the CN substep, E_pot = sum V |psi|^2 dV, E_int = g/2 sum |psi|^4 dV,
  E = E_kin + E_pot + E_int,   mu = E_kin + E_pot + 2 E_int,
  rms_a = sqrt(sum a^2 |psi|^2 dV / norm),   rms_r = sqrt(rms_x^2 + rms_y^2 + rms_z^2).
They are checked against dense matrices (Kronecker-sum Laplacian) and direct
numpy marginals, and against the closed forms of a Gaussian.
"""
import numpy as np
import pytest


def lap(n):
    return np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)


def coords(n, h):
    return (np.arange(n) - (n - 1) / 2.0) * h


@pytest.fixture
def tiny(orc):
    p = orc.Problem(5, 4, 3, 0.3, 0.25, 0.4, 0.01, gamma=1.1, nu=1.7, lam=0.6, g=7.0)
    rng = np.random.default_rng(42)
    psi = rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)
    return p, psi


def test_energy_functional_matches_dense_hamiltonian(orc, tiny):
    p, psi = tiny
    dV = p.hx * p.hy * p.hz
    Ix, Iy, Iz = np.eye(p.nx), np.eye(p.ny), np.eye(p.nz)
    lap3 = (np.kron(Iz, np.kron(Iy, lap(p.nx) / p.hx ** 2))
            + np.kron(Iz, np.kron(lap(p.ny) / p.hy ** 2, Ix))
            + np.kron(lap(p.nz) / p.hz ** 2, np.kron(Iy, Ix)))
    z, y, x = np.meshgrid(coords(p.nz, p.hz), coords(p.ny, p.hy), coords(p.nx, p.hx), indexing="ij")
    V = 0.5 * (p.gamma ** 2 * x ** 2 + p.nu ** 2 * y ** 2 + p.lam ** 2 * z ** 2)
    v = psi.reshape(-1)
    ekin = np.vdot(v, -0.5 * lap3 @ v).real * dV
    epot = np.sum(V * np.abs(psi) ** 2) * dV
    eint = 0.5 * p.g * np.sum(np.abs(psi) ** 4) * dV
    norm = np.sum(np.abs(psi) ** 2) * dV
    o = orc.observables(p, psi)
    assert o["norm"] == pytest.approx(norm, rel=1e-14)
    assert o["ekin"] == pytest.approx(ekin, rel=1e-13)
    assert o["epot"] == pytest.approx(epot, rel=1e-14)
    assert o["eint"] == pytest.approx(eint, rel=1e-14)
    assert o["energy"] == pytest.approx(ekin + epot + eint, rel=1e-13)
    assert o["mu"] == pytest.approx(ekin + epot + 2 * eint, rel=1e-13)
    for name, c in (("rms_x", x), ("rms_y", y), ("rms_z", z)):
        assert o[name] == pytest.approx(np.sqrt(np.sum(c ** 2 * np.abs(psi) ** 2) * dV / norm), rel=1e-14)
    assert o["rms_r"] == pytest.approx(np.sqrt(o["rms_x"] ** 2 + o["rms_y"] ** 2 + o["rms_z"] ** 2), rel=1e-14)


def test_real_field_observables_equal_complex_ones(orc, tiny):
    p, psi = tiny
    a = orc.observables(p, psi.real)
    b = orc.observables(p, psi.real.astype(complex))
    for k in a:
        assert a[k] == pytest.approx(b[k], rel=1e-15, abs=1e-300)


def test_gaussian_closed_forms(orc):
    """A wide, fine grid: sampled Gaussian sums equal the integrals up to
    exponentially small aliasing, so rms_a = 1/sqrt(2 w_a) and E_pot = sum w_a / 4."""
    p = orc.Problem(96, 80, 64, 0.15, 0.15, 0.15, 0.01, gamma=1.0, nu=1.41, lam=2.0, g=0.0)
    psi = orc.init_gaussian(p)
    o = orc.observables(p, psi)
    w = (1.0, 1.41, 2.0)
    assert o["norm"] == pytest.approx(1.0, rel=1e-14)
    for name, wa in zip(("rms_x", "rms_y", "rms_z"), w):
        assert o[name] == pytest.approx(1 / np.sqrt(2 * wa), rel=1e-11)
    assert o["epot"] == pytest.approx(sum(w) / 4, rel=1e-11)
    # FD kinetic energy of a Gaussian: sum_a (1 - exp(-w_a h^2 / 4)) / h^2, exactly
    # (every edge term is a shifted Gaussian product), up to aliasing.
    ek = sum((1 - np.exp(-wa * p.hx ** 2 / 4)) / p.hx ** 2 for wa in w)
    assert o["ekin"] == pytest.approx(ek, rel=1e-11)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_density1d_brute_force_and_sum_rule(orc, tiny, axis):
    p, psi = tiny
    d = np.abs(psi) ** 2
    w = [p.hy * p.hz, p.hx * p.hz, p.hx * p.hy][axis]
    sum_axes = {0: (0, 1), 1: (0, 2), 2: (1, 2)}[axis]
    want = d.sum(axis=sum_axes) * w
    got = orc.density1d(p, psi, axis)
    assert np.allclose(got, want, rtol=1e-14, atol=0)
    h = [p.hx, p.hy, p.hz][axis]
    assert np.sum(got) * h == pytest.approx(orc.observables(p, psi)["norm"], rel=1e-14)


@pytest.mark.parametrize("plane", [0, 1, 2])
def test_density2d_brute_force_and_marginals(orc, tiny, plane):
    p, psi = tiny
    d = np.abs(psi) ** 2
    if plane == 0:
        want = d.sum(axis=0) * p.hz                     # [j, i]
    elif plane == 1:
        want = d.sum(axis=1) * p.hy                     # [k, i]
    else:
        want = d.sum(axis=2) * p.hx                     # [k, j]
    got = orc.density2d(p, psi, plane)
    assert got.shape == want.shape
    assert np.allclose(got, want, rtol=1e-14, atol=0)
    # integrating the 2D density over one more axis gives the 1D density
    if plane == 0:
        assert np.allclose(got.sum(axis=0) * p.hy, orc.density1d(p, psi, 0), rtol=1e-14)
        assert np.allclose(got.sum(axis=1) * p.hx, orc.density1d(p, psi, 1), rtol=1e-14)
    elif plane == 1:
        assert np.allclose(got.sum(axis=1) * p.hx, orc.density1d(p, psi, 2), rtol=1e-14)
    else:
        assert np.allclose(got.sum(axis=1) * p.hy, orc.density1d(p, psi, 2), rtol=1e-14)
        assert np.allclose(got.sum(axis=0) * p.hz, orc.density1d(p, psi, 1), rtol=1e-14)
