"""Pins of the oracle's 2D problems (nz = 1: the imag2d / real2d programs' equation
in the xy plane, CN solves along x and y only, cell area hx hy).

* one Lie step against dense linear algebra: the pointwise factor, then the Kronecker
  factors I (x) C_x and C_y (x) I with C = (I + aL)^-1 (I - aL) built as dense
  matrices (numpy solve, not the Thomas recurrence), then the renormalisation;
* the g = 0 imaginary-time fixed point against the product of the dominant
  eigenvectors of the two 1D step matrices;
* g = 0 chemical potential near (gamma + nu) / 2 (O(h^2 + dt));
* large g: the 2D Thomas-Fermi value mu = sqrt(g gamma nu / pi), approached from above.
"""
import numpy as np
import pytest


def p2(orc, nx, ny, h, dt, g, w=(1.0, 1.6)):
    return orc.Problem(nx, ny, 1, h, 1.17 * h, 0.5, dt, gamma=w[0], nu=w[1], lam=3.0, g=g)


def cn_dense(n, a):
    L = -2 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    return np.linalg.solve(np.eye(n) - a * L, np.eye(n) + a * L)


@pytest.mark.parametrize("mode", ["imag", "real"])
@pytest.mark.parametrize("shape", [(5, 4), (6, 3), (7, 7)])
def test_2d_step_equals_dense_kronecker_step(orc, shape, mode):
    nx, ny = shape
    p = p2(orc, nx, ny, 0.4, 0.02, 7.0)
    x, y = p.coords(0), p.coords(1)
    V = 0.5 * (p.gamma ** 2 * x[None, :] ** 2 + p.nu ** 2 * y[:, None] ** 2)
    rng = np.random.default_rng(nx * 10 + ny)
    if mode == "imag":
        psi = rng.uniform(0.2, 1.0, (1, ny, nx))
        got = orc.step_imag(p, psi, 1)
        tau = p.dt
    else:
        psi = 0.5 * (rng.standard_normal((1, ny, nx)) + 1j * rng.standard_normal((1, ny, nx)))
        got = orc.step_real(p, psi, 1)
        tau = 1j * p.dt
    f = psi[0] * np.exp(-tau * (V + p.g * np.abs(psi[0]) ** 2))
    Cx = cn_dense(nx, tau / (4 * p.hx ** 2))
    Cy = cn_dense(ny, tau / (4 * p.hy ** 2))
    want = Cy @ (f @ Cx.T)
    if mode == "imag":
        want = want / np.sqrt(np.sum(np.abs(want) ** 2) * p.hx * p.hy)
    assert np.max(np.abs(got[0] - want)) <= 1e-13


def test_2d_g0_fixed_point_is_product_of_1d_eigenvectors(orc):
    p = p2(orc, 24, 20, 0.3, 0.01, 0.0)
    psi = orc.step_imag(p, orc.init_gaussian(p), 4000)
    vecs = []
    for n, h, w, c in ((p.nx, p.hx, p.gamma, p.coords(0)), (p.ny, p.hy, p.nu, p.coords(1))):
        C = cn_dense(n, p.dt / (4 * h * h))
        M = C * np.exp(-p.dt * 0.5 * w * w * c ** 2)[None, :]   # C diag(exp(-dt V_a))
        ev, V = np.linalg.eig(M)
        v = np.real(V[:, np.argmax(np.abs(ev))])
        vecs.append(v * np.sign(v[n // 2]))
    want = np.outer(vecs[1], vecs[0])
    want /= np.sqrt(np.sum(want ** 2) * p.hx * p.hy)
    assert np.max(np.abs(psi[0] - want)) <= 1e-10


def test_2d_mu_at_g0_is_the_trap_zero_point_energy(orc):
    p = p2(orc, 48, 40, 0.2, 0.002, 0.0)
    psi = orc.step_imag(p, orc.init_gaussian(p), 3000)
    mu = orc.observables(p, psi)["mu"]
    assert abs(mu - 0.5 * (p.gamma + p.nu)) <= 0.02 * 0.5 * (p.gamma + p.nu)
    assert orc.observables(p, psi)["rms_z"] == 0.0


def test_2d_thomas_fermi_limit(orc):
    for g in (400.0, 1600.0):
        p = p2(orc, 64, 56, 0.25, 0.005, g)
        psi = orc.step_imag(p, orc.init_gaussian(p), 3000)
        mu = orc.observables(p, psi)["mu"]
        tf = np.sqrt(g * p.gamma * p.nu / np.pi)
        assert tf < mu < 1.08 * tf, (g, mu, tf)
