"""Closed-form and exact-discrete physics pins of the oracle.

The paper prints no numeric physics result (its only numbers are the timings of
Table 1), so the oracle is pinned by what the mathematics fixes:
  (a) at g = 0 the step matrix is a Kronecker product of 1D matrices, so the
      imaginary-time fixed point is the tensor product of their dominant
      eigenvectors (numpy eig, independent of the oracle);
  (b) at g = 0 the chemical potential tends to the continuum (gamma+nu+lambda)/2,
      shifted by the finite-difference error -h^2 (gamma^2+nu^2+lambda^2)/32, and
      equals the lowest eigenvalue of the discrete Hamiltonian up to O(dt^2);
  (c) real time: every substep is unitary, so the norm is conserved to rounding,
      and the energy drift is first order in dt;
  (d) large g: mu approaches the Thomas-Fermi value (15 g gamma nu lambda / 4 pi)^(2/5) / 2
      from above, with a relative gap shrinking as g grows;
  (e) virial identity 2 E_kin - 2 E_pot + 3 E_int = 0 of the stationary state;
  (f) g = 0 breathing: a Gaussian of frequency w0 in a trap of frequency w has
      <x^2>(t) = cos^2(w t) / (2 w0) + w0 sin^2(w t) / (2 w^2), frequency 2 w;
  (g) real time from an eigenvector of the 1D real-time step matrices is stationary.
"""
import numpy as np
import pytest


def lap(n):
    return np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)


def coords(n, h):
    return (np.arange(n) - (n - 1) / 2.0) * h


def step_matrix_1d(n, h, w, dt, real_time):
    """One SSCN step restricted to one axis at g = 0: CN(al) after exp(-tau V_a)."""
    tau = 1j * dt if real_time else dt
    a = tau / (4 * h * h)
    I = np.eye(n)
    C = np.linalg.solve(I - a * lap(n), I + a * lap(n))
    D = np.diag(np.exp(-tau * 0.5 * w * w * coords(n, h) ** 2))
    return C @ D


def dominant_eigvec(S):
    vals, vecs = np.linalg.eig(S)
    v = vecs[:, np.argmax(np.abs(vals))].real
    return v * np.sign(v[len(v) // 2])


def tensor(ez, ey, ex):
    return np.einsum("k,j,i->kji", ez, ey, ex)


def test_g0_fixed_point_is_tensor_product_of_1d_eigvecs(orc):
    p = orc.Problem(20, 16, 12, 0.3, 0.35, 0.4, 0.02, gamma=1.0, nu=1.3, lam=1.7, g=0.0)
    psi = orc.step_imag(p, orc.init_gaussian(p, 0.8, 1.0, 1.2), 1500)
    ex = dominant_eigvec(step_matrix_1d(p.nx, p.hx, p.gamma, p.dt, False))
    ey = dominant_eigvec(step_matrix_1d(p.ny, p.hy, p.nu, p.dt, False))
    ez = dominant_eigvec(step_matrix_1d(p.nz, p.hz, p.lam, p.dt, False))
    want = tensor(ez, ey, ex)
    want /= np.sqrt(np.sum(want ** 2) * p.hx * p.hy * p.hz)
    assert np.max(np.abs(psi - want)) <= 1e-12


def lowest_discrete_energy(n, h, w):
    H = -0.5 * lap(n) / (h * h) + np.diag(0.5 * w * w * coords(n, h) ** 2)
    return np.linalg.eigvalsh(H)[0]


@pytest.mark.slow
def test_g0_mu_continuum_and_discrete(orc):
    """C1 geometry at g = 0: 64x48x32, h = 0.2, trap (1, 1.5, 2).  Larger dt than C1
    so that 12 time units of relaxation stay cheap; the dt bias is checked to be
    second order."""
    h, n, w = 0.2, (64, 48, 32), (1.0, 1.5, 2.0)
    e0 = sum(lowest_discrete_energy(m, h, wa) for m, wa in zip(n, w))
    mus = {}
    for dt in (0.02, 0.01):
        p = orc.Problem(*n, h, h, h, dt, gamma=w[0], nu=w[1], lam=w[2], g=0.0)
        psi = orc.step_imag(p, orc.init_gaussian(p, 0.9, 1.4, 2.1), int(12.0 / dt))
        mus[dt] = orc.observables(p, psi)["mu"]
    # variational: the O(dt) splitting bias of the state gives O(dt^2) in mu
    assert 0 < mus[0.01] - e0 <= 0.01 ** 2
    assert 3.6 < (mus[0.02] - e0) / (mus[0.01] - e0) < 4.4
    # continuum (gamma+nu+lambda)/2 with the finite-difference shift -h^2 sum(w^2)/32
    predicted = 0.5 * sum(w) - h * h * sum(wa * wa for wa in w) / 32
    assert abs(mus[0.01] - predicted) <= 0.1 * h ** 4 + 0.01 ** 2
    # the shift is second order in h (exact 1D spectra, independent of the oracle)
    e_half = sum(lowest_discrete_energy(2 * m, h / 2, wa) for m, wa in zip(n, w))
    assert 3.8 < (0.5 * sum(w) - e0) / (0.5 * sum(w) - e_half) < 4.2


def test_real_time_norm_and_energy(orc):
    p = orc.Problem(24, 20, 16, 0.3, 0.3, 0.3, 0.004, gamma=1.0, nu=1.41, lam=2.0, g=30.0)
    ground = orc.step_imag(p, orc.init_gaussian(p), 1500)
    drifts = []
    for dt in (0.004, 0.002):
        q = orc.Problem(24, 20, 16, 0.3, 0.3, 0.3, dt, gamma=1.0, nu=1.41, lam=2.0, g=60.0)
        psi = ground.astype(complex)
        e0 = orc.observables(q, psi)["energy"]
        n_steps = int(round(1.0 / dt))
        worst = 0.0
        for _ in range(10):
            psi = orc.step_real(q, psi, n_steps // 10)
            obs = orc.observables(q, psi)
            assert abs(obs["norm"] - 1.0) <= 1e-12
            worst = max(worst, abs(obs["energy"] - e0))
        drifts.append(worst)
    assert drifts[0] < 1e-2 * abs(e0)
    assert 1.5 < drifts[0] / drifts[1] < 2.6  # first order in dt


def thomas_fermi_mu(g, w):
    return 0.5 * (15.0 * g * w[0] * w[1] * w[2] / (4 * np.pi)) ** 0.4


@pytest.mark.slow
def test_thomas_fermi_limit(orc):
    w = (1.0, 1.41, 2.0)
    gaps = {}
    for g in (100.0, 2000.0):
        p = orc.Problem(64, 48, 32, 0.25, 0.25, 0.25, 0.02, gamma=w[0], nu=w[1], lam=w[2], g=g)
        psi = orc.step_imag(p, orc.init_gaussian(p), 1000)
        mu = orc.observables(p, psi)["mu"]
        tf = thomas_fermi_mu(g, w)
        gaps[g] = (mu - tf) / tf
        assert gaps[g] > 0
    assert gaps[2000.0] < 0.05
    assert gaps[2000.0] < gaps[100.0]


def test_virial_identity(orc):
    p = orc.Problem(48, 40, 32, 0.2, 0.2, 0.2, 0.01, gamma=1.0, nu=1.41, lam=2.0, g=100.0)
    psi = orc.step_imag(p, orc.init_gaussian(p), 1500)
    o = orc.observables(p, psi)
    residual = 2 * o["ekin"] - 2 * o["epot"] + 3 * o["eint"]
    assert abs(residual) <= 5e-3 * o["energy"]


def breathing_run(orc, h, n, dt, w, w0):
    p = orc.Problem(n, 6, 6, h, 0.5, 0.5, dt, gamma=w, nu=1.0, lam=1.0, g=0.0)
    psi = orc.init_gaussian(p, w0, 1.0, 1.0).astype(complex)
    chunk = int(round(0.05 / dt))
    ts, x2 = [0.0], [orc.observables(p, psi)["rms_x"] ** 2]
    for _ in range(64):  # t up to 3.2 > one breathing period pi / w
        psi = orc.step_real(p, psi, chunk)
        ts.append(ts[-1] + chunk * dt)
        x2.append(orc.observables(p, psi)["rms_x"] ** 2)
    return np.array(ts), np.array(x2)


def fitted_breathing_frequency(ts, x2):
    """W of the least-squares fit <x^2>(t) = A + B cos(2 W t), by a fine scan."""
    best = None
    for W in np.linspace(0.97, 1.03, 6001):
        M = np.stack([np.ones_like(ts), np.cos(2 * W * ts)], 1)
        coef, *_ = np.linalg.lstsq(M, x2, rcond=None)
        r = np.sum((M @ coef - x2) ** 2)
        if best is None or r < best[0]:
            best = (r, W)
    return best[1]


def test_breathing_mode_g0(orc):
    """x-axis dynamics decouple exactly at g = 0; Gaussian of w0 = 1.6 w released in
    the trap.  Curve and frequency errors are the O(h^2) finite-difference
    dispersion (the dt part is far smaller at these steps), so both must drop ~4x
    when h halves."""
    w, w0 = 1.0, 1.6
    errs, ferrs = [], []
    for h, n in ((0.15, 80), (0.075, 160)):
        ts, x2 = breathing_run(orc, h, n, 0.001, w, w0)
        exact = np.cos(w * ts) ** 2 / (2 * w0) + w0 * np.sin(w * ts) ** 2 / (2 * w * w)
        errs.append(np.max(np.abs(x2 - exact)))
        ferrs.append(abs(fitted_breathing_frequency(ts, x2) - w) / w)
        assert errs[-1] <= 0.35 * h * h
        assert ferrs[-1] <= 0.3 * h * h
    assert 3.0 < errs[0] / errs[1] < 5.0
    assert 3.0 < ferrs[0] / ferrs[1] < 5.0


def test_real_time_eigenstate_is_stationary_g0(orc):
    p = orc.Problem(14, 12, 10, 0.35, 0.35, 0.35, 0.01, gamma=1.0, nu=1.3, lam=1.8, g=0.0)
    vecs = []
    for n, h, w in ((p.nx, p.hx, p.gamma), (p.ny, p.hy, p.nu), (p.nz, p.hz, p.lam)):
        S = step_matrix_1d(n, h, w, p.dt, True)
        vals, V = np.linalg.eig(S)
        gauss = np.exp(-0.5 * w * coords(n, h) ** 2)
        v = V[:, np.argmax(np.abs(V.conj().T @ gauss))]
        vecs.append(v / np.linalg.norm(v))
    psi0 = tensor(vecs[2], vecs[1], vecs[0])
    psi0 /= np.sqrt(np.sum(np.abs(psi0) ** 2) * p.hx * p.hy * p.hz)
    psi = orc.step_real(p, psi0, 200)
    d0, d1 = np.abs(psi0) ** 2, np.abs(psi) ** 2
    assert np.max(np.abs(d1 - d0)) <= 1e-12 * np.max(d0)
