"""Pins of the full-length oracle fixtures (tests/golden/*.json, written by
make_golden.py from the oracle alone) against what the mathematics fixes, so that the
GPU tests that read them compare with pinned values:
  C2, g = 0      psi at the sampled points equals the exact discrete fixed point (tensor
                 product of the dominant eigenvectors of the 1D step matrices, numpy);
                 mu within O(h^4 + dt^2) of the continuum value shifted by the
                 finite-difference error, (gamma+nu+lambda)/2 - h^2 (gamma^2+nu^2+lambda^2)/32
  C2, g > 0      Thomas-Fermi limit approached from above, gap < 5 % at g = 2000 and
                 smaller than at g = 100; virial identity 2 E_kin - 2 E_pot + 3 E_int = 0
                 to O(h^2)
  all            sum rules: sum_i n_1D(x_i) h = norm = 1 on every axis
  C3             the real-time steps are unitary: norm conserved to rounding along the
                 trajectory; the start state is the C2 g = 100 state (its g-independent
                 observables agree exactly); the quench excites a breathing motion
"""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")


def fixture(name):
    path = os.path.join(GOLD, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated (python tests/golden/make_golden.py)")
    with open(path) as f:
        return json.load(f)


def lap(n):
    return np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)


def fixed_point_1d(n, h, w, dt):
    a = dt / (4 * h * h)
    I = np.eye(n)
    C = np.linalg.solve(I - a * lap(n), I + a * lap(n))
    x = (np.arange(n) - (n - 1) / 2.0) * h
    S = C @ np.diag(np.exp(-dt * 0.5 * w * w * x * x))
    vals, vecs = np.linalg.eig(S)
    v = vecs[:, np.argmax(np.abs(vals))].real
    return v * np.sign(v[n // 2])


def test_c2_g0_oracle_is_the_exact_discrete_fixed_point():
    fx = fixture("c2_g0.json")
    nx, ny, nz = fx["grid"]
    h, (wx, wy, wz), dt = fx["h"], fx["trap"], fx["dt"]
    ex, ey, ez = (fixed_point_1d(nx, h, wx, dt), fixed_point_1d(ny, h, wy, dt),
                  fixed_point_1d(nz, h, wz, dt))
    norm = math.sqrt(np.sum(ex ** 2) * np.sum(ey ** 2) * np.sum(ez ** 2) * h ** 3)
    idx = np.array(fx["sample_index"])
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    want = ex[i] * ey[j] * ez[k] / norm
    assert np.max(np.abs(np.array(fx["psi_samples"]) - want)) <= 1e-10
    mu = fx["observables"]["mu"]
    cont = 0.5 * (wx + wy + wz) - h * h * (wx ** 2 + wy ** 2 + wz ** 2) / 32.0
    assert abs(mu - cont) <= 0.1 * h ** 4 + 10 * dt ** 2, (mu, cont)


def test_c2_thomas_fermi_and_virial():
    gap = {}
    for g in (100, 2000):
        fx = fixture(f"c2_g{g}.json")
        o = fx["observables"]
        w = fx["trap"]
        mu_tf = 0.5 * (15.0 * g * w[0] * w[1] * w[2] / (4.0 * math.pi)) ** 0.4
        assert o["mu"] > mu_tf
        gap[g] = (o["mu"] - mu_tf) / mu_tf
        virial = 2 * o["ekin"] - 2 * o["epot"] + 3 * o["eint"]
        assert abs(virial) <= 5e-3 * o["energy"], (g, virial)
    assert gap[2000] < 0.05 and gap[2000] < gap[100], gap


@pytest.mark.parametrize("name", ["c2_g0.json", "c2_g100.json", "c2_g2000.json", "c3_quench.json"])
def test_sum_rules(name):
    fx = fixture(name)
    h = fx["h"]
    norm = fx["observables"]["norm"] if "observables" in fx else fx["trajectory"]["norm"][-1]
    for a in range(3):
        assert abs(np.sum(fx["density1d"][a]) * h - norm) <= 1e-12
    assert abs(norm - 1.0) <= 1e-11


def test_c3_quench_trajectory_physics():
    fx = fixture("c3_quench.json")
    gs = fixture("c2_g100.json")
    tr = {k: np.array(v) for k, v in fx["trajectory"].items()}
    # unitary steps: the norm stays 1 to rounding over 2*10^4 steps
    assert np.max(np.abs(tr["norm"] - 1.0)) <= 1e-11
    # the start is the g = 100 ground state (g-independent observables equal)
    for k in ("norm", "epot", "ekin", "rms_x", "rms_y", "rms_z", "rms_r"):
        assert tr[k][0] == gs["observables"][k], k
    # doubling g pushes the cloud outward: a breathing motion of the rms sizes
    for k in ("rms_x", "rms_y", "rms_z"):
        assert np.max(tr[k]) > tr[k][0] * 1.01, k
    # the Lie split step conserves energy to O(dt) per unit time: bounded drift
    assert np.max(np.abs(tr["energy"] - tr["energy"][0])) <= 1e-2 * abs(tr["energy"][0])
