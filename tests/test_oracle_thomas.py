"""Pins of the oracle's Thomas solver and its precomputed elimination coefficients.

The CN kinetic substep along one grid line solves the constant-coefficient
tridiagonal system (1+2a) u_j - a (u_{j-1}+u_{j+1}) = (1-2a) v_j + a (v_{j-1}+v_{j+1})
with zero ghosts (Solution method: split-step Crank-Nicolson).  These tests check
the oracle against LAPACK's dense LU solve and against the LU factorisation the
coefficients stand for, on every size 1..12 and on real (imaginary time) and
complex (real time) coefficients.
"""
import numpy as np
import pytest

ALPHAS = [0.025, 0.7, 3.0, 0.005j, 0.3j, 2.0j, 0.1 + 0.2j]


def lap(n):
    return np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("n", list(range(1, 13)))
def test_cn_line_matches_dense_lu(orc, n, alpha):
    rng = np.random.default_rng(1000 * n + int(abs(alpha) * 100))
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    L = lap(n)
    I = np.eye(n)
    want = np.linalg.solve(I - alpha * L, (I + alpha * L) @ v)
    got = orc.cn_line(v, alpha)
    assert np.max(np.abs(got - want)) <= 1e-14 * max(1.0, np.max(np.abs(want))) * (1 + abs(alpha))


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("n", [1, 2, 3, 7, 12, 40])
def test_coefficients_are_the_lu_factors(orc, n, alpha):
    """Lower bidiagonal (diag 1/m_j, sub -a) times unit upper bidiagonal (super cp_j)
    reproduces I - a L exactly up to rounding: the coefficients are Thomas' LU."""
    cp, m = orc.thomas_coeffs(n, alpha)
    lower = np.diag(1.0 / m) + np.diag(-alpha * np.ones(n - 1), -1)
    upper = np.eye(n, dtype=complex) + np.diag(cp[:-1], 1)
    want = np.eye(n) - alpha * lap(n)
    assert np.max(np.abs(lower @ upper - want)) <= 1e-14 * (1 + 4 * abs(alpha))


def test_single_point_line_closed_form(orc):
    for alpha in ALPHAS:
        got = orc.cn_line(np.array([1.0 + 0.5j]), alpha)
        want = (1 - 2 * alpha) / (1 + 2 * alpha) * (1.0 + 0.5j)
        assert abs(got[0] - want) <= 1e-15 * 4


def test_real_time_line_is_unitary(orc):
    """For purely imaginary a the CN matrix is a Cayley transform of a Hermitian
    matrix, hence unitary: the line norm is conserved."""
    rng = np.random.default_rng(7)
    v = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    for alpha in [0.005j, 0.3j, 2.0j]:
        u = orc.cn_line(v, alpha)
        assert abs(np.vdot(u, u).real - np.vdot(v, v).real) <= 1e-13 * np.vdot(v, v).real


def test_elimination_coefficients_converge_geometrically(orc):
    """cp_j tends to the smaller root of a c^2 + (1+2a) c + a = 0 (the Toeplitz limit)."""
    a = 0.025
    cp, m = orc.thomas_coeffs(30, a)
    root = (-(1 + 2 * a) + np.sqrt((1 + 2 * a) ** 2 - 4 * a * a)) / (2 * a)
    assert abs(cp[-1] - root) < 1e-16 * 10
    assert abs(m[-1] - 1.0 / (1 + 2 * a + a * root)) < 1e-15
