"""Pins of the oracle's Strang-split steps (half pointwise substep, CN solves, half
pointwise substep), against properties that the Lie step does not have:

* real time: the Strang step is time-reversible — n steps with -dt undo n steps with
  dt to rounding (the pointwise phase keeps |psi|, so its halves commute with their
  reversal, and CN with -a is the inverse of CN with a); the Lie step is not;
* second order: the state after a fixed time converges like dt^2 (error ratio near 4
  when dt halves, against a fine-step solution of the same scheme), the Lie step like
  dt (ratio near 2);
* with V = 0 and g = 0 both splittings reduce to the CN solves alone.
"""
import numpy as np
import pytest


def prob(orc, dt, g=40.0, w=(1.0, 1.3, 1.7)):
    return orc.Problem(12, 10, 8, 0.3, 0.35, 0.4, dt, gamma=w[0], nu=w[1], lam=w[2], g=g)


def start(orc, p):
    rng = np.random.default_rng(3)
    psi = orc.init_gaussian(p).astype(complex)
    return psi * np.exp(1j * 0.3 * rng.standard_normal(p.shape))


def test_real_strang_is_time_reversible_and_lie_is_not(orc):
    p, q = prob(orc, 0.01), prob(orc, -0.01)
    psi0 = start(orc, p)
    back = orc.step_real_strang(q, orc.step_real_strang(p, psi0, 25), 25)
    assert np.max(np.abs(back - psi0)) <= 1e-12
    back_lie = orc.step_real(q, orc.step_real(p, psi0, 25), 25)
    assert np.max(np.abs(back_lie - psi0)) > 1e-6


@pytest.mark.parametrize("mode", ["real", "imag"])
def test_strang_is_second_order_lie_first(orc, mode):
    """Imaginary time at g = 0: renormalising after every step commutes with a linear
    step, so the splitting's own order shows; with g != 0 the per-step projection
    onto unit norm is itself a first-order step of the normalised flow."""
    T = 0.08
    fine = 2 ** 7
    g = 40.0 if mode == "real" else 0.0

    def prob_(dt):
        return prob(orc, dt, g=g)

    pf = prob_(T / fine)
    psi0 = start(orc, pf) if mode == "real" else orc.init_gaussian(pf)
    S = orc.step_real_strang if mode == "real" else orc.step_imag_strang
    L = orc.step_real if mode == "real" else orc.step_imag
    ref_s, ref_l = S(pf, psi0, fine), L(pf, psi0, fine)
    err = {}
    for name, f, ref in (("strang", S, ref_s), ("lie", L, ref_l)):
        e = []
        for n in (4, 8, 16):
            e.append(np.max(np.abs(f(prob_(T / n), psi0, n) - ref)))
        err[name] = e
    rs = [err["strang"][i] / err["strang"][i + 1] for i in range(2)]
    rl = [err["lie"][i] / err["lie"][i + 1] for i in range(2)]
    assert all(3.3 < r < 4.7 for r in rs), (rs, err)
    assert all(1.6 < r < 2.5 for r in rl), (rl, err)


def test_without_potential_and_nonlinearity_both_splittings_are_the_cn_solves(orc):
    p = prob(orc, 0.02, g=0.0, w=(1e-9, 1e-9, 1e-9))
    psi0 = start(orc, p)
    a = orc.step_real_strang(p, psi0, 7)
    b = orc.step_real(p, psi0, 7)
    assert np.max(np.abs(a - b)) <= 1e-13
