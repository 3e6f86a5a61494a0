"""Plain FP64 CPU oracle for the 3D split-step Crank-Nicolson Gross-Pitaevskii step.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import this package.
It shares no code with the CUDA library in ``paper_1605_03958_gb300``; the two are
checked against each other.

The arithmetic lives in ``gp_oracle.c`` (see its header for the method statement
and the readings of the paper); this module only marshals numpy arrays through
ctypes.  Layout of every field: ``psi[k, j, i]`` (x fastest); complex fields are
numpy complex128 arrays.

Parity status of each function (what pins it, in tests/):
  thomas_coeffs, cn_line  - dense LU / matrix inverse on n <= 12 (test_oracle_thomas)
  step_imag, step_real    - dense Kronecker brute force on tiny grids, exact discrete
                            fixed point at g = 0, closed-form physics
                            (test_oracle_step, test_oracle_physics)
  observables             - dense <psi|H_h|psi> and closed forms (test_oracle_observables)
  density1d, density2d    - brute-force marginals and sum rules (test_oracle_observables)
  g_physical              - scaling invariants only: the paper prints no worked value
  init_gaussian           - separable closed form on the grid
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double), ("nu", ctypes.c_double), ("lam", ctypes.c_double),
        ("g", ctypes.c_double),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Problem)
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_g_physical.argtypes = [ctypes.c_double] * 3
        L.orc_g_physical.restype = ctypes.c_double
        L.orc_coord.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_coord.restype = ctypes.c_double
        L.orc_thomas_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_thomas_coeffs.restype = None
        L.orc_cn_line.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        L.orc_cn_line.restype = None
        L.orc_init_gaussian.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.orc_init_gaussian.restype = None
        L.orc_step_imag.argtypes = [pp, dp, ctypes.c_long]
        L.orc_step_imag.restype = ctypes.c_int
        L.orc_step_real.argtypes = [pp, dp, ctypes.c_long]
        L.orc_step_imag_strang.restype = ctypes.c_int
        L.orc_step_imag_strang.argtypes = [pp, dp, ctypes.c_long]
        L.orc_step_real_strang.restype = ctypes.c_int
        L.orc_step_real_strang.argtypes = [pp, dp, ctypes.c_long]
        L.orc_step_real.restype = ctypes.c_int
        L.orc_observables.argtypes = [pp, dp, ctypes.c_int, dp]
        L.orc_observables.restype = None
        L.orc_density1d.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int, dp]
        L.orc_density1d.restype = None
        L.orc_density2d.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int, dp]
        L.orc_density2d.restype = None
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


OBS_NAMES = ("norm", "mu", "energy", "ekin", "epot", "eint", "rms_x", "rms_y", "rms_z", "rms_r")


@dataclass
class Problem:
    """Grid, trap and nonlinearity of one solve (see gp_oracle.h)."""
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    dt: float
    gamma: float = 1.0
    nu: float = 1.0
    lam: float = 1.0
    g: float = 0.0

    def _c(self) -> _Problem:
        return _Problem(self.nx, self.ny, self.nz, self.hx, self.hy, self.hz, self.dt,
                        self.gamma, self.nu, self.lam, self.g)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def coords(self, axis: int) -> np.ndarray:
        n, h = [(self.nx, self.hx), (self.ny, self.hy), (self.nz, self.hz)][axis]
        return np.array([lib().orc_coord(i, n, h) for i in range(n)])


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def g_physical(natoms: float, a_s: float, l_osc: float) -> float:
    return lib().orc_g_physical(natoms, a_s, l_osc)


def thomas_coeffs(n: int, alpha: complex):
    cp = np.zeros(n, np.complex128)
    m = np.zeros(n, np.complex128)
    lib().orc_thomas_coeffs(n, alpha.real, alpha.imag, _dp(cp), _dp(m))
    return cp, m


def cn_line(v: np.ndarray, alpha: complex) -> np.ndarray:
    out = np.ascontiguousarray(v, dtype=np.complex128).copy()
    lib().orc_cn_line(out.size, complex(alpha).real, complex(alpha).imag, _dp(out))
    return out


def init_gaussian(p: Problem, wx=None, wy=None, wz=None) -> np.ndarray:
    psi = np.zeros(p.shape, np.float64)
    lib().orc_init_gaussian(ctypes.byref(p._c()),
                            p.gamma if wx is None else wx,
                            p.nu if wy is None else wy,
                            p.lam if wz is None else wz, _dp(psi))
    return psi


def step_imag(p: Problem, psi: np.ndarray, nsteps: int) -> np.ndarray:
    out = np.ascontiguousarray(psi, dtype=np.float64).copy()
    assert out.shape == p.shape
    rc = lib().orc_step_imag(ctypes.byref(p._c()), _dp(out), int(nsteps))
    if rc != 0:
        raise FloatingPointError(f"oracle imaginary-time step failed ({rc})")
    return out


def step_real(p: Problem, psi: np.ndarray, nsteps: int) -> np.ndarray:
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    assert out.shape == p.shape
    rc = lib().orc_step_real(ctypes.byref(p._c()), _dp(out), int(nsteps))
    if rc != 0:
        raise FloatingPointError(f"oracle real-time step failed ({rc})")
    return out


def step_imag_strang(p: Problem, psi: np.ndarray, nsteps: int) -> np.ndarray:
    out = np.ascontiguousarray(psi, dtype=np.float64).copy()
    assert out.shape == p.shape
    rc = lib().orc_step_imag_strang(ctypes.byref(p._c()), _dp(out), int(nsteps))
    if rc != 0:
        raise FloatingPointError(f"oracle imaginary-time Strang step failed ({rc})")
    return out


def step_real_strang(p: Problem, psi: np.ndarray, nsteps: int) -> np.ndarray:
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    assert out.shape == p.shape
    rc = lib().orc_step_real_strang(ctypes.byref(p._c()), _dp(out), int(nsteps))
    if rc != 0:
        raise FloatingPointError(f"oracle real-time Strang step failed ({rc})")
    return out


def observables(p: Problem, psi: np.ndarray) -> dict:
    cplx = np.iscomplexobj(psi)
    a = np.ascontiguousarray(psi, dtype=np.complex128 if cplx else np.float64)
    out = np.zeros(10)
    lib().orc_observables(ctypes.byref(p._c()), _dp(a), int(cplx), _dp(out))
    return dict(zip(OBS_NAMES, out.tolist()))


def density1d(p: Problem, psi: np.ndarray, axis: int) -> np.ndarray:
    cplx = np.iscomplexobj(psi)
    a = np.ascontiguousarray(psi, dtype=np.complex128 if cplx else np.float64)
    out = np.zeros([p.nx, p.ny, p.nz][axis])
    lib().orc_density1d(ctypes.byref(p._c()), _dp(a), int(cplx), axis, _dp(out))
    return out


def density2d(p: Problem, psi: np.ndarray, plane: int) -> np.ndarray:
    cplx = np.iscomplexobj(psi)
    a = np.ascontiguousarray(psi, dtype=np.complex128 if cplx else np.float64)
    shape = [(p.ny, p.nx), (p.nz, p.nx), (p.nz, p.ny)][plane]
    out = np.zeros(shape)
    lib().orc_density2d(ctypes.byref(p._c()), _dp(a), int(cplx), plane, _dp(out))
    return out


__all__ = ["Problem", "OBS_NAMES", "lib", "set_threads", "g_physical", "thomas_coeffs",
           "cn_line", "init_gaussian", "step_imag", "step_real", "observables",
           "density1d", "density2d"]
