"""ctypes binding of the C ABI in include/gp.h (libgp_sscn.so).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  The functions carry the C names (gp_create, gp_step_imag, ...); the
``Solver`` class is a convenience wrapper over them that can place the device
workspace in a PyTorch tensor and run on PyTorch's current stream.

There is no CPU fallback: importing this module raises when the library has not
been built, and every call that fails raises ``GPError`` with the library's message.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("GP_SSCN_LIB") or os.path.join(_HERE, "_build", "libgp_sscn.so")

GP_OK = 0
GP_ERR_ARG = -1
GP_ERR_NOMEM = -2
GP_ERR_CUDA = -3
GP_ERR_NONFINITE = -4
GP_ERR_TIMEOUT = -5
GP_ERR_STATE = -6
GP_ERR_BOUNDS = -7
GP_F64 = 0
GP_F32 = 1


class GpParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double), ("nu", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("use_physical", ctypes.c_int),
        ("g", ctypes.c_double),
        ("natoms", ctypes.c_double), ("a_s", ctypes.c_double), ("l_osc", ctypes.c_double),
        ("prec", ctypes.c_int),
    ]


class GpObs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("norm", "mu", "energy", "ekin", "epot", "eint", "rms_x", "rms_y", "rms_z", "rms_r")]


OBS_NAMES = tuple(n for n, _ in GpObs._fields_)


class GPError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{message} (code {code})")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgp_sscn.so; raise if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()' "
            "or python paper_1605_03958_gb300/build.py); there is no CPU fallback")
    L = ctypes.CDLL(path)
    vp, i, d, l, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_longlong
    dp = ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(GpParams)
    sig = {
        "gp_workspace_bytes": (i, [pp, ctypes.POINTER(ctypes.c_size_t)]),
        "gp_create": (i, [pp, vp, ctypes.POINTER(vp)]),
        "gp_create_on": (i, [pp, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
        "gp_destroy": (None, [vp]),
        "gp_init_gaussian": (i, [vp, d, d, d]),
        "gp_set_psi": (i, [vp, vp, i]),
        "gp_get_psi": (i, [vp, vp, i]),
        "gp_set_psi_f32": (i, [vp, vp, i]),
        "gp_get_psi_f32": (i, [vp, vp, i]),
        "gp_get_psi_f32_async": (i, [vp, vp, i]),
        "gp_set_psi_f32_async": (i, [vp, vp, i]),
        "gp_step_imag": (i, [vp, l]),
        "gp_step_real": (i, [vp, l]),
        "gp_set_g": (i, [vp, d]),
        "gp_set_splitting": (i, [vp, i]),
        "gp_get_g": (i, [vp, dp]),
        "gp_observables": (i, [vp, ctypes.POINTER(GpObs)]),
        "gp_density1d": (i, [vp, i, dp]),
        "gp_density2d": (i, [vp, i, dp]),
        "gp_sync": (i, [vp]),
        "gp_set_wait_limit": (i, [vp, ctypes.c_longlong]),
        "gp_set_timing": (i, [vp, i]),
        "gp_get_timing": (i, [vp, dp, ctypes.POINTER(ll)]),
        "gp_get_info": (i, [vp, ctypes.POINTER(ll)]),
        "gp_observables_noalloc": (i, [vp, i, i, i, ll, i, i, d, d, d, d, d, d, d, vp, vp]),
        "gp_last_error": (ctypes.c_char_p, [vp]),
        "gp_strerror": (ctypes.c_char_p, [i]),
        "gp_units_g": (i, [d, d, d, dp]),
        "gp_units_l_osc": (i, [d, d, dp]),
        "gp_pool_slot_bytes": (i, [pp, ctypes.POINTER(ctypes.c_size_t)]),
        "gp_pool_create": (i, [ctypes.c_size_t, i, vp, ctypes.POINTER(vp)]),
        "gp_pool_destroy": (None, [vp]),
        "gp_pool_free_bytes": (i, [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
        "gp_pool_add": (i, [vp, pp, ctypes.POINTER(i)]),
        "gp_pool_remove": (i, [vp, i]),
        "gp_pool_set_real_time": (i, [vp, i]),
        "gp_pool_set_g": (i, [vp, i, d]),
        "gp_pool_step": (i, [vp, l]),
        "gp_pool_observables": (i, [vp, i, ctypes.POINTER(GpObs)]),
        "gp_pool_get_psi": (i, [vp, i, vp, i]),
        "gp_pool_set_psi": (i, [vp, i, vp, i]),
        "gp_pool_set_shape": (i, [vp, i, i]),
        "gp_pool_tune": (i, [vp, i, dp]),
        "gp_pool_set_graph": (i, [vp, i]),
        "gp_pool_info": (i, [vp, ctypes.POINTER(ll)]),
        "gp_pool_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc: int, handle=None) -> None:
    if rc != GP_OK:
        msg = load_library().gp_last_error(handle).decode()
        raise GPError(rc, msg)


def make_params(nx, ny, nz, dx, dy=None, dz=None, dt=None, gamma=1.0, nu=1.0, lam=1.0,
                g=0.0, natoms=None, a_s=None, l_osc=None, prec="f64") -> GpParams:
    """gp_params from keyword values; g = 4 pi N a_s / l_osc when natoms is given."""
    dy = dx if dy is None else dy
    dz = dx if dz is None else dz
    dt = 0.1 * dx * dx if dt is None else dt
    phys = natoms is not None
    return GpParams(nx, ny, nz, dx, dy, dz, dt, gamma, nu, lam, int(phys), 0.0 if phys else g,
                    natoms or 0.0, a_s or 0.0, l_osc or 1.0,
                    {"f64": GP_F64, "f32": GP_F32}[prec])


# --------------------------------------------------------------- C-named calls

def gp_workspace_bytes(p: GpParams) -> int:
    n = ctypes.c_size_t()
    _check(load_library().gp_workspace_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def gp_create(p: GpParams, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().gp_create(ctypes.byref(p), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def gp_create_on(p: GpParams, dev_ptr: int, nbytes: int, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().gp_create_on(ctypes.byref(p), ctypes.c_void_p(dev_ptr), nbytes,
                                       ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def gp_destroy(h) -> None:
    load_library().gp_destroy(h)


def gp_init_gaussian(h, wx: float, wy: float, wz: float) -> None:
    _check(load_library().gp_init_gaussian(h, wx, wy, wz), h)


def gp_set_psi(h, host: np.ndarray) -> None:
    """host: numpy float64 (real field) or complex128 (complex field), C-contiguous,
    shape (nz, ny, nx); or any object with a host address via ``host_ptr`` (pinned)."""
    a = np.ascontiguousarray(host)
    cplx = np.iscomplexobj(a)
    a = a.astype(np.complex128 if cplx else np.float64, copy=False)
    _check(load_library().gp_set_psi(h, a.ctypes.data_as(ctypes.c_void_p), int(cplx)), h)


def gp_set_psi_ptr(h, host_ptr: int, is_complex: bool) -> None:
    """Same as gp_set_psi from a raw host address (e.g. a pinned torch tensor)."""
    _check(load_library().gp_set_psi(h, ctypes.c_void_p(host_ptr), int(is_complex)), h)


def gp_get_psi(h, shape, as_complex: bool = False) -> np.ndarray:
    out = np.empty(shape, np.complex128 if as_complex else np.float64)
    _check(load_library().gp_get_psi(h, out.ctypes.data_as(ctypes.c_void_p), int(as_complex)), h)
    return out


def gp_get_psi_ptr(h, host_ptr: int, as_complex: bool) -> None:
    _check(load_library().gp_get_psi(h, ctypes.c_void_p(host_ptr), int(as_complex)), h)


def gp_set_psi_f32(h, host: np.ndarray) -> None:
    """FP32 solvers: host float32 (real field) or complex64 (complex field), shape
    (nz, ny, nx), copied straight into the device field."""
    a = np.ascontiguousarray(host)
    cplx = np.iscomplexobj(a)
    a = a.astype(np.complex64 if cplx else np.float32, copy=False)
    _check(load_library().gp_set_psi_f32(h, a.ctypes.data_as(ctypes.c_void_p), int(cplx)), h)


def gp_get_psi_f32(h, shape, as_complex: bool = False) -> np.ndarray:
    out = np.empty(shape, np.complex64 if as_complex else np.float32)
    _check(load_library().gp_get_psi_f32(h, out.ctypes.data_as(ctypes.c_void_p), int(as_complex)), h)
    return out


def gp_set_psi_f32_ptr(h, host_ptr: int, is_complex: bool) -> None:
    """gp_set_psi_f32 from a raw host address (e.g. a pinned torch float32 tensor)."""
    _check(load_library().gp_set_psi_f32(h, ctypes.c_void_p(host_ptr), int(is_complex)), h)


def gp_get_psi_f32_ptr(h, host_ptr: int, as_complex: bool) -> None:
    _check(load_library().gp_get_psi_f32(h, ctypes.c_void_p(host_ptr), int(as_complex)), h)


def gp_set_psi_f32_async_ptr(h, host_ptr: int, is_complex: bool) -> None:
    """Overlapped write from caller host memory (page-locked for overlap), taken into
    the field by the next call that touches it; the buffer may be changed once a
    synchronising call (gp_sync(h), a synchronous read, observables) has returned."""
    _check(load_library().gp_set_psi_f32_async(h, ctypes.c_void_p(host_ptr), int(is_complex)), h)


def gp_get_psi_f32_async_ptr(h, host_ptr: int, as_complex: bool) -> None:
    """Overlapped read into caller host memory (page-locked for overlap); the buffer
    is complete after gp_sync(h)."""
    _check(load_library().gp_get_psi_f32_async(h, ctypes.c_void_p(host_ptr), int(as_complex)), h)


def gp_step_imag(h, nsteps: int) -> None:
    _check(load_library().gp_step_imag(h, int(nsteps)), h)


def gp_step_real(h, nsteps: int) -> None:
    _check(load_library().gp_step_real(h, int(nsteps)), h)


def gp_set_g(h, g: float) -> None:
    _check(load_library().gp_set_g(h, float(g)), h)


GP_SPLIT_LIE = 0
GP_SPLIT_STRANG = 1


def gp_set_splitting(h, scheme: int) -> None:
    _check(load_library().gp_set_splitting(h, int(scheme)), h)


def gp_get_g(h) -> float:
    v = ctypes.c_double()
    _check(load_library().gp_get_g(h, ctypes.byref(v)), h)
    return v.value


def gp_observables(h) -> dict:
    o = GpObs()
    _check(load_library().gp_observables(h, ctypes.byref(o)), h)
    return {n: getattr(o, n) for n in OBS_NAMES}


def gp_density1d(h, axis: int, n: int) -> np.ndarray:
    out = np.empty(n)
    _check(load_library().gp_density1d(h, axis, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), h)
    return out


def gp_density2d(h, plane: int, shape) -> np.ndarray:
    out = np.empty(shape)
    _check(load_library().gp_density2d(h, plane, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), h)
    return out


def gp_sync(h) -> None:
    _check(load_library().gp_sync(h), h)


def gp_set_wait_limit(h, first_wait_ns: int) -> None:
    _check(load_library().gp_set_wait_limit(h, int(first_wait_ns)), h)


def gp_set_timing(h, enable: bool) -> None:
    _check(load_library().gp_set_timing(h, int(enable)), h)


def gp_get_timing(h):
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_longlong * 3)()
    _check(load_library().gp_get_timing(h, ms, n), h)
    return list(ms), list(n)


def gp_get_info(h) -> dict:
    v = (ctypes.c_longlong * 8)()
    _check(load_library().gp_get_info(h, v), h)
    keys = ("pitch", "is_complex", "lines_x", "lines_y", "lines_z", "bytes", "fast_mask",
            "trunc")
    d = dict(zip(keys, list(v)))
    d["band_mask"] = (d["fast_mask"] >> 3) & 7
    d["band_w"] = (d["fast_mask"] >> 8) & 15
    d["line64_mask"] = (d["fast_mask"] >> 12) & 7
    d["x_reg"] = (d["fast_mask"] >> 15) & 1
    d["fast_mask"] &= 7
    return d


def gp_observables_noalloc(psi_ptr: int, nx: int, ny: int, nz: int, pitch: int, prec: int,
                           is_complex: bool, dx: float, dy: float, dz: float, gamma: float,
                           nu: float, lam: float, g: float, out_ptr: int, stream: int = 0) -> None:
    """Observables of a field in the caller's device memory into 10 doubles of the
    caller's device memory, without any device allocation (see include/gp.h)."""
    rc = load_library().gp_observables_noalloc(
        ctypes.c_void_p(psi_ptr), nx, ny, nz, pitch, prec, int(is_complex), dx, dy, dz,
        gamma, nu, lam, g, ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))
    _check(rc)


def gp_last_error(h=None) -> str:
    return load_library().gp_last_error(h).decode()


def gp_strerror(code: int) -> str:
    return load_library().gp_strerror(code).decode()


# ------------------------------------------------------------------ wrapper

@dataclass
class Solver:
    """One GP solve on the current CUDA device.

    By default the workspace is a PyTorch uint8 tensor and the stream is PyTorch's
    current stream (``use_torch=True``); with ``use_torch=False`` the library
    allocates with cudaMalloc and uses the legacy default stream.
    """
    nx: int
    ny: int
    nz: int
    dx: float
    dy: Optional[float] = None
    dz: Optional[float] = None
    dt: Optional[float] = None
    gamma: float = 1.0
    nu: float = 1.0
    lam: float = 1.0
    g: float = 0.0
    natoms: Optional[float] = None
    a_s: Optional[float] = None
    l_osc: Optional[float] = None
    prec: str = "f64"
    use_torch: bool = True
    stream: Optional[int] = None
    handle: ctypes.c_void_p = field(init=False, default=None)
    _buf: object = field(init=False, default=None, repr=False)

    def __post_init__(self):
        self.params = make_params(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.dt,
                                  self.gamma, self.nu, self.lam, self.g, self.natoms, self.a_s,
                                  self.l_osc, self.prec)
        if self.use_torch:
            import torch
            nbytes = gp_workspace_bytes(self.params)
            self._buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            st = torch.cuda.current_stream().cuda_stream if self.stream is None else self.stream
            self.handle = gp_create_on(self.params, self._buf.data_ptr(), nbytes, st)
        else:
            self.handle = gp_create(self.params, self.stream or 0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def close(self):
        if self.handle:
            gp_destroy(self.handle)
            self.handle = None
            self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_gaussian(self, wx=None, wy=None, wz=None):
        p = self.params
        gp_init_gaussian(self.handle, p.gamma if wx is None else wx, p.nu if wy is None else wy,
                         p.lambda_ if wz is None else wz)

    def set_psi(self, psi):
        gp_set_psi(self.handle, psi)

    def get_psi(self, as_complex=False):
        return gp_get_psi(self.handle, self.shape, as_complex)

    def step_imag(self, n):
        gp_step_imag(self.handle, n)

    def step_real(self, n):
        gp_step_real(self.handle, n)

    def set_g(self, g):
        gp_set_g(self.handle, g)

    def set_splitting(self, scheme: str):
        gp_set_splitting(self.handle, {"lie": GP_SPLIT_LIE, "strang": GP_SPLIT_STRANG}[scheme])

    def get_g(self):
        return gp_get_g(self.handle)

    def observables(self):
        return gp_observables(self.handle)

    def density1d(self, axis):
        return gp_density1d(self.handle, axis, [self.nx, self.ny, self.nz][axis])

    def density2d(self, plane):
        shape = [(self.ny, self.nx), (self.nz, self.nx), (self.nz, self.ny)][plane]
        return gp_density2d(self.handle, plane, shape)

    def sync(self):
        gp_sync(self.handle)

    def info(self):
        return gp_get_info(self.handle)


# --------------------------------------------------------------------- units

def gp_units_g(natoms: float, a_s_bohr: float, l_osc_m: float) -> float:
    """g = 4 pi N a_s / l_osc, a_s in Bohr radii, l_osc in metres."""
    v = ctypes.c_double()
    _check(load_library().gp_units_g(float(natoms), float(a_s_bohr), float(l_osc_m), ctypes.byref(v)))
    return v.value


def gp_units_l_osc(mass_amu: float, omega: float) -> float:
    """Oscillator length sqrt(hbar / (m omega)) in metres (mass in u, omega in rad/s)."""
    v = ctypes.c_double()
    _check(load_library().gp_units_l_osc(float(mass_amu), float(omega), ctypes.byref(v)))
    return v.value


# --------------------------------------------------------------------- pools

def _pcheck(rc: int, pool=None) -> None:
    if rc != GP_OK:
        raise GPError(rc, load_library().gp_pool_last_error(pool).decode())


def gp_pool_slot_bytes(p: GpParams) -> int:
    n = ctypes.c_size_t()
    _check(load_library().gp_pool_slot_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def gp_pool_create(arena_bytes: int, max_slots: int, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().gp_pool_create(arena_bytes, max_slots, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def gp_pool_destroy(pool) -> None:
    load_library().gp_pool_destroy(pool)


def gp_pool_free_bytes(pool):
    f, g = ctypes.c_size_t(), ctypes.c_size_t()
    _pcheck(load_library().gp_pool_free_bytes(pool, ctypes.byref(f), ctypes.byref(g)), pool)
    return f.value, g.value


def gp_pool_add(pool, p: GpParams) -> int:
    slot = ctypes.c_int()
    _pcheck(load_library().gp_pool_add(pool, ctypes.byref(p), ctypes.byref(slot)), pool)
    return slot.value


def gp_pool_remove(pool, slot: int) -> None:
    _pcheck(load_library().gp_pool_remove(pool, slot), pool)


def gp_pool_set_real_time(pool, slot: int) -> None:
    _pcheck(load_library().gp_pool_set_real_time(pool, slot), pool)


def gp_pool_set_g(pool, slot: int, g: float) -> None:
    _pcheck(load_library().gp_pool_set_g(pool, slot, float(g)), pool)


def gp_pool_step(pool, nsteps: int) -> None:
    _pcheck(load_library().gp_pool_step(pool, int(nsteps)), pool)


def gp_pool_observables(pool, slot: int) -> dict:
    o = GpObs()
    _pcheck(load_library().gp_pool_observables(pool, slot, ctypes.byref(o)), pool)
    return {n: getattr(o, n) for n in OBS_NAMES}


def gp_pool_get_psi(pool, slot: int, shape, as_complex: bool = False) -> np.ndarray:
    out = np.empty(shape, np.complex128 if as_complex else np.float64)
    _pcheck(load_library().gp_pool_get_psi(pool, slot, out.ctypes.data_as(ctypes.c_void_p), int(as_complex)), pool)
    return out


def gp_pool_set_psi(pool, slot: int, host: np.ndarray) -> None:
    a = np.ascontiguousarray(host)
    cplx = np.iscomplexobj(a)
    a = a.astype(np.complex128 if cplx else np.float64, copy=False)
    _pcheck(load_library().gp_pool_set_psi(pool, slot, a.ctypes.data_as(ctypes.c_void_p), int(cplx)), pool)


def gp_pool_set_shape(pool, x_stages: int, seg_turns: int) -> None:
    _pcheck(load_library().gp_pool_set_shape(pool, x_stages, seg_turns), pool)


def gp_pool_tune(pool, steps_per_candidate: int = 5) -> float:
    ms = ctypes.c_double()
    _pcheck(load_library().gp_pool_tune(pool, steps_per_candidate, ctypes.byref(ms)), pool)
    return ms.value


def gp_pool_set_graph(pool, enable: bool) -> None:
    _pcheck(load_library().gp_pool_set_graph(pool, int(enable)), pool)


def gp_pool_info(pool) -> dict:
    v = (ctypes.c_longlong * 8)()
    _pcheck(load_library().gp_pool_info(pool, v), pool)
    keys = ("live", "bytes_used", "x_stages", "seg_turns", "graph", "launches_per_step",
            "free_bytes", "largest_free")
    d = dict(zip(keys, list(v)))
    d["x_reg"] = (d["graph"] >> 1) & 1
    d["x_reg_complex"] = (d["graph"] >> 2) & 1
    d["graph"] &= 1
    return d


class Pool:
    """Resident FP32 solves of different grids stepped together (see include/gp.h).
    Slots are added with the keyword parameters of ``make_params``."""

    def __init__(self, arena_bytes: int, max_slots: int = 256, stream: Optional[int] = None):
        self.handle = gp_pool_create(int(arena_bytes), int(max_slots), stream or 0)
        self.shapes = {}

    def close(self):
        if self.handle:
            gp_pool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def slot_bytes(**kw) -> int:
        kw.setdefault("prec", "f32")
        return gp_pool_slot_bytes(make_params(**kw))

    def add(self, **kw) -> int:
        kw.setdefault("prec", "f32")
        p = make_params(**kw)
        slot = gp_pool_add(self.handle, p)
        self.shapes[slot] = (p.nz, p.ny, p.nx)
        return slot

    def remove(self, slot):
        gp_pool_remove(self.handle, slot)
        self.shapes.pop(slot, None)

    def set_real_time(self, slot):
        gp_pool_set_real_time(self.handle, slot)

    def set_g(self, slot, g):
        gp_pool_set_g(self.handle, slot, g)

    def step(self, n):
        gp_pool_step(self.handle, n)

    def observables(self, slot):
        return gp_pool_observables(self.handle, slot)

    def get_psi(self, slot, as_complex=False):
        return gp_pool_get_psi(self.handle, slot, self.shapes[slot], as_complex)

    def set_psi(self, slot, psi):
        gp_pool_set_psi(self.handle, slot, psi)

    def set_shape(self, x_stages, seg_turns):
        gp_pool_set_shape(self.handle, x_stages, seg_turns)

    def tune(self, steps_per_candidate=5):
        return gp_pool_tune(self.handle, steps_per_candidate)

    def set_graph(self, enable):
        gp_pool_set_graph(self.handle, enable)

    def free_bytes(self):
        return gp_pool_free_bytes(self.handle)

    def info(self):
        return gp_pool_info(self.handle)
