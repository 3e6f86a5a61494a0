"""C-ABI checks that need no GPU: the library builds, loads, exports every symbol
include/gp.h declares, and its host-only logic (parameter validation, workspace
size, error strings) behaves as documented.  No call here reaches a kernel.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gp.h")


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03958_gb300 as pkg
    return pkg


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("gp_create", "gp_create_on", "gp_destroy", "gp_step_imag", "gp_step_real",
                     "gp_observables", "gp_density1d", "gp_density2d", "gp_set_g",
                     "gp_init_gaussian", "gp_set_psi", "gp_get_psi", "gp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(P):
    lib = ctypes.CDLL(P.gp.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_only_declared_names(P):
    declared = set(declared_functions())
    bound = {n for n in dir(P.gp) if n.startswith("gp_") and not n.endswith("_ptr")}
    assert bound <= declared, bound - declared


def test_params_struct_layout_matches_header(P):
    # gp_params: 3 ints, 7 doubles, int, 4 doubles, int -> natural alignment
    assert ctypes.sizeof(P.gp.GpParams) == 4 * 3 + 4 + 8 * 7 + 4 + 4 + 8 * 4 + 4 + 4
    assert ctypes.sizeof(P.gp.GpObs) == 10 * 8


@pytest.mark.parametrize("bad", [
    dict(nx=2), dict(ny=2049), dict(dx=0.0), dict(dt=-1.0), dict(gamma=0.0),
    dict(g=float("nan")), dict(prec="f16"),
])
def test_invalid_params_are_rejected_on_the_host(P, bad):
    kw = dict(nx=16, ny=12, nz=10, dx=0.2, dt=0.004, gamma=1.0, nu=1.5, lam=2.0, g=5.0, prec="f64")
    kw.update(bad)
    if kw["prec"] not in ("f64", "f32"):
        p = P.make_params(kw["nx"], kw["ny"], kw["nz"], kw["dx"], dt=kw["dt"], g=kw["g"])
        p.prec = 7
    else:
        p = P.make_params(kw["nx"], kw["ny"], kw["nz"], kw["dx"], dt=kw["dt"], gamma=kw["gamma"],
                          nu=kw["nu"], lam=kw["lam"], g=kw["g"], prec=kw["prec"])
    with pytest.raises(P.GPError) as e:
        P.gp_workspace_bytes(p)
    assert e.value.code == P.gp.GP_ERR_ARG
    with pytest.raises(P.GPError) as e:
        P.gp_create(p)   # validation precedes any CUDA call
    assert e.value.code == P.gp.GP_ERR_ARG
    assert P.gp_last_error(None) != ""


def test_workspace_bytes_covers_field_and_staging(P):
    for prec, rb in (("f64", 8), ("f32", 4)):
        p = P.make_params(240, 200, 160, 0.1, gamma=1.0, nu=1.41, lam=2.0, g=100.0, prec=prec)
        n = P.gp_workspace_bytes(p)
        N = 240 * 200 * 160
        assert n >= N * 2 * rb + N * 16      # complex-capable field + FP64 staging
        assert n <= N * 2 * rb * 1.05 + N * 16 + (1 << 22)


def test_physical_units_validation(P):
    p = P.make_params(16, 12, 10, 0.2, natoms=1000.0, a_s=0.005, l_osc=1.0)
    assert P.gp_workspace_bytes(p) > 0
    p.l_osc = 0.0
    with pytest.raises(P.GPError):
        P.gp_workspace_bytes(p)


def test_strerror(P):
    assert P.gp_strerror(0) == "ok"
    assert "non-finite" in P.gp_strerror(P.gp.GP_ERR_NONFINITE)
    assert P.gp_strerror(-99) == "unknown error"


def test_pool_slot_bytes_on_the_host(P):
    """gp_pool_slot_bytes needs no device: field and staging sized for the complex field
    plus the trap tables; invalid parameters are rejected like gp_workspace_bytes."""
    p = P.make_params(96, 80, 64, 0.2, gamma=1.0, nu=1.5, lam=2.0, g=10.0, prec="f32")
    n = P.gp.gp_pool_slot_bytes(p)
    rows = 80 * 64
    assert n >= 2 * 96 * 8 * rows + (96 * 12 + rows * 12)
    assert n < 2 * 96 * 8 * rows * 1.2
    assert n % 256 == 0
    bad = P.make_params(2, 80, 64, 0.2, prec="f32")
    with pytest.raises(P.GPError) as e:
        P.gp.gp_pool_slot_bytes(bad)
    assert e.value.code == P.gp.GP_ERR_ARG


def test_units_helpers(P):
    """Physical units -> g.  Pins independent of the formula's own constants: the
    oscillator length of 87Rb (86.909 u) in a 2 pi x 100 Hz trap is 1.078 um (the
    textbook value for rubidium in such a trap), and g is linear in N and a_s and
    inversely proportional to l_osc; a_s given in metres through gp_params gives the
    same g as a_s in Bohr radii through the helper."""
    import math
    l = P.gp.gp_units_l_osc(86.909, 2 * math.pi * 100.0)
    assert abs(l - 1.0785e-6) / 1.0785e-6 < 1e-3
    g1 = P.gp.gp_units_g(1e4, 100.0, l)
    assert abs(P.gp.gp_units_g(2e4, 100.0, l) - 2 * g1) <= 1e-12 * g1
    assert abs(P.gp.gp_units_g(1e4, 50.0, l) - g1 / 2) <= 1e-12 * g1
    assert abs(P.gp.gp_units_g(1e4, 100.0, 2 * l) - g1 / 2) <= 1e-12 * g1
    assert P.gp.gp_units_g(1e4, -10.0, l) < 0
    # the same-unit path of gp_params: 4 pi N a_s / l_osc with a_s = 100 a0 in metres
    assert abs(g1 - 4 * math.pi * 1e4 * 100 * 5.29177210903e-11 / l) <= 1e-12 * g1
    for bad in ((-1.0, 100.0, l), (1e4, float("nan"), l), (1e4, 100.0, 0.0)):
        with pytest.raises(P.GPError):
            P.gp.gp_units_g(*bad)
    with pytest.raises(P.GPError):
        P.gp.gp_units_l_osc(0.0, 1.0)
