"""gp_observables_noalloc: observables of a field in the caller's device memory with
no device allocation, for callers that cannot call cudaMalloc (it synchronises the
device, it can fail while another allocator holds the free memory, and some plugin
hosts forbid it).  Its scratch is a fixed array inside the library shared by all
calls, so this test makes two calls in a row and checks that each one matches the
FP64 CPU oracle on the same (rounded) field and the solver's own gp_observables, on
3D fields and on 2D fields (nz = 1), real and complex, FP64 and FP32.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FIELDS = [((37, 29, 23), 0.3, 0.25, 0.4), ((64, 48, 32), 0.2, 0.2, 0.2),
          ((40, 33, 1), 0.2, 0.25, 0.3)]
TOL = 1e-13


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03958_gb300 as pkg
    return pkg


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("cplx", [False, True])
def test_two_calls_match_oracle_and_gp_observables(P, orc, prec, cplx):
    import torch
    rng = np.random.default_rng(2024)
    trap, g = (1.1, 1.7, 0.6), 9.0
    stream = torch.cuda.current_stream()
    for (nx, ny, nz), hx, hy, hz in FIELDS:
        psi = rng.standard_normal((nz, ny, nx))
        if cplx:
            psi = psi + 1j * rng.standard_normal((nz, ny, nx))
        if prec == "f32":  # the oracle sees exactly the values the device holds
            psi = psi.astype(np.complex64 if cplx else np.float32).astype(psi.dtype)
        p = orc.Problem(nx, ny, nz, hx, hy, hz, 0.01, gamma=trap[0], nu=trap[1], lam=trap[2], g=g)
        ref = orc.observables(p, psi)
        # the existing entry point, on a solver holding the same field
        s = P.Solver(nx, ny, nz, hx, hy, hz, 0.01, *trap, g=g, prec=prec)
        s.set_psi(psi)
        want = s.observables()
        s.close()
        # the same field in a caller-owned device buffer, padded pitch
        pitch = nx + 3
        host = np.zeros((nz, ny, pitch), psi.dtype)
        host[:, :, :nx] = psi
        if prec == "f32":
            host = host.astype(np.complex64 if cplx else np.float32)
        dev = torch.from_numpy(host).cuda()
        for call in range(2):
            out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
            P.gp.gp_observables_noalloc(dev.data_ptr(), nx, ny, nz, pitch,
                                        P.gp.GP_F64 if prec == "f64" else P.gp.GP_F32, cplx,
                                        hx, hy, hz, *trap, g, out.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            got = dict(zip(P.gp.OBS_NAMES, out.cpu().tolist()))
            for k in P.gp.OBS_NAMES:
                if nz == 1 and k == "rms_z":
                    assert got[k] == 0.0 and ref[k] == 0.0
                    continue
                assert abs(got[k] - ref[k]) <= TOL * abs(ref[k]), (call, nz, k, got[k], ref[k])
                assert abs(got[k] - want[k]) <= TOL * abs(want[k]), (call, nz, k, got[k], want[k])


@pytest.mark.parametrize("shape", [(4096, 3, 3), (2, 3, 3), (3, 2, 3), (3, 3, 2)])
def test_rejects_extents_outside_the_solver_range(P, shape):
    import torch
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    dev = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    nx, ny, nz = shape
    with pytest.raises(P.GPError) as e:
        P.gp.gp_observables_noalloc(dev.data_ptr(), nx, ny, nz, nx, P.gp.GP_F64, False,
                                    0.1, 0.1, 0.1, 1.0, 1.0, 1.0, 0.0, out.data_ptr(), 0)
    assert e.value.code == P.gp.GP_ERR_ARG
    assert "2048" in P.gp_last_error(None)
