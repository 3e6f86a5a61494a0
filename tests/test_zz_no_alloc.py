"""gp_observables_noalloc: observables of a field in the caller's device memory with
no device allocation, for callers that cannot call cudaMalloc (it synchronises the
device, it can fail while another allocator holds the free memory, and some plugin
hosts forbid it).  Its scratch is a fixed array inside the library shared by all
calls, so this test makes two calls in a row and checks that each one matches the
solver's own gp_observables on the same field.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FIELDS = [((37, 29, 23), 0.3, 0.25, 0.4), ((64, 48, 32), 0.2, 0.2, 0.2)]


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
def test_two_calls_match_gp_observables(P, prec, cplx):
    import torch
    rng = np.random.default_rng(2024)
    trap, g = (1.1, 1.7, 0.6), 9.0
    stream = torch.cuda.current_stream()
    for (nx, ny, nz), hx, hy, hz in FIELDS:
        psi = rng.standard_normal((nz, ny, nx))
        if cplx:
            psi = psi + 1j * rng.standard_normal((nz, ny, nx))
        # the existing entry point, on a solver holding the same field
        s = P.Solver(nx, ny, nz, hx, hy, hz, 0.01, *trap, g=g, prec=prec)
        s.set_psi(psi)
        want = s.observables()
        s.close()
        # the same field (same rounding) in a caller-owned device buffer, padded pitch
        pitch = nx + 3
        host = np.zeros((nz, ny, pitch), psi.dtype)
        host[:, :, :nx] = psi
        if prec == "f32":
            host = host.astype(np.complex64 if cplx else np.float32)
        dev = torch.from_numpy(host).cuda()
        out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
        P.gp.gp_observables_noalloc(dev.data_ptr(), nx, ny, nz, pitch,
                                    P.gp.GP_F64 if prec == "f64" else P.gp.GP_F32, cplx,
                                    hx, hy, hz, *trap, g, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = dict(zip(P.gp.OBS_NAMES, out.cpu().tolist()))
        for k in P.gp.OBS_NAMES:
            assert abs(got[k] - want[k]) <= 1e-13 * abs(want[k]), (k, got[k], want[k])


def test_rejects_sizes_beyond_the_maximum(P):
    import torch
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    dev = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(P.GPError) as e:
        P.gp.gp_observables_noalloc(dev.data_ptr(), 4096, 2, 2, 4096, P.gp.GP_F64, False,
                                    0.1, 0.1, 0.1, 1.0, 1.0, 1.0, 0.0, out.data_ptr(), 0)
    assert e.value.code == P.gp.GP_ERR_ARG
    assert "2048" in P.gp_last_error(None)
