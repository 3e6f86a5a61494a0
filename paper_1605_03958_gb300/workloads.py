"""Seeded synthetic workloads of the batched and serving configurations.

Parameter draws only (grids, trap ratios, nonlinearities, arrival times, step
counts); nothing here computes any part of the method.  Both the benchmark and the
tests draw their instances from here.
"""
import numpy as np

H = 0.2
DT = 0.1 * H * H


def batch_instances(count: int = 64, seed: int = 1605):
    """Uneven imaginary-time solves: each extent drawn uniformly from {32, 48, ..., 160},
    trap ratios uniform in [0.5, 3], g log-uniform in [1, 5000]; h = 0.2, dt = 0.1 h^2."""
    rng = np.random.default_rng(seed)
    dims = np.arange(32, 161, 16)
    out = []
    for _ in range(count):
        nx, ny, nz = (int(rng.choice(dims)) for _ in range(3))
        gamma, nu, lam = (float(rng.uniform(0.5, 3.0)) for _ in range(3))
        g = float(np.exp(rng.uniform(0.0, np.log(5000.0))))
        out.append(dict(nx=nx, ny=ny, nz=nz, dx=H, dt=DT, gamma=gamma, nu=nu, lam=lam, g=g))
    return out


def serve_requests(count: int = 2000, rate: float = 200.0, seed: int = 3958):
    """Poisson arrivals (mean `rate` per second): 70 % ground-state requests (2000
    imaginary-time steps), 30 % quench requests (the g = 0 trap Gaussian evolved in
    real time at the request's g for a uniform 500..5000 steps).  Extents: multiples of
    16 in [32, 128] x [32, 96] x [32, 64]; g log-uniform in [1, 1000]; trap ratios
    uniform in [0.5, 3]; h = 0.2, dt = 0.1 h^2."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        ground = bool(rng.uniform() < 0.7)
        nx = int(rng.choice(np.arange(32, 129, 16)))
        ny = int(rng.choice(np.arange(32, 97, 16)))
        nz = int(rng.choice(np.arange(32, 65, 16)))
        gamma, nu, lam = (float(rng.uniform(0.5, 3.0)) for _ in range(3))
        g = float(np.exp(rng.uniform(0.0, np.log(1000.0))))
        steps = 2000 if ground else int(rng.integers(500, 5001))
        reqs.append(dict(id=i, arrival=t, kind="ground" if ground else "quench", steps=steps,
                         params=dict(nx=nx, ny=ny, nz=nz, dx=H, dt=DT, gamma=gamma, nu=nu,
                                     lam=lam, g=g)))
    return reqs
