"""Write the full-length oracle fixtures of the paper-scale configurations.

Calls only the FP64 CPU oracle (``oracle/``); no value here comes from the CUDA
library.  Each fixture is a JSON file beside this script:

  c2_g{0,100,2000}.json  imaginary-time ground state, 240x200x160, h = 0.1,
                         dt = 0.1 h^2, trap (1, 1.41, 2), 10^4 steps from the
                         normalised trap Gaussian (paper: "Solution method",
                         imaginary-time propagation with renormalisation);
  c3_quench.json         the g = 100 state above, then g -> 200 and 2*10^4
                         real-time steps at dt = 0.02 h^2 (paper: "Summary of
                         revisions", the NRUN quench of the nonlinearity), with the
                         observables every 100 steps.

Each file holds the observables, the three 1D integrated densities (Eq. 1 and its
analogues), and psi on a fixed sub-lattice (every 10th x, 10th y and 8th z point)
plus 512 seeded random points, with the sha256 of the oracle's source files.

Usage (about 4 hours on 8 cores): python tests/golden/make_golden.py [--threads 8]
A fixture whose oracle hash matches the current sources is not recomputed.
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

GRID = (240, 200, 160)
H = 0.1
TRAP = (1.0, 1.41, 2.0)
DT_IMAG = 0.1 * H * H
DT_REAL = 0.02 * H * H
STEPS_IMAG = 10_000
STEPS_REAL = 20_000
RECORD_EVERY = 100
SUB = (10, 10, 8)  # sub-lattice strides along x, y, z
N_RANDOM = 512
SEED = 1605


def oracle_hash() -> str:
    h = hashlib.sha256()
    for name in ("gp_oracle.c", "gp_oracle.h"):
        with open(os.path.join(ROOT, "oracle", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def problem(dt, g):
    nx, ny, nz = GRID
    return oracle.Problem(nx, ny, nz, H, H, H, dt, gamma=TRAP[0], nu=TRAP[1], lam=TRAP[2], g=g)


def sample_points():
    """Flat indices (k*ny + j)*nx + i of the sub-lattice, then the random points."""
    nx, ny, nz = GRID
    k, j, i = np.meshgrid(np.arange(0, nz, SUB[2]), np.arange(0, ny, SUB[1]),
                          np.arange(0, nx, SUB[0]), indexing="ij")
    lattice = ((k * ny + j) * nx + i).ravel()
    rng = np.random.default_rng(SEED)
    rand = rng.integers(0, nx * ny * nz, N_RANDOM)
    return np.concatenate([lattice, rand]).astype(np.int64)


def pack(a):
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return {"re": [float(x) for x in a.real.ravel()], "im": [float(x) for x in a.imag.ravel()]}
    return [float(x) for x in a.ravel()]


def summary(p, psi, idx):
    return {
        "observables": oracle.observables(p, psi),
        "density1d": [pack(oracle.density1d(p, psi, a)) for a in range(3)],
        "psi_samples": pack(psi.ravel()[idx]),
    }


def write(name, payload):
    path = os.path.join(HERE, name)
    with open(path + ".tmp", "w") as f:
        json.dump(payload, f, separators=(",", ":"))
    os.replace(path + ".tmp", path)
    print(f"wrote {path}", flush=True)


def up_to_date(name, ohash):
    path = os.path.join(HERE, name)
    if not os.path.exists(path):
        return False
    with open(path) as f:
        return json.load(f).get("oracle_sha256") == ohash


def common(ohash, idx):
    return {"oracle_sha256": ohash, "grid": list(GRID), "h": H, "trap": list(TRAP),
            "sub_lattice_strides_xyz": list(SUB), "n_random": N_RANDOM, "seed": SEED,
            "sample_index": [int(x) for x in idx],
            "command": "python tests/golden/make_golden.py"}


def ground_state(g):
    p = problem(DT_IMAG, g)
    t0 = time.time()
    psi = oracle.step_imag(p, oracle.init_gaussian(p), STEPS_IMAG)
    print(f"g = {g}: {STEPS_IMAG} imaginary steps in {time.time() - t0:.0f} s", flush=True)
    return p, psi


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--only", nargs="*", default=None)
    args = ap.parse_args()
    oracle.set_threads(args.threads)
    ohash = oracle_hash()
    idx = sample_points()
    want = args.only or ["c2_g100", "c3_quench", "c2_g2000", "c2_g0"]
    gs100 = None
    for case in want:
        name = case + ".json"
        if up_to_date(name, ohash):
            print(f"{name} is up to date", flush=True)
            continue
        if case.startswith("c2_g"):
            g = float(case[4:])
            p, psi = ground_state(g)
            if g == 100.0:
                gs100 = psi
            write(name, dict(common(ohash, idx), config="imag3d ground state", g=g,
                             dt=DT_IMAG, steps=STEPS_IMAG, **summary(p, psi, idx)))
        elif case == "c3_quench":
            if gs100 is None:
                _, gs100 = ground_state(100.0)
            q = problem(DT_REAL, 200.0)
            psi = gs100.astype(np.complex128)
            traj = [oracle.observables(q, psi)]
            t0 = time.time()
            for _ in range(STEPS_REAL // RECORD_EVERY):
                psi = oracle.step_real(q, psi, RECORD_EVERY)
                traj.append(oracle.observables(q, psi))
            print(f"quench: {STEPS_REAL} real steps in {time.time() - t0:.0f} s", flush=True)
            write(name, dict(common(ohash, idx), config="real3d quench", g_imag=100.0,
                             dt_imag=DT_IMAG, steps_imag=STEPS_IMAG, g=200.0, dt=DT_REAL,
                             steps=STEPS_REAL, record_every=RECORD_EVERY,
                             trajectory={k: [o[k] for o in traj] for k in oracle.OBS_NAMES},
                             **summary(q, psi, idx)))
        else:
            raise SystemExit(f"unknown case {case}")


if __name__ == "__main__":
    main()
