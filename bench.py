"""Benchmark: grid-point SSCN steps per second of the 3D Gross-Pitaevskii solver.

Workload (paper-scale imaginary-time ground state): grid 240 x 200 x 160, h = 0.1
(box centred on the origin), dt = 0.1 h^2, trap ratios (1, 1.41, 2), g = 100, field
stored in FP32 (default) or FP64 with FP64 reductions, started from the g = 0 trap
Gaussian.  One benchmark step is one full SSCN time step: pointwise substep, CN
sweeps along x, y and z, norm and renormalisation factor.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the
solver's stream; between timed steps (outside the events) a 256 MiB device buffer is
written and another 256 MiB read, so that every step starts with a cold L2 (the FP32
field is 31 MB, below the 129 MB L2).  Per-sweep durations come from a second pass
with the library's own events on the same stream.
`value` = (ranks x grid points x K) / max over ranks of the summed step time.

Multi-GPU: every rank runs an independent replica of the solve (the solve itself
does not shard), so scaling is weak and no collective touches the data path.

`--impl reference` times the CPU oracle (plain FP64 C, OpenMP over independent
line solves) on the same metric, each step a z-slab sample of the same grid.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY, NZ, H = 240, 200, 160, 0.1
DT = 0.1 * H * H
TRAP = (1.0, 1.41, 2.0)
G = 100.0
NPTS = NX * NY * NZ
FLUSH_BYTES = 256 << 20
WORKLOAD = "imag3d 240x200x160, h=0.1, dt=0.1h^2, trap (1,1.41,2), g=100, imaginary time"


def parse():
    global NX, NY, NZ, NPTS, WORKLOAD, DT
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--prec", choices=["f32", "f64"], default="f32")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--f64-steps", type=int, default=300,
                    help="context: timed steps of the FP64 imaginary-time solve (complex128 "
                         "real time: a third of them)")
    ap.add_argument("--no-context", dest="context", action="store_false",
                    help="skip the context lines (paper precision, DRAM-bound grid, shortened "
                         "batched and served workloads)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["single", "batch", "serve", "c1"], default="single",
                    help="single: the 240x200x160 solve (default); batch: 64 uneven FP32 "
                         "solves resident in one pool; serve: the continuous-batching server "
                         "on a Poisson request stream; c1: the plain FP64 64x48x32 ground "
                         "state (2000 steps, L2-resident, steps/s and observables vs the oracle)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-compare", type=int, default=100,
                    help="serve: leading requests also served one at a time in FP64 and FP32")
    ap.add_argument("--batch-single-steps", type=int, default=200,
                    help="batch: steps per instance timed for the one-at-a-time baselines")
    ap.add_argument("--splitting", choices=["lie", "strang"], default="lie",
                    help="splitting of a step (single workload)")
    ap.add_argument("--mode", choices=["imag", "real"], default="imag",
                    help="single workload: imag (ground state, default) or real: the quench "
                         "dynamics workload (dt = 0.02 h^2; 300 imaginary steps at g = 100 from "
                         "the Gaussian, then g = 200 and timed real-time steps on the complex field)")
    ap.add_argument("--grid", type=int, nargs=3, default=None,
                    help="override the grid (profiling of out-of-L2 cases); h and dt unchanged")
    args = ap.parse_args()
    if args.mode == "real":
        DT = 0.02 * H * H
        WORKLOAD = ("real3d 240x200x160, h=0.1, dt=0.02h^2, trap (1,1.41,2), ground state at "
                    "g=100 then quench to g=200, real time")
    if args.grid:
        NX, NY, NZ = args.grid
        NPTS = NX * NY * NZ
        WORKLOAD = WORKLOAD.replace("240x200x160", f"{NX}x{NY}x{NZ}")
        if NZ == 1:
            WORKLOAD = WORKLOAD.replace("imag3d", "imag2d")
    return args


# ------------------------------------------------------------------ helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.06)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash():
    """Hash of the code (comments and blank space removed) of the files that define the
    sweep kernels and their launch shapes: ncu figures stay tied to the code they were
    taken on, and an edit of a comment does not void them."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("gp_sweeps.cu", "gp_sweeps64.cu", "gp_device.cuh", "gp_internal.h", "gp_api.cu"):
        with open(os.path.join(ROOT, "paper_1605_03958_gb300", "csrc", f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch_full_size")


def replica_throughput(local_ms, units_per_rank, group=None, device=None):
    """Whole-job throughput of independent replicas: every rank processed
    `units_per_rank` units in `local_ms`; the job took the slowest rank's time.
    Returns (units / s over all ranks, max ms over ranks)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    ms = float(local_ms)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        ms = float(t.item())
    return world * units_per_rank / (ms / 1e3), ms


# ------------------------------------------------------------ shared helpers

def sweep_kernel_names(info, prec, real):
    """Kernel (template) names of the x, y, z sweeps a solver with gp_get_info `info` runs."""
    rt = "float" if prec == "f32" else "double"
    L = info["trunc"]
    W = info["band_w"]
    c = "true" if real else "false"     # complex field
    nm = "false" if real else "true"    # the z sweep sums the norm in imaginary time only
    if info.get("line64_mask", 0) == 7:
        return {"sweep_x": f"k_sweep_x64<{c}>", "sweep_y": f"k_sweep_line64<{c},1,false>",
                "sweep_z": f"k_sweep_line64<{c},2,{nm}>"}
    return {
        "sweep_x": (f"k_sweep_x_reg<{c},{W}>" if info.get("x_reg") else
                    f"k_sweep_x_band<float,{c},{W}>" if info["band_mask"] & 1 else
                    f"k_sweep_x_stream<float,{c},{L}>" if info["fast_mask"] & 1 else f"k_sweep_x<{rt},{c}>"),
        "sweep_y": (f"k_sweep_band_line<float,{c},1,false,{W}>" if info["band_mask"] & 2 else
                    f"k_sweep_stream<float,{c},1,false,{L}>" if info["fast_mask"] & 2 else f"k_sweep_y<{rt},{c}>"),
        "sweep_z": (f"k_sweep_band_line<float,{c},2,{nm},{W}>" if info["band_mask"] & 4 else
                    f"k_sweep_stream<float,{c},2,{nm},{L}>" if info["fast_mask"] & 4 else f"k_sweep_z<{rt},{c},{nm}>")}


def make_workload_solver(P, prec, mode, grid, splitting="lie"):
    """The bench's solve on `grid`: imaginary time (dt = 0.1 h^2, g = 100, from the
    Gaussian) or the quench (dt = 0.02 h^2: 300 imaginary steps at g = 100, then
    g = 200 in real time).  Returns (solver, step function)."""
    real = mode == "real"
    dt = (0.02 if real else 0.1) * H * H
    so = P.Solver(*grid, H, dt=dt, gamma=TRAP[0], nu=TRAP[1], lam=TRAP[2], g=G, prec=prec)
    so.set_splitting(splitting)
    so.init_gaussian()
    if real:
        so.step_imag(300)
        so.set_g(2 * G)
    return so, (so.step_real if real else so.step_imag)


def time_steps(P, so, step, steps, flush):
    """Per-step CUDA-event times (L2 flushed between steps, outside the events), then
    per-sweep times from the library's events over the same number of steps.
    Returns (ms per step, [avg ms of the x, y, z sweeps], launches per sweep)."""
    import torch
    for _ in range(3):
        step(1)
        flush()
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        e0[k].record()
        step(1)
        e1[k].record()
        flush()
    torch.cuda.synchronize()
    ms = sum(e0[k].elapsed_time(e1[k]) for k in range(steps)) / steps
    P.gp_set_timing(so.handle, True)
    for _ in range(steps):
        step(1)
        flush()
    kms, kn = P.gp_get_timing(so.handle)
    P.gp_set_timing(so.handle, False)
    so.sync()
    return ms, [kms[i] / max(kn[i], 1) for i in range(3)], kn


# FP64 lane operations (DADD, DMUL, DFMA: one each; the FP64 pipe takes them at the
# same rate) per grid point of each sweep, counted from the arithmetic of the FP64
# kernels (gp_sweeps64.cu) at the bench workloads: x = pointwise substep (real: 8 at
# the degree-4 exp polynomial; complex: 21 with the degree-4/5 cos/sin polynomials)
# + forward (4 / 14) + back substitution (1 / 4); y and z: 5 / 18; the imaginary-time
# z sweep adds 1 for the norm.
FP64_OPS = {"imag": (13, 5, 6), "real": (39, 18, 18)}


def fp64_peak():
    """Measured FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul, 4096^3, best of 3),
    as FP64 operations per second (one fused multiply-add = one operation)."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    return n ** 3 / (best / 1e3)


def fp64_pipe_peak(sm_mhz):
    """FP64 ALU peak from unit counts and the clock: 2 FP64 lane operations per clock
    per SM (the rate ncu's sm__inst_executed_pipe_fp64 peak implies on this part, and
    the nominal 1.25 TFLOP/s at 2.07 GHz over 152 SMs), at the SM clock sampled during
    the run."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    return 2.0 * nsm * sm_mhz * 1e6, nsm


def paper_precision(P, args, flush, hbm, sm_mhz):
    """FP64 imaginary time on the bench grid and complex128 real time on the quench
    workload, each with per-sweep times, HBM fractions and FP64 ALU fractions."""
    grid = (NX, NY, NZ)
    npts = NX * NY * NZ
    peak, nsm = fp64_pipe_peak(sm_mhz)
    out = {"fp64_peak": {"value": round(peak / 1e12, 4), "unit": "T FP64 op/s",
                         "source": f"derived: 2 FP64 lane op/clk/SM x {nsm} SMs x {sm_mhz:.0f} MHz "
                                   "(sampled SM clock)",
                         "dgemm_measured": round(fp64_peak() / 1e12, 4)}}
    for mode, steps in (("imag", max(args.f64_steps, 3)), ("real", max(args.f64_steps // 3, 3))):
        so, st = make_workload_solver(P, "f64", mode, grid)
        ms, sw, kn = time_steps(P, so, st, steps, flush)
        names = sweep_kernel_names(so.info(), "f64", mode == "real")
        so.close()
        ops = FP64_OPS[mode]
        sb = 16 if mode == "real" else 8
        per = {}
        for i, n in enumerate(("sweep_x", "sweep_y", "sweep_z")):
            achieved = ops[i] * npts / (sw[i] / 1e3)
            per[n] = {"kernel": names[n], "avg_ms": round(sw[i], 5),
                      "fp64_ops_per_point": ops[i],
                      "alu_frac": round(achieved / peak, 3),
                      "hbm_frac": round(2 * npts * sb / (sw[i] / 1e3) / 1e9 / hbm, 3)}
        dom = max(per, key=lambda n: per[n]["avg_ms"])
        out["imag_f64" if mode == "imag" else "real_c128"] = {
            "workload": (f"imag3d {NX}x{NY}x{NZ}, h=0.1, dt=0.1h^2, trap (1,1.41,2), g=100, "
                         "imaginary time, FP64 field" if mode == "imag" else
                         f"real3d {NX}x{NY}x{NZ}, h=0.1, dt=0.02h^2, trap (1,1.41,2), ground state "
                         "at g=100 then quench to g=200, real time, complex128 field"),
            "value": round(npts / (ms / 1e3), 1), "unit": "grid-point-steps/s",
            "ms_per_step": round(ms, 5), "steps": steps, "sweeps": per,
            "roofline_alu": {"bound": "alu", "kernel": per[dom]["kernel"],
                             "achieved": round(ops[("sweep_x", "sweep_y", "sweep_z").index(dom)] * npts
                                               / (per[dom]["avg_ms"] / 1e3) / 1e12, 4),
                             "peak": round(peak / 1e12, 4), "unit": "T FP64 op/s",
                             "frac": per[dom]["alu_frac"]}}
    return out


def link_bandwidth(host_in, host_out, reps=10):
    """Host-device copy rates of the e2e loop's pinned buffers (one field each way):
    host-to-device alone, device-to-host alone, and both at once on two streams (GB/s
    per direction), CUDA events around each repetition set."""
    import torch
    n = host_in.numel()
    d_a = torch.empty(n, dtype=host_in.dtype, device="cuda")
    d_b = torch.zeros(n, dtype=host_in.dtype, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nbytes = n * host_in.element_size()

    def rate(h2d, d2h):
        def once():
            if h2d:
                with torch.cuda.stream(s1):
                    d_a.copy_(host_in, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s2):
                    host_out.copy_(d_b, non_blocking=True)
        once()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            once()
        torch.cuda.synchronize()
        return round(nbytes * reps / (time.perf_counter() - t0) / 1e9, 1)

    out = {"bytes": nbytes, "h2d_gbs": rate(True, False), "d2h_gbs": rate(False, True),
           "both_per_direction_gbs": rate(True, True)}
    del d_a, d_b
    return out


def dram_bound(P, args, flush, hbm):
    """The same FP32 imaginary-time step on 512 x 400 x 320 (a 262 MB field, twice the
    L2): every sweep streams from and to DRAM."""
    grid = (512, 400, 320)
    npts = grid[0] * grid[1] * grid[2]
    so, st = make_workload_solver(P, "f32", "imag", grid)
    ms, sw, kn = time_steps(P, so, st, 20, flush)
    names = sweep_kernel_names(so.info(), "f32", False)
    so.close()
    per = {}
    for i, n in enumerate(("sweep_x", "sweep_y", "sweep_z")):
        gbs = 2 * npts * 4 / (sw[i] / 1e3) / 1e9
        per[n] = {"kernel": names[n], "avg_ms": round(sw[i], 5), "achieved_gbs": round(gbs, 1),
                  "frac": round(gbs / hbm, 3)}
    return {"workload": WORKLOAD.replace("240x200x160", "512x400x320"),
            "value": round(npts / (ms / 1e3), 1), "unit": "grid-point-steps/s",
            "ms_per_step": round(ms, 5), "steps": 20,
            "step_frac_of_hbm": round(6 * npts * 4 / (ms / 1e3) / 1e9 / hbm, 3),
            "sweeps": per, "traffic": ncu_traffic_512()}


def ncu_traffic_512():
    """DRAM bytes per launch of the 512x400x320 sweeps from the committed ncu summary,
    when it was taken on the current kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != source_hash():
        return None
    return d.get("dram_bound_512x400x320")


def batch_short(P, args):
    """A shortened batched workload: the 64 uneven FP32 solves, 200 steps each, one pool,
    against the same instances one at a time in FP64 and FP32 (100 steps each, scaled),
    with the mu error against the FP64 solves on four instances."""
    import torch
    from paper_1605_03958_gb300 import workloads
    inst = workloads.batch_instances()
    K = 200
    need = sum(P.Pool.slot_bytes(**k) for k in inst)
    pool = P.Pool(int(need * 1.05) + (64 << 20), max_slots=len(inst))
    ids = [pool.add(**k) for k in inst]
    pool.tune(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pool.step(K)
    batch_s = time.perf_counter() - t0
    obs = [pool.observables(i) for i in ids[:4]]
    pool.close()
    single = {}
    for prec in ("f64", "f32"):
        tot = 0.0
        for k in inst:
            so = P.Solver(k["nx"], k["ny"], k["nz"], k["dx"], dt=k["dt"], gamma=k["gamma"],
                          nu=k["nu"], lam=k["lam"], g=k["g"], prec=prec)
            so.init_gaussian()
            so.step_imag(2)
            so.sync()
            t0 = time.perf_counter()
            so.step_imag(100)
            so.sync()
            tot += (time.perf_counter() - t0) * K / 100
            so.close()
        single[prec] = len(inst) / tot
    err = []
    for k, o in zip(inst[:4], obs):
        so = P.Solver(k["nx"], k["ny"], k["nz"], k["dx"], dt=k["dt"], gamma=k["gamma"],
                      nu=k["nu"], lam=k["lam"], g=k["g"], prec="f64")
        so.init_gaussian()
        so.step_imag(K)
        ref = so.observables()
        so.close()
        err.append(abs(o["mu"] - ref["mu"]) / abs(ref["mu"]))
    v = len(inst) / batch_s
    return {"workload": "64 uneven imag3d solves (extents {32..160}, trap U[0.5,3], g log-U[1,5000], "
                        "h=0.2, dt=0.1h^2, seed 1605), 200 steps each",
            "value": round(v, 3), "unit": "solves/s",
            "one_at_a_time_f64": round(single["f64"], 3), "one_at_a_time_f32": round(single["f32"], 3),
            "speedup_vs_f64": round(v / single["f64"], 2),
            "mu_rel_vs_f64_max": max(err), "accuracy_instances": len(err)}


def serve_summary(done):
    """solves / s over the run (first arrival to last finish), latency percentiles, the
    offered rate and the p99 latency by quarter of the request index (flat quarters: the
    server keeps up; growing ones: the queue grows)."""
    import numpy as np
    lat = sorted(d["latency"] for d in done)
    span = max(d["finished"] for d in done) - min(d["arrival"] for d in done)
    arr = sorted(d["arrival"] for d in done)
    out = {"solves": len(done), "solves_per_s": round(len(done) / span, 3),
           "p50_s": round(float(np.percentile(lat, 50)), 4),
           "p99_s": round(float(np.percentile(lat, 99)), 4), "makespan_s": round(span, 3)}
    if len(done) >= 8 and arr[-1] > arr[0]:
        out["offered_per_s"] = round((len(arr) - 1) / (arr[-1] - arr[0]), 3)
        by_id = [d["latency"] for d in sorted(done, key=lambda d: d["id"])]
        q = len(by_id) // 4
        out["p99_by_quarter_s"] = [round(float(np.percentile(by_id[i * q:(i + 1) * q if i < 3 else None], 99)), 4)
                                   for i in range(4)]
    return out


def serve_short(P, args):
    """The serving workload in the default line's context: the seeded request stream
    (--serve-requests, Poisson at 200 / s) through the continuous-batching server, and
    the leading 50 requests one at a time with FP64 single solvers (arrivals on the wall
    clock in both)."""
    import numpy as np
    from paper_1605_03958_gb300 import workloads
    from paper_1605_03958_gb300.serve import Server, serve_one_at_a_time

    summary = serve_summary
    reqs = workloads.serve_requests(args.serve_requests)
    srv = Server(quantum=100)
    done = srv.run(reqs, realtime=True)
    srv.close()
    head = reqs[:50]
    f64 = serve_one_at_a_time(head, prec="f64", realtime=True)
    by = {d["id"]: d for d in f64}
    gerr = qerr = 0.0
    for d in done:
        if d["id"] not in by:
            continue
        w = by[d["id"]]["obs"]
        if d["kind"] == "ground":
            gerr = max(gerr, abs(d["obs"]["mu"] - w["mu"]) / abs(w["mu"]))
        else:
            qerr = max(qerr, abs(d["obs"]["energy"] - w["energy"]) / abs(w["energy"]))
    return {"workload": f"{len(reqs)} requests, Poisson arrivals at 200/s (seed 3958): 70 % ground "
                        "state (2000 imaginary steps), 30 % quench (500..5000 real steps)",
            "batched": summary(done),
            "one_at_a_time_f64_first_50": summary(f64),
            "accuracy_vs_f64_first_50": {"ground_mu_rel_max": gerr, "quench_energy_rel_max": qerr}}


# ------------------------------------------------------------ CUDA arm

def run_cuda(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03958_gb300 as P

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x):
        return replica_throughput(x, 1, device="cuda")[1]

    real = args.mode == "real"
    sbytes = (4 if args.prec == "f32" else 8) * (2 if real else 1)   # bytes per stored point

    def make_solver(prec):
        so = P.Solver(NX, NY, NZ, H, dt=DT, gamma=TRAP[0], nu=TRAP[1], lam=TRAP[2], g=G, prec=prec)
        so.set_splitting(args.splitting)
        so.init_gaussian()
        if real:   # the quench: ground state at g, then 2 g in real time
            so.step_imag(300)
            so.set_g(2 * G)
        return so, (so.step_real if real else so.step_imag)

    s, step = make_solver(args.prec)
    flush_w = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    flush_r = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def flush():
        # evict the field: write 256 MiB, then read another 256 MiB so that L2 holds
        # clean unrelated lines (the write-back of the written buffer happens here,
        # outside the timed step, not in the next step's first sweep)
        flush_w.zero_()
        flush_r.sum()

    for _ in range(max(args.warmup, 3)):
        step(1)
        flush()
    s.sync()
    torch.cuda.synchronize()
    barrier()

    K = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        for k in range(K):
            ev0[k].record()
            step(1)
            ev1[k].record()
            flush()
        torch.cuda.synchronize()
        barrier()
    s.sync()
    step_ms = sum(ev0[k].elapsed_time(ev1[k]) for k in range(K))
    value, total_ms = replica_throughput(step_ms, NPTS * K, device="cuda")

    # second timed region: the same steps with every sweep bracketed by the library's
    # CUDA events on the solver stream (these events keep consecutive sweeps from
    # overlapping, so the step timing above is taken without them)
    K2 = min(K, 500)
    P.gp_set_timing(s.handle, True)
    torch.cuda.synchronize()
    for k in range(K2):
        step(1)
        flush()
    kms, kn = P.gp_get_timing(s.handle)
    P.gp_set_timing(s.handle, False)
    s.sync()

    # per-sweep roofline: algorithmic bytes = one read + one write of the field
    hbm, peak_kind = peaks()
    names = ["sweep_x", "sweep_y", "sweep_z"]
    info = s.info()
    kernels = sweep_kernel_names(info, args.prec, real)
    per = {}
    for i, n in enumerate(names):
        if kn[i] == 0:   # a 2D solve has no z sweep
            continue
        avg = kms[i] / kn[i]
        gbs = 2 * NPTS * sbytes / (avg / 1e3) / 1e9
        per[n] = {"kernel": kernels[n], "avg_ms": round(avg, 5), "launches": kn[i],
                  "achieved_gbs": round(gbs, 1), "frac": round(gbs / hbm, 3)}
    dom = max(per, key=lambda n: per[n]["avg_ms"])
    traffic = ncu_traffic(kernels[dom])
    roofline = {"bound": "hbm", "kernel": kernels[dom], "achieved": per[dom]["achieved_gbs"],
                "peak": hbm, "unit": "GB/s", "frac": per[dom]["frac"], "traffic": traffic,
                "algorithmic_bytes_per_launch": 2 * NPTS * sbytes,
                "peak_source": f"{peak_kind} hbm_gbs (copy, MEASURED_PEAKS.json)"
                if peak_kind == "measured" else "fallback 6.8 TB/s"}
    if args.prec == "f64" and info.get("line64_mask", 0) == 7 and NZ > 1:
        # the FP64 sweeps are bound by GB300's FP64 unit, not by HBM: report the
        # dominant sweep against the FP64 ALU peak (the HBM figures stay in `sweeps`)
        sm_mhz = (clk.summary() or {}).get("sm_mhz") or 2070.0
        fpk, nsm = fp64_pipe_peak(sm_mhz)
        ops = FP64_OPS["real" if real else "imag"][names.index(dom)]
        ach = ops * NPTS / (per[dom]["avg_ms"] / 1e3)
        roofline = {"bound": "alu", "kernel": kernels[dom], "achieved": round(ach / 1e12, 4),
                    "peak": round(fpk / 1e12, 4), "unit": "T FP64 op/s",
                    "frac": round(ach / fpk, 3), "traffic": traffic,
                    "fp64_ops_per_point": ops,
                    "hbm_frac": per[dom]["frac"],
                    "peak_source": f"derived: 2 FP64 lane op/clk/SM x {nsm} SMs x "
                                   f"{sm_mhz:.0f} MHz (sampled SM clock)"}

    # end to end through the public API: H2D of the step's input field from pinned
    # host memory, one step, D2H of the resulting field into pinned host memory; the
    # host buffers are in the field's own precision (FP32 I/O for an FP32 solve).
    # FP32: the read is the overlapped one (its device-to-host copy runs beside the next
    # step's host-to-device copy and the next step) and gp_sync completes the last read
    # before the clock stops.
    e2e = None
    if args.e2e_steps > 0:
        f32 = args.prec == "f32"
        hdt = torch.float32 if f32 else torch.float64
        get = P.gp.gp_get_psi_f32_async_ptr if f32 else P.gp.gp_get_psi_ptr
        nh = NPTS * (2 if real else 1)
        host_in = torch.empty(nh, dtype=hdt, pin_memory=True)
        host_out = torch.empty(nh, dtype=hdt, pin_memory=True)
        get(s.handle, host_in.data_ptr(), real)
        P.gp.gp_sync(s.handle)

        def e2e_run(put, nsteps):
            for _ in range(3):
                put(s.handle, host_in.data_ptr(), real)
                step(1)
                get(s.handle, host_out.data_ptr(), real)
            P.gp.gp_sync(s.handle)
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for _ in range(nsteps):
                put(s.handle, host_in.data_ptr(), real)
                step(1)
                get(s.handle, host_out.data_ptr(), real)
            P.gp.gp_sync(s.handle)
            torch.cuda.synchronize()
            barrier()
            return max_over_ranks(time.perf_counter() - t0)

        # FP32: the overlapped write (its host-to-device copy beside the previous step
        # and the previous read's packing) and, for comparison, the synchronous one
        put = P.gp.gp_set_psi_f32_async_ptr if f32 else P.gp.gp_set_psi_ptr
        e2e_s = e2e_run(put, args.e2e_steps)
        name = "_f32" if f32 else ""
        e2e = {"value": round(world * NPTS * args.e2e_steps / e2e_s, 1), "unit": "grid-point-steps/s",
               "h2d_bytes_per_step": NPTS * sbytes, "d2h_bytes_per_step": NPTS * sbytes,
               "steps": args.e2e_steps,
               "api": (f"gp_set_psi{name}{'_async' if f32 else ''}(pinned host field) + "
                       f"gp_step_{args.mode}(1) + gp_get_psi{name}{'_async' if f32 else ''}(pinned)"
                       + ("; gp_sync after the last step" if f32 else ""))}
        if f32:
            e2e["value_synchronous_write"] = round(
                world * NPTS * args.e2e_steps / e2e_run(P.gp.gp_set_psi_f32_ptr, args.e2e_steps), 1)
        e2e["link"] = link_bandwidth(host_in, host_out)

    # context: the same step back to back with L2 kept warm (no flush), one call
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    step(K)
    b.record()
    torch.cuda.synchronize()
    warm_ms = a.elapsed_time(b) / K

    # context (after the timed regions): the paper's precision (FP64 imaginary time on
    # this grid, complex128 real time on the quench workload) with its per-sweep FP64
    # ALU roofline; the same solve on a DRAM-bound grid; shortened batched and served
    # workloads
    paper = dram = batched = served = None
    if args.context and world == 1:
        csum = clk.summary()
        paper = paper_precision(P, args, flush, hbm, (csum or {}).get("sm_mhz") or 2070.0)
        dram = dram_bound(P, args, flush, hbm)
        batched = batch_short(P, args)
        served = serve_short(P, args)
    obs = s.observables()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(real)

    line = {
        "metric": "grid-point SSCN steps/s", "value": round(value, 1),
        "unit": "grid-point-steps/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(total_ms / K, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f32": "c64", "f64": "c128"}[args.prec] if real else args.prec,
        "data": "synthetic",
        "config": {"workload": WORKLOAD + ("" if args.splitting == "lie" else ", Strang splitting"),
                   "grid": [NX, NY, NZ], "field": {"f32": "c64", "f64": "c128"}[args.prec] if real else args.prec,
                   "reductions": "f64", "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write + 256 MiB read, untimed)",
                   "steps_per_sample": 1},
        "roofline": roofline, "sweeps": per,
        "e2e": e2e, "gpu_launches": (6 if args.splitting == "strang" else 3) * K,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "context": {"warm_l2_ms_per_step": round(warm_ms, 5),
                    "warm_l2_value": round(NPTS / (warm_ms / 1e3), 1),
                    "paper_precision": paper, "dram_bound": dram,
                    "batched": batched, "served": served,
                    "mu_after_run": obs["mu"], "norm_after_run": obs["norm"]},
    }
    s.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


# ------------------------------------------------------- CPU oracle timings

def _oracle_sample(nz_s, steps, threads, real=False):
    import oracle
    oracle.set_threads(threads)
    p = oracle.Problem(NX, NY, nz_s, H, H, H, DT, gamma=TRAP[0], nu=TRAP[1], lam=TRAP[2],
                       g=2 * G if real else G)
    psi = oracle.init_gaussian(p)
    if real:
        psi = psi.astype(complex)
    t0 = time.perf_counter()
    (oracle.step_real if real else oracle.step_imag)(p, psi, steps)
    return time.perf_counter() - t0


def cpu_baseline(real=False):
    """The oracle as it stands on this host's cores, full grid, bounded to ~20 s."""
    threads = os.cpu_count() or 1
    t1 = _oracle_sample(NZ, 1, threads, real)
    steps = max(1, min(100, int(20.0 / max(t1, 1e-3))))
    t = _oracle_sample(NZ, steps, threads, real)
    ts = _oracle_sample(NZ, 1, 1, real)
    kind = "real-time" if real else "imaginary-time"
    return {"value": round(NPTS * steps / t, 1), "unit": "grid-point-steps/s", "cores": threads,
            "kind": "oracle",
            "sample": f"{steps} FP64 {kind} steps of the full 240x200x160 grid, "
                      f"OpenMP over line solves on {threads} threads",
            "single_thread": {"value": round(NPTS / ts, 1), "unit": "grid-point-steps/s",
                              "cores": 1, "sample": f"1 FP64 {kind} step of the full grid"}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.lib()
    threads = os.cpu_count() or 1
    # each step: one oracle SSCN step on a 240x200xnz_s slab of the grid, nz_s sized so
    # that the whole warm-up + timed run stays near 90 s of CPU time
    real = args.mode == "real"
    probe = _oracle_sample(16, 1, threads, real) / 16.0    # seconds per z-plane-step
    budget = 90.0 / max(args.steps + args.warmup, 1)
    nz_s = int(max(3, min(NZ, budget / max(probe, 1e-9))))
    if args.warmup:
        _oracle_sample(nz_s, args.warmup, threads, real)
    t = _oracle_sample(nz_s, args.steps, threads, real)
    value = NX * NY * nz_s * args.steps / t
    line = {"impl": "reference", "metric": "grid-point SSCN steps/s", "value": round(value, 1),
            "unit": "grid-point-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128" if real else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [NX, NY, NZ], "sample_grid": [NX, NY, nz_s]},
            "cpu_baseline": {"value": round(value, 1), "unit": "grid-point-steps/s",
                             "cores": threads, "kind": "oracle",
                             "sample": f"each step one FP64 SSCN step of a 240x200x{nz_s} slab, "
                                       f"OpenMP over line solves on {threads} threads"},
            "e2e": {"value": round(value, 1), "unit": "grid-point-steps/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------ plain FP64 ground state

def run_c1(args):
    """The small plain-FP64 ground state: 64 x 48 x 32, h = 0.2, dt = 0.1 h^2, trap
    (1, 1.5, 2), g = 20, 2000 imaginary steps from the Gaussian.  The field (0.8 MB)
    lives in L2 and a step is a few launches, so the figure is steps/s of back-to-back
    steps (one call of 2000 steps, and 2000 single-step calls replaying the step's
    graph), not a fraction of HBM bandwidth.  The observables after 2000 steps are set
    beside the oracle's, computed on the host cores in the same run."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03958_gb300 as P
    import oracle
    nx, ny, nz, h, dt, trap, g, K = 64, 48, 32, 0.2, 0.004, (1.0, 1.5, 2.0), 20.0, 2000
    prec = "f64"   # the plain FP64 workload
    npts = nx * ny * nz

    def solver():
        so = P.Solver(nx, ny, nz, h, dt=dt, gamma=trap[0], nu=trap[1], lam=trap[2], g=g, prec=prec)
        so.init_gaussian()
        return so

    s = solver()
    s.step_imag(20)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        s2 = solver()
        torch.cuda.synchronize()
        a.record()
        s2.step_imag(K)
        b.record()
        torch.cuda.synchronize()
        one_call_ms = a.elapsed_time(b)
        s3 = solver()
        torch.cuda.synchronize()
        a.record()
        for _ in range(K):
            s3.step_imag(1)
        b.record()
        torch.cuda.synchronize()
        single_ms = a.elapsed_time(b)
    obs = s2.observables()
    same = bool(np.array_equal(s2.get_psi(), s3.get_psi()))
    oracle.set_threads(os.cpu_count() or 1)
    p = oracle.Problem(nx, ny, nz, h, h, h, dt, gamma=trap[0], nu=trap[1], lam=trap[2], g=g)
    t0 = time.perf_counter()
    ref = oracle.step_imag(p, oracle.init_gaussian(p), K)
    cpu_s = time.perf_counter() - t0
    ro = oracle.observables(p, ref)
    keys = ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z", "rms_r")
    line = {"metric": "grid-point SSCN steps/s", "value": round(npts * K / (one_call_ms / 1e3), 1),
            "unit": "grid-point-steps/s", "n_gpus": 1, "steps": K, "warmup": 20,
            "ms_per_step": round(one_call_ms / K, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": "imag3d 64x48x32, h=0.2, dt=0.1h^2, trap (1,1.5,2), g=20, "
                                   "2000 imaginary steps from the Gaussian",
                       "l2": "resident (0.8 MB field): steps back to back, no flush"},
            "steps_per_s": {"one_call": round(K / (one_call_ms / 1e3), 1),
                            "single_step_calls_graph": round(K / (single_ms / 1e3), 1)},
            "single_calls_same_bits": same,
            "observables": {k: obs[k] for k in keys},
            "oracle_observables": {k: ro[k] for k in keys},
            "mu_rel_vs_oracle": abs(obs["mu"] - ro["mu"]) / abs(ro["mu"]),
            "cpu_baseline": {"value": round(npts * K / cpu_s, 1), "unit": "grid-point-steps/s",
                             "cores": os.cpu_count() or 1, "kind": "oracle",
                             "sample": "the same 2000 FP64 steps, OpenMP over line solves"},
            "clocks": clk.summary()}
    for so in (s, s2, s3):
        so.close()
    print(json.dumps(line))


# ------------------------------------------------------------ batched solves

def run_batch(args):
    """64 uneven imaginary-time FP32 solves resident in one pool, every one stepped
    `--steps` steps by one batched launch per sweep direction (graph replay, shape
    autotuned first).  value = solves / s.  Baselines: the same instances one at a time
    with the single-solve library in FP64 and FP32 (each instance timed over
    --batch-single-steps steps, scaled to --steps)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03958_gb300 as P
    from paper_1605_03958_gb300 import workloads

    inst = workloads.batch_instances()
    K = args.steps
    points = sum(k["nx"] * k["ny"] * k["nz"] for k in inst)
    need = sum(P.Pool.slot_bytes(**k) for k in inst)
    pool = P.Pool(int(need * 1.05) + (64 << 20), max_slots=len(inst))
    ids = [pool.add(**k) for k in inst]
    tuned_ms = pool.tune(5)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        pool.step(K)
        batch_s = time.perf_counter() - t0
    info = pool.info()
    obs = [pool.observables(s) for s in ids[:4]]
    pool.close()

    # one at a time through the single-solve library
    n1 = min(args.batch_single_steps, K)
    single = {}
    for prec in ("f64", "f32"):
        tot = 0.0
        for k in inst:
            s = P.Solver(k["nx"], k["ny"], k["nz"], k["dx"], dt=k["dt"], gamma=k["gamma"],
                         nu=k["nu"], lam=k["lam"], g=k["g"], prec=prec)
            s.init_gaussian()
            s.step_imag(2)
            s.sync()
            t0 = time.perf_counter()
            s.step_imag(n1)
            s.sync()
            tot += time.perf_counter() - t0
            s.close()
        single[prec] = len(inst) / (tot * K / n1)

    # accuracy of the batched FP32 solves against FP64 one-at-a-time solves (first 4)
    acc = []
    for k, o in zip(inst[:4], obs):
        s = P.Solver(k["nx"], k["ny"], k["nz"], k["dx"], dt=k["dt"], gamma=k["gamma"],
                     nu=k["nu"], lam=k["lam"], g=k["g"], prec="f64")
        s.init_gaussian()
        s.step_imag(K)
        ref = s.observables()
        s.close()
        acc.append(abs(o["mu"] - ref["mu"]) / abs(ref["mu"]))

    value = len(inst) / batch_s
    line = {
        "metric": "batched solves/s", "value": round(value, 3), "unit": "solves/s",
        "n_gpus": 1, "steps": K, "warmup": 0, "ms_per_step": round(batch_s / K * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "64 uneven imag3d solves: extents from {32,48,...,160}, trap "
                               "U[0.5,3], g log-uniform [1,5000], h=0.2, dt=0.1h^2, seed 1605",
                   "grid_points": points, "parallelism": "one pool, one batched launch per sweep",
                   "launch_shape": {"x_stages": info["x_stages"], "seg_turns": info["seg_turns"],
                                    "graph": bool(info["graph"]),
                                    "launches_per_step": info["launches_per_step"]},
                   "l2": "not flushed (the batch's 1 GB of fields exceeds L2)"},
        "grid_point_steps_per_s": round(points * K / batch_s, 1),
        "one_at_a_time": {"f64_solves_per_s": round(single["f64"], 3),
                          "f32_solves_per_s": round(single["f32"], 3),
                          "timed_steps_per_instance": n1,
                          "speedup_vs_f64": round(value / single["f64"], 2)},
        "accuracy": {"mu_rel_vs_f64_single_max": max(acc), "instances": len(acc)},
        "tuned_ms_per_step": round(tuned_ms, 5),
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


# ------------------------------------------------------------------- serving

def run_serve(args):
    """The continuous-batching server on the seeded request stream (Poisson arrivals,
    mean 200 / s; 70 % ground-state, 30 % quench requests), arrivals on the wall clock.
    value = completed solves / s over the run; latency = finish - arrival.  The leading
    --serve-compare requests are also served one at a time (FP64 and FP32 single
    solvers, FIFO, same arrival times) and by the batched server alone."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03958_gb300  # noqa: F401  (loads the library)
    from paper_1605_03958_gb300 import workloads
    from paper_1605_03958_gb300.serve import Server, serve_one_at_a_time

    summary = serve_summary

    import numpy as np
    reqs = workloads.serve_requests(args.serve_requests)
    srv = Server(quantum=100)
    with ClockSampler(0) as clk:
        done = srv.run(reqs, realtime=True)
    full = summary(done)
    stats = dict(srv.stats)
    srv.close()

    head = reqs[:args.serve_compare]
    compare = None
    if head:
        srv = Server(quantum=100)
        b = srv.run(head, realtime=True)
        srv.close()
        f64 = serve_one_at_a_time(head, prec="f64", realtime=True)
        f32 = serve_one_at_a_time(head, prec="f32", realtime=True)
        by = {d["id"]: d for d in f64}
        err = {"ground_mu_rel_max": 0.0, "quench_energy_rel_max": 0.0}
        for d in b:
            w = by[d["id"]]["obs"]
            if d["kind"] == "ground":
                err["ground_mu_rel_max"] = max(err["ground_mu_rel_max"],
                                               abs(d["obs"]["mu"] - w["mu"]) / abs(w["mu"]))
            else:
                err["quench_energy_rel_max"] = max(err["quench_energy_rel_max"],
                                                   abs(d["obs"]["energy"] - w["energy"]) / abs(w["energy"]))
        compare = {"requests": len(head), "batched": summary(b), "one_at_a_time_f64": summary(f64),
                   "one_at_a_time_f32": summary(f32), "accuracy_vs_f64": err}
    line = {
        "metric": "served solves/s", "value": full["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(reqs)} requests, Poisson arrivals at 200/s (seed 3958): 70 % "
                               "ground state (2000 imaginary steps), 30 % quench (500..5000 real "
                               "steps from the g=0 Gaussian); extents multiples of 16 in "
                               "[32,128]x[32,96]x[32,64], g log-uniform [1,1000], h=0.2, dt=0.1h^2",
                   "quantum_steps": 100,
                   "admission": "arrival order with backfill past a request that does not fit "
                                "(head wait bound 1 s); arena = half of free HBM"},
        "latency": {"p50_s": full["p50_s"], "p99_s": full["p99_s"]},
        "run": full, "server": stats,
        "compare_first_requests": compare,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c1":
        run_c1(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
