"""The multi-GPU form of the benchmark runs independent replicas (one solve per rank,
no collective on the data path) and reports units over all ranks divided by the
slowest rank's time.  Checked here with two gloo processes on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1200.0, 1500.0][rank]          # rank 1 is the slower replica
    value, ms = bench.replica_throughput(local_ms, units_per_rank=7_680_000 * 100)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, ms = res[rank]
        assert ms == 1500.0                     # max over ranks
        assert value == pytest.approx(2 * 7_680_000 * 100 / 1.5)


def test_single_process_is_identity():
    import bench
    value, ms = bench.replica_throughput(250.0, 1000)
    assert ms == 250.0 and value == pytest.approx(4000.0)


def test_source_hash_ignores_comments_and_follows_code(tmp_path, monkeypatch):
    """The ncu figures in profiles/ncu_traffic.json are keyed to the code of the kernel
    sources: a comment edit keeps the key, a code edit changes it."""
    import shutil
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(tmp_path, "paper_1605_03958_gb300", "csrc")
    os.makedirs(csrc)
    for f in ("gp_sweeps.cu", "gp_sweeps64.cu", "gp_device.cuh", "gp_internal.h", "gp_api.cu"):
        shutil.copy(os.path.join(root, "paper_1605_03958_gb300", "csrc", f), csrc)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_hash()
    api = os.path.join(csrc, "gp_api.cu")
    src = open(api).read()
    open(api, "w").write(src + "\n// a comment\n/* another\n   one */\n")
    assert bench.source_hash() == h0
    open(api, "w").write(src + "\nstatic int an_extra_definition = 1;\n")
    assert bench.source_hash() != h0


def test_reference_arm_line(monkeypatch, capsys):
    """`bench.py --impl reference` prints one JSON line with the contract's keys, the
    oracle timed on this host's cores (a z-slab sample of the grid)."""
    import json
    import sys
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1",
                                      "--warmup", "0"])
    monkeypatch.setattr(bench, "_oracle_sample",
                        lambda nz_s, steps, threads, real=False: 1e-3 * nz_s * max(steps, 1))
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
