"""Multi-rank host logic of bench.py on CPU: world size 2 over gloo.

The replicas' figures combine as the slowest rank's time and the sum of the
particle-steps; under --impl reference only rank 0 works and prints."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, ps, ms2, ps2 = [(10.0, 100.0, 20.0, 110.0), (12.0, 90.0, 19.0, 95.0)][rank]
    r = bench.combine_ranks(ms, ps, ms2, ps2, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, r))


def test_combine_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert res[r] == (12.0, 190.0, 20.0, 205.0)


def test_reference_arm_other_ranks_do_no_work():
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=3, order=1, theta=0.0)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert bench.run_reference_plasma(args, rank=1, world=2) is None


def test_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(1.0, 2.0, 3.0, 4.0, 1, "cpu") == (1.0, 2.0, 3.0, 4.0)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints
    one JSON line with the contract's keys, the workload of the GPU arm and
    a cpu_baseline describing the sample it timed."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "256x256x512" in d["config"]["workload"] and "oracle" in d["cpu_baseline"]["sample"]


def test_batched_runs_cpu_baseline_is_a_scaled_oracle_sample():
    """The batched runs' oracle baseline times a few of the same runs and
    scales by cells: positive rates, cell-updates = particle-steps x mean
    cells per run (one particle per run)."""
    import bench
    from paper_2201_09084_gb300 import inputs as I
    ps, cu, desc = bench.cpu_batch_sample(nruns=16, sample=2, steps=2)
    r = I.batched_runs(16)
    cells = int(((r["nx"] + 2 * r["npml"]) * (r["nz"] + 2 * r["npml"])).sum())
    assert ps > 0 and cu > 0 and "oracle" in desc
    assert abs(cu / ps - cells / 16) < 1e-6 * cells


def test_single_particle_cpu_baseline_counts_the_mover_until_removal():
    """The 2D single-particle oracle baseline runs the whole workload: the
    electron (u_z = 10, 64 cells from the +z interface at 0.70 cells per
    step) is pushed until it is removed at the outer PML edge, ~115 steps."""
    import bench
    ps, cu, desc = bench.cpu_single_particle(200)
    pushes = 25600 * 200 * ps / cu
    assert 100 <= round(pushes) <= 130, pushes
    assert bench.single_particle_bytes() == (120 * 128 * 128 + 200 * (160 * 160 - 128 * 128), 25600)
