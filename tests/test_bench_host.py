"""Host-side logic of bench.py on CPU: the reference (oracle) arm's JSON line and its rank
handling under torchrun, and the max-over-ranks reduction of the multi-rank path (gloo,
world size 2, loopback rendezvous)."""
import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def run_bench(args, env_extra=None, timeout=300):
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], env=env, cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_line():
    r = run_bench(["--impl", "reference", "--steps", "2", "--warmup", "3", "--nvec", "4", "--n", "65536",
                   "--ref-budget", "2"])
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config"):
        assert k in line, k
    assert line["value"] > 0 and line["unit"] == "GB/s" and line["warmup"] >= 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same config dict as the GPU arm's line for the same arguments (one workload, one config)
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    args = argparse.Namespace(fmt="frsz2", bits=32, n=65536, nvec=4)
    assert line["config"] == bench.step_config(args, line["config"]["workload"], 1)


def test_reference_arm_other_ranks_exit_quietly():
    r = run_bench(["--impl", "reference", "--gpus", "2", "--steps", "2", "--ref-budget", "2"],
                  env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def _max_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    got = bench.max_over_ranks(dist, 1.5 + rank, torch.device("cpu"))
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    port = 29400 + os.getpid() % 500
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_max_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        assert dict(out) == {0: 2.5, 1: 2.5}


def test_max_over_ranks_single_process():
    import bench

    assert bench.max_over_ranks(None, 3.25, None) == 3.25


def test_oracle_solve_rate_scales_one_cycle():
    """cpu_baseline.solves times one whole restart cycle of the oracle at a reduced size and scales
    its time per Arnoldi step by the row count; with a 5-step cycle on the power-law operator."""
    sys.path.insert(0, ROOT)
    import bench

    r = bench.oracle_solve_rate("c4", restart=5)
    assert r["s_per_step_full_size"] > 0 and r["cores"] == 1 and r["unit"] == "s per Arnoldi step"
    assert "one restart cycle (5 steps" in r["sample"] and "x16" in r["sample"]
