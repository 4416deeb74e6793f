"""Host logic of the multi-GPU bench on CPU with world_size-2 gloo ranks: the slowest rank's time
is the job's time, throughput counts every replica's rays, and under torchrun the reference arm
prints exactly one line from rank 0 while the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dev = torch.device("cpu")
    pg = bench.init_ranks(world, dev)
    mine = 10.0 + 5.0 * rank  # rank 1 is the slow replica
    ms = bench.max_over_ranks(mine, pg, dev)
    out[rank] = (ms, bench.job_mrays(world, 4_194_304, ms))
    pg.barrier()
    pg.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    ms, mrays = res[0]
    assert ms == 15.0
    assert mrays == pytest.approx(2 * 4_194_304 / 0.015 / 1e6)


def test_single_rank_has_no_process_group():
    import bench
    assert bench.init_ranks(1, torch.device("cpu")) is None
    assert bench.max_over_ranks(3.5, None, torch.device("cpu")) == 3.5


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-rays", "8192"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
