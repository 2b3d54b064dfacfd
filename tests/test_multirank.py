"""The N>1 path on CPU (gloo, world size 2): every rank aligns its own batch
of the same size (weak scaling, no collective on the data path), the job's
step time is the slowest rank's and its cells are every rank's; under
torchrun only rank 0 prints the reference arm's line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, cfg = bench.make_workload("dna_short_read_extension_1M", 400, rank)
        ms, cells = bench.combine_ranks(10.0 + rank, b.cells, dist)
        out.put((rank, b.npairs, int(b.cells), int(b.q.sum() + 7 * b.t.sum()), ms, cells))
    finally:
        dist.destroy_process_group()


def test_ranks_combine_max_time_and_total_cells():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, c0, h0, ms0, cells0), (r1, n1, c1, h1, ms1, cells1) = got
    assert n0 == n1 == 400          # same batch size on every rank (weak scaling)
    assert h0 != h1                 # but each rank's own seeded batch
    assert ms0 == ms1 == 11.0       # the slowest rank's time
    assert cells0 == cells1 == c0 + c1


def test_single_rank_combine_is_identity():
    import bench
    assert bench.combine_ranks(3.5, 1234) == (3.5, 1234)


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--workload", "dna_1k_100x1000", "--ref-pairs", "16"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
