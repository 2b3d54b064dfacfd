"""The N>1 path on CPU (gloo, world size 2): every rank aligns its own batch
of the same size (weak scaling, no collective on the data path), the job's
step time is the slowest rank's and its cells are every rank's; under
torchrun only rank 0 prints the reference arm's line.  The split of one job
(--split): pairs assigned to ranks by cells (LPT), each rank aligns its shard
(the oracle stands in for the GPU here), and rank 0's gathered records equal
the single-rank records of the whole job, CIGARs included."""
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


def _split_rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _split_job()
        parts = bench.lpt_partition(b.q_len.astype(np.int64) * b.t_len, world)
        s = b.subset(parts[rank])
        rec, cig = _oracle_records(s)
        merged = bench.gather_shards(dist, rank, world, parts[rank], rec, cig, b.npairs)
        if rank == 0:
            out.put(("merged", merged, [int(s.cells) for s in (b.subset(x) for x in parts)],
                     [len(x) for x in parts]))
    finally:
        dist.destroy_process_group()


def _split_job():
    from paper_1208_6350_gb300 import workloads as wl
    # short-read extensions with a few long reads mixed in: uneven work
    sb = wl.config2(300, seed=11)
    lb = wl.dna_long_reads(6, 800, 2000, seed=12)
    b = wl.concat([sb.subset(np.arange(sb.npairs)), lb])
    return wl.Batch("split", b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, lb.W, lb.gap_open, lb.gap_extend,
                    "ACGT")


def _oracle_records(b):
    """The oracle's results as the library's records plus a flat CIGAR buffer."""
    import oracle
    from paper_1208_6350_gb300 import gsw
    stride = int(b.q_len.max() + b.t_len.max() + 2)
    ores, ocg, _ = oracle.align_batch(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, b.gap_open,
                                      b.gap_extend, cigar_stride=stride, nthreads=2)
    rec = np.zeros(b.npairs, gsw.RESULT_DTYPE)
    words = []
    at = 0
    for p in range(b.npairs):
        for f in ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2",
                  "cigar_len"):
            rec[f][p] = ores[f][p]
        n = int(ores["cigar_len"][p])
        rec["cigar_off"][p] = at if n > 0 else -1
        words.append(ocg[p, :n])
        at += n
    return rec, np.concatenate(words).astype(np.uint32)


def test_lpt_partition_balances_and_covers():
    import bench
    rng = np.random.default_rng(5)
    cells = rng.integers(30_000, 250_000, 20_000)
    parts = bench.lpt_partition(cells, 8)
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(len(cells)))   # every pair exactly once
    loads = np.array([cells[x].sum() for x in parts])
    assert loads.max() / loads.mean() - 1 < 0.001
    # one pair heavier than the rest together: it gets a rank of its own
    cells = np.array([10, 20, 30, 10_000, 15], np.int64)
    parts = bench.lpt_partition(cells, 2)
    assert any(list(x) == [3] for x in parts)


def test_split_job_gathers_the_single_rank_records():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    _, (rec, cig), cells, sizes = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sum(sizes) == len(rec) and min(sizes) > 0
    assert max(cells) / (sum(cells) / 2) - 1 < 0.01          # cells balanced within 1 %
    whole = _split_job()
    ref, ref_cig = _oracle_records(whole)
    for f in ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2", "cigar_len"):
        assert np.array_equal(rec[f], ref[f]), f
    for p in range(len(rec)):
        n = int(rec["cigar_len"][p])
        got = cig[rec["cigar_off"][p]: rec["cigar_off"][p] + n] if n > 0 else []
        want = ref_cig[ref["cigar_off"][p]: ref["cigar_off"][p] + n] if n > 0 else []
        assert list(got) == list(want), p
