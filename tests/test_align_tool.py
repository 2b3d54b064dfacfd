"""The FASTA-in / SAM-out tool: helpers on CPU; on the GPU its best-target
records equal the oracle's for (query, every target)."""
import io
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1208_6350_gb300 import align  # noqa: E402


def _write(path, recs):
    with open(path, "w") as f:
        for name, s in recs:
            f.write(f">{name} description\n")
            for k in range(0, len(s), 60):
                f.write(s[k:k + 60] + "\n")


def test_fasta_encoding_and_cigar_string(tmp_path):
    p = tmp_path / "a.fa"
    _write(p, [("r1", "ACGTNacgt"), ("r2", "GGA" * 50)])
    recs = align.read_fasta(p)
    assert [n for n, _ in recs] == ["r1", "r2"] and len(recs[1][1]) == 150
    assert list(align.encode("ACGTNacgt", "ACGTN")) == [0, 1, 2, 3, 4, 0, 1, 2, 3]
    # 3M1D2M with two clipped query letters at each end of a 9-letter query
    assert align.cigar_string([3 << 4, (1 << 4) | 2, 2 << 4], 9, 2, 6) == "2S3M1D2M2S"
    W = align.dna_matrix(2, -3)
    assert W[4].tolist() == [0] * 5 and W[0, 0] == 2 and W[0, 1] == -3


@pytest.mark.gpu
def test_tool_best_target_equals_oracle(tmp_path, capsys):
    import oracle
    from paper_1208_6350_gb300 import workloads as wl
    rng = np.random.default_rng(91)
    letters = np.array(list("ACGT"))
    targets = [("chrA", "".join(letters[rng.integers(0, 4, 3000)])),
               ("chrB", "".join(letters[rng.integers(0, 4, 5000)]))]
    queries = []
    for k in range(12):
        t = targets[k % 2][1]
        o = int(rng.integers(0, len(t) - 150))
        q = list(t[o:o + 150])
        for x in rng.integers(0, 150, 3):
            q[x] = "ACGT"[(("ACGT".index(q[x])) + 1) % 4]
        queries.append((f"q{k}", "".join(q)))
    queries.append(("rand", "".join(letters[rng.integers(0, 4, 120)])))
    tf, qf = tmp_path / "t.fa", tmp_path / "q.fa"
    _write(tf, targets)
    _write(qf, queries)
    align.main([str(tf), str(qf), "--table", "-m", "2", "-x", "3", "-o", "5", "-e", "2"])
    lines = capsys.readouterr().out.strip().split("\n")
    assert len(lines) == len(queries)
    W = wl.dna_matrix(2, -3)
    for line, (qn, qs) in zip(lines, queries):
        f = line.split("\t")
        assert f[0] == qn
        qc = align.encode(qs, "ACGT")
        best = None
        for tn, ts in targets:
            tc = align.encode(ts, "ACGT")
            res, cg, _ = oracle.align_batch(qc, np.array([0]), np.array([len(qc)], np.int32), tc, np.array([0]),
                                            np.array([len(tc)], np.int32), W, 5, 2,
                                            cigar_stride=len(qc) + len(tc) + 2)
            if best is None or res["score1"][0] > best[0]["score1"][0]:
                best = (res, cg, tn)
        res, cg, tn = best
        assert int(f[2]) == int(res["score1"][0]) and int(f[3]) == int(res["score2"][0])
        if res["score1"][0] > 0:
            assert f[1] == tn
            assert [int(x) for x in f[4:9]] == [int(res[k][0]) for k in
                                                ("ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2")]
            want = align.cigar_string(cg[0, : res["cigar_len"][0]], len(qc), int(res["read_begin1"][0]),
                                      int(res["read_end1"][0]))
            assert f[10] == want
