"""Seeded synthetic workloads for the alignment hot path.

This module only draws sequences; it holds none of the alignment arithmetic,
so that the CUDA path and the CPU oracle can both be fed from it.  Every draw
comes from numpy's PCG64 seeded through ``SeedSequence(seed)``.

Workloads (sizes and mixes follow the paper's experiments; its datasets --
UniProt, human chr1/chr8, simulated Illumina reads, real ABI / Ion Torrent /
Illumina read sets -- are not available, so these stand in for their shapes):

``dna_short_reads``   queries of uniform length, targets containing a mutated
                      copy of the query (the 1,000 simulated 100 bp reads of
                      the genome benchmark, and short-read extension).
``dna_long_reads``    log-uniform long queries at 10 % error against targets
                      1.2x longer that contain the source (the long-read rows).
``protein_search``    queries against a shared database with a few homologs
                      (the protein database search) with a seeded synthetic
                      symmetric 20x20 matrix in a BLOSUM-like range.
``serving_trace``     Poisson arrivals of requests mixing the DNA workloads.

DNA codes are A=0, C=1, G=2, T=3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DNA = "ACGT"
PROTEIN = "ARNDCQEGHILKMFPSTWYV"


@dataclass
class Batch:
    """Pairs as two code arenas with offsets and lengths (query p is
    ``q[q_off[p]:q_off[p]+q_len[p]]``, target p likewise)."""
    name: str
    q: np.ndarray
    q_off: np.ndarray
    q_len: np.ndarray
    t: np.ndarray
    t_off: np.ndarray
    t_len: np.ndarray
    W: np.ndarray
    gap_open: int
    gap_extend: int
    alphabet: str
    meta: dict = field(default_factory=dict)

    @property
    def npairs(self) -> int:
        return int(len(self.q_len))

    @property
    def cells(self) -> int:
        return int(np.dot(self.q_len.astype(np.int64), self.t_len.astype(np.int64)))

    def query(self, p):
        return self.q[self.q_off[p]:self.q_off[p] + self.q_len[p]]

    def target(self, p):
        return self.t[self.t_off[p]:self.t_off[p] + self.t_len[p]]

    def subset(self, idx, name=None) -> "Batch":
        """Pairs ``idx`` (in that order), re-packed into fresh arenas."""
        idx = np.asarray(idx, dtype=np.int64)
        q, qo, ql = _gather(self.q, self.q_off, self.q_len, idx)
        t, to, tl = _gather(self.t, self.t_off, self.t_len, idx)
        meta = {k: (v[idx] if isinstance(v, np.ndarray) and len(v) == self.npairs else v)
                for k, v in self.meta.items()}
        return Batch(name or self.name, q, qo, ql, t, to, tl, self.W, self.gap_open,
                     self.gap_extend, self.alphabet, meta)


def _offsets(lengths):
    off = np.zeros(len(lengths), dtype=np.int64)
    if len(lengths) > 1:
        off[1:] = np.cumsum(lengths[:-1], dtype=np.int64)
    return off


def _gather(arena, off, length, idx):
    ln = length[idx].astype(np.int32)
    no = _offsets(ln)
    total = int(ln.sum(dtype=np.int64))
    if total == 0:
        return np.zeros(0, np.uint8), no, ln
    src = np.repeat(off[idx] - no, ln) + np.arange(total, dtype=np.int64)
    return arena[src], no, ln


def dna_matrix(match: int, mismatch: int) -> np.ndarray:
    W = np.full((4, 4), mismatch, dtype=np.int8)
    np.fill_diagonal(W, match)
    return W


def encode(s: str, alphabet: str = DNA) -> np.ndarray:
    lut = {c: k for k, c in enumerate(alphabet)}
    return np.array([lut[c] for c in s], dtype=np.uint8)


def decode(codes, alphabet: str = DNA) -> str:
    return "".join(alphabet[int(c)] for c in codes)


def mutate(rng, arena, off, length, p_sub, p_ins, p_del, max_indel=1, alpha=4):
    """Mutation walk over every sequence of an arena.

    Per source position, independently: substitution with probability
    ``p_sub`` (to one of the other letters, uniformly), insertion of
    U{1..max_indel} random letters after it with probability ``p_ins``, or
    deletion of it and the next U{1..max_indel}-1 positions (within the same
    sequence) with probability ``p_del``.  Returns (arena, off, len).
    """
    n = int(length.sum(dtype=np.int64))
    src = _gather(arena, off, length, np.arange(len(length)))[0].copy()
    if n == 0:
        return src, _offsets(length), length.astype(np.int32)
    seq = np.repeat(np.arange(len(length)), length)
    seq_end = np.repeat(_offsets(length) + length, length)
    u = rng.random(n, dtype=np.float32)
    k = rng.integers(1, max_indel + 1, n, dtype=np.int8).astype(np.int64) if max_indel > 1 else np.ones(n, np.int64)
    sub = u < p_sub
    ins = (u >= p_sub) & (u < p_sub + p_ins)
    dele = (u >= p_sub + p_ins) & (u < p_sub + p_ins + p_del)
    src[sub] = (src[sub] + rng.integers(1, alpha, int(sub.sum()), dtype=np.uint8)) % alpha
    pos = np.arange(n, dtype=np.int64)
    diff = np.zeros(n + 1, dtype=np.int64)
    dpos = pos[dele]
    np.add.at(diff, dpos, 1)
    np.add.at(diff, np.minimum(dpos + k[dele], seq_end[dele]), -1)
    deleted = np.cumsum(diff[:n]) > 0
    ins_len = np.where(ins, k, 0)
    counts = (~deleted).astype(np.int64) + ins_len
    total = int(counts.sum())
    owner = np.repeat(pos, counts)
    first = np.repeat(np.cumsum(counts) - counts, counts)
    rank = np.arange(total, dtype=np.int64) - first
    out = rng.integers(0, alpha, total, dtype=np.uint8)
    keep_slot = (rank == 0) & ~deleted[owner]
    out[keep_slot] = src[owner[keep_slot]]
    new_len = np.bincount(seq[owner], minlength=len(length)).astype(np.int32)
    return out, _offsets(new_len), new_len


def _random_arena(rng, lengths, alpha=4):
    ln = np.asarray(lengths, dtype=np.int32)
    return rng.integers(0, alpha, int(ln.sum(dtype=np.int64)), dtype=np.uint8), _offsets(ln), ln


def _implant_vec(rng, bg, bg_off, bg_len, ins, ins_off, ins_len, rows):
    """Overwrites background row rows[k] with insert k at a uniform offset."""
    rows = np.asarray(rows, dtype=np.int64)
    room = bg_len[rows].astype(np.int64) - ins_len.astype(np.int64)
    assert (room >= 0).all()
    o = (rng.random(len(rows)) * (room + 1)).astype(np.int64)
    total = int(ins_len.sum(dtype=np.int64))
    if total:
        rep = np.repeat(np.arange(len(rows)), ins_len)
        within = np.arange(total, dtype=np.int64) - np.repeat(ins_off, ins_len)
        bg[bg_off[rows][rep] + o[rep] + within] = ins[np.repeat(ins_off, ins_len) + within]
    return o


def dna_short_reads(npairs=1000, qlen=(100, 100), tlen=(1000, 1000), p_sub=0.02,
                    p_indel=0.002, max_indel=3, decoy_frac=0.0, match=2, mismatch=-2,
                    gap_open=3, gap_extend=1, seed=0, name="dna_short_reads") -> Batch:
    """Query q uniform ACGT of length U[qlen]; target uniform ACGT of length
    U[tlen] holding a mutated copy of q at a uniform offset (indels half
    insertions, half deletions, lengths U{1..max_indel}).  A fraction of pairs,
    chosen by permutation, are decoys: target and query unrelated."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    ql = rng.integers(qlen[0], qlen[1] + 1, npairs).astype(np.int32)
    tl = rng.integers(tlen[0], tlen[1] + 1, npairs).astype(np.int32)
    q, qo, ql = _random_arena(rng, ql)
    n_decoy = int(round(decoy_frac * npairs))
    decoy = np.zeros(npairs, dtype=bool)
    decoy[rng.permutation(npairs)[:n_decoy]] = True
    true_rows = np.nonzero(~decoy)[0]
    mq, mo, ml = mutate(rng, q, qo, ql, p_sub, p_indel / 2, p_indel / 2, max_indel)
    mq2, mo2, ml2 = _gather(mq, mo, ml, true_rows)
    tl[true_rows] = np.maximum(tl[true_rows], ml2)   # the target holds the whole copy
    t, to, tl = _random_arena(rng, tl)
    offs = _implant_vec(rng, t, to, tl, mq2, mo2, ml2, true_rows)
    implant = np.full(npairs, -1, dtype=np.int64)
    implant[true_rows] = offs
    return Batch(name, q, qo, ql, t, to, tl, dna_matrix(match, mismatch), gap_open, gap_extend,
                 DNA, {"decoy": decoy, "implant_offset": implant, "seed": seed})


def config1(seed=0) -> Batch:
    """1,000 pairs: 100 nt queries, 1,000 nt targets, 2 % substitutions, 0.2 %
    1-3 nt indels, +2/-2, open 3, extend 1."""
    return dna_short_reads(1000, (100, 100), (1000, 1000), 0.02, 0.002, 3, 0.0, 2, -2, 3, 1,
                           seed, "dna_1k_100x1000")


def config2(npairs=1_000_000, seed=1) -> Batch:
    """Short-read extension: queries U[100, 250], targets U[300, 1000] holding
    the query at 1 % substitutions and 0.1 % indels; 10 % decoys."""
    return dna_short_reads(npairs, (100, 250), (300, 1000), 0.01, 0.001, 3, 0.10, 2, -2, 3, 1,
                           seed, f"dna_{npairs}_short_extension")


def dna_long_reads(npairs=10_000, lmin=1000, lmax=20000, p_sub=0.06, p_ins=0.02, p_del=0.02,
                   flank=1.2, match=2, mismatch=-4, gap_open=4, gap_extend=2, seed=2,
                   name=None) -> Batch:
    """Source s of length L = round(exp(U[ln lmin, ln lmax])); query = s with
    single-letter substitutions / insertions / deletions at the given rates;
    target = random flanks around s, round(flank * L) long, s at a uniform
    offset."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    L = np.rint(np.exp(rng.uniform(np.log(lmin), np.log(lmax), npairs))).astype(np.int32)
    s, so, sl = _random_arena(rng, L)
    q, qo, ql = mutate(rng, s, so, sl, p_sub, p_ins, p_del, 1)
    tl = np.rint(flank * L).astype(np.int32)
    t, to, tl = _random_arena(rng, tl)
    offs = _implant_vec(rng, t, to, tl, s, so, sl, np.arange(npairs))
    return Batch(name or f"dna_{npairs}_long_reads", q, qo, ql, t, to, tl,
                 dna_matrix(match, mismatch), gap_open, gap_extend, DNA,
                 {"source_offset": offs, "seed": seed})


def config3(npairs=10_000, seed=2) -> Batch:
    return dna_long_reads(npairs, seed=seed)


def synthetic_protein_matrix(seed=4) -> np.ndarray:
    """Seeded symmetric 20x20 int8 matrix with BLOSUM-like ranges: diagonal in
    [4, 11], off-diagonal in [-4, 3].  A stand-in, not BLOSUM values."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    W = rng.integers(-4, 4, (20, 20))
    W = np.triu(W, 1)
    W = W + W.T
    np.fill_diagonal(W, rng.integers(4, 12, 20))
    return W.astype(np.int8)


def load_matrix(path: str, alphabet: str = PROTEIN) -> np.ndarray:
    """Reads a whitespace matrix file (header row of letters, then one row per
    letter) restricted to ``alphabet``."""
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    cols = rows[0]
    table = {r[0]: dict(zip(cols, map(int, r[1:]))) for r in rows[1:]}
    return np.array([[table[a][b] for b in alphabet] for a in alphabet], dtype=np.int8)


@dataclass
class ProteinSearch:
    queries: Batch  # q arena holds the queries; t arena the database
    n_queries: int
    n_db: int

    def pairs(self, qidx, didx, name=None) -> Batch:
        """Batch of (query qidx[k], database didx[k]) pairs sharing the arenas."""
        b = self.queries
        qidx = np.asarray(qidx, np.int64)
        didx = np.asarray(didx, np.int64)
        return Batch(name or b.name, b.q, b.q_off[qidx], b.q_len[qidx], b.t, b.t_off[didx],
                     b.t_len[didx], b.W, b.gap_open, b.gap_extend, b.alphabet,
                     {"query": qidx, "db": didx})


def protein_search(n_queries=1000, n_db=10_000, homolog_frac=0.05, identity=0.40,
                   gap_open=11, gap_extend=1, W=None, seed=3) -> ProteinSearch:
    """Queries of length U[50, 1000] from a uniform background over 20 letters;
    a database of lengths clip(round(LogNormal(ln 300, 0.6)), 20, 5000), of
    which a fraction are homologs: copies of distinct random queries with each
    position redrawn from the background with probability 1 - identity."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    ql = rng.integers(50, 1001, n_queries).astype(np.int32)
    q, qo, ql = _random_arena(rng, ql, 20)
    dl = np.clip(np.rint(rng.lognormal(np.log(300), 0.6, n_db)), 20, 5000).astype(np.int32)
    n_h = int(round(homolog_frac * n_db))
    hom_db = rng.permutation(n_db)[:n_h]
    hom_q = rng.permutation(n_queries)[:n_h]
    dl[hom_db] = ql[hom_q]
    t, to, dl = _random_arena(rng, dl, 20)
    for d, qq in zip(hom_db, hom_q):
        src = q[qo[qq]: qo[qq] + ql[qq]].copy()
        redraw = rng.random(len(src)) >= identity
        src[redraw] = rng.integers(0, 20, int(redraw.sum()))
        t[to[d]: to[d] + dl[d]] = src
    W = synthetic_protein_matrix() if W is None else W
    b = Batch(f"protein_{n_queries}x{n_db}", q, qo, ql, t, to, dl, W, gap_open, gap_extend,
              PROTEIN, {"homolog_db": hom_db, "homolog_query": hom_q, "seed": seed})
    return ProteinSearch(b, n_queries, n_db)


@dataclass
class Request:
    arrival_s: float
    kind: int  # 1, 2 or 3: which DNA workload the pairs come from
    batch: Batch


def serving_trace(rate_per_s: float, n_requests=20_000, mix=(0.7, 0.2, 0.1), max_pairs=64,
                  seed=5, long_scale=1.0):
    """Poisson arrivals; each request draws its kind from ``mix`` and
    U{1..max_pairs} pairs of that kind (short 100x1000, short-read extension,
    long reads; ``long_scale`` shrinks the long-read lengths)."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    kinds = rng.choice(3, n_requests, p=np.asarray(mix) / sum(mix)) + 1
    npairs = rng.integers(1, max_pairs + 1, n_requests)
    seeds = rng.integers(0, 2**31 - 1, n_requests)
    reqs = []
    for a, k, n, s in zip(arrivals, kinds, npairs, seeds):
        if k == 1:
            b = dna_short_reads(int(n), (100, 100), (1000, 1000), 0.02, 0.002, 3, 0.0,
                                seed=int(s), name="req_short")
        elif k == 2:
            b = dna_short_reads(int(n), (100, 250), (300, 1000), 0.01, 0.001, 3, 0.10,
                                seed=int(s), name="req_extension")
        else:
            b = dna_long_reads(int(n), int(1000 * long_scale), int(20000 * long_scale),
                               seed=int(s), name="req_long")
        reqs.append(Request(float(a), int(k), b))
    return reqs


def reads_vs_reference(n_reads=1000, read_len=100, ref_len=10_000_000, p_sub=0.01, p_indel=0.001, seed=6):
    """One random reference of ref_len letters and n_reads reads of read_len
    sampled from it at uniform positions with substitutions and 1-3 nt indels
    (stands in for simulated Illumina reads of a chromosome region).  Returns
    (reads, ref): reads a Batch whose targets are unused (t of one letter)."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    ref = rng.integers(0, 4, ref_len).astype(np.uint8)
    starts = rng.integers(0, max(1, ref_len - read_len - 8), n_reads)
    src = np.concatenate([ref[s:s + read_len + 8] for s in starts])
    so = np.arange(n_reads, dtype=np.int64) * (read_len + 8)
    sl = np.full(n_reads, read_len + 8, np.int32)
    q, qo, ql = mutate(rng, src, so, sl, p_sub, p_indel / 2, p_indel / 2, 3)
    ql = np.minimum(ql, read_len).astype(np.int32)
    z = np.zeros(1, np.uint8)
    reads = Batch("reads", q, qo, ql, z, np.zeros(n_reads, np.int64), np.zeros(n_reads, np.int32),
                  dna_matrix(2, -2), 3, 1, DNA, {"starts": starts})
    return reads, ref


def overlap_reads(n_reads=22543, read_len=70, coverage=10.0, p_sub=0.01, seed=7):
    """Reads of read_len sampled at uniform positions of one random genome
    (length n_reads * read_len / coverage) with substitutions: the input of an
    all-vs-all read-overlap computation (stands in for a 22,543 x 70 bp read
    set).  Returns (seq arena, offsets, lengths)."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    g_len = max(read_len + 1, int(n_reads * read_len / coverage))
    genome = rng.integers(0, 4, g_len).astype(np.uint8)
    starts = rng.integers(0, g_len - read_len, n_reads)
    idx = starts[:, None] + np.arange(read_len)[None, :]
    seq = genome[idx].reshape(-1).copy()
    mut = rng.random(len(seq)) < p_sub
    seq[mut] = (seq[mut] + rng.integers(1, 4, int(mut.sum()))) % 4
    off = np.arange(n_reads, dtype=np.int64) * read_len
    return seq.astype(np.uint8), off, np.full(n_reads, read_len, np.int32)


def concat(batches, name="concat") -> Batch:
    """Concatenates batches that share scoring."""
    b0 = batches[0]
    q = np.concatenate([b.q for b in batches])
    t = np.concatenate([b.t for b in batches])
    qo = np.concatenate([b.q_off + s for b, s in zip(batches, np.cumsum([0] + [len(b.q) for b in batches[:-1]]))])
    to = np.concatenate([b.t_off + s for b, s in zip(batches, np.cumsum([0] + [len(b.t) for b in batches[:-1]]))])
    return Batch(name, q, qo.astype(np.int64), np.concatenate([b.q_len for b in batches]), t,
                 to.astype(np.int64), np.concatenate([b.t_len for b in batches]), b0.W,
                 b0.gap_open, b0.gap_extend, b0.alphabet)
