"""Stand-alone alignment tool: FASTA in, SAM (or a plain table) out.

    python -m paper_1208_6350_gb300.align [options] target.fa query.fa > out.sam

Every query is aligned against every target sequence on the GPU through the
library's batched path (gsw_align_batch; a target longer than --long letters
goes through gsw_align_to_reference's exact windows), and each query's best
target (largest score1, then the earlier target) is reported.  With -c the
reverse complement of each DNA query is aligned too and the better strand is
kept (SAM flag 16).  The tool mirrors the usage the paper describes: a
practical aligner for whole viral or bacterial genomes, and a validator of
read mappers (Results, Usage).

Output: SAM (default): QNAME FLAG RNAME POS MAPQ CIGAR * 0 0 SEQ * with tags
AS:i (score1), ZS:i (score2, the suboptimal score), and soft clips for the
query letters outside the alignment; unaligned queries (score1 = 0) get flag
4.  With --table: one line per query with the record's fields.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np

from . import gsw

DNA = "ACGT"
COMP = {0: 3, 1: 2, 2: 1, 3: 0}


def read_fasta(path):
    """[(name, sequence string)] of a FASTA file."""
    out, name, parts = [], None, []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith(">"):
                if name is not None:
                    out.append((name, "".join(parts)))
                name, parts = line[1:].split()[0] if len(line) > 1 else "", []
            else:
                parts.append(line)
    if name is not None:
        out.append((name, "".join(parts)))
    return out


def dna_matrix(match, mismatch):
    """4-letter DNA, plus N (code 4) scoring 0 against everything."""
    W = np.full((5, 5), mismatch, np.int8)
    np.fill_diagonal(W, match)
    W[4, :] = 0
    W[:, 4] = 0
    return W


def encode(seq, alphabet):
    lut = np.full(256, alphabet.index("N") if "N" in alphabet else 0, np.uint8)
    for k, a in enumerate(alphabet):
        lut[ord(a)] = k
        lut[ord(a.lower())] = k
    return lut[np.frombuffer(seq.encode(), np.uint8)]


def load_matrix(path, alphabet):
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    cols = rows[0]
    table = {r[0]: dict(zip(cols, map(int, r[1:]))) for r in rows[1:]}
    return np.array([[table[a][b] for b in alphabet] for a in alphabet], np.int8)


def arena(seqs):
    lens = np.array([len(s) for s in seqs], np.int32)
    offs = np.zeros(len(seqs), np.int64)
    if len(seqs):
        offs[1:] = np.cumsum(lens.astype(np.int64))[:-1]
    return (np.concatenate(seqs) if seqs else np.zeros(0, np.uint8)), offs, lens


def cigar_string(words, qlen, qb, qe):
    ops = "MID"
    s = f"{qb}S" if qb > 0 else ""
    s += "".join(f"{int(w) >> 4}{ops[int(w) & 15]}" for w in words)
    tail = qlen - 1 - qe
    return s + (f"{tail}S" if tail > 0 else "")


def align(targets, queries, W, O, X, alphabet, revcomp, long_cut, ctx):
    """Best (record, cigar words, target index, strand) per query."""
    t_codes = [encode(s, alphabet) for _, s in targets]
    q_codes = [encode(s, alphabet) for _, s in queries]
    strands = [q_codes]
    if revcomp:
        strands.append([np.array([COMP.get(int(x), int(x)) for x in c[::-1]], np.uint8) for c in q_codes])
    nq = len(q_codes)
    best = [None] * nq
    qarena, qoff, qlen = None, None, None
    for strand, qs in enumerate(strands):
        qarena, qoff, qlen = arena(qs)
        for ti, tc in enumerate(t_codes):
            if len(tc) > long_cut:
                res, cig, rc = ctx.align_to_reference(qarena, qoff, qlen, tc, W, O, X, gsw.GSW_CIGAR)
            else:
                toff = np.zeros(nq, np.int64)
                tlen = np.full(nq, len(tc), np.int32)
                res, cig, _, rc = ctx.align_host(qarena, qoff, qlen, tc, toff, tlen, W, O, X, gsw.GSW_CIGAR, -1,
                                                 int(qlen.sum() + nq * (len(tc) + 2) + 64))
            if rc != gsw.GSW_OK:
                raise SystemExit(f"alignment failed: {gsw.load().gsw_strerror(rc).decode()}")
            for p in range(nq):
                r = res[p]
                words = cig[r["cigar_off"]: r["cigar_off"] + r["cigar_len"]].copy() if r["cigar_len"] > 0 else []
                if best[p] is None or r["score1"] > best[p][0]["score1"]:
                    best[p] = (r.copy(), words, ti, strand, qs[p])
    return best


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("target")
    ap.add_argument("query")
    ap.add_argument("-m", "--match", type=int, default=2)
    ap.add_argument("-x", "--mismatch", type=int, default=2, help="mismatch penalty (positive)")
    ap.add_argument("-o", "--gap-open", type=int, default=3)
    ap.add_argument("-e", "--gap-extend", type=int, default=1)
    ap.add_argument("-p", "--protein", action="store_true", help="protein sequences (needs -a)")
    ap.add_argument("-a", "--matrix", help="score matrix file (protein)")
    ap.add_argument("-c", "--revcomp", action="store_true", help="also align the reverse complement (DNA)")
    ap.add_argument("-f", "--filter", type=int, default=0, help="report only alignments with score1 >= this")
    ap.add_argument("--table", action="store_true", help="plain table instead of SAM")
    ap.add_argument("--long", type=int, default=200000, help="targets longer than this use reference windows")
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args(argv)
    if args.protein:
        if not args.matrix:
            raise SystemExit("protein alignment needs a matrix file (-a)")
        alphabet = "ARNDCQEGHILKMFPSTWYV"
        W = load_matrix(args.matrix, alphabet)
    targets = read_fasta(args.target)
    queries = read_fasta(args.query)
    if not args.protein:
        # the 4-letter path unless a sequence holds another letter (then N, scoring 0)
        pure = all(set(s.upper()) <= set(DNA) for _, s in targets + queries)
        alphabet = DNA if pure else DNA + "N"
        W = dna_matrix(args.match, -abs(args.mismatch))
        if pure:
            W = np.ascontiguousarray(W[:4, :4])
    ctx = gsw.Context(args.device, 8 << 30)
    try:
        best = align(targets, queries, W, args.gap_open, args.gap_extend, alphabet,
                     args.revcomp and not args.protein, args.long, ctx)
    finally:
        ctx.close()
    out = sys.stdout
    if not args.table:
        out.write("@HD\tVN:1.6\tSO:unsorted\n")
        for name, seq in targets:
            out.write(f"@SQ\tSN:{name}\tLN:{len(seq)}\n")
        out.write("@PG\tID:gsw\tPN:paper_1208_6350_gb300.align\n")
    for (qname, qseq), b in zip(queries, best):
        r, words, ti, strand, qc = b
        s1 = int(r["score1"])
        shown = "".join(alphabet[int(x)] for x in qc)
        if args.table:
            out.write(f"{qname}\t{targets[ti][0]}\t{s1}\t{int(r['score2'])}\t{int(r['ref_begin1'])}\t"
                      f"{int(r['ref_end1'])}\t{int(r['read_begin1'])}\t{int(r['read_end1'])}\t{int(r['ref_end2'])}\t"
                      f"{'-' if strand else '+'}\t"
                      f"{cigar_string(words, len(qc), int(r['read_begin1']), int(r['read_end1'])) if s1 > 0 else '*'}\n")
            continue
        if s1 <= 0 or s1 < args.filter:
            out.write(f"{qname}\t4\t*\t0\t0\t*\t*\t0\t0\t{shown}\t*\n")
            continue
        flag = 16 if strand else 0
        cig = cigar_string(words, len(qc), int(r["read_begin1"]), int(r["read_end1"]))
        out.write(f"{qname}\t{flag}\t{targets[ti][0]}\t{int(r['ref_begin1']) + 1}\t255\t{cig}\t*\t0\t0\t{shown}\t*\t"
                  f"AS:i:{s1}\tZS:i:{int(r['score2'])}\n")


if __name__ == "__main__":
    main()
