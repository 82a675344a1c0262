"""Seeded synthetic seed-extension workloads.

The paper evaluates X-Drop on PacBio HiFi overlaps extracted from the ELBA assembler
(E. coli, C. elegans) and on metaclust proteins in PASTIS (Sec. 5.2-5.3, Table 2).  Those
datasets are not available here, so every workload below is synthetic and seeded.  The
construction follows the paper's own synthetic generator idea (equal treatment of all
positions, uniform random mutations outside the seed, Sec. 5.2) and the shapes of the
long-read and protein workloads:

* ``dna_tiny``      1,000 pairs, query uniform ACGT of length U[1000, 5000], target =
                    query mutated at 5% substitutions / 5% insertions / 5% deletions, one
                    exact k=17 seed at a uniform surviving position, +1/-1/-1, X = 15.
* ``dna_longread``  100,000 dovetail pairs, read lengths lognormal (median 8 kbp,
                    sigma 0.6) clipped to [1 kbp, 30 kbp], overlap U[20%, 100%] of the
                    shorter read, per-pair error U[8%, 18%] with ins:del:sub = 1:1:1,
                    10% unrelated pairs, k = 17, +1/-1/-1, X in {10, 20, 50}.
* ``protein``       1,000,000 pairs, residues i.i.d. from background frequencies,
                    lengths lognormal (median 300, sigma 0.6) clipped to [50, 2000],
                    60% homologs (substitutions from a BLOSUM62-derived model at a
                    target identity U[30%, 90%] plus 2% indels of geometric length with
                    mean 2), 40% unrelated, k = 6, BLOSUM62, gap -2, X = 49.
* ``uneven``        200,000 DNA pairs, lengths log-uniform in [500, 100,000], error
                    U[5%, 20%] (ins:del:sub = 1:1:1), k = 17, X = 20, optional
                    memory-restricted window delta_b.

A workload is a :class:`Batch`: a flat array of residue codes (0..3 for DNA, 0..19 for
protein), per-sequence offsets and lengths, and per-pair seed tuples
``(h_id, v_id, h_seed, v_seed, seed_len)`` -- the paper's seed-extension tuple
e_c = (H, V, H_s, V_s) (Sec. 4.4) plus the seed length.  This module holds no alignment
arithmetic: it only draws sequences and seed positions.
"""
from dataclasses import dataclass, field
import ctypes
import hashlib
import os
import subprocess

import numpy as np

from .tables import BLOSUM62, BACKGROUND, substitution_model

DNA = "dna"
PROTEIN = "protein"
X_INF = 2**31 - 1   # "no pruning": any X >= 2**30 behaves as X = infinity


@dataclass
class Batch:
    alphabet: str
    codes: np.ndarray          # uint8, concatenated residue codes
    offsets: np.ndarray        # uint64 [n_seqs]
    lengths: np.ndarray        # uint32 [n_seqs]
    pairs: np.ndarray          # uint32 [n_pairs, 5]: h_id, v_id, h_seed, v_seed, seed_len
    match: int = 1
    mismatch: int = -1
    gap: int = -1
    matrix: np.ndarray = None  # int8 [20, 20] for protein
    X: int = 15
    delta: int = 0             # 0 = unrestricted
    name: str = ""
    meta: dict = field(default_factory=dict)
    zdrop: int = 0             # > 0: the Z-Drop rule with Z = zdrop on top of X-Drop

    @property
    def n_pairs(self):
        return int(self.pairs.shape[0])

    @property
    def n_seqs(self):
        return int(self.lengths.shape[0])

    def digest(self):
        """sha256 over every input byte (codes, layout, seeds, scoring, X, delta)."""
        h = hashlib.sha256()
        for a in (self.codes, self.offsets, self.lengths, self.pairs):
            h.update(np.ascontiguousarray(a).tobytes())
        h.update(np.array([self.match, self.mismatch, self.gap, self.X, self.delta, self.zdrop],
                          dtype=np.int64).tobytes())
        if self.matrix is not None:
            h.update(np.ascontiguousarray(self.matrix).tobytes())
        h.update(self.alphabet.encode())
        return h.hexdigest()

    def subset(self, idx):
        """Batch holding only the pairs ``idx`` (sequences re-packed, order kept)."""
        idx = np.asarray(idx, dtype=np.int64)
        p = self.pairs[idx]
        seq_ids = np.stack([p[:, 0], p[:, 1]], axis=1).reshape(-1).astype(np.int64)
        lens = self.lengths[seq_ids]
        offs = np.zeros(len(seq_ids), dtype=np.uint64)
        if len(seq_ids):
            offs[1:] = np.cumsum(lens[:-1], dtype=np.uint64)
        codes = _gather_segments(self.codes, self.offsets[seq_ids], lens)
        new_pairs = p.copy()
        new_pairs[:, 0] = np.arange(0, 2 * len(idx), 2, dtype=np.uint32)
        new_pairs[:, 1] = np.arange(1, 2 * len(idx), 2, dtype=np.uint32)
        return Batch(self.alphabet, codes, offs, lens.astype(np.uint32), new_pairs,
                     self.match, self.mismatch, self.gap, self.matrix, self.X, self.delta,
                     self.name + "[subset]", dict(self.meta), self.zdrop)

    def pair_range(self, a, b):
        """Batch of the pairs [a, b) sharing this batch's arrays where possible.

        Needs the generator layout (pair p uses sequences 2p and 2p+1, stored in order), so
        the codes of the range are one contiguous view; offsets and ids are rebased."""
        a, b = int(a), int(b)
        if not (0 <= a <= b <= self.n_pairs):
            raise ValueError("pair range out of bounds")
        ids = self.pairs[a:b, :2]
        if b > a and not (np.array_equal(ids[:, 0], np.arange(2 * a, 2 * b, 2)) and
                          np.array_equal(ids[:, 1], np.arange(2 * a + 1, 2 * b, 2))):
            raise ValueError("pair_range needs the generator's sequence layout")
        lens = self.lengths[2 * a:2 * b]
        base = int(self.offsets[2 * a]) if b > a else 0
        end = base + int(lens.astype(np.int64).sum())
        offs = self.offsets[2 * a:2 * b] - np.uint64(base)
        pairs = self.pairs[a:b].copy()
        pairs[:, :2] -= np.uint32(2 * a)
        return Batch(self.alphabet, self.codes[base:end], offs, lens, pairs,
                     self.match, self.mismatch, self.gap, self.matrix, self.X, self.delta,
                     f"{self.name}[{a}:{b}]", dict(self.meta), self.zdrop)

    def with_params(self, X=None, delta=None, zdrop=None):
        b = Batch(self.alphabet, self.codes, self.offsets, self.lengths, self.pairs,
                  self.match, self.mismatch, self.gap, self.matrix,
                  self.X if X is None else int(X), self.delta if delta is None else int(delta),
                  self.name, dict(self.meta), self.zdrop if zdrop is None else int(zdrop))
        return b


def _gather_segments(src, starts, lens):
    starts = np.asarray(starts, dtype=np.int64)
    lens = np.asarray(lens, dtype=np.int64)
    total = int(lens.sum())
    if total == 0:
        return np.zeros(0, dtype=np.uint8)
    seg_off = np.zeros(len(lens), dtype=np.int64)
    seg_off[1:] = np.cumsum(lens[:-1])
    idx = np.arange(total, dtype=np.int64) - np.repeat(seg_off - starts, lens)
    return src[idx]


def _segment_starts(lens):
    s = np.zeros(len(lens), dtype=np.int64)
    if len(lens):
        s[1:] = np.cumsum(lens[:-1])
    return s


_GEN = None


def _gen_lib():
    """Compile (once) and load the C pair constructor that lives beside this module."""
    global _GEN
    if _GEN is not None:
        return _GEN
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "_gen.c")
    out_dir = os.path.join(here, "_build")
    so = os.path.join(out_dir, "libsynthgen.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        os.makedirs(out_dir, exist_ok=True)
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, src])
        os.replace(tmp, so)
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    lib.gen_pairs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, P, P, ctypes.c_uint64,
                              P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]
    lib.gen_pairs.restype = ctypes.c_int
    _GEN = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _build(alphabet, k, seed, kind, lh, lv, ov, p_sub, p_ins, p_del, seeds_per_pair=1):
    """Construct all pairs with the C generator: sizing pass, layout, writing pass.

    Sequences are laid out H0, V0, H1, V1, ... so pair p uses ids (2p, 2p+1).  With two
    seeds per pair, tuples 2p and 2p+1 are the two seeds of pair p (same sequences)."""
    lib = _gen_lib()
    n = len(kind)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    lh = np.ascontiguousarray(lh, dtype=np.uint32)
    lv = np.ascontiguousarray(lv, dtype=np.uint32)
    ov = np.ascontiguousarray(ov, dtype=np.uint32)
    p_sub = np.ascontiguousarray(p_sub, dtype=np.float64)
    p_ins = np.ascontiguousarray(p_ins, dtype=np.float64)
    p_del = np.ascontiguousarray(p_del, dtype=np.float64)
    bg_cdf = np.ascontiguousarray(np.cumsum(BACKGROUND), dtype=np.float64)
    sub_cdf = np.ascontiguousarray(np.cumsum(substitution_model(), axis=1).reshape(-1), dtype=np.float64)
    alpha = 0 if alphabet == DNA else 1
    out_lv = np.zeros(n, dtype=np.uint32)
    hs = np.zeros(n, dtype=np.uint32)
    vs = np.zeros(n, dtype=np.uint32)
    hs2 = np.zeros(n, dtype=np.uint32) if seeds_per_pair == 2 else None
    vs2 = np.zeros(n, dtype=np.uint32) if seeds_per_pair == 2 else None
    threads = max(1, min(64, os.cpu_count() or 1))
    args = (alpha, k, seed, _ptr(bg_cdf), _ptr(sub_cdf), n, _ptr(kind), _ptr(lh), _ptr(lv), _ptr(ov),
            _ptr(p_sub), _ptr(p_ins), _ptr(p_del), _ptr(out_lv), _ptr(hs), _ptr(vs), _ptr(hs2), _ptr(vs2))
    lib.gen_pairs(*args, None, None, None, threads)
    lens = np.empty(2 * n, dtype=np.uint32)
    lens[0::2] = lh
    lens[1::2] = out_lv
    offs = _segment_starts(lens.astype(np.int64)).astype(np.uint64)
    codes = np.empty(int(lens.astype(np.int64).sum()), dtype=np.uint8)
    h_off = np.ascontiguousarray(offs[0::2])
    v_off = np.ascontiguousarray(offs[1::2])
    lib.gen_pairs(*args, _ptr(codes), _ptr(h_off), _ptr(v_off), threads)
    pairs = np.empty((n, 5), dtype=np.uint32)
    pairs[:, 0] = np.arange(0, 2 * n, 2)
    pairs[:, 1] = np.arange(1, 2 * n, 2)
    pairs[:, 2] = hs
    pairs[:, 3] = vs
    pairs[:, 4] = k
    if seeds_per_pair == 2:
        two = np.empty((2 * n, 5), dtype=np.uint32)
        two[0::2] = pairs
        two[1::2] = pairs
        two[1::2, 2] = hs2
        two[1::2, 3] = vs2
        pairs = two
    return codes, offs, lens, pairs


def _choose(rng, n, n_special):
    mask = np.zeros(n, dtype=bool)
    mask[rng.permutation(n)[:n_special]] = True
    return mask


def dna_tiny(n_pairs=1000, seed=42, X=15):
    """Plain-method DNA workload (5% sub / 5% ins / 5% del, k = 17, +1/-1/-1)."""
    rng = np.random.default_rng(seed)
    k = 17
    lh = rng.integers(1000, 5001, size=n_pairs)
    e = np.full(n_pairs, 0.05)
    z = np.zeros(n_pairs)
    codes, offs, lens, pairs = _build(DNA, k, seed, np.zeros(n_pairs), lh, z, z, e, e, e)
    return Batch(DNA, codes, offs, lens, pairs, 1, -1, -1, None, X, 0,
                 f"dna_tiny_{n_pairs}", {"seed": seed, "k": k})


def _lognormal_lengths(rng, n, median, sigma, lo, hi):
    return np.clip(np.exp(rng.normal(np.log(median), sigma, size=n)), lo, hi).astype(np.int64)


def dna_longread(n_pairs=100_000, seed=43, X=20, unrelated_frac=0.10, seeds_per_pair=1):
    """Long-read dovetail overlaps: query = read A, target = read B whose prefix is A's
    suffix (overlap U[20%, 100%] of the shorter read) carrying U[8%, 18%] error.  With
    seeds_per_pair = 2 every overlap gives two seed tuples on the same two stored reads (the
    two-seeds-per-overlap shape of the assembly and search pipelines; the sequences are the
    same as with one seed)."""
    rng = np.random.default_rng(seed)
    k = 17
    unrel = _choose(rng, n_pairs, int(round(n_pairs * unrelated_frac)))
    la = _lognormal_lengths(rng, n_pairs, 8000, 0.6, 1000, 30000)
    lb = _lognormal_lengths(rng, n_pairs, 8000, 0.6, 1000, 30000)
    ov = np.maximum(k + 1, (rng.uniform(0.2, 1.0, size=n_pairs) * np.minimum(la, lb)).astype(np.int64))
    e3 = rng.uniform(0.08, 0.18, size=n_pairs) / 3.0
    kind = np.where(unrel, 2, 1)
    codes, offs, lens, pairs = _build(DNA, k, seed, kind, la, lb, ov, e3, e3, e3, seeds_per_pair)
    name = f"dna_longread_{n_pairs}_x{X}" + ("_2seeds" if seeds_per_pair == 2 else "")
    return Batch(DNA, codes, offs, lens, pairs, 1, -1, -1, None, X, 0, name,
                 {"seed": seed, "k": k, "seeds_per_pair": seeds_per_pair})


def protein(n_pairs=1_000_000, seed=44, X=49, homolog_frac=0.60):
    """Protein-search pairs: BLOSUM62 homologs at 30-90% identity with 2% indels (half
    insertions, half deletions, geometric length with mean 2), plus unrelated pairs,
    k = 6, gap -2, X = 49."""
    rng = np.random.default_rng(seed)
    k = 6
    unrel = _choose(rng, n_pairs, n_pairs - int(round(n_pairs * homolog_frac)))
    lh = _lognormal_lengths(rng, n_pairs, 300, 0.6, 50, 2000)
    lv = _lognormal_lengths(rng, n_pairs, 300, 0.6, 50, 2000)
    p_sub = 1.0 - rng.uniform(0.30, 0.90, size=n_pairs)
    p_indel = np.full(n_pairs, 0.01)
    kind = np.where(unrel, 2, 0)
    codes, offs, lens, pairs = _build(PROTEIN, k, seed, kind, lh, lv, np.zeros(n_pairs),
                                      p_sub, p_indel, p_indel)
    return Batch(PROTEIN, codes, offs, lens, pairs, 0, 0, -2, np.array(BLOSUM62), X, 0,
                 f"protein_{n_pairs}", {"seed": seed, "k": k})


def uneven(n_pairs=200_000, seed=45, X=20, delta=0):
    """Uneven-length DNA homologs: log-uniform lengths in [500, 100000], U[5%, 20%] error."""
    rng = np.random.default_rng(seed)
    k = 17
    lh = np.exp(rng.uniform(np.log(500), np.log(100_000), size=n_pairs)).astype(np.int64)
    e3 = rng.uniform(0.05, 0.20, size=n_pairs) / 3.0
    z = np.zeros(n_pairs)
    codes, offs, lens, pairs = _build(DNA, k, seed, np.zeros(n_pairs), lh, z, z, e3, e3, e3)
    return Batch(DNA, codes, offs, lens, pairs, 1, -1, -1, None, X, int(delta),
                 f"uneven_{n_pairs}_d{delta}", {"seed": seed, "k": k})


def from_strings(pairs, alphabet=DNA, match=1, mismatch=-1, gap=-1, matrix=None, X=15, delta=0):
    """Small hand-made batch: ``pairs`` is a list of (H, V, h_seed, v_seed, seed_len) with
    H and V as strings over ACGT (DNA) or the 20 amino-acid letters (protein)."""
    letters = "ACGT" if alphabet == DNA else "ARNDCQEGHILKMFPSTWYV"
    lut = {c: i for i, c in enumerate(letters)}
    seqs, tup = [], []
    for n, (h, v, hs, vs, k) in enumerate(pairs):
        seqs.append(np.array([lut[c] for c in h], dtype=np.uint8))
        seqs.append(np.array([lut[c] for c in v], dtype=np.uint8))
        tup.append((2 * n, 2 * n + 1, hs, vs, k))
    lens = np.array([len(s) for s in seqs], dtype=np.uint32)
    offs = _segment_starts(lens.astype(np.int64)).astype(np.uint64)
    codes = np.concatenate(seqs) if seqs else np.zeros(0, dtype=np.uint8)
    p = np.array(tup, dtype=np.uint32).reshape(-1, 5)
    if alphabet == PROTEIN and matrix is None:
        matrix = np.array(BLOSUM62)
    return Batch(alphabet, codes, offs, lens, p, match, mismatch, gap, matrix, X, delta, "strings")


WORKLOADS = {
    "dna_tiny": dna_tiny,
    "dna_longread": dna_longread,
    "protein": protein,
    "uneven": uneven,
}
