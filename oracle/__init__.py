"""CPU oracle for batched X-Drop seed extension (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  The CUDA library never loads it and shares no code with it.

The arithmetic lives in ``xdrop_oracle.c`` (plain single-threaded C, int64 scores, the
paper's Sec. 2.2 recurrence and X-Drop rule swept by anti-diagonals as in Algorithm 1).
This module only compiles it with gcc and marshals numpy arrays.  ``run_batch`` can run
independent pair ranges on several host threads (each call is single-threaded C; ctypes
releases the GIL), which is how large parity checks finish in reasonable time.

Parity status of each function (what pins it, all in ``tests/test_oracle_pins.py``):
  * orc_extend  -- pinned: X = inf equals the brute-force full DP maximum and cell count
                   (m+1)(n+1); identical sequences; all-mismatch closed forms; H/V swap;
                   exact integer scaling; left = right on reversed strings; restricted =
                   unrestricted without overflow; hand-derived traces in tests/golden.
                   The end-cell tie-break and the band rule are fixed readings (R3, R4);
                   between alternative readings they are pinned only by the hand traces.
  * orc_extend_z (Z-Drop, z > 0) -- pinned: against a dense-matrix restatement of the same
                   rules on random small inputs (several Z), equal to orc_extend when Z is
                   never reached, and identical sequences never trigger it.  Mutants of the
                   Z test are caught.
  * orc_batch   -- pinned through orc_extend plus the seed-score closed form: for DNA
                   (pin_pair_total, pin_left_is_right_on_reversed) and for protein
                   (pin_protein_batch: each side against orc_extend with a BLOSUM62 table
                   the test builds from the published entries, and the total against the
                   seed's BLOSUM62 sum computed in the test).
"""
import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xdrop_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")

SIDE_DTYPE = np.dtype([("score", np.int32), ("h_ext", np.uint32), ("v_ext", np.uint32),
                       ("flags", np.uint32), ("cells", np.uint64)])
assert SIDE_DTYPE.itemsize == 24

_LIB = None


def build(src=_SRC, so=_SO, extra_flags=()):
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(os.path.dirname(so), exist_ok=True)
    tmp = so + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra_flags,
                           "-o", tmp, src])
    os.replace(tmp, so)
    return so


def load(so=None):
    """Load (building if needed) the oracle shared library."""
    global _LIB
    if so is None:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            build()
        so = _SO
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    lib.orc_extend.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int64,
                               P, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, P]
    lib.orc_extend.restype = ctypes.c_int
    lib.orc_batch.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_uint64, ctypes.c_uint64,
                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P,
                              ctypes.c_int32, ctypes.c_uint32, P, P, P]
    lib.orc_batch.restype = ctypes.c_int
    lib.orc_extend_z.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int64,
                                 P, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32, P]
    lib.orc_extend_z.restype = ctypes.c_int
    lib.orc_batch_z.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P,
                                ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32, P, P, P]
    lib.orc_batch_z.restype = ctypes.c_int
    if so == _SO:
        _LIB = lib
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def sim_table(alphabet, match=1, mismatch=-1, matrix=None):
    """Dense similarity table as the oracle's C code expects it (int32, row-major)."""
    if alphabet == "dna":
        t = np.full((4, 4), mismatch, dtype=np.int32)
        np.fill_diagonal(t, match)
        return t
    return np.ascontiguousarray(np.asarray(matrix, dtype=np.int32).reshape(20, 20))


def extend(h_side, v_side, sim, gap, X, delta=0, lib=None, zdrop=0):
    """One side extension on already-oriented side strings (codes as uint8 arrays);
    zdrop > 0 adds the Z-Drop rule with Z = zdrop.

    Returns a dict with score, h_ext, v_ext, flags, cells."""
    lib = lib or load()
    h = np.ascontiguousarray(np.asarray(h_side, dtype=np.uint8))
    v = np.ascontiguousarray(np.asarray(v_side, dtype=np.uint8))
    sim = np.ascontiguousarray(np.asarray(sim, dtype=np.int32))
    hb = h if h.size else np.zeros(1, np.uint8)
    vb = v if v.size else np.zeros(1, np.uint8)
    out = np.zeros(1, dtype=SIDE_DTYPE)
    if zdrop:
        rc = lib.orc_extend_z(_p(hb), 1, h.size, _p(vb), 1, v.size, _p(sim), sim.shape[0],
                              int(gap), int(X), int(delta), int(zdrop), _p(out))
    else:
        rc = lib.orc_extend(_p(hb), 1, h.size, _p(vb), 1, v.size, _p(sim), sim.shape[0],
                            int(gap), int(X), int(delta), _p(out))
    if rc != 0:
        raise RuntimeError(f"orc_extend failed ({rc})")
    r = out[0]
    return {k: int(r[k]) for k in SIDE_DTYPE.names}


def run_batch(batch, first=0, count=None, threads=1, lib=None):
    """Oracle results for pairs [first, first+count) of a synth.Batch.

    Returns (left, right, total): two SIDE_DTYPE arrays and an int64 array, indexed from 0."""
    lib = lib or load()
    n = batch.n_pairs if count is None else int(count)
    alpha = 4 if batch.alphabet == "dna" else 20
    codes = np.ascontiguousarray(batch.codes, dtype=np.uint8)
    if codes.size == 0:
        codes = np.zeros(1, np.uint8)
    offs = np.ascontiguousarray(batch.offsets, dtype=np.uint64)
    lens = np.ascontiguousarray(batch.lengths, dtype=np.uint32)
    pairs = np.ascontiguousarray(batch.pairs, dtype=np.uint32)
    matrix = None if batch.matrix is None else np.ascontiguousarray(batch.matrix, dtype=np.int8)
    left = np.zeros(batch.n_pairs, dtype=SIDE_DTYPE)
    right = np.zeros(batch.n_pairs, dtype=SIDE_DTYPE)
    total = np.zeros(batch.n_pairs, dtype=np.int64)

    zdrop = int(getattr(batch, "zdrop", 0) or 0)

    def work(lo, hi):
        if zdrop:
            rc = lib.orc_batch_z(alpha, _p(codes), _p(offs), _p(lens), _p(pairs), lo, hi - lo,
                                 batch.match, batch.mismatch, batch.gap,
                                 None if matrix is None else _p(matrix), batch.X, batch.delta, zdrop,
                                 _p(left), _p(right), _p(total))
        else:
            rc = lib.orc_batch(alpha, _p(codes), _p(offs), _p(lens), _p(pairs), lo, hi - lo,
                               batch.match, batch.mismatch, batch.gap,
                               None if matrix is None else _p(matrix), batch.X, batch.delta,
                               _p(left), _p(right), _p(total))
        if rc != 0:
            raise RuntimeError(f"orc_batch failed ({rc})")

    threads = max(1, int(threads))
    if threads == 1 or n < 2 * threads:
        work(first, first + n)
    else:
        # many small ranges so that uneven pair costs balance across threads
        n_chunks = min(n, threads * 16)
        bounds = [first + (n * c) // n_chunks for c in range(n_chunks + 1)]
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda c: work(bounds[c], bounds[c + 1]), range(n_chunks)))
    return left[first:first + n], right[first:first + n], total[first:first + n]
