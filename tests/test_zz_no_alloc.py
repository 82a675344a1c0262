"""The allocation-free entry point against xd_run_device and the oracle, through the C ABI.

xd_run_device_noalloc serves callers that cannot allocate device memory; it keeps its
scratch rows in a fixed array inside the library.  Its results must equal xd_run_device's
bit for bit (all outputs are integers), on two calls in a row (the second call reuses
whatever the first left in the shared array), and the oracle's.  Invalid pairs must be
flagged, not computed.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import X_INF

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402


def _device_batch(b):
    dev = torch.device("cuda", 0)
    codes = torch.from_numpy(b.codes).to(dev)
    offs = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
    lens = torch.from_numpy(b.lengths.view(np.int32)).to(dev)
    pairs = torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)
    return xdrop.BatchArgs(b.alphabet, codes, offs, lens, pairs, b.match, b.mismatch, b.gap,
                           b.matrix, b.X, b.delta, b.zdrop)


@pytest.mark.parametrize("make", [
    lambda: synth.dna_longread(n_pairs=300),
    lambda: synth.protein(n_pairs=1500),
    lambda: synth.uneven(n_pairs=40, delta=256),
    lambda: synth.from_strings([("ACGT", "ACGT", 0, 0, 4), ("A" * 50, "A" * 50, 25, 25, 1)], X=3),
    lambda: synth.dna_longread(n_pairs=200).with_params(X=50, zdrop=20),
], ids=["dna_longread", "protein", "uneven_restricted", "edges", "zdrop"])
def test_noalloc_matches_run_device_on_two_calls(make):
    b = make()
    args = _device_batch(b)
    n_bytes = b.n_pairs * xdrop.RESULT_DTYPE.itemsize
    ref = torch.zeros(n_bytes, dtype=torch.uint8, device="cuda")
    ctx = xdrop.xd_create(0)
    try:
        xdrop.xd_run_device(ctx, args, ref, None)
        torch.cuda.synchronize()
        assert xdrop.xd_device_status(ctx) == 0
    finally:
        xdrop.xd_destroy(ctx)
    max_side = int(b.lengths.max())
    for call in range(2):
        out = torch.full((n_bytes,), 0xAB, dtype=torch.uint8, device="cuda")
        assert xdrop.xd_run_device_noalloc(args, max_side, out, None) == xdrop.XD_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(xdrop.RESULT_DTYPE)
        want = ref.cpu().numpy().view(xdrop.RESULT_DTYPE)
        assert np.array_equal(got, want), f"call {call} differs from xd_run_device"
    L, R, T = oracle.run_batch(b, threads=8)
    for side, o in (("left", L), ("right", R)):
        for f in ("score", "h_ext", "v_ext", "flags", "cells"):
            assert np.array_equal(got[side][f], o[f]), (side, f)
    assert np.array_equal(got["total"], T)


def _noalloc(b, max_side, args=None):
    args = args or _device_batch(b)
    out = torch.full((b.n_pairs * xdrop.RESULT_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device="cuda")
    assert xdrop.xd_run_device_noalloc(args, max_side, out, None) == xdrop.XD_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().view(xdrop.RESULT_DTYPE)


INVALID = 0x80000000


def test_noalloc_flags_invalid_pairs_on_both_sides():
    rows = [("ACGTACGTAC", "ACGTACGTAC", 3, 3, 4)] * 4
    b = synth.from_strings(rows, X=5)
    b.pairs[1, 0] = b.n_seqs + 7                 # a sequence id past the table
    b.codes[int(b.offsets[4]) + 1] = 9           # a code outside the DNA alphabet (pair 2's H)
    got = _noalloc(b, 16)
    for p in (1, 2):
        assert got["left"]["flags"][p] & INVALID and got["right"]["flags"][p] & INVALID, p
    for p in (0, 3):
        assert not (got["left"]["flags"][p] & INVALID) and not (got["right"]["flags"][p] & INVALID), p
    # a side longer than max_side_len: H's right side is 10 - 3 - 4 = 3, its left side 3
    got = _noalloc(b.subset(np.array([0])), 2)
    assert got["left"]["flags"][0] & INVALID and got["right"]["flags"][0] & INVALID


def test_noalloc_single_warp_blocks_when_few_warps_fit():
    # three rows of 2,000,001 scores take about 24 MB: two warps fit the 64 MiB array, fewer
    # than a block of four, so the entry point launches single-warp blocks
    b = synth.dna_longread(n_pairs=40)
    L, R, T = oracle.run_batch(b, threads=8)
    for call in range(2):
        got = _noalloc(b, 2_000_000)
        for side, o in (("left", L), ("right", R)):
            for f in ("score", "h_ext", "v_ext", "flags", "cells"):
                assert np.array_equal(got[side][f], o[f]), (call, side, f)
        assert np.array_equal(got["total"], T), call


def test_noalloc_x_infinite_against_oracle():
    rng = np.random.default_rng(5)
    rows = []
    for _ in range(30):
        m, n = int(rng.integers(0, 60)), int(rng.integers(0, 60))
        h = "".join(rng.choice(list("ACGT"), m + 3))
        v = "".join(rng.choice(list("ACGT"), n + 3))
        rows.append((h, v, int(rng.integers(0, m + 1)), int(rng.integers(0, n + 1)), 3))
    for X in (1 << 30, X_INF):
        b = synth.from_strings(rows, X=X)
        got = _noalloc(b, 64)
        L, R, T = oracle.run_batch(b)
        for side, o in (("left", L), ("right", R)):
            for f in ("score", "h_ext", "v_ext", "flags", "cells"):
                assert np.array_equal(got[side][f], o[f]), (X, side, f)
        assert np.array_equal(got["total"], T)


def test_noalloc_rejects_sides_beyond_its_scratch():
    b = synth.from_strings([("ACGT", "ACGT", 0, 0, 2)], X=3)
    args = _device_batch(b)
    out = torch.zeros(xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    assert xdrop.xd_run_device_noalloc(args, 1 << 30, out, None) == xdrop.XD_EINVAL
