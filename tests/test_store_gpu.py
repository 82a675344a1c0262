"""Resident sequence store through the C ABI: sequences packed once per context, shared by
any number of later seed-tuple batches (xd_submit_pairs), deduplicated by content.

Results on the store must equal the same tuples submitted with their sequences
(xd_submit_batch) bit for bit.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402


def _poll(ctx, t, n):
    out = np.zeros(n, dtype=xdrop.RESULT_DTYPE)
    assert xdrop.xd_poll(ctx, t, out, -1) == xdrop.XD_OK
    return out


@pytest.mark.parametrize("make", [lambda: synth.dna_longread(n_pairs=1500),
                                  lambda: synth.protein(n_pairs=4000)], ids=["dna", "protein"])
def test_store_pairs_equal_host_batches(make):
    b = make()
    ctx = xdrop.xd_create(0)
    try:
        ref = xdrop.extend_host(ctx, b)
        h = xdrop.xd_store_add(ctx, b.alphabet, b.codes, b.offsets, b.lengths)
        n1, bytes1 = xdrop.xd_store_info(ctx, b.alphabet)
        assert n1 == len(np.unique(h))
        again = xdrop.xd_store_add(ctx, b.alphabet, b.codes, b.offsets, b.lengths)
        assert np.array_equal(again, h)                   # deduplicated: same handles
        assert xdrop.xd_store_info(ctx, b.alphabet) == (n1, bytes1)
        pairs = b.pairs.copy()
        pairs[:, 0] = h[b.pairs[:, 0]]
        pairs[:, 1] = h[b.pairs[:, 1]]
        kw = dict(match=b.match, mismatch=b.mismatch, gap=b.gap, matrix=b.matrix, X=b.X, delta=b.delta)
        # several requests in a row: they may be merged into one launch
        parts = np.array_split(np.arange(b.n_pairs), 5)
        tickets = [xdrop.xd_submit_pairs(ctx, b.alphabet, pairs[idx], **kw) for idx in parts]
        got = np.concatenate([_poll(ctx, t, len(idx)) for t, idx in zip(tickets, parts)])
        assert got.tobytes() == ref.tobytes()
        # the same reads with the seeds moved: a new batch on the stored sequences
        moved = b.pairs.copy()
        moved[:, 2] //= 2
        moved[:, 3] //= 2
        mb = synth.Batch(b.alphabet, b.codes, b.offsets, b.lengths, moved, b.match, b.mismatch, b.gap,
                         b.matrix, b.X, b.delta)
        ref2 = xdrop.extend_host(ctx, mb)
        pm = moved.copy()
        pm[:, 0] = h[moved[:, 0]]
        pm[:, 1] = h[moved[:, 1]]
        got2 = _poll(ctx, xdrop.xd_submit_pairs(ctx, b.alphabet, pm, **kw), b.n_pairs)
        assert got2.tobytes() == ref2.tobytes()
    finally:
        xdrop.xd_destroy(ctx)


def test_store_duplicates_within_one_call_and_bad_handles():
    seqs = ["ACGTACGTAC", "TTTTGGGGCC", "ACGTACGTAC", ""]
    codes = np.array(["ACGT".index(c) for c in "".join(seqs)], dtype=np.uint8)
    lens = np.array([len(x) for x in seqs], dtype=np.uint32)
    offs = np.concatenate([[0], np.cumsum(lens[:-1])]).astype(np.uint64)
    ctx = xdrop.xd_create(0)
    try:
        h = xdrop.xd_store_add(ctx, "dna", codes, offs, lens)
        assert h[0] == h[2] and len(set(h.tolist())) == 3
        pairs = np.array([[h[0], h[1], 0, 0, 0], [h[0], h[2], 2, 2, 3]], dtype=np.uint32)
        out = _poll(ctx, xdrop.xd_submit_pairs(ctx, "dna", pairs, X=5), 2)
        assert out["right"]["score"][1] == 5       # identical sequences: the rest matches
        with pytest.raises(xdrop.XdError) as e:
            xdrop.xd_submit_pairs(ctx, "dna", np.array([[h[0], 999, 0, 0, 0]], dtype=np.uint32), X=5)
        assert e.value.status == xdrop.XD_EINVAL
    finally:
        xdrop.xd_destroy(ctx)
