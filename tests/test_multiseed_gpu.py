"""Several seeds per overlap on the same stored reads (two per overlap, as in assembly and
protein-search pipelines), through the C ABI.

The tuples of one overlap share their two sequences in the batch's sequence table; each
tuple is an independent seed extension.  The first seed's results must equal the one-seed
batch's bit for bit, and every tuple must match the oracle.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402


@pytest.mark.parametrize("X", [10, 20])
def test_two_seeds_per_overlap(X):
    one = synth.dna_longread(n_pairs=2000, X=X)
    two = synth.dna_longread(n_pairs=2000, X=X, seeds_per_pair=2)
    ctx = xdrop.xd_create(0)
    try:
        r1 = xdrop.extend_host(ctx, one)
        r2 = xdrop.extend_host(ctx, two)
    finally:
        xdrop.xd_destroy(ctx)
    assert r2[0::2].tobytes() == r1.tobytes()
    idx = np.arange(1, two.n_pairs, 2)[::8]
    L, R, T = oracle.run_batch(two.subset(idx), threads=8)
    for side, ref in (("left", L), ("right", R)):
        for f in ("score", "h_ext", "v_ext", "flags", "cells"):
            assert np.array_equal(r2[side][f][idx], ref[f]), (side, f)
    assert np.array_equal(r2["total"][idx], T)
