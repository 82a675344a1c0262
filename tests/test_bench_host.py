"""Host-side helpers of bench.py that need no GPU: the bench labels a batch as running on
16-bit packed scores (its roofline peak and dtype) by the same bound the library applies,
-127 <= gap <= 0 and (1022 - X - s_max) - (2 (s_max - gap) + 1) >= 64 with
s_max = max(similarity, 0); the GPU parity tests exercise both sides of that bound."""
import numpy as np
import pytest

import synth
from synth import X_INF

bench = pytest.importorskip("bench")


def _dna(X, gap=-1, match=1, mismatch=-1):
    return synth.from_strings([("ACGT", "ACGT", 0, 0, 1)], gap=gap, match=match, mismatch=mismatch, X=X)


def _prot(X, gap=-2):
    return synth.from_strings([("ARND", "ARND", 0, 0, 1)], alphabet="protein", gap=gap, X=X)


@pytest.mark.parametrize("X,gap,match,mismatch,packed", [
    (0, -1, 1, -1, True), (952, -1, 1, -1, True), (953, -1, 1, -1, False),
    (322, -127, 127, -127, True), (323, -127, 127, -127, False),
    (40, 0, 2, -3, True), (40, -128, 5, -4, False), (X_INF, -1, 1, -1, False),
    (40, -1, -1, -2, True)])
def test_packed_bound_dna(X, gap, match, mismatch, packed):
    assert bench.packed_scores(_dna(X, gap, match, mismatch)) is packed


@pytest.mark.parametrize("X,packed", [(49, True), (920, True), (921, False)])
def test_packed_bound_protein(X, packed):
    b = _prot(X)
    assert int(np.max(b.matrix)) == 11   # BLOSUM62's largest entry sets s_max
    assert bench.packed_scores(b) is packed
