"""Synthetic workloads: seeded, valid seed tuples, and the documented shapes."""
import numpy as np
import pytest

import synth


def _seeds_exact(b, n=500):
    p = b.pairs.astype(np.int64)
    for r in p[:n]:
        h = b.codes[b.offsets[r[0]]:b.offsets[r[0]] + b.lengths[r[0]]]
        v = b.codes[b.offsets[r[1]]:b.offsets[r[1]] + b.lengths[r[1]]]
        k = r[4]
        assert r[2] + k <= len(h) and r[3] + k <= len(v)
        assert np.array_equal(h[r[2]:r[2] + k], v[r[3]:r[3] + k])


def test_dna_tiny_shape_and_determinism():
    b = synth.dna_tiny()
    assert b.n_pairs == 1000 and b.X == 15 and b.alphabet == "dna"
    h_len = b.lengths[0::2]
    assert h_len.min() >= 1000 and h_len.max() <= 5000
    assert b.codes.max() < 4
    _seeds_exact(b)
    assert synth.dna_tiny().digest() == b.digest()
    assert synth.dna_tiny(seed=1).digest() != b.digest()


def test_longread_and_protein_small():
    b = synth.dna_longread(n_pairs=2000)
    assert b.lengths.min() >= 17 and b.lengths.max() <= 60000
    _seeds_exact(b)
    p = synth.protein(n_pairs=5000)
    assert p.codes.max() < 20 and p.gap == -2 and p.X == 49 and p.matrix.shape == (20, 20)
    _seeds_exact(p)
    u = synth.uneven(n_pairs=300, delta=256)
    assert u.delta == 256
    _seeds_exact(u)


def test_blosum62_invariants():
    m = synth.BLOSUM62.astype(int)
    assert m.shape == (20, 20) and (m == m.T).all()
    assert m.min() >= -4 and m.max() <= 11
    d = np.diag(m)
    assert (d > 0).all()
    for a in range(20):
        assert all(d[a] > m[a, b] for b in range(20) if b != a)
    assert abs(synth.BACKGROUND.sum() - 1) < 1e-12


def test_subset_roundtrip():
    b = synth.dna_tiny(n_pairs=50)
    s = b.subset([3, 7, 11])
    assert s.n_pairs == 3
    for new, old in enumerate([3, 7, 11]):
        for side in (0, 1):
            o = b.pairs[old, side]
            n_ = s.pairs[new, side]
            assert np.array_equal(b.codes[b.offsets[o]:b.offsets[o] + b.lengths[o]],
                                  s.codes[s.offsets[n_]:s.offsets[n_] + s.lengths[n_]])


def test_pair_range_matches_subset():
    b = synth.dna_longread(n_pairs=200)
    for a, e in ((0, 0), (0, 1), (17, 90), (150, 200)):
        r = b.pair_range(a, e)
        s = b.subset(np.arange(a, e))
        assert np.array_equal(r.codes, s.codes)
        assert np.array_equal(r.offsets, s.offsets)
        assert np.array_equal(r.lengths, s.lengths)
        assert np.array_equal(r.pairs, s.pairs)
    with pytest.raises(ValueError):
        b.pair_range(5, 201)
    with pytest.raises(ValueError):
        b.pair_range(-1, 2)
    with pytest.raises(ValueError):
        _swap(b).pair_range(0, 2)      # not the generator's layout


def _swap(b):
    p = b.pairs.copy()
    p[:, [0, 1]] = p[:, [1, 0]]
    return synth.Batch(b.alphabet, b.codes, b.offsets, b.lengths, p)


def test_two_seeds_per_overlap_share_the_reads():
    one = synth.dna_longread(n_pairs=300)
    two = synth.dna_longread(n_pairs=300, seeds_per_pair=2)
    assert np.array_equal(one.codes, two.codes) and np.array_equal(one.offsets, two.offsets)
    assert two.n_pairs == 2 * one.n_pairs
    assert np.array_equal(two.pairs[0::2], one.pairs)
    assert np.array_equal(two.pairs[1::2, :2], one.pairs[:, :2])
    p = two.pairs.astype(np.int64)
    k = 17
    h = two.codes[(two.offsets[p[:, 0]].astype(np.int64) + p[:, 2])[:, None] + np.arange(k)]
    v = two.codes[(two.offsets[p[:, 1]].astype(np.int64) + p[:, 3])[:, None] + np.arange(k)]
    assert (h == v).all()                                  # every seed is an exact k-mer match
    d = np.abs(p[1::2, 2] - p[0::2, 2])
    assert ((d == 0) | (d >= k)).all()                     # second seeds do not overlap the first
    assert (d > 0).mean() > 0.5
