"""The 16-bit packed score representation of the register levels, modelled step by step
on the CPU and checked against the oracle (no GPU).

The model follows the representation the kernels use (not their code): a score S of
anti-diagonal d is carried as 32 z with z = S - (B0 + gap d); a cell is
max(max(up, left), diag + 32 (Sim - 2 gap)); dead cells hold -1; a cell is live when its
value minus 32 theta is not negative, theta = T - X - (B0 + gap d); every value is
rebased (B0 += delta) once theta passes theta1 = 1022 - X - s_max, back to
theta0 = 2 (|gap| + s_max) + 1; the best cell comes from value + (31 - slot) keys.  Every
intermediate must fit a signed 16-bit half, and the results must equal the oracle's, at
the bound of the packed range (X, gap and scores at their extremes) and on inputs that
rebase often."""
import numpy as np
import pytest

import oracle
import synth

LO16, HI16 = -32768, 32767


def _h(x):
    assert LO16 <= x <= HI16, x
    return x


def packed_extend(H, V, sim, gap, X, delta=0):
    m, n = len(H), len(V)
    smax = max(int(sim.max()), 0)
    th0, th1 = 2 * (smax - gap) + 1, 1022 - X - smax
    assert th1 - th0 >= 64 and -127 <= gap <= 0
    sp_max = int(sim.max()) - 2 * gap
    B0 = -X - gap - th0
    P2, P1 = {}, {0: _h(-32 * B0)}        # anti-diagonals d-2, d-1: cell i -> value (absent: -1)
    T = best = bi = bj = barg = flags = 0
    L = U = 0
    cells, rebases, d = 1, 0, 1
    while True:
        lo, hi = max(L, d - n, 0), min(U + 1, m, d)
        if delta and hi - lo + 1 > delta:
            # memory-restricted window (Sec. 3): delta cells centred on d-1's best cell
            flags |= 1
            lo = max(lo, min(barg - delta // 2, hi - delta + 1))
            hi = lo + delta - 1
        zb = B0 + gap * d
        theta = T - X - zb
        if theta > th1:
            shift = theta - th0
            for row in (P1, P2):
                for k in row:
                    row[k] = max(_h(row[k] - _h(32 * shift)), -1)
            B0, zb, theta, rebases = B0 + shift, zb + shift, theta - shift, rebases + 1
        new, first, last, kmax = {}, None, None, -1
        for i in range(lo, hi + 1):
            j = d - i
            up, lf, dg = P1.get(i - 1, -1), P1.get(i, -1), P2.get(i - 1, -1)
            # outside the matrix the table holds whatever residue the slice carries: take the
            # largest similarity (the diagonal term is then dead-derived and must stay dead)
            sp = int(sim[H[i - 1], V[j - 1]]) - 2 * gap if i >= 1 and j >= 1 else sp_max
            raw = max(max(up, lf), _h(dg + _h(32 * sp)))
            live = _h(raw - 32 * _h(theta)) >= 0
            v = raw if live else -1
            if live:
                new[i] = v
                first = i if first is None else first
                last = i
                key = _h(v + 31)            # the largest slot key (slot 0)
                if v > kmax:
                    kmax, karg = v, i
        cells += hi - lo + 1
        if first is None:
            break
        assert kmax % 32 == 0
        wmax = kmax // 32 + zb
        if wmax > T:
            T = best = wmax
            bi, bj = karg, d - karg
        barg = karg
        L, U = first, last
        P2, P1 = P1, new
        if d == m + n:
            break
        d += 1
    return {"score": best, "h_ext": bi, "v_ext": bj, "flags": flags, "cells": cells}, rebases


def _cases(rng, alphabet, n, max_len):
    letters = synth.AMINO_ACIDS if alphabet == "protein" else "ACGT"
    lut = {c: k for k, c in enumerate(letters)}
    for _ in range(n):
        lh = int(rng.integers(1, max_len + 1))
        h = rng.choice(list(letters), lh)
        v = h.copy()
        flip = rng.random(lh) < rng.uniform(0.0, 0.35)
        v[flip] = rng.choice(list(letters), int(flip.sum()))
        if rng.random() < 0.3:
            v = rng.choice(list(letters), int(rng.integers(1, max_len + 1)))
        yield (np.array([lut[c] for c in h], np.uint8), np.array([lut[c] for c in v], np.uint8))


@pytest.mark.parametrize("match,mismatch,gap,X", [
    (1, -1, -1, 0), (1, -1, -1, 20), (1, -1, -1, 952),          # 952: the bound for 1/-1/-1
    (127, -127, -127, 322), (127, -127, -127, 40),             # 322: the bound at the extremes
    (2, -3, 0, 40), (-1, -2, -1, 30)])
def test_packed_model_dna(match, mismatch, gap, X):
    rng = np.random.default_rng(abs(match) * 1000 + X - gap)
    sim = oracle.sim_table("dna", match, mismatch)
    lib = oracle.load()
    n_rebased = 0
    for H, V in _cases(rng, "dna", 25, 160):
        got, rebases = packed_extend(H, V, sim, gap, X)
        want = oracle.extend(H, V, sim, gap, X, lib=lib)
        for k in ("score", "h_ext", "v_ext", "flags", "cells"):
            assert got[k] == want[k], (k, got, want)
        n_rebased += rebases > 0
    if X in (952, 322):
        assert n_rebased > 0   # the bound cases rebase within these lengths


@pytest.mark.parametrize("X", [49, 920])
def test_packed_model_protein(X):
    rng = np.random.default_rng(X)
    sim = oracle.sim_table("protein", matrix=synth.BLOSUM62)
    lib = oracle.load()
    for H, V in _cases(rng, "protein", 15, 120):
        got, _ = packed_extend(H, V, sim, -2, X)
        want = oracle.extend(H, V, sim, -2, X, lib=lib)
        for k in ("score", "h_ext", "v_ext", "cells"):
            assert got[k] == want[k], (k, got, want)


@pytest.mark.parametrize("delta", [1, 3, 8, 33])
def test_packed_model_restricted(delta):
    """The restricted window re-centres on the previous anti-diagonal's best cell, the one
    the value + (31 - slot) keys select (lowest i on ties)."""
    rng = np.random.default_rng(500 + delta)
    sim = oracle.sim_table("dna", 1, -1)
    lib = oracle.load()
    for X in (5, 30):
        for H, V in _cases(rng, "dna", 20, 150):
            got, _ = packed_extend(H, V, sim, -1, X, delta)
            want = oracle.extend(H, V, sim, -1, X, delta, lib=lib)
            for k in ("score", "h_ext", "v_ext", "flags", "cells"):
                assert got[k] == want[k], (k, got, want)
