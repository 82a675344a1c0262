"""Pins for the CPU oracle: facts fixed by the paper or by mathematics, not by the oracle.

Each ``pin_*`` function checks the oracle library it is given against something other
than the oracle itself: hand-derived traces (tests/golden), the textbook full dynamic
program (X = infinity, Sec. 2.2: "if X is large, the computation approaches filling the
entire dynamic programming matrix"), closed forms, symmetries and exact invariances, and
a structurally different dense-matrix restatement of the same rules.  ``test_mutants``
plants plausible mistakes in copies of the oracle source and checks that every one of
them breaks at least one pin.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from synth import X_INF

HERE = os.path.dirname(os.path.abspath(__file__))
DNA_SIM = oracle.sim_table("dna", 1, -1)
PROT_SIM = oracle.sim_table("protein", matrix=synth.BLOSUM62)
LUT = {c: i for i, c in enumerate("ACGT")}


def enc(s):
    return np.array([LUT[c] for c in s], dtype=np.uint8)


def ext(lib, h, v, sim, gap, X, delta=0, zdrop=0):
    r = oracle.extend(h, v, sim, gap, X, delta, lib=lib, zdrop=zdrop)
    return (r["score"], r["h_ext"], r["v_ext"], r["flags"], r["cells"])


# ---------------------------------------------------------------- independent references

def full_dp(h, v, sim, gap):
    """Textbook prefix DP over the whole (m+1) x (n+1) matrix (Sec. 2.2), S(0,0) = 0,
    off-matrix -inf.  Returns (max, i, j) with the end cell chosen as the smallest
    anti-diagonal i+j reaching the maximum, then the smallest i."""
    m, n = len(h), len(v)
    S = np.zeros((m + 1, n + 1), dtype=np.int64)
    for i in range(m + 1):
        for j in range(n + 1):
            if i == 0 and j == 0:
                continue
            c = []
            if i > 0 and j > 0:
                c.append(S[i - 1, j - 1] + sim[h[i - 1], v[j - 1]])
            if i > 0:
                c.append(S[i - 1, j] + gap)
            if j > 0:
                c.append(S[i, j - 1] + gap)
            S[i, j] = max(c)
    best = S.max()
    cells = [(i + j, i) for i in range(m + 1) for j in range(n + 1) if S[i, j] == best]
    d, i = min(cells)
    return int(best), i, d - i


def dense_xdrop(h, v, sim, gap, X, delta=0, zdrop=0):
    """The same rules restated on a dense matrix with per-cell live flags: the band of
    anti-diagonal d is read off the live flags of anti-diagonal d-1 in the full matrix,
    and predecessors are read from the full matrix.  No band bookkeeping is shared with
    the C oracle's three rotating arrays.  zdrop > 0: after each anti-diagonal, stop when
    the best cell so far beats the anti-diagonal's best live cell (lowest i) by more than
    zdrop + |gap| times the difference of their diagonals (minimap2's Z-Drop)."""
    m, n = len(h), len(v)
    S = np.zeros((m + 1, n + 1), dtype=np.int64)
    live = np.zeros((m + 1, n + 1), dtype=bool)
    live[0, 0] = True
    T, best, cells, flags = 0, (0, 0, 0), 1, 0
    for d in range(1, m + n + 1):
        prev = [i for i in range(0, m + 1) if 0 <= d - 1 - i <= n and live[i, d - 1 - i]]
        lo, hi = max(min(prev), d - n, 0), min(max(prev) + 1, m, d)
        if delta and hi - lo + 1 > delta:
            flags = 1
            b = min(prev, key=lambda i: (-S[i, d - 1 - i], i))
            lo = max(lo, min(b - delta // 2, hi - delta + 1))
            hi = lo + delta - 1
        new_t, any_live = T, False
        for i in range(lo, hi + 1):
            j = d - i
            c = []
            if i > 0 and j > 0 and live[i - 1, j - 1]:
                c.append(S[i - 1, j - 1] + sim[h[i - 1], v[j - 1]])
            if i > 0 and live[i - 1, j]:
                c.append(S[i - 1, j] + gap)
            if j > 0 and live[i, j - 1]:
                c.append(S[i, j - 1] + gap)
            cells += 1
            if c and max(c) >= T - X:
                live[i, j] = True
                S[i, j] = max(c)
                any_live = True
                if S[i, j] > new_t:
                    new_t, best = int(S[i, j]), (int(S[i, j]), i, j)
        if not any_live:
            break
        T = new_t
        if zdrop:
            on_d = [(int(S[i, d - i]), i) for i in range(lo, hi + 1) if live[i, d - i]]
            top = max(v_ for v_, _ in on_d)
            zi = min(i for v_, i in on_d if v_ == top)
            diag_shift = abs((zi - best[1]) - ((d - zi) - best[2]))
            if best[0] - top > zdrop + abs(gap) * diag_shift:
                flags |= 2
                break
    return best[0], best[1], best[2], flags, cells


# ---------------------------------------------------------------- pins

def _golden_cases():
    cases, cur = [], None
    for ln in open(os.path.join(HERE, "golden", "hand_traces.txt")):
        ln = ln.rstrip("\n")
        if ln.startswith("case "):
            cur = {"name": ln[5:].strip()}
            cases.append(cur)
        elif cur is not None and not ln.startswith("#") and ln.strip():
            key, _, val = ln.partition(" ")
            cur[key] = val
    return cases


def pin_hand_traces(lib):
    for c in _golden_cases():
        got = ext(lib, enc(c["H"].strip()), enc(c["V"].strip()), DNA_SIM, -1, int(c["X"]),
                  int(c["delta"]))
        want = tuple(int(x) for x in c["expect"].split())
        assert got == want, (c["name"], got, want)


def pin_x_infinite_is_full_dp(lib, trials=120, seed=7):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        prot = t % 3 == 2
        m, n = int(rng.integers(0, 11)), int(rng.integers(0, 11))
        a = 20 if prot else 4
        h, v = rng.integers(0, a, m), rng.integers(0, a, n)
        sim, gap = (PROT_SIM, -2) if prot else (DNA_SIM, -1)
        got = ext(lib, h, v, sim, gap, X_INF)
        assert got[:3] == full_dp(h, v, sim, gap), (h, v)
        assert got[3] == 0 and got[4] == (m + 1) * (n + 1)


def pin_identical_sequences(lib, seed=3):
    """Identical strings: the diagonal dominates every other path, so once the gap cells
    next to it on odd anti-diagonals survive (X >= |gap|) the best is l*match at (l, l).
    With X < |gap| both cells of anti-diagonal 1 are gap cells below T - X = -X and the
    sweep ends there: score 0 at (0, 0) after 3 cells."""
    rng = np.random.default_rng(seed)
    for ell in (1, 2, 7, 40, 300):
        h = rng.integers(0, 4, ell)
        for X in (1, 5, 100):
            got = ext(lib, h, h, DNA_SIM, -1, X)
            assert got[:3] == (ell, ell, ell), (ell, X, got)
        assert ext(lib, h, h, DNA_SIM, -1, 0) == (0, 0, 0, 0, 3)
        p = rng.integers(0, 20, ell)
        for X in (2, 49):
            got = ext(lib, p, p, PROT_SIM, -2, X)
            assert got[:3] == (sum(int(synth.BLOSUM62[c, c]) for c in p), ell, ell)
        assert ext(lib, p, p, PROT_SIM, -2, 1) == (0, 0, 0, 0, 3)


def pin_closed_forms(lib):
    # all-mismatch with X = 0: both cells of d = 1 fall below T - X = 0
    for ell in (1, 5, 30):
        assert ext(lib, enc("A" * ell), enc("C" * ell), DNA_SIM, -1, 0) == (0, 0, 0, 0, 3)
    # one empty side: gap cells (0, j) = j*gap live while j*|gap| <= X, plus one dead cell
    for n in (0, 1, 3, 20):
        for X in (0, 1, 4, 9):
            for gap in (-1, -3):
                got = ext(lib, enc(""), np.zeros(n, np.uint8), DNA_SIM, gap, X)
                assert got == (0, 0, 0, 0, 1 + min(n, X // -gap + 1)), (n, X, gap, got)


def pin_swap_symmetry(lib, trials=150, seed=11):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        prot = t % 2 == 1
        a = 20 if prot else 4
        m, n = int(rng.integers(0, 40)), int(rng.integers(0, 40))
        h, v = rng.integers(0, a, m), rng.integers(0, a, n)
        sim, gap, X = (PROT_SIM, -2, int(rng.integers(0, 30))) if prot else (DNA_SIM, -1, int(rng.integers(0, 8)))
        a1, a2 = ext(lib, h, v, sim, gap, X), ext(lib, v, h, sim, gap, X)
        assert (a1[0], a1[4]) == (a2[0], a2[4]), (h, v, X)


def pin_integer_scaling(lib, trials=100, seed=13):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        m, n = int(rng.integers(0, 40)), int(rng.integers(0, 40))
        h, v = rng.integers(0, 4, m), rng.integers(0, 4, n)
        X, c = int(rng.integers(0, 8)), int(rng.integers(2, 6))
        a1 = ext(lib, h, v, DNA_SIM, -1, X)
        a2 = ext(lib, h, v, DNA_SIM * c, -c, X * c)
        assert (a1[0] * c,) + a1[1:] == a2


def _pair_batch(rows, X, delta=0):
    return synth.from_strings(rows, X=X, delta=delta)


def pin_left_is_right_on_reversed(lib, trials=60, seed=17):
    rng = np.random.default_rng(seed)
    rows, rev = [], []
    for _ in range(trials):
        m, n, k = int(rng.integers(0, 60)), int(rng.integers(0, 60)), int(rng.integers(1, 6))
        h = "".join(rng.choice(list("ACGT"), m + k))
        v = "".join(rng.choice(list("ACGT"), n + k))
        hs, vs = int(rng.integers(0, m + 1)), int(rng.integers(0, n + 1))
        v = v[:vs] + h[hs:hs + k] + v[vs + k:]
        rows.append((h, v, hs, vs, k))
        rev.append((h[::-1], v[::-1], len(h) - hs - k, len(v) - vs - k, k))
    for X in (2, 6):
        L1, R1, T1 = oracle.run_batch(_pair_batch(rows, X), lib=lib)
        L2, R2, T2 = oracle.run_batch(_pair_batch(rev, X), lib=lib)
        assert np.array_equal(L1, R2) and np.array_equal(R1, L2) and np.array_equal(T1, T2)


def pin_pair_total(lib, seed=19):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(40):
        h = "".join(rng.choice(list("ACGT"), 50))
        v = "".join(rng.choice(list("ACGT"), 50))
        hs, vs, k = int(rng.integers(0, 40)), int(rng.integers(0, 40)), int(rng.integers(1, 10))
        rows.append((h, v, hs, vs, k))          # seed need not match: its score is summed
    b = _pair_batch(rows, 4)
    L, R, T = oracle.run_batch(b, lib=lib)
    for p, (h, v, hs, vs, k) in enumerate(rows):
        seed_score = sum(1 if h[hs + t] == v[vs + t] else -1 for t in range(k))
        assert T[p] == L[p]["score"] + R[p]["score"] + seed_score
        hl, vl = enc(h[:hs][::-1]), enc(v[:vs][::-1])
        hr, vr = enc(h[hs + k:]), enc(v[vs + k:])
        assert tuple(L[p]) == ext(lib, hl, vl, DNA_SIM, -1, 4)
        assert tuple(R[p]) == ext(lib, hr, vr, DNA_SIM, -1, 4)


PROT_LETTERS = "ARNDCQEGHILKMFPSTWYV"


def pin_protein_batch(lib, seed=31):
    """orc_batch on protein tuples (Sec. 2.2 scoring with a substitution matrix; Sec. 5.3:
    BLOSUM62, gap -2).  Each side must equal orc_extend on side strings cut out here, scored
    with a table built here from the published BLOSUM62 entries, and the pair total must add
    the seed's BLOSUM62 sum computed here; the seeds are random residues, so negative
    entries of the matrix take part."""
    rng = np.random.default_rng(seed)
    blosum = [[int(x) for x in row] for row in synth.BLOSUM62]
    table = np.array(blosum, dtype=np.int32)
    lut = {c: i for i, c in enumerate(PROT_LETTERS)}
    rows = []
    for t in range(50):
        m, n, k = int(rng.integers(0, 50)), int(rng.integers(0, 50)), int(rng.integers(1, 8))
        h = "".join(rng.choice(list(PROT_LETTERS), m + k))
        v = "".join(rng.choice(list(PROT_LETTERS), n + k))
        if t % 2 == 0 and min(m, n) > 0:
            # a related pair: V copies H around the seed with a few substitutions
            v = list(h[:n + k] + "".join(rng.choice(list(PROT_LETTERS), max(0, n + k - len(h)))))
            for q in rng.integers(0, len(v), len(v) // 5):
                v[q] = PROT_LETTERS[int(rng.integers(0, 20))]
            v = "".join(v)
        hs, vs = int(rng.integers(0, m + 1)), int(rng.integers(0, n + 1))
        rows.append((h, v, hs, vs, k))
    codes = lambda s: np.array([lut[c] for c in s], dtype=np.uint8)  # noqa: E731
    for X in (5, 49):
        b = synth.from_strings(rows, alphabet="protein", gap=-2, X=X)
        L, R, T = oracle.run_batch(b, lib=lib)
        for p, (h, v, hs, vs, k) in enumerate(rows):
            seed_score = sum(blosum[lut[h[hs + t]]][lut[v[vs + t]]] for t in range(k))
            assert T[p] == L[p]["score"] + R[p]["score"] + seed_score, (p, X)
            assert tuple(L[p]) == ext(lib, codes(h[:hs][::-1]), codes(v[:vs][::-1]), table, -2, X), (p, X)
            assert tuple(R[p]) == ext(lib, codes(h[hs + k:]), codes(v[vs + k:]), table, -2, X), (p, X)


def pin_dense_restatement(lib, trials=400, seed=23):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        prot = t % 4 == 3
        a = 20 if prot else 4
        m, n = int(rng.integers(0, 13)), int(rng.integers(0, 13))
        h, v = rng.integers(0, a, m), rng.integers(0, a, n)
        sim, gap = (PROT_SIM, -2) if prot else (DNA_SIM, -1)
        X = int(rng.integers(0, 12 if prot else 5))
        delta = int(rng.choice([0, 0, 1, 2, 3, 5]))
        assert ext(lib, h, v, sim, gap, X, delta) == dense_xdrop(h, v, sim, gap, X, delta), \
            (h, v, X, delta)


def pin_zdrop_dense_restatement(lib, trials=500, seed=37):
    """Z-Drop (the variant the paper names in Sec. 1; minimap2's definition) against the
    dense restatement, on random and related small inputs, several Z and X."""
    rng = np.random.default_rng(seed)
    hits = 0
    for t in range(trials):
        prot = t % 5 == 4
        a = 20 if prot else 4
        m, n = int(rng.integers(0, 15)), int(rng.integers(0, 15))
        h = rng.integers(0, a, m)
        v = rng.integers(0, a, n)
        if t % 2 == 0 and m and n:
            # a matching prefix followed by noise, where the anti-diagonal maxima fall away
            k = min(m, n, int(rng.integers(1, 8)))
            v[:k] = h[:k]
        sim, gap = (PROT_SIM, -2) if prot else (DNA_SIM, -1)
        X = int(rng.integers(3, 40 if prot else 12))
        z = int(rng.integers(1, 6))
        delta = int(rng.choice([0, 0, 0, 4]))
        got = ext(lib, h, v, sim, gap, X, delta, zdrop=z)
        assert got == dense_xdrop(h, v, sim, gap, X, delta, zdrop=z), (h, v, X, z, delta)
        hits += bool(got[3] & 2)
    assert hits > trials // 10, hits   # the rule fires in a good share of the cases


def pin_zdrop_closed_forms(lib, seed=41):
    """Z beyond any reachable drop changes nothing; identical sequences never trigger it
    (each anti-diagonal's best cell lies on the main diagonal, at most one gap below the
    best); a long matching prefix followed by all mismatches triggers it as soon as the
    drop exceeds Z + |gap| x the shift."""
    rng = np.random.default_rng(seed)
    for _ in range(40):
        m, n = int(rng.integers(0, 30)), int(rng.integers(0, 30))
        h, v = rng.integers(0, 4, m), rng.integers(0, 4, n)
        X = int(rng.integers(0, 8))
        assert ext(lib, h, v, DNA_SIM, -1, X, zdrop=1 << 29) == ext(lib, h, v, DNA_SIM, -1, X)
        g = rng.integers(0, 4, m)
        for z in (1, 2, 5):
            assert ext(lib, g, g, DNA_SIM, -1, 50, zdrop=z) == ext(lib, g, g, DNA_SIM, -1, 50)
    # A^8 then C^8 against A^8 then G^8, X large: the best is 8 at (8, 8) (d = 16); on
    # d = 16 + k the best cell is 8 - ceil(k/2) (k/2 mismatches down the diagonal, or one
    # more gap), on the diagonal for even k and one off it for odd k.  With Z = 2 the first
    # anti-diagonal whose drop exceeds 2 + shift is d = 22 (drop 3, shift 0): stop there.
    h = enc("A" * 8 + "C" * 8)
    v = enc("A" * 8 + "G" * 8)
    got = ext(lib, h, v, DNA_SIM, -1, 100, zdrop=2)
    assert got[:4] == (8, 8, 8, 2), got


def pin_restricted_without_overflow(lib, trials=120, seed=29):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        m, n = int(rng.integers(0, 80)), int(rng.integers(0, 80))
        h = rng.integers(0, 4, m)
        v = h[:n].copy() if n <= m else np.concatenate([h, rng.integers(0, 4, n - m)])
        flip = rng.random(len(v)) < 0.2
        v[flip] = rng.integers(0, 4, int(flip.sum()))
        X = int(rng.integers(0, 10))
        full = ext(lib, h, v, DNA_SIM, -1, X)
        for delta in (1, 4, 8, 16, 200):
            r = ext(lib, h, v, DNA_SIM, -1, X, delta)
            if r[3] == 0:
                assert r == full, (delta, r, full)
            else:
                assert delta < min(m, n) + 1


PINS = [pin_hand_traces, pin_x_infinite_is_full_dp, pin_identical_sequences, pin_closed_forms,
        pin_swap_symmetry, pin_integer_scaling, pin_left_is_right_on_reversed, pin_pair_total,
        pin_protein_batch, pin_dense_restatement, pin_restricted_without_overflow,
        pin_zdrop_dense_restatement, pin_zdrop_closed_forms]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.load())


def test_regression_pairs_not_monotone_in_x():
    lines = open(os.path.join(HERE, "golden", "regression_x_nonmonotone.txt")).read().splitlines()
    h = v = None
    n = 0
    for ln in lines:
        if ln.startswith("H "):
            h = enc(ln[2:])
        elif ln.startswith("V "):
            v = enc(ln[2:])
        elif ln.startswith("scores"):
            want = [int(x) for x in ln.split()[1:]]
            got = [ext(oracle.load(), h, v, DNA_SIM, -1, X)[0] for X in range(5)]
            assert got == want
            assert any(got[i] > got[i + 1] for i in range(4))
            n += 1
    assert n == 2


# ---------------------------------------------------------------- mutation check

MUTANTS = {
    "nonstrict_xdrop": ("int live = has && !(c < T - (int64_t)X);", "int live = has && !(c <= T - (int64_t)X);"),
    "running_T": ("int live = has && !(c < T - (int64_t)X);", "int live = has && !(c < T_new - (int64_t)X);"),
    "band_no_plus_one": ("int64_t lo = L, hi = U + 1;", "int64_t lo = L, hi = U;"),
    "band_wider_low": ("int64_t lo = L, hi = U + 1;", "int64_t lo = L - 1, hi = U + 1;"),
    "diag_from_P1": ("diag_live(P2, i - 1)) {", "diag_live(P1, i - 1)) {"),
    "gap_subtracted": ("int64_t t = P1->val[i - 1] + gap;", "int64_t t = P1->val[i - 1] - gap;"),
    "tie_break_last": ("if (c > T_new) {", "if (c >= T_new) {"),
    "cells_live_only": ("cells++;\n            int live = has && !(c < T - (int64_t)X);",
                        "int live = has && !(c < T - (int64_t)X); cells += live;"),
    "left_offset": ("rc = orc_extend_z(hs > 0 ? H + hs - 1 : H,", "rc = orc_extend_z(hs > 0 ? H + hs : H,"),
    "restricted_last_on_tie": ("(b < 0 || P1->val[i] > bv)", "(b < 0 || P1->val[i] >= bv)"),
    "restricted_no_flag": ("flags |= 1u;", ";"),
    "seed_not_scored": ("+ (int64_t)right[p].score + seed_score;", "+ (int64_t)right[p].score;"),
    "no_origin_cell": ("uint64_t cells = 1;", "uint64_t cells = 0;"),
    "centre_on_hi": ("int64_t centred = b - (int64_t)(delta / 2);", "int64_t centred = b;"),
    "matrix_sign_dropped": ("(int32_t)matrix[a * 20 + b]", "(int32_t)(uint8_t)matrix[a * 20 + b]"),
    "zdrop_nonstrict": ("if (best - zv > (int64_t)z + (-(int64_t)gap) * shift)",
                        "if (best - zv >= (int64_t)z + (-(int64_t)gap) * shift)"),
    "zdrop_no_shift_term": ("(int64_t)z + (-(int64_t)gap) * shift)", "(int64_t)z)"),
    "zdrop_last_on_tie": ("if (C->live[i] && (zi < 0 || C->val[i] > zv))",
                          "if (C->live[i] && (zi < 0 || C->val[i] >= zv))"),
    "zdrop_no_flag": ("{ flags |= 2u; break; }", "{ break; }"),
    "protein_scored_as_dna": ("alpha == 20 ? (int32_t)matrix[a * 20 + b] : (a == b ? match : mismatch)",
                              "(a == b ? match : mismatch)"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutants(name, tmp_path):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    mutated = src.replace(old, new)
    path = tmp_path / "mutant.c"
    path.write_text(mutated)
    so = oracle.build(str(path), str(tmp_path / "libmutant.so"))
    lib = oracle.load(so)
    failed = []
    for pin in PINS:
        try:
            pin(lib)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passes every pin"
