"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle, bit for bit.

Every field is integer (score, h_ext, v_ext, flags, cells, total), so the tolerance is
zero.  Cases cover the hand traces, random tiny and ragged inputs, empty and length-1
sides, X = 0 and X = infinity, tiny and large restricted windows, every workload shape
at reduced size, and the long-read workload at full size (every pair) through the device
entry point in the launch configuration the bench times.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from synth import X_INF

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402

THREADS = max(1, os.cpu_count() or 1)
FIELDS = ("score", "h_ext", "v_ext", "flags", "cells")


# tiered: the default choice (batches this small take the latency chain, a warp per side);
# throughput / split: the X-based chains of large batches, fused or one launch per level;
# generic: every side in the generic tier
MODES = {"tiered": {}, "generic": {"XD_TIERS": "generic"},
         "throughput": {"XD_LATENCY_UNITS": "0"},
         "split": {"XD_LATENCY_UNITS": "0", "XD_FUSED": "0"},
         # DNA through the four-role fused grid (windows 32, 128, 256, 512)
         "four_roles": {"XD_LATENCY_UNITS": "0", "XD_CHAIN": "1,3,4,5,6", "XD_EVERY1": "16"},
         # the chains of launches with a million or more sides (1 x 32, 4 x 32, 8 x 32 and
         # 32 x 32 in the four-role three-block grid), here on every batch size
         "huge": {"XD_LATENCY_UNITS": "0", "XD_HUGE_UNITS": "0", "XD_EVERY1": "4", "XD_EVERY3": "8"}}
ENV_KEYS = ("XD_TIERS", "XD_FUSED", "XD_FUSED_PROT", "XD_LATENCY_UNITS", "XD_CHAIN", "XD_CHAIN_PROT",
            "XD_CHAIN_SMALL", "XD_EVERY1", "XD_EVERY3", "XD_HUGE_UNITS", "XD_BAND_WARPS")


def _ctx(mode, env=None):
    keys = ENV_KEYS
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ.pop(k, None)
    os.environ.update(MODES[mode] if env is None else env)
    try:
        return xdrop.xd_create(0)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module", params=["tiered", "throughput", "split", "generic", "four_roles", "huge"])
def ctx(request):
    c = _ctx(request.param)
    yield c
    xdrop.xd_destroy(c)


@pytest.fixture(scope="module")
def tiered():
    c = _ctx("tiered")
    yield c
    xdrop.xd_destroy(c)


def assert_parity(got, batch, idx=None):
    L, R, T = oracle.run_batch(batch, threads=THREADS)
    if idx is not None:
        L, R, T = L[idx], R[idx], T[idx]
    for side, ref in (("left", L), ("right", R)):
        for f in FIELDS:
            g = got[side][f]
            bad = np.nonzero(g != ref[f])[0]
            assert bad.size == 0, (f"{side}.{f} differs at pairs {bad[:10].tolist()}: "
                                   f"gpu {g[bad[:5]].tolist()} oracle {ref[f][bad[:5]].tolist()}")
    bad = np.nonzero(got["total"] != T)[0]
    assert bad.size == 0, f"total differs at {bad[:10].tolist()}"


def random_pairs(rng, n, alphabet, max_len, k_max=8, related=True):
    letters = "ACGT" if alphabet == "dna" else synth.AMINO_ACIDS
    rows = []
    for _ in range(n):
        lh, lv = int(rng.integers(1, max_len + 1)), int(rng.integers(1, max_len + 1))
        k = int(rng.integers(1, min(k_max, lh, lv) + 1))
        h = rng.choice(list(letters), lh)
        if related:
            v = h.copy()
            v = v[:lv] if lv <= lh else np.concatenate([v, rng.choice(list(letters), lv - lh)])
            flip = rng.random(lv) < rng.uniform(0.0, 0.4)
            v[flip] = rng.choice(list(letters), int(flip.sum()))
        else:
            v = rng.choice(list(letters), lv)
        hs, vs = int(rng.integers(0, lh - k + 1)), int(rng.integers(0, lv - k + 1))
        v[vs:vs + k] = h[hs:hs + k]
        rows.append(("".join(h), "".join(v), hs, vs, k))
    return rows


def test_hand_traces(ctx):
    """The hand-derived traces of tests/golden, run as right extensions with an empty seed."""
    here = os.path.dirname(os.path.abspath(__file__))
    cases, cur = [], None
    for ln in open(os.path.join(here, "golden", "hand_traces.txt")):
        ln = ln.rstrip("\n")
        if ln.startswith("case "):
            cur = {}
            cases.append(cur)
        elif cur is not None and ln and not ln.startswith("#"):
            k, _, v = ln.partition(" ")
            cur[k] = v.strip()
    for c in cases:
        b = synth.from_strings([(c["H"], c["V"], 0, 0, 0)], X=int(c["X"]), delta=int(c["delta"]))
        got = xdrop.extend_host(ctx, b)
        want = [int(x) for x in c["expect"].split()]
        assert [int(got["right"][0][f]) for f in FIELDS] == want, c
        assert_parity(got, b)


@pytest.mark.parametrize("alphabet", ["dna", "protein"])
@pytest.mark.parametrize("X", [0, 1, 3, 10, 49, X_INF])
def test_random_tiny(ctx, alphabet, X):
    rng = np.random.default_rng(100 + X % 1000 + (alphabet == "protein"))
    rows = random_pairs(rng, 300, alphabet, 40)
    gap = -1 if alphabet == "dna" else -2
    b = synth.from_strings(rows, alphabet=alphabet, gap=gap, X=X)
    assert_parity(xdrop.extend_host(ctx, b), b)


# DNA register levels keep scores in 16-bit halves when -127 <= gap <= 0 and
# 1022 - X - s_max - (2 (|gap| + s_max) + 1) >= 64, s_max = max(match, mismatch, 0)
# (else 32-bit levels): both sides of that bound for two scorings, and a gap of 0
@pytest.mark.parametrize("X,gap,match,mismatch", [
    (952, -1, 1, -1), (953, -1, 1, -1), (322, -127, 127, -127), (323, -127, 127, -127),
    (40, -127, 127, -127), (15000, -1, 1, -1), (40, 0, 2, -3), (40, -128, 5, -4)])
def test_score_ranges(ctx, X, gap, match, mismatch):
    rng = np.random.default_rng(7 + X - gap + match)
    rows = random_pairs(rng, 120, "dna", 500)
    b = synth.from_strings(rows, gap=gap, match=match, mismatch=mismatch, X=X)
    assert_parity(xdrop.extend_host(ctx, b), b)


@pytest.mark.parametrize("X", [500, 920, 921])
def test_protein_score_ranges(ctx, X):
    """BLOSUM62 with gap -2: packed levels up to X = 920, 32-bit beyond."""
    rng = np.random.default_rng(11 + X)
    rows = random_pairs(rng, 60, "protein", 400)
    b = synth.from_strings(rows, alphabet="protein", gap=-2, X=X)
    assert_parity(xdrop.extend_host(ctx, b), b)


@pytest.mark.parametrize("delta", [1, 2, 3, 7, 32, 33, 100])
def test_random_restricted(ctx, delta):
    rng = np.random.default_rng(delta)
    rows = random_pairs(rng, 200, "dna", 300)
    for X in (5, 30):
        b = synth.from_strings(rows, X=X, delta=delta)
        assert_parity(xdrop.extend_host(ctx, b), b)


def test_edges(ctx):
    rows = [
        ("ACGT", "ACGT", 0, 0, 4),          # both sides empty
        ("ACGTA", "ACGT", 0, 0, 4),         # right side m = 1, n = 0
        ("AACGT", "ACGT", 1, 0, 4),         # left side m = 1, n = 0
        ("A", "A", 0, 0, 1),
        ("CA", "GA", 1, 1, 1),              # left side 1 x 1 mismatch
        ("ACCCCCCCCCC", "AGGGGGGGGGG", 0, 0, 1),
        ("T" * 200, "T" * 200, 100, 100, 1),
        ("ACGT" * 50, "TGCA" * 50, 0, 0, 1),
    ]
    for X in (0, 1, 2, 15, X_INF):
        for delta in (0, 1, 4):
            b = synth.from_strings(rows, X=X, delta=delta)
            assert_parity(xdrop.extend_host(ctx, b), b)


@pytest.mark.parametrize("zdrop", [1, 3, 8, 40])
def test_zdrop_random(ctx, zdrop):
    """The Z-Drop rule (Sec. 1 names it; minimap2's definition) on top of X-Drop: random
    tiny and ragged pairs, DNA and protein, several X, unrestricted and restricted."""
    rng = np.random.default_rng(300 + zdrop)
    for alphabet, gap in (("dna", -1), ("protein", -2)):
        rows = random_pairs(rng, 250, alphabet, 120)
        for X in (5, 30, X_INF):
            for delta in (0, 16):
                b = synth.from_strings(rows, alphabet=alphabet, gap=gap, X=X, delta=delta).with_params(zdrop=zdrop)
                got = xdrop.extend_host(ctx, b)
                assert_parity(got, b)


@pytest.mark.parametrize("zdrop", [10, 50, 200])
def test_zdrop_workloads(ctx, zdrop):
    """Z-Drop on the workload shapes: long reads at X = 50 (wide random-walk bands that
    Z-Drop ends early), protein, and the uneven batch with a memory-restricted window."""
    batches = [synth.dna_longread(n_pairs=1500).with_params(X=50, zdrop=zdrop),
               synth.protein(n_pairs=5000).with_params(zdrop=zdrop),
               synth.uneven(n_pairs=60, delta=256).with_params(zdrop=zdrop)]
    fired = 0
    for b in batches:
        got = xdrop.extend_host(ctx, b)
        assert_parity(got, b)
        fired += int(((got["left"]["flags"] | got["right"]["flags"]) & 2).sum())
    # every live cell is at least T - X, so no anti-diagonal drops by more than X: with
    # Z >= X (X = 20, 49, 50 here) the rule can never end a side
    assert fired > 0 if zdrop < 20 else fired == 0


def test_dna_tiny_workload(ctx):
    b = synth.dna_tiny()
    assert_parity(xdrop.extend_host(ctx, b), b)


@pytest.mark.parametrize("X", [10, 20, 50])
def test_longread_shape(ctx, X):
    b = synth.dna_longread(n_pairs=1500).with_params(X=X)
    assert_parity(xdrop.extend_host(ctx, b), b)


def test_protein_shape(ctx):
    b = synth.protein(n_pairs=20000)
    assert_parity(xdrop.extend_host(ctx, b), b)


@pytest.mark.parametrize("delta", [0, 256, 1024, 4096])
def test_uneven_restricted_shape(ctx, delta):
    b = synth.uneven(n_pairs=150, delta=delta)
    assert_parity(xdrop.extend_host(ctx, b), b)


# Every compiled (lanes per side, slots per lane) variant, as a level of some chain, fused
# and as separate launches, on a mix of narrow and wide bands (DNA ids: 0 G1C16, 1 G1C32,
# 2 G4C16, 3 G8C16, 4 G16C16, 5 G32C16, 6 G32C32, 7 G4C32, 8 G8C32, 9 G16C32, 10 G4C8,
# 11 G8C8, 12 G16C8, 13 G32C8, 14 G1C24, 15 G1C20).
CHAINS_DNA = ["1,4,5,6", "0,2,4,6", "1,7,8,6", "1,3,5,6", "10,11,12,13,6", "0,3,9,6", "13,6", "2,4,6",
              "14,4,5,6", "15,4,5,6", "0,1,4,5,6", "1,13,5,6"]
CHAINS_PROT = ["2,4,6", "0,2,4,6", "3,5,6", "11,13,6", "13,6", "1,3,6", "14,4,6", "10,4,6"]


@pytest.fixture(scope="module")
def chain_batches():
    rng = np.random.default_rng(808)
    dna = [synth.dna_longread(n_pairs=200).with_params(X=X) for X in (10, 50)]
    dna.append(synth.from_strings(random_pairs(rng, 150, "dna", 400), X=30))
    # bands wider than every register window (X = infinity): these sides pass through all
    # levels to the band tier
    dna.append(synth.from_strings(random_pairs(rng, 12, "dna", 1600), X=X_INF))
    prot = [synth.protein(n_pairs=500),
            synth.from_strings(random_pairs(rng, 150, "protein", 300), alphabet="protein", gap=-2, X=80),
            synth.from_strings(random_pairs(rng, 10, "protein", 1400), alphabet="protein", gap=-2, X=X_INF)]
    return dna, prot


@pytest.mark.parametrize("fused", ["1", "0"])
@pytest.mark.parametrize("chain", CHAINS_DNA + ["p" + c for c in CHAINS_PROT])
def test_every_variant_chain(chain_batches, chain, fused):
    prot = chain.startswith("p")
    env = {"XD_LATENCY_UNITS": "0", "XD_FUSED": fused, "XD_FUSED_PROT": fused}
    env["XD_CHAIN_PROT" if prot else "XD_CHAIN"] = chain.lstrip("p")
    c = _ctx("tiered", env)
    try:
        for b in chain_batches[1 if prot else 0]:
            assert_parity(xdrop.extend_host(c, b), b)
    finally:
        xdrop.xd_destroy(c)


@pytest.mark.parametrize("nw", ["1", "2", "4", "16", "32"])
def test_band_tier_warps_per_side(chain_batches, nw):
    """The band tier with 1 - 32 warps per side (32 - 1024 threads per alignment): with a
    single 16-slot register level most sides reach it."""
    env = {"XD_LATENCY_UNITS": "0", "XD_CHAIN": "0", "XD_CHAIN_PROT": "0", "XD_BAND_WARPS": nw}
    c = _ctx("tiered", env)
    try:
        for b in chain_batches[0] + chain_batches[1]:
            assert_parity(xdrop.extend_host(c, b), b)
    finally:
        xdrop.xd_destroy(c)


def test_uneven_small_window_overflows(tiered):
    b = synth.uneven(n_pairs=100, delta=24, X=50)
    got = xdrop.extend_host(tiered, b)
    assert (got["left"]["flags"] | got["right"]["flags"]).any()
    assert_parity(got, b)


def _device_args(b):
    dev = torch.device("cuda", 0)
    codes = torch.from_numpy(b.codes).to(dev)
    offs = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
    lens = torch.from_numpy(b.lengths.view(np.int32)).to(dev)
    pairs = torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)
    args = xdrop.BatchArgs(b.alphabet, codes, offs, lens, pairs, b.match, b.mismatch, b.gap,
                           b.matrix, b.X, b.delta, b.zdrop)
    out = torch.zeros(b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    return args, out


def _results(out):
    return out.cpu().numpy().view(xdrop.RESULT_DTYPE)


def test_device_entry_matches_host_entry(tiered):
    b = synth.dna_longread(n_pairs=800)
    args, out = _device_args(b)
    xdrop.xd_run_device(tiered, args, out, None)
    torch.cuda.synchronize()
    assert xdrop.xd_device_status(tiered) == 0
    got = _results(out)
    host = xdrop.extend_host(tiered, b)
    assert np.array_equal(got, host)
    assert_parity(got, b)


def test_full_size_longread_all_pairs(tiered, oracle_all):
    """100,000 long-read pairs, X = 20, through xd_run_device as the bench runs it: every
    pair against the oracle, and every result for properties that hold at any size."""
    b = synth.dna_longread()
    args, out = _device_args(b)
    xdrop.xd_reserve(tiered, b.codes.size, b.n_seqs, b.n_pairs, int(b.lengths.max()))
    xdrop.xd_run_device(tiered, args, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert xdrop.xd_device_status(tiered) == 0
    got = _results(out)
    L, R, T = oracle_all(b)
    for side, ref in (("left", L), ("right", R)):
        for f in FIELDS:
            bad = np.nonzero(got[side][f] != ref[f])[0]
            assert bad.size == 0, f"{side}.{f} differs at {bad.size} pairs, first {bad[:10].tolist()}"
    assert np.array_equal(got["total"], T)
    p = b.pairs.astype(np.int64)
    lh, lv = b.lengths[p[:, 0]].astype(np.int64), b.lengths[p[:, 1]].astype(np.int64)
    r, l = got["right"], got["left"]
    assert (r["score"] >= 0).all() and (l["score"] >= 0).all()
    assert (r["h_ext"] <= lh - p[:, 2] - p[:, 4]).all() and (l["h_ext"] <= p[:, 2]).all()
    assert (r["v_ext"] <= lv - p[:, 3] - p[:, 4]).all() and (l["v_ext"] <= p[:, 3]).all()
    assert (r["cells"] >= 1).all() and (r["flags"] == 0).all()
    assert (got["total"] == r["score"].astype(np.int64) + l["score"] + p[:, 4]).all()


def test_invalid_inputs_rejected(tiered):
    good = synth.from_strings([("ACGT", "ACGT", 0, 0, 2)], X=3)
    bad_code = synth.from_strings([("ACGT", "ACGT", 0, 0, 2)], X=3)
    bad_code.codes = bad_code.codes.copy()
    bad_code.codes[1] = 7
    with pytest.raises(xdrop.XdError) as e:
        xdrop.extend_host(tiered, bad_code)
    assert e.value.status == xdrop.XD_EINVAL
    bad_seed = synth.from_strings([("ACGT", "ACGT", 3, 0, 2)], X=3)
    with pytest.raises(xdrop.XdError):
        xdrop.extend_host(tiered, bad_seed)
    neg_x = good.with_params(X=-1)
    with pytest.raises(xdrop.XdError):
        xdrop.extend_host(tiered, neg_x)
    prot = synth.from_strings([("ACDE", "ACDE", 0, 0, 2)], alphabet="protein", X=3)
    prot.matrix = None
    with pytest.raises(xdrop.XdError):
        xdrop.extend_host(tiered, prot)
    # the context stays usable
    assert_parity(xdrop.extend_host(tiered, good), good)


def test_poll_unknown_ticket(tiered):
    out = np.zeros(1, dtype=xdrop.RESULT_DTYPE)
    with pytest.raises(xdrop.XdError) as e:
        xdrop.xd_poll(tiered, 987654321, out, 0)
    assert e.value.status == xdrop.XD_ENOTFOUND
