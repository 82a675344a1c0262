"""Full-size parity of every workload, through xd_run_device in the launch configuration
the bench times: every pair of every batch against the oracle (run on all host cores),
all five result fields and the total, bit for bit.

Batches: DNA tiny (1,000 pairs, X = 15), DNA long-read (100,000 pairs) at X = 10, 20 and
50, protein (1,000,000 pairs, BLOSUM62, X = 49), and the uneven batch (200,000 pairs)
unrestricted and with the memory-restricted window delta_b = 256, 1024, 4096.  Every pair
is also checked for properties that hold at any size (score and extension bounds, the
total), and the restricted runs for equality with the unrestricted one wherever the
window was never exceeded (the paper's claim for the memory-restricted variant, Sec. 3).
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402

THREADS = max(1, os.cpu_count() or 1)
FIELDS = ("score", "h_ext", "v_ext", "flags", "cells")


def _run_device(ctx, b):
    dev = torch.device("cuda", 0)
    codes = torch.from_numpy(b.codes).to(dev)
    offs = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
    lens = torch.from_numpy(b.lengths.view(np.int32)).to(dev)
    pairs = torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)
    args = xdrop.BatchArgs(b.alphabet, codes, offs, lens, pairs, b.match, b.mismatch, b.gap,
                           b.matrix, b.X, b.delta)
    out = torch.zeros(b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    xdrop.xd_reserve(ctx, b.codes.size, b.n_seqs, b.n_pairs, int(b.lengths.max()))
    xdrop.xd_run_device(ctx, args, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert xdrop.xd_device_status(ctx) == 0
    res = out.cpu().numpy().view(xdrop.RESULT_DTYPE).copy()
    del codes, offs, lens, pairs, out
    return res


def _all_parity(got, b, ref):
    L, R, T = ref
    assert len(L) == b.n_pairs == len(got)
    for side, o in (("left", L), ("right", R)):
        for f in FIELDS:
            bad = np.nonzero(got[side][f] != o[f])[0]
            assert bad.size == 0, f"{side}.{f} differs at {bad.size} pairs, first {bad[:10].tolist()}"
    bad = np.nonzero(got["total"] != T)[0]
    assert bad.size == 0, f"total differs at {bad.size} pairs, first {bad[:10].tolist()}"


def _seed_scores(b):
    p = b.pairs.astype(np.int64)
    k = int(p[0, 4]) if len(p) else 0
    assert (p[:, 4] == k).all()
    h = b.codes[(b.offsets[p[:, 0]].astype(np.int64) + p[:, 2])[:, None] + np.arange(k)]
    v = b.codes[(b.offsets[p[:, 1]].astype(np.int64) + p[:, 3])[:, None] + np.arange(k)]
    if b.alphabet == "dna":
        sim = np.where(h == v, b.match, b.mismatch)
    else:
        sim = np.asarray(b.matrix, dtype=np.int64)[h, v]
    return sim.sum(axis=1)


def _properties(got, b):
    p = b.pairs.astype(np.int64)
    lh, lv = b.lengths[p[:, 0]].astype(np.int64), b.lengths[p[:, 1]].astype(np.int64)
    r, l = got["right"], got["left"]
    assert (r["score"] >= 0).all() and (l["score"] >= 0).all()
    assert (r["h_ext"] <= lh - p[:, 2] - p[:, 4]).all() and (l["h_ext"] <= p[:, 2]).all()
    assert (r["v_ext"] <= lv - p[:, 3] - p[:, 4]).all() and (l["v_ext"] <= p[:, 3]).all()
    assert (r["cells"] >= 1).all() and (l["cells"] >= 1).all()
    assert (got["total"] == r["score"].astype(np.int64) + l["score"] + _seed_scores(b)).all()


@pytest.fixture(scope="module")
def ctx():
    c = xdrop.xd_create(0)
    yield c
    xdrop.xd_destroy(c)


def test_full_size_dna_tiny_all_pairs(ctx, oracle_all):
    """1,000 pairs, 1-5 kbp, 15% error, X = 15."""
    b = synth.dna_tiny()
    got = _run_device(ctx, b)
    _properties(got, b)
    _all_parity(got, b, oracle_all(b))


@pytest.mark.parametrize("X", [10, 20, 50])
def test_full_size_longread_all_pairs(ctx, oracle_all, X):
    """100,000 long-read pairs (lognormal lengths, median 8 kbp, 8-18% error)."""
    b = synth.dna_longread().with_params(X=X)
    got = _run_device(ctx, b)
    _properties(got, b)
    assert (got["right"]["flags"] == 0).all() and (got["left"]["flags"] == 0).all()
    _all_parity(got, b, oracle_all(b))


def test_full_size_protein_all_pairs(ctx, oracle_all):
    """1,000,000 protein pairs, BLOSUM62, gap -2, X = 49."""
    b = synth.protein()
    got = _run_device(ctx, b)
    _properties(got, b)
    assert (got["right"]["flags"] == 0).all() and (got["left"]["flags"] == 0).all()
    _all_parity(got, b, oracle_all(b))


@pytest.fixture(scope="module")
def uneven():
    return synth.uneven()


@pytest.fixture(scope="module")
def uneven_unrestricted(ctx, uneven):
    return _run_device(ctx, uneven)


def test_full_size_uneven_unrestricted_all_pairs(uneven, uneven_unrestricted, oracle_all):
    """200,000 DNA pairs, lengths log-uniform in [500, 100,000], X = 20."""
    _properties(uneven_unrestricted, uneven)
    _all_parity(uneven_unrestricted, uneven, oracle_all(uneven))


@pytest.mark.parametrize("delta", [256, 1024, 4096])
def test_full_size_uneven_restricted_all_pairs(ctx, uneven, uneven_unrestricted, oracle_all, delta):
    b = uneven.with_params(delta=delta)
    got = _run_device(ctx, b)
    _properties(got, b)
    for side in ("left", "right"):
        f = got[side]["flags"]
        assert ((f == 0) | (f == 1)).all()
        clear = f == 0
        for fld in FIELDS:
            assert np.array_equal(got[side][fld][clear], uneven_unrestricted[side][fld][clear]), (side, fld)
    _all_parity(got, b, oracle_all(b))


def _ctx_env(env):
    keys = ("XD_FUSED", "XD_FUSED_PROT", "XD_EVERY1", "XD_EVERY2", "XD_EVERY3", "XD_LONG_PERMILLE", "XD_CHAIN",
            "XD_FUSED_MINB", "XD_FUSED4", "XD_CHAIN_PROT")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ.pop(k, None)
    os.environ.update(env)
    try:
        return xdrop.xd_create(0)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("X,chain,minb,roles", [(10, None, None, 4), (20, None, None, 4), (50, None, None, 4),
                                                (20, "1,3,4,5,6", None, 4), (20, "1,7,8,6", "3", 4),
                                                (10, "1,7,8,6", "3", 4), (50, "1,7,8,6", "3", 4),
                                                (20, "1,7,8,6", "3", 3), (20, "1,7,8,9", "3", 4),
                                                (20, "1,7,8,5", "3", 4), (20, "1,7,8,6", "4", 3),
                                                (10, "15,7,8,6", "4", 3), (20, "14,7,8,6", "4", 3)])
def test_full_size_fused_grid_equals_level_launches(X, chain, minb, roles):
    """Every one of the 100,000 long-read pairs: the persistent grid whose warps run
    different group shapes at once (and the long-side role) must give exactly the results of
    one launch per register level; also the four-role grids (windows 32, 128, 256, 512 and the
    32-slot wide levels followed by 16 x 32, 32 x 32 or 32 x 16), and the three-role grid
    followed by a separate launch of the fourth level."""
    b = synth.dna_longread().with_params(X=X)
    extra = {"XD_CHAIN": chain, "XD_EVERY3": "8"} if chain else {}
    if minb:
        extra["XD_FUSED_MINB"] = minb
    if roles == 3:
        extra["XD_FUSED4"] = "0"
    fused = _ctx_env({"XD_EVERY1": "2", "XD_EVERY2": "4", "XD_LONG_PERMILLE": "5", **extra})
    split = _ctx_env({"XD_FUSED": "0", **({"XD_CHAIN": chain} if chain else {})})
    try:
        a = _run_device(fused, b)
        c = _run_device(split, b)
    finally:
        xdrop.xd_destroy(fused)
        xdrop.xd_destroy(split)
    diff = np.nonzero((a.view(np.uint8).reshape(len(a), -1) != c.view(np.uint8).reshape(len(c), -1)).any(axis=1))[0]
    assert diff.size == 0, f"{diff.size} pairs differ, first {diff[:10].tolist()}"


@pytest.mark.parametrize("X", [10, 20, 50])
def test_full_size_longread_ten_batches_per_launch_all_pairs(ctx, oracle_all, X):
    """Ten long-read batches of 100,000 pairs in one pass (xd_run_device_many), the launch
    the bench times by default: every pair of every batch against the oracle."""
    b = synth.dna_longread().with_params(X=X)
    dev = torch.device("cuda", 0)
    keep = [torch.from_numpy(b.codes).to(dev), torch.from_numpy(b.offsets.view(np.int64)).to(dev),
            torch.from_numpy(b.lengths.view(np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)]
    args = xdrop.BatchArgs(b.alphabet, *keep, b.match, b.mismatch, b.gap, b.matrix, b.X, b.delta)
    k = 10
    out = torch.zeros(k * b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    xdrop.xd_reserve(ctx, k * b.codes.size, k * b.n_seqs, k * b.n_pairs, int(b.lengths.max()))
    xdrop.xd_run_device_many(ctx, [args] * k, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert xdrop.xd_device_status(ctx) == 0
    res = out.cpu().numpy().view(xdrop.RESULT_DTYPE)
    ref = oracle_all(b)
    for j in range(k):
        _all_parity(res[j * b.n_pairs:(j + 1) * b.n_pairs].copy(), b, ref)


def test_full_size_protein_fused_grid_all_pairs(oracle_all):
    """1,000,000 protein pairs through the persistent grid of the 16-slot protein levels
    (4 x 16 -> 8 x 16 -> 16 x 16, then 32 x 32): every pair against the oracle."""
    b = synth.protein()
    ctx = _ctx_env({"XD_FUSED_PROT": "1", "XD_CHAIN_PROT": "2,3,4,6", "XD_FUSED4": "0"})
    try:
        got = _run_device(ctx, b)
    finally:
        xdrop.xd_destroy(ctx)
    _all_parity(got, b, oracle_all(b))
