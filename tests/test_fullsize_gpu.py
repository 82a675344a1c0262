"""Full-size parity for the protein and uneven/restricted workloads, through xd_run_device
in the launch configuration the bench times.

At these sizes the oracle cannot recompute every pair within a test, so each batch is
checked (a) on sampled pairs recomputed by the oracle one by one, and (b) on every pair
through properties that hold at any size: score and extension bounds, the total, and for
the memory-restricted variant (Sec. 3) equality with the unrestricted run wherever the
window was never exceeded (overflow flag clear).
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


def _sampled_parity(got, b, n, seed):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(b.n_pairs, min(n, b.n_pairs), replace=False))
    L, R, T = oracle.run_batch(b.subset(idx), threads=THREADS)
    for side, ref in (("left", L), ("right", R)):
        for f in FIELDS:
            g = got[side][f][idx]
            bad = np.nonzero(g != ref[f])[0]
            assert bad.size == 0, f"{side}.{f} differs at pairs {idx[bad[:10]].tolist()}"
    assert np.array_equal(got["total"][idx], T)


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


def test_full_size_protein_sampled(ctx):
    """1,000,000 protein pairs, BLOSUM62, gap -2, X = 49."""
    b = synth.protein()
    got = _run_device(ctx, b)
    _properties(got, b)
    assert (got["right"]["flags"] == 0).all() and (got["left"]["flags"] == 0).all()
    _sampled_parity(got, b, 600, seed=31)


@pytest.fixture(scope="module")
def uneven():
    return synth.uneven()


@pytest.fixture(scope="module")
def uneven_unrestricted(ctx, uneven):
    return _run_device(ctx, uneven)


def test_full_size_uneven_unrestricted_sampled(ctx, uneven, uneven_unrestricted):
    """200,000 DNA pairs, lengths log-uniform in [500, 100,000], X = 20."""
    _properties(uneven_unrestricted, uneven)
    _sampled_parity(uneven_unrestricted, uneven, 150, seed=32)


@pytest.mark.parametrize("delta", [256, 1024, 4096])
def test_full_size_uneven_restricted(ctx, uneven, uneven_unrestricted, delta):
    b = uneven.with_params(delta=delta)
    got = _run_device(ctx, b)
    _properties(got, b)
    for side in ("left", "right"):
        f = got[side]["flags"]
        assert ((f == 0) | (f == 1)).all()
        clear = f == 0
        for fld in FIELDS:
            assert np.array_equal(got[side][fld][clear], uneven_unrestricted[side][fld][clear]), (side, fld)
    _sampled_parity(got, b, 100, seed=33 + delta)


def _ctx_env(env):
    keys = ("XD_FUSED", "XD_FUSED_PROT", "XD_EVERY1", "XD_EVERY2", "XD_EVERY3", "XD_LONG_PERMILLE", "XD_CHAIN")
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


@pytest.mark.parametrize("X,chain", [(10, None), (20, None), (50, None), (20, "1,3,4,5,6")])
def test_full_size_fused_grid_equals_level_launches(X, chain):
    """Every one of the 100,000 long-read pairs: the persistent grid whose warps run
    different group shapes at once (and the long-side role) must give exactly the results of
    one launch per register level; also the four-role grid (windows 32, 128, 256, 512)."""
    b = synth.dna_longread().with_params(X=X)
    extra = {"XD_CHAIN": chain, "XD_EVERY3": "8"} if chain else {}
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
