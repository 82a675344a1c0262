"""Several device batches in one pass of the hot path (xd_run_device_many).

The batches share one packed store, one cost-ordered unit list and one persistent
extension grid; every batch's results must be exactly those of running it alone, in the
launch configurations that large batches use (fused grid) and small ones use.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402

KEYS = ("XD_LATENCY_UNITS",)


def _ctx(env):
    old = {k: os.environ.get(k) for k in KEYS}
    for k in KEYS:
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


def _dev(b):
    dev = torch.device("cuda", 0)
    keep = [torch.from_numpy(b.codes).to(dev), torch.from_numpy(b.offsets.view(np.int64)).to(dev),
            torch.from_numpy(b.lengths.view(np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)]
    return xdrop.BatchArgs(b.alphabet, *keep, b.match, b.mismatch, b.gap, b.matrix, b.X, b.delta)


def _alone(ctx, b):
    out = torch.zeros(max(1, b.n_pairs) * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    xdrop.xd_run_device(ctx, _dev(b), out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert xdrop.xd_device_status(ctx) == 0
    return out.cpu().numpy().view(xdrop.RESULT_DTYPE)[:b.n_pairs].copy()


def _many(ctx, batches):
    n = sum(b.n_pairs for b in batches)
    out = torch.zeros(max(1, n) * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    args = [_dev(b) for b in batches]
    xdrop.xd_run_device_many(ctx, args, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert xdrop.xd_device_status(ctx) == 0
    res = out.cpu().numpy().view(xdrop.RESULT_DTYPE)[:n].copy()
    parts, k = [], 0
    for b in batches:
        parts.append(res[k:k + b.n_pairs])
        k += b.n_pairs
    return parts


@pytest.mark.parametrize("env", [{"XD_LATENCY_UNITS": "0"}, {}], ids=["fused", "default"])
@pytest.mark.parametrize("make", [
    lambda: [synth.dna_longread(n_pairs=3000), synth.dna_longread(n_pairs=5000, seed=101),
             synth.from_strings([("ACGT", "ACGT", 0, 0, 4)], X=20), synth.dna_longread(n_pairs=2000, seed=102)],
    lambda: [synth.protein(n_pairs=4000), synth.protein(n_pairs=9000, seed=7)],
    lambda: [synth.uneven(n_pairs=300, delta=256), synth.uneven(n_pairs=200, seed=9, delta=256)],
], ids=["dna", "protein", "uneven_restricted"])
def test_many_equals_each_alone(env, make):
    batches = make()
    ctx = _ctx(env)
    try:
        parts = _many(ctx, batches)
        for k, b in enumerate(batches):
            assert np.array_equal(parts[k], _alone(ctx, b)), f"batch {k} differs from its own run"
        # the same call twice in a row (scratch reuse)
        again = _many(ctx, batches)
        for k in range(len(batches)):
            assert np.array_equal(parts[k], again[k])
    finally:
        xdrop.xd_destroy(ctx)
    b = batches[0]
    L, R, T = oracle.run_batch(b, threads=8)
    for side, o in (("left", L), ("right", R)):
        for f in ("score", "h_ext", "v_ext", "flags", "cells"):
            assert np.array_equal(parts[0][side][f], o[f]), (side, f)
    assert np.array_equal(parts[0]["total"], T)


def test_many_rejects_mixed_parameters_and_takes_none():
    ctx = xdrop.xd_create(0)
    try:
        a, b = synth.dna_longread(n_pairs=50), synth.dna_longread(n_pairs=50).with_params(X=10)
        out = torch.zeros(100 * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        with pytest.raises(xdrop.XdError) as e:
            xdrop.xd_run_device_many(ctx, [_dev(a), _dev(b)], out)
        assert e.value.status == xdrop.XD_EINVAL
        xdrop.xd_run_device_many(ctx, [], out)
        # the context still runs a valid call
        parts = _many(ctx, [a, a])
        assert np.array_equal(parts[0], parts[1])
    finally:
        xdrop.xd_destroy(ctx)
