"""Per-side timeline (xd_set_trace / xd_get_trace) on the GPU.

Tracing must not change a result, and its records must tell a consistent story: every
side extension is finished by exactly one level, every level that escalated a side is
followed by a later level that took it, and the clocks fall inside the batch.
"""
import os
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402

KEYS = ("XD_LATENCY_UNITS", "XD_TIERS")


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


def _run(ctx, b):
    dev = torch.device("cuda", 0)
    keep = [torch.from_numpy(b.codes).to(dev), torch.from_numpy(b.offsets.view(np.int64)).to(dev),
            torch.from_numpy(b.lengths.view(np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)]
    args = xdrop.BatchArgs(b.alphabet, *keep, b.match, b.mismatch, b.gap, b.matrix, b.X, b.delta)
    out = torch.zeros(b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    xdrop.xd_run_device(ctx, args, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert xdrop.xd_device_status(ctx) == 0
    return out.cpu().numpy().view(xdrop.RESULT_DTYPE).copy()


@pytest.mark.parametrize("env,make", [
    ({"XD_LATENCY_UNITS": "0"}, lambda: synth.dna_longread(n_pairs=20000)),
    ({"XD_LATENCY_UNITS": "0"}, lambda: synth.protein(n_pairs=40000)),
    ({}, lambda: synth.dna_longread(n_pairs=500)),
    ({"XD_TIERS": "generic"}, lambda: synth.dna_tiny(n_pairs=200)),
], ids=["fused_dna", "protein_levels", "small_batch", "generic"])
def test_trace_is_consistent_and_changes_nothing(env, make):
    b = make()
    ctx = _ctx(env)
    try:
        plain = _run(ctx, b)
        xdrop.xd_set_trace(ctx, True)
        t0 = time.time_ns()
        traced = _run(ctx, b)
        tr = xdrop.xd_get_trace(ctx)
        xdrop.xd_set_trace(ctx, False)
    finally:
        xdrop.xd_destroy(ctx)
    assert np.array_equal(plain, traced)
    assert tr.shape == (2 * b.n_pairs, xdrop.TRACE_VISITS)
    seen = tr["start_ns"] != 0
    assert (tr["level"][seen] == np.nonzero(seen)[1]).all()
    finished = (tr["outcome"] == 1).sum(axis=1)
    assert (finished == 1).all(), f"{int((finished != 1).sum())} sides without exactly one finishing level"
    starts = tr["start_ns"][seen].astype(np.int64)
    ends = starts + tr["dur_ns"][seen]
    assert ends.max() - starts.min() < 60e9
    for u in np.nonzero((tr["outcome"] == 2).any(axis=1))[0][:2000]:
        lv = np.nonzero(tr["outcome"][u] == 2)[0]
        fin = int(np.nonzero(tr["outcome"][u] == 1)[0][0])
        # the finishing visit starts after every escalating one began
        assert all(int(tr["start_ns"][u, fin]) >= int(tr["start_ns"][u, k]) for k in lv), u
    reg = seen & (np.arange(xdrop.TRACE_VISITS)[None, :] < 5)
    assert (tr["window"][reg] >= 16).all()
    del t0
