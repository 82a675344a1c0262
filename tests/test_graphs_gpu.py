"""CUDA-graph replay of the device entry point, through the C ABI.

A call to xd_run_device that repeats the previous call's arguments is captured as a CUDA
graph, and later identical calls replay it.  Replays must read the buffers' current
contents and give the same results as a direct run, bit for bit.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402


def _device(b):
    dev = torch.device("cuda", 0)
    t = {"codes": torch.from_numpy(b.codes).to(dev),
         "offs": torch.from_numpy(b.offsets.view(np.int64)).to(dev),
         "lens": torch.from_numpy(b.lengths.view(np.int32)).to(dev),
         "pairs": torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)}
    args = xdrop.BatchArgs(b.alphabet, t["codes"], t["offs"], t["lens"], t["pairs"], b.match, b.mismatch,
                           b.gap, b.matrix, b.X, b.delta)
    return t, args


def _run(ctx, args, n_pairs, stream):
    out = torch.zeros(n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    xdrop.xd_run_device(ctx, args, out, stream.cuda_stream)
    stream.synchronize()
    assert xdrop.xd_device_status(ctx) == 0
    return out.cpu().numpy().view(xdrop.RESULT_DTYPE).copy()


def test_replay_matches_direct_and_reads_current_contents():
    b = synth.dna_longread(n_pairs=400)
    stream = torch.cuda.Stream()
    ctx = xdrop.xd_create(0)
    try:
        t, args = _device(b)
        first = _run(ctx, args, b.n_pairs, stream)          # direct
        second = _run(ctx, args, b.n_pairs, stream)         # captured, then launched
        third = _run(ctx, args, b.n_pairs, stream)          # replayed
        st = xdrop.xd_get_stats(ctx)
        assert st["graph_captures"] == 1 and st["graph_replays"] == 1, st
        assert first.tobytes() == second.tobytes() == third.tobytes()
        # same buffers, new contents: move every seed to half its position (still inside
        # its sequences); the replay must see the new seeds
        moved = b.pairs.copy()
        moved[:, 2] //= 2
        moved[:, 3] //= 2
        t["pairs"].copy_(torch.from_numpy(np.ascontiguousarray(moved).view(np.int32)))
        replayed = _run(ctx, args, b.n_pairs, stream)
        assert xdrop.xd_get_stats(ctx)["graph_replays"] == 2
    finally:
        xdrop.xd_destroy(ctx)
    changed = synth.Batch(b.alphabet, b.codes, b.offsets, b.lengths, moved, X=b.X)
    fresh = xdrop.xd_create(0)
    try:
        _, a2 = _device(changed)
        direct = _run(fresh, a2, b.n_pairs, torch.cuda.Stream())
    finally:
        xdrop.xd_destroy(fresh)
    assert replayed.tobytes() == direct.tobytes()
    assert replayed.tobytes() != first.tobytes()


def test_changed_arguments_run_directly():
    b = synth.protein(n_pairs=600)
    stream = torch.cuda.Stream()
    ctx = xdrop.xd_create(0)
    try:
        _, args = _device(b)
        a = _run(ctx, args, b.n_pairs, stream)
        a2 = _run(ctx, args, b.n_pairs, stream)
        small = b.pair_range(0, 300)
        _, sargs = _device(small)
        s1 = _run(ctx, sargs, small.n_pairs, stream)
        a3 = _run(ctx, args, b.n_pairs, stream)
        assert a.tobytes() == a2.tobytes() == a3.tobytes()
        assert s1.tobytes() == a[:300].tobytes()
    finally:
        xdrop.xd_destroy(ctx)
