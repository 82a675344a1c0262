"""Failure detection without a GPU fault: a bounded device wait that runs out.

The fused grid's consumers wait for their producers with a bounded, progress-based wait.
With a short limit and a producer that never finishes (a test setting of the library),
the consumers' waits run out, the kernel raises the wait-error flag and returns, the host
reports XD_EDEVICE for the batch, and the GPU context stays usable.
"""
import os
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402

KEYS = ("XD_TEST_WAIT_MS", "XD_TEST_PHANTOM_PRODUCER", "XD_LATENCY_UNITS")


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


def test_wait_that_runs_out_is_reported_and_context_survives():
    b = synth.dna_longread(n_pairs=3000)
    bad = _ctx({"XD_TEST_WAIT_MS": "50", "XD_TEST_PHANTOM_PRODUCER": "1", "XD_LATENCY_UNITS": "0"})
    try:
        t0 = time.perf_counter()
        with pytest.raises(xdrop.XdError) as e:
            xdrop.extend_host(bad, b)
        assert e.value.status == xdrop.XD_EDEVICE
        assert "flags 8" in str(e.value)                 # bit 3: a bounded device wait gave up
        assert time.perf_counter() - t0 < 20
        # the same context still runs batches that do not use a fused grid (DNA at X > 30 runs
        # one launch per register level)
        p = synth.dna_longread(n_pairs=300).with_params(X=50)
        out = xdrop.extend_host(bad, p)
        L, R, T = oracle.run_batch(p, threads=8)
        assert np.array_equal(out["total"], T)
    finally:
        assert xdrop.xd_destroy(bad) == xdrop.XD_OK
    good = _ctx({"XD_LATENCY_UNITS": "0"})
    try:
        out = xdrop.extend_host(good, b)
        idx = np.arange(0, b.n_pairs, 25)
        L, R, T = oracle.run_batch(b.subset(idx), threads=8)
        assert np.array_equal(out["total"][idx], T)
        assert np.array_equal(out["left"]["cells"][idx], L["cells"])
    finally:
        xdrop.xd_destroy(good)


def test_device_entry_flags_a_sequence_past_the_codes():
    """xd_run_device validates on the device: a sequence whose offset + length passes
    n_codes is reported in the validation word (bit 1) instead of being read clamped."""
    b = synth.dna_tiny(n_pairs=8)
    dev = torch.device("cuda", 0)
    offs = b.offsets.copy()
    offs[3] = np.uint64(b.codes.size - 5)        # sequence 3 now runs past the end
    codes = torch.from_numpy(b.codes).to(dev)
    lens = torch.from_numpy(b.lengths.view(np.int32)).to(dev)
    pairs = torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)
    args = xdrop.BatchArgs(b.alphabet, codes, torch.from_numpy(offs.view(np.int64)).to(dev), lens, pairs,
                           b.match, b.mismatch, b.gap, b.matrix, b.X, b.delta)
    out = torch.zeros(b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    ctx = xdrop.xd_create(0)
    try:
        xdrop.xd_run_device(ctx, args, out, None)
        torch.cuda.synchronize()
        assert xdrop.xd_device_status(ctx) & 2
        # the same context then runs a valid batch cleanly
        good = xdrop.BatchArgs(b.alphabet, codes, torch.from_numpy(b.offsets.view(np.int64)).to(dev),
                               lens, pairs, b.match, b.mismatch, b.gap, b.matrix, b.X, b.delta)
        xdrop.xd_run_device(ctx, good, out, None)
        torch.cuda.synchronize()
        assert xdrop.xd_device_status(ctx) == 0
    finally:
        xdrop.xd_destroy(ctx)
