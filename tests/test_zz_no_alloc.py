"""The allocation-free entry point against xd_run_device, through the C ABI.

xd_run_device_noalloc serves callers that cannot allocate device memory; it keeps its
scratch rows in a fixed array inside the library.  Its results must equal xd_run_device's
bit for bit (all outputs are integers), on two calls in a row (the second call reuses
whatever the first left in the shared array).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402


def _device_batch(b):
    dev = torch.device("cuda", 0)
    codes = torch.from_numpy(b.codes).to(dev)
    offs = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
    lens = torch.from_numpy(b.lengths.view(np.int32)).to(dev)
    pairs = torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)
    return xdrop.BatchArgs(b.alphabet, codes, offs, lens, pairs, b.match, b.mismatch, b.gap,
                           b.matrix, b.X, b.delta)


@pytest.mark.parametrize("make", [
    lambda: synth.dna_longread(n_pairs=300),
    lambda: synth.protein(n_pairs=1500),
    lambda: synth.uneven(n_pairs=40, delta=256),
    lambda: synth.from_strings([("ACGT", "ACGT", 0, 0, 4), ("A" * 50, "A" * 50, 25, 25, 1)], X=3),
], ids=["dna_longread", "protein", "uneven_restricted", "edges"])
def test_noalloc_matches_run_device_on_two_calls(make):
    b = make()
    args = _device_batch(b)
    n_bytes = b.n_pairs * xdrop.RESULT_DTYPE.itemsize
    ref = torch.zeros(n_bytes, dtype=torch.uint8, device="cuda")
    ctx = xdrop.xd_create(0)
    try:
        xdrop.xd_run_device(ctx, args, ref, None)
        torch.cuda.synchronize()
        assert xdrop.xd_device_status(ctx) == 0
    finally:
        xdrop.xd_destroy(ctx)
    max_side = int(b.lengths.max())
    for call in range(2):
        out = torch.full((n_bytes,), 0xAB, dtype=torch.uint8, device="cuda")
        assert xdrop.xd_run_device_noalloc(args, max_side, out, None) == xdrop.XD_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(xdrop.RESULT_DTYPE)
        want = ref.cpu().numpy().view(xdrop.RESULT_DTYPE)
        assert np.array_equal(got, want), f"call {call} differs from xd_run_device"


def test_noalloc_rejects_sides_beyond_its_scratch():
    b = synth.from_strings([("ACGT", "ACGT", 0, 0, 2)], X=3)
    args = _device_batch(b)
    out = torch.zeros(xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    assert xdrop.xd_run_device_noalloc(args, 1 << 30, out, None) == xdrop.XD_EINVAL
