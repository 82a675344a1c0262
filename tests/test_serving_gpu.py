"""Continuous batching through the C ABI: each request's results are the same alone and in
the mix.

A request is one host batch (xd_submit_batch).  The context's dispatcher merges requests
that wait for a launch slot into one launch (those with the same parameters into one batch
of the hot path, up to four parameter sets side by side), and launches on different slots
overlap on the device.  Merging must not change any result: every
field is an integer, so "the same" means bit-identical, here and against the oracle.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402

FIELDS = ("score", "h_ext", "v_ext", "flags", "cells")


@pytest.fixture(scope="module")
def pools():
    dna = synth.dna_longread(n_pairs=3000)
    prot = synth.protein(n_pairs=6000)
    return dna, prot


def _requests(pools, n, seed, max_pairs=200):
    """Mixed DNA (X in {10, 20, 50}) and protein (X = 49) requests, log-uniform sizes."""
    dna, prot = pools
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        pool = dna if rng.random() < 0.5 else prot
        size = int(np.exp(rng.uniform(0, np.log(max_pairs))))
        a = int(rng.integers(0, pool.n_pairs - size + 1))
        b = pool.pair_range(a, a + size)
        if pool is dna:
            b = b.with_params(X=int(rng.choice([10, 20, 50])))
        out.append(b)
    return out


def _alone(batches):
    """Each request run by itself: one launch per request, one launch in flight."""
    ctx = xdrop.xd_create(0, max_inflight=1, batching=-1)
    try:
        return [xdrop.extend_host(ctx, b) for b in batches]
    finally:
        assert xdrop.xd_destroy(ctx) == xdrop.XD_OK


def _assert_same(a, b, what):
    assert a.tobytes() == b.tobytes(), what


def test_mix_equals_alone(pools):
    batches = _requests(pools, 60, seed=5)
    ref = _alone(batches)
    ctx = xdrop.xd_create(0, max_inflight=2)
    try:
        tickets = []
        rng = np.random.default_rng(7)
        for b in batches:
            tickets.append(xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(b)))
            if rng.random() < 0.2:
                time.sleep(0.002)
        got = []
        for b, t in zip(batches, tickets):
            out = np.zeros(b.n_pairs, dtype=xdrop.RESULT_DTYPE)
            assert xdrop.xd_poll(ctx, t, out, -1) == xdrop.XD_OK
            got.append(out)
        st = xdrop.xd_get_stats(ctx)
    finally:
        assert xdrop.xd_destroy(ctx) == xdrop.XD_OK
    for k, (g, r) in enumerate(zip(got, ref)):
        _assert_same(g, r, f"request {k} ({batches[k].name}, X={batches[k].X}) differs in the mix")
    # requests were merged: fewer launches than requests
    assert st["host_launches"] < len(batches), st
    assert st["host_requests"] == len(batches)


def test_mixed_parameter_launch(pools):
    """Requests of several parameter sets in one launch: DNA at X = 10, 20 and 50 (one with
    Z-Drop), protein, a memory-restricted DNA request.  One slot, so the requests sent while
    the first launch runs wait together and leave in launches of up to four sets whose
    kernels run side by side; every result equals the request's run alone, bit for bit, and
    a sample of them the oracle."""
    dna, prot = pools
    blocker = dna.pair_range(0, 2000)
    mixed = [dna.pair_range(2000, 2100), prot.pair_range(0, 300), dna.pair_range(2100, 2150).with_params(X=10),
             dna.pair_range(2150, 2400), prot.pair_range(300, 340), dna.pair_range(2400, 2500).with_params(X=50),
             dna.pair_range(2500, 2600).with_params(delta=64), dna.pair_range(2600, 2700).with_params(zdrop=5),
             prot.pair_range(340, 1340), dna.pair_range(2700, 2710).with_params(X=10)]
    batches = [blocker] + mixed
    ref = _alone(batches)
    ctx = xdrop.xd_create(0, max_inflight=1)
    try:
        tickets = [xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(b)) for b in batches]
        got = []
        for b, t in zip(batches, tickets):
            out = np.zeros(b.n_pairs, dtype=xdrop.RESULT_DTYPE)
            assert xdrop.xd_poll(ctx, t, out, -1) == xdrop.XD_OK
            got.append(out)
        st = xdrop.xd_get_stats(ctx)
    finally:
        assert xdrop.xd_destroy(ctx) == xdrop.XD_OK
    for k, (g, r) in enumerate(zip(got, ref)):
        _assert_same(g, r, f"request {k} ({batches[k].name}) differs in a mixed launch")
    assert st["mixed_launches"] >= 1, st
    assert st["host_launches"] < len(batches), st
    for k in (1, 2, 7):
        b = batches[k]
        L, R, T = oracle.run_batch(b, threads=8)
        for side, refs in (("left", L), ("right", R)):
            for f in FIELDS:
                assert np.array_equal(got[k][side][f], refs[f]), (b.name, side, f)
        assert np.array_equal(got[k]["total"], T)


def test_mix_matches_oracle(pools):
    batches = _requests(pools, 24, seed=11, max_pairs=60)
    ctx = xdrop.xd_create(0, max_inflight=3)
    try:
        tickets = [xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(b)) for b in batches]
        for b, t in zip(batches, tickets):
            out = np.zeros(b.n_pairs, dtype=xdrop.RESULT_DTYPE)
            assert xdrop.xd_poll(ctx, t, out, -1) == xdrop.XD_OK
            L, R, T = oracle.run_batch(b, threads=8)
            for side, refs in (("left", L), ("right", R)):
                for f in FIELDS:
                    assert np.array_equal(out[side][f], refs[f]), (b.name, side, f)
            assert np.array_equal(out["total"], T)
    finally:
        xdrop.xd_destroy(ctx)


def test_concurrent_submitters_and_pollers(pools):
    batches = _requests(pools, 48, seed=13, max_pairs=120)
    ref = _alone(batches)
    ctx = xdrop.xd_create(0, max_inflight=3)
    got = [None] * len(batches)
    errors = []

    def worker(ids):
        try:
            for k in ids:
                t = xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(batches[k]))
                out = np.zeros(batches[k].n_pairs, dtype=xdrop.RESULT_DTYPE)
                while xdrop.xd_poll(ctx, t, out, 1) != xdrop.XD_OK:
                    pass
                got[k] = out
        except Exception as e:  # surfaced below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(range(w, len(batches), 4),)) for w in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    xdrop.xd_destroy(ctx)
    assert not errors, errors
    for k in range(len(batches)):
        _assert_same(got[k], ref[k], f"request {k} differs under concurrent submitters")


def test_admission_by_memory_cap(pools):
    dna, _ = pools
    b = dna.pair_range(0, 200)        # several MB of residues
    ctx = xdrop.xd_create(0, store_bytes_cap=1 << 20)
    try:
        with pytest.raises(xdrop.XdError) as e:
            xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(b))
        assert e.value.status == xdrop.XD_ENOMEM
        small = dna.pair_range(0, 1)
        out = xdrop.extend_host(ctx, small)
        assert out.shape == (1,)
    finally:
        xdrop.xd_destroy(ctx)


def test_destroy_with_unpolled_and_pending_requests(pools):
    batches = _requests(pools, 20, seed=17)
    ctx = xdrop.xd_create(0, max_inflight=1)
    for b in batches:
        xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(b))
    assert xdrop.xd_destroy(ctx) == xdrop.XD_OK


def test_poll_timeout_and_pending(pools):
    dna, _ = pools
    ctx = xdrop.xd_create(0, max_inflight=1)
    try:
        big = xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(dna.pair_range(0, 3000)))
        small = xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(dna.pair_range(0, 1)))
        out = np.zeros(1, dtype=xdrop.RESULT_DTYPE)
        rc = xdrop.xd_poll(ctx, small, out, 0)
        assert rc in (xdrop.XD_PENDING, xdrop.XD_OK)
        if rc == xdrop.XD_PENDING:
            assert xdrop.xd_poll(ctx, small, out, -1) == xdrop.XD_OK
        assert xdrop.xd_poll(ctx, big, None, -1) == xdrop.XD_OK
        with pytest.raises(xdrop.XdError):
            xdrop.xd_poll(ctx, big, None, 0)   # retired
    finally:
        xdrop.xd_destroy(ctx)
