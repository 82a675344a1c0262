"""Autotuner through the C ABI: tuning changes speed, never results.

xd_autotune times candidate register-level configurations (lanes per side and window of
each level, queue chunk, fused role mix, band-tier warps) on a sample and keeps the fastest
per alphabet, X, length, size and window bucket; the table it writes is loaded by xd_create.  Every candidate
is the same method, so the library itself checks that all candidates agree bit for bit;
here a context built from the table must give the default context's results.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2304_08662_gb300 import xdrop  # noqa: E402


def _entries(path):
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        rows.append(dict(tok.split("=", 1) for tok in line.split()))
    return rows


@pytest.mark.parametrize("make,bucket", [
    (lambda: synth.dna_longread(n_pairs=3000), {"alpha": "4", "xb": "1"}),
    (lambda: synth.protein(n_pairs=20000), {"alpha": "20", "xb": "2"}),
], ids=["dna_x20", "protein_x49"])
def test_tuned_table_gives_default_results(tmp_path, make, bucket):
    b = make()
    sample, check = b.pair_range(0, b.n_pairs // 2), b.pair_range(b.n_pairs // 2, b.n_pairs)
    table = tmp_path / "tune.txt"
    ctx = xdrop.xd_create(0)
    try:
        ms = xdrop.xd_autotune(ctx, xdrop.BatchArgs.from_host(sample), table)
        assert ms > 0
        ref = xdrop.extend_host(ctx, check)       # the winner already applies to this context
    finally:
        xdrop.xd_destroy(ctx)
    rows = _entries(table)
    assert len(rows) == 1 and all(rows[0][k] == v for k, v in bucket.items()), rows
    plain = xdrop.xd_create(0)
    tuned = xdrop.xd_create(0, tune_table=str(table))
    try:
        a = xdrop.extend_host(plain, check)
        t = xdrop.extend_host(tuned, check)
    finally:
        xdrop.xd_destroy(plain)
        xdrop.xd_destroy(tuned)
    assert a.tobytes() == t.tobytes() == ref.tobytes()
    idx = np.arange(0, check.n_pairs, max(1, check.n_pairs // 200))
    L, R, T = oracle.run_batch(check.subset(idx), threads=8)
    assert np.array_equal(t["left"]["score"][idx], L["score"])
    assert np.array_equal(t["right"]["cells"][idx], R["cells"])
    assert np.array_equal(t["total"][idx], T)


def test_table_merges_buckets(tmp_path):
    table = tmp_path / "tune.txt"
    dna = synth.dna_longread(n_pairs=1000)
    ctx = xdrop.xd_create(0)
    try:
        xdrop.xd_autotune(ctx, xdrop.BatchArgs.from_host(dna.with_params(X=10)), table)
        xdrop.xd_autotune(ctx, xdrop.BatchArgs.from_host(dna.with_params(X=50)), table)
        xdrop.xd_autotune(ctx, xdrop.BatchArgs.from_host(dna.with_params(X=12)), table)   # same bucket as X=10
    finally:
        xdrop.xd_destroy(ctx)
    rows = _entries(table)
    assert sorted(r["xb"] for r in rows) == ["0", "2"]


def test_table_keys_the_restricted_window(tmp_path):
    """Memory-restricted batches (Sec. 3.3) are tuned per window bucket: the uneven batch at
    delta_b = 256 and 4096 gives two entries, and each tuned context keeps the results."""
    table = tmp_path / "tune.txt"
    u = synth.uneven(n_pairs=80)
    ctx = xdrop.xd_create(0)
    try:
        for d in (256, 4096, 300):      # 300 falls in the bucket of 256 and replaces its entry
            xdrop.xd_autotune(ctx, xdrop.BatchArgs.from_host(u.with_params(delta=d)), table)
    finally:
        xdrop.xd_destroy(ctx)
    rows = _entries(table)
    assert sorted(r["db"] for r in rows) == ["1", "3"], rows
    plain = xdrop.xd_create(0)
    tuned = xdrop.xd_create(0, tune_table=str(table))
    try:
        for d in (256, 4096):
            b = u.with_params(delta=d)
            assert xdrop.extend_host(plain, b).tobytes() == xdrop.extend_host(tuned, b).tobytes()
    finally:
        xdrop.xd_destroy(plain)
        xdrop.xd_destroy(tuned)


def test_malformed_table_is_rejected(tmp_path):
    bad = tmp_path / "bad.txt"
    for line in ("alpha=4 xb=1 lb=1 chain=1,99\n", "alpha=4 xb=1 lb=1 db=4 chain=1,6\n"):
        bad.write_text(line)
        with pytest.raises(xdrop.XdError) as e:
            xdrop.xd_create(0, tune_table=str(bad))
        assert e.value.status == xdrop.XD_EINVAL
    with pytest.raises(xdrop.XdError):
        xdrop.xd_create(0, tune_table=str(tmp_path / "missing.txt"))
