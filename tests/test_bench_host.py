"""Host-side helpers of bench.py that need no GPU: the bench labels a batch as running on
16-bit packed scores (its roofline peak and dtype) by the same bound the library applies,
-127 <= gap <= 0 and (1022 - X - s_max) - (2 (s_max - gap) + 1) >= 64 with
s_max = max(similarity, 0); the GPU parity tests exercise both sides of that bound."""
import numpy as np
import pytest

import synth
from synth import X_INF

bench = pytest.importorskip("bench")


def _dna(X, gap=-1, match=1, mismatch=-1):
    return synth.from_strings([("ACGT", "ACGT", 0, 0, 1)], gap=gap, match=match, mismatch=mismatch, X=X)


def _prot(X, gap=-2):
    return synth.from_strings([("ARND", "ARND", 0, 0, 1)], alphabet="protein", gap=gap, X=X)


@pytest.mark.parametrize("X,gap,match,mismatch,packed", [
    (0, -1, 1, -1, True), (952, -1, 1, -1, True), (953, -1, 1, -1, False),
    (322, -127, 127, -127, True), (323, -127, 127, -127, False),
    (40, 0, 2, -3, True), (40, -128, 5, -4, False), (X_INF, -1, 1, -1, False),
    (40, -1, -1, -2, True)])
def test_packed_bound_dna(X, gap, match, mismatch, packed):
    assert bench.packed_scores(_dna(X, gap, match, mismatch)) is packed


@pytest.mark.parametrize("X,packed", [(49, True), (920, True), (921, False)])
def test_packed_bound_protein(X, packed):
    b = _prot(X)
    assert int(np.max(b.matrix)) == 11   # BLOSUM62's largest entry sets s_max
    assert bench.packed_scores(b) is packed


# ---- the replicated (N > 1) path of bench.py on CPU ranks (gloo, world size 2)

def _job_worker(rank, world, port, q):
    import os
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank cells and pairs differ (each rank extends its own seeded batch)
        sums, slowest = bench.job_totals(dist, "cpu", [1000.0 * (rank + 1), 7.0], [0.25 + rank])
        q.put((rank, sums, slowest))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_totals_two_ranks():
    """Whole-job value = every rank's cells over the slowest rank's time, on every rank."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_job_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, sums, slowest in got:
        assert sums == [3000.0, 14.0]
        assert slowest == [1.25]


def test_job_totals_single_process():
    assert bench.job_totals(None, "cpu", [5, 2], [0.5]) == ([5.0, 2.0], [0.5])


def test_reference_arm_ranks(monkeypatch, capsys):
    """--impl reference under torchrun: rank 0 alone times the oracle and prints one line;
    the other ranks exit without work."""
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--workload", "dna_tiny",
                                     "--pairs", "40", "--steps", "1", "--warmup", "1", "--cpu-pairs", "160"])
    a = bench.parse()
    assert bench.run_reference(a, 1, 2) is None
    assert capsys.readouterr().out == ""
    bench.run_reference(a, 0, 2)
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    import json
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_baseline_fields():
    """The bench's CPU baseline: the oracle on every core and on one core (host only)."""
    b = synth.dna_tiny(n_pairs=40)
    d = bench.cpu_baseline(b, 40, 2)
    assert d["kind"] == "oracle" and d["cores"] == 2 and d["unit"] == "GCUPS"
    assert d["value"] > 0 and d["value_1_core"] > 0
    assert d["sample"].startswith("40 ") and d["sample_1_core"].startswith("2 ")


# ---- the serving loop's host side, against a fake library (no GPU)

class _FakeLib:
    """Stands in for the binding: each request finishes `delay` seconds after it is sent;
    the first submit of every third request is refused for memory (the loop retries)."""
    XD_OK, XD_PENDING, XD_ENOMEM = 0, 1, 3
    RESULT_DTYPE = np.dtype([("left", [("cells", np.uint64)]), ("right", [("cells", np.uint64)])])

    class XdError(Exception):
        def __init__(self, status):
            super().__init__(status)
            self.status = status

    def __init__(self, delay):
        self.delay = delay
        self.sent = {}
        self.refused = 0
        self.n = 0

    def submit(self, b):
        self.n += 1
        if self.n % 3 == 0 and self.refused < self.n // 3:
            self.refused += 1
            raise self.XdError(self.XD_ENOMEM)
        tk = len(self.sent) + 1
        self.sent[tk] = (bench.time.perf_counter(), b.n_pairs)
        return tk

    def xd_poll(self, ctx, tk, out, wait_ms):
        t, n = self.sent[tk]
        if bench.time.perf_counter() - t < self.delay:
            return self.XD_PENDING
        out["left"]["cells"] = 2
        out["right"]["cells"] = 3
        return self.XD_OK


class _CountingMix:
    def __init__(self):
        self.drawn = 0

    def next(self):
        self.drawn += 1
        return synth.from_strings([("ACGT", "ACGT", 0, 0, 1)] * (1 + self.drawn % 4))


@pytest.mark.parametrize("rate", [200.0, float("inf")])
def test_serve_run_host_loop(rate):
    lib = _FakeLib(delay=0.004)
    mix = _CountingMix()
    r = bench.serve_run(lib, None, mix, rate, 0.2, max_requests=40, submit=lib.submit)
    n = r["requests"]
    assert mix.drawn == n > 0 and lib.refused > 0
    assert r["pairs"] == sum(1 + k % 4 for k in range(1, n + 1))
    # every request took at least the fake's delay from its scheduled arrival
    assert r["p50_ms"] >= 4.0 and r["p99_ms"] >= r["p50_ms"]
    assert r["gcups"] > 0 and r["pairs_per_s"] > 0
