"""Benchmark of batched X-Drop seed extension on GB300.

A step is one pass of the whole hot path over one batch: pack the residue codes, build
the work units (left and right extension per pair), order them by cost, run the
alignment tiers, and form the pair totals.  The default workload is the DNA long-read
batch: 100,000 dovetail pairs, lengths lognormal (median 8 kbp) in [1, 30] kbp, 8-18%
error, 10% unrelated, k = 17, +1/-1/-1, X = 20, unrestricted.

The timed steps run as launches of --batches-per-launch batches each (default 10, through
xd_run_device_many): the batches of a launch share one persistent grid, so the long serial
chains of one batch overlap the bulk work of the others; every batch is computed in full and
checked against its single-batch results.

value = computed-cell GCUPS (sum of evaluated DP cells / device time) with the inputs
resident in HBM; e2e = the same through xd_submit_batch / xd_poll with host buffers
(host-to-device and device-to-host copies inside the timed region).  --impl reference
times the CPU oracle (the plain definition of the method) on a bounded sample of the
same workload.  Under torchrun every rank runs its own batch of the same size (weak
scaling; no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# Integer operations of one cell of the method as Algorithm 1 writes it: two gap adds, the
# similarity lookup and add, two maxima for the three-way maximum, the X-Drop compare and
# conditional assignment, and the running maximum T'.
ALG_OPS_PER_CELL = 9
SM_COUNT_GB300 = 152
# Integer ALU-pipe lanes per SM per clock: max, DPX, logic, select and byte-permute
# instructions all issue there (measured: 60-61 per clock at 1.99 GHz for each of them);
# plain adds and multiply-adds can also use the FMA pipe.  The DNA register levels compute
# (and protein) register levels compute on 16-bit halves (16x2 DPX at the same instruction
# rate) when the scores allow, so their peak counts two 16-bit lanes per ALU lane.
ALU_LANES_PER_SM = 64
# DRAM bytes (read + write) per computed cell of the dominant kernel, from one ncu capture of
# the same kernel build on the same workload (profiles/k_fused_dna_longread_100k_x20.md: the
# fused grid of ten-batch launches, 1 x 32 -> 4 x 32 -> 8 x 32, captured on 40,000 pairs);
# roofline.traffic = that figure x the cells of one launch.  Reported only for that workload
# with the default configuration, and only while the kernel is the build the counters were
# taken on (empty: the kernel has changed since).
DOMINANT_KERNEL_TRAFFIC_PER_CELL = {
    ("dna_longread_100000_x20", 10): (92_125_696 + 8_757_760) / 8_761_163_347,
}


def save_trace(path, tr):
    """Compact per-side timeline: one row per (side extension, level) that ran, times in
    microseconds from the batch's first start, written with numpy's compressed format."""
    seen = tr["start_ns"] != 0
    u, lv = np.nonzero(seen)
    r = tr[u, lv]
    t0 = int(r["start_ns"].min()) if r.size else 0
    np.savez_compressed(path, unit=u.astype(np.uint32), level=lv.astype(np.uint8),
                        start_us=((r["start_ns"].astype(np.int64) - t0) / 1e3).astype(np.float32),
                        dur_us=(r["dur_ns"] / 1e3).astype(np.float32), diags=r["diags"], window=r["window"],
                        smid=r["smid"], lanes=r["lanes"], outcome=r["outcome"].astype(np.uint8),
                        n_units=np.array([tr.shape[0]]))


def packed_scores(b):
    """True when the library runs this batch's register levels on 16-bit scores (the bound
    of the packed representation: -127 <= gap <= 0 and theta1 - theta0 >= 64)."""
    if not (-127 <= b.gap <= 0) or not (0 <= b.X <= 1022):
        return False
    sm = max(b.match, b.mismatch, 0) if b.alphabet == "dna" else max(int(np.max(b.matrix)), 0)
    return (1022 - b.X - sm) - (2 * (sm - b.gap) + 1) >= 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="batches timed (in launches of --batches-per-launch)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dna_longread", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--x", type=int, default=None, help="X (default: the workload's)")
    ap.add_argument("--delta", type=int, default=0)
    ap.add_argument("--pairs", type=int, default=None, help="pairs (default: the workload's full size)")
    ap.add_argument("--seeds", type=int, default=1, choices=[1, 2],
                    help="seed tuples per overlap on the same reads (dna_longread only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the short record of the other workloads (configs sub-object)")
    ap.add_argument("--cpu-pairs", type=int, default=100_000,
                    help="oracle sample of the cpu_baseline (about 10 s on 16 cores for the long-read "
                         "workload); the reference arm times a quarter of it per step")
    ap.add_argument("--serve", type=float, default=5.0,
                    help="seconds per offered load of the serving run (0 = skip)")
    ap.add_argument("--serve-loads", default="0.25,0.5,0.9")
    ap.add_argument("--serve-inflight", type=int, default=3)
    ap.add_argument("--slots", type=int, default=1,
                    help="launch slots of the main context (0: the library's default, 3); with one slot, "
                         "host batches that wait while it runs leave together in one merged launch")
    ap.add_argument("--e2e-inflight", type=int, default=20,
                    help="host batches the e2e measurement keeps submitted ahead of the one it polls "
                         "(measured: 2 -> 397, 10 -> 615-654, 20 -> 667-736 GCUPS with one slot)")
    ap.add_argument("--serve-modes", default="continuous,per_batch,continuous_resident",
                    help="serving modes to run (e.g. --serve 600 --serve-modes continuous for ten "
                         "minutes per offered load)")
    ap.add_argument("--tune-table", default=None, help="tuning table written by xd_autotune")
    ap.add_argument("--configs-tune-table", default=os.path.join(ROOT, "paper_2304_08662_gb300", "tuning", "gb300.txt"),
                    help="tuning table under which the memory-restricted uneven batches of the configs "
                         "record are also timed (skipped if the file does not exist)")
    ap.add_argument("--autotune", default=None, help="run xd_autotune on the workload first and write "
                                                      "the table to this path")
    ap.add_argument("--batches-per-launch", type=int, default=10,
                    help="batches of the workload that share one pass of the hot path (xd_run_device_many): "
                         "the timed steps run as launches of this many batches each (1: one launch per batch)")
    ap.add_argument("--trace", default=None, help="after the timed region, run one traced batch and save "
                                                  "its per-side timeline (compressed numpy .npz) to this path")
    return ap.parse_args()


def make_batch(a, rank):
    gen = synth.WORKLOADS[a.workload]
    kw = {}
    if a.pairs is not None:
        kw["n_pairs"] = a.pairs
    if a.workload == "uneven":
        kw["delta"] = a.delta
    if a.seeds == 2 and a.workload == "dna_longread":
        kw["seeds_per_pair"] = 2
    b = gen(**kw) if rank == 0 else gen(seed=1000 + rank, **kw)
    if a.x is not None:
        b = b.with_params(X=a.x)
    if a.delta and a.workload != "uneven":
        b = b.with_params(delta=a.delta)
    return b


def workload_config(a, b):
    seeds = b.meta.get("seeds_per_pair", 1)
    bpl = max(1, getattr(a, "batches_per_launch", 1))
    return {"workload": f"{a.workload}_{b.n_pairs // seeds}_x{b.X}" + (f"_delta{b.delta}" if b.delta else "") +
                        (f"_{seeds}seeds" if seeds > 1 else ""),
            "batches_per_launch": bpl,
            "pairs": b.n_pairs, "residues": int(b.codes.size), "X": b.X, "delta_b": b.delta,
            "alphabet": b.alphabet, "scoring": ("BLOSUM62" if b.alphabet == "protein" else
                                                f"{b.match}/{b.mismatch}/{b.gap}"),
            "l2": "inputs larger than L2 (codes %.2f GB)" % (b.codes.size / 1e9),
            "parallelism": "replicas (one batch per GPU)"}


def paper_cells(b):
    p = b.pairs.astype(np.int64)
    return float((b.lengths[p[:, 0]].astype(np.float64) * b.lengths[p[:, 1]]).sum())


def job_totals(dist, dev, per_rank, slowest):
    """Whole-job figures over the ranks of a replicated run: the sums of `per_rank` (cells,
    pairs) and the maximum of `slowest` (seconds).  Without a process group: the inputs."""
    if dist is None:
        return [float(x) for x in per_rank], [float(x) for x in slowest]
    import torch
    s = torch.tensor([float(x) for x in per_rank], dtype=torch.float64, device=dev)
    m = torch.tensor([float(x) for x in slowest], dtype=torch.float64, device=dev)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return s.tolist(), m.tolist()


def cpu_oracle(b, n_sample, threads):
    import oracle
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(b.n_pairs, min(n_sample, b.n_pairs), replace=False))
    sub = b.subset(idx)
    t0 = time.perf_counter()
    L, R, _ = oracle.run_batch(sub, threads=threads)
    dt = time.perf_counter() - t0
    cells = float(L["cells"].sum() + R["cells"].sum())
    return cells, dt, len(idx)


def cpu_baseline(b, n_pairs, threads):
    """The oracle timed on the host: on every core (one pair range per thread) over n_pairs
    seeded pairs of the workload, and on one core over a twentieth of them."""
    c, dt, n = cpu_oracle(b, n_pairs, threads)
    c1, dt1, n1 = cpu_oracle(b, max(1, n_pairs // 20), 1)
    return {"value": c / dt / 1e9, "unit": "GCUPS", "cores": threads, "kind": "oracle",
            "sample": f"{n} seeded-random pairs of the same workload ({c:.3g} cells, {dt:.1f} s)",
            "value_1_core": c1 / dt1 / 1e9,
            "sample_1_core": f"{n1} seeded-random pairs ({c1:.3g} cells, {dt1:.1f} s)"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- per-config record

CONFIG_SET = [("dna_tiny", {}), ("dna_longread", {"X": 10}), ("dna_longread", {"X": 50}),
              ("protein", {}), ("uneven", {"delta": 0}), ("uneven", {"delta": 256}),
              ("uneven", {"delta": 1024}), ("uneven", {"delta": 4096})]


def device_args(xdrop, torch, dev, b):
    keep = [torch.from_numpy(b.codes).to(dev), torch.from_numpy(b.offsets.view(np.int64)).to(dev),
            torch.from_numpy(b.lengths.view(np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)]
    return xdrop.BatchArgs(b.alphabet, *keep, b.match, b.mismatch, b.gap, b.matrix, b.X, b.delta)


def single_batch_record(xdrop, torch, ctx, dev, b, args, out, reps=3):
    """One batch per launch on device-resident inputs: the results (after warm-up launches)
    and the time per launch (CUDA events on the launching stream)."""
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        xdrop.xd_run_device(ctx, args, out, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    if xdrop.xd_device_status(ctx) != 0:
        raise RuntimeError(f"device validation failed for {b.name}")
    res = out[:b.n_pairs * xdrop.RESULT_DTYPE.itemsize].cpu().numpy().view(xdrop.RESULT_DTYPE).copy()
    cells = float(res["left"]["cells"].sum() + res["right"]["cells"].sum())
    ev0.record(stream)
    for _ in range(reps):
        xdrop.xd_run_device(ctx, args, out, stream.cuda_stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / reps
    return res, {"ms_per_batch": ms, "gcups": cells / (ms * 1e-3) / 1e9, "pairs_per_s": b.n_pairs / (ms * 1e-3)}


def config_record(xdrop, torch, ctx, dev, b, bpl, launches, oracle_pairs, peak_16, peak_32, tuned_ctx=None):
    """Short measurement of one workload: one batch per launch and bpl batches per launch
    (device-resident inputs, CUDA events on the launching stream), the dominant stage's
    fraction of the integer roofline, and the oracle on a bounded sample.  With tuned_ctx
    (a context built from a tuning table) the single-batch launch is also timed there and
    its results must equal the default's bit for bit."""
    stream = torch.cuda.current_stream(dev)
    args = device_args(xdrop, torch, dev, b)
    out = torch.zeros(bpl * b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    xdrop.xd_reserve(ctx, bpl * b.codes.size, bpl * b.n_seqs, bpl * b.n_pairs, int(b.lengths.max()))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rec = {"pairs": b.n_pairs, "X": b.X, "delta_b": b.delta, "batches_per_launch": bpl}
    # one batch per launch
    res, rec["single_batch"] = single_batch_record(xdrop, torch, ctx, dev, b, args, out)
    cells = float(res["left"]["cells"].sum() + res["right"]["cells"].sum())
    if tuned_ctx is not None:
        t_res, t_rec = single_batch_record(xdrop, torch, tuned_ctx, dev, b, args, out)
        t_rec["identical_to_default"] = bool(np.array_equal(t_res, res))
        if not t_rec["identical_to_default"]:
            raise RuntimeError(f"{b.name}: the tuned configuration changed the results")
        rec["single_batch_tuned"] = t_rec
    # bpl batches per launch, timed with the stage events
    xdrop.xd_run_device_many(ctx, [args] * bpl, out, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    xdrop.xd_set_timing(ctx, True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(launches):
        xdrop.xd_run_device_many(ctx, [args] * bpl, out, stream.cuda_stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    tim = xdrop.xd_get_timing(ctx)
    xdrop.xd_set_timing(ctx, False)
    if xdrop.xd_device_status(ctx) != 0:
        raise RuntimeError(f"device validation failed for {b.name}")
    got = out.cpu().numpy().view(xdrop.RESULT_DTYPE)
    for k in range(bpl):
        if not np.array_equal(got[k * b.n_pairs:(k + 1) * b.n_pairs], res):
            raise RuntimeError(f"{b.name}: batch {k} of a shared launch differs from its single-batch run")
    ms = ev0.elapsed_time(ev1) / (launches * bpl)
    nb = max(1, tim["batches"])
    tier_ms = [x / nb for x in tim["tier_ms"]]
    top = int(np.argmax(tier_ms))
    top_cells = tim["tier_cells"][top] / nb
    packed = packed_scores(b)
    peak = peak_16 if packed else peak_32
    achieved = ALG_OPS_PER_CELL * top_cells / (tier_ms[top] * 1e-3) / 1e12 if tier_ms[top] > 0 else 0.0
    rec.update({"gcups": cells / (ms * 1e-3) / 1e9, "pairs_per_s": b.n_pairs / (ms * 1e-3), "ms_per_batch": ms,
                "paper_gcups": paper_cells(b) / (ms * 1e-3) / 1e9, "cells_per_batch": cells,
                "roofline_frac": achieved / peak if peak else None, "dominant_stage_ms_per_launch": tier_ms[top],
                "dtype": "int16" if packed else "int32",
                "register_window_fill": (tim["register_band_cells"] / tim["register_slot_cells"]
                                         if tim["register_slot_cells"] else None)})
    del args, out
    if oracle_pairs:
        c, dt, n = cpu_oracle(b, oracle_pairs, os.cpu_count() or 1)
        rec["cpu_baseline"] = {"value": c / dt / 1e9, "unit": "GCUPS", "cores": os.cpu_count() or 1, "kind": "oracle",
                               "sample": f"{n} seeded-random pairs ({c:.3g} cells, {dt:.1f} s)"}
    return rec


def configs_bench(xdrop, torch, ctx, dev, bpl, peak_16, peak_32, headline, tune_table=None):
    """The other workloads, a few launches each; the headline's batch object is reused for
    its X variants.  With a tuning table, the memory-restricted uneven batches are also timed
    under it (single-batch launches, the size the table was tuned at)."""
    out = {}
    uneven = None
    tuned_ctx = xdrop.xd_create(dev.index or 0, tune_table=tune_table) if tune_table else None
    for name, kw in CONFIG_SET:
        if name == "dna_longread":
            b = headline.with_params(X=kw["X"])
        elif name == "uneven":
            uneven = uneven if uneven is not None else synth.uneven()
            b = uneven.with_params(delta=kw["delta"])
        else:
            b = synth.WORKLOADS[name]()
        k = f"{name}_{b.n_pairs}_x{b.X}" + (f"_delta{b.delta}" if b.delta else "")
        # large batches need fewer batches per launch to fill the GPU; the oracle sample is
        # sized to a few seconds of host work
        per = bpl if b.n_pairs <= 200_000 else max(1, bpl // 5)
        sample = {"dna_tiny": 1000, "protein": 50_000, "uneven": 5000}.get(name, 20_000)
        tc = tuned_ctx if name == "uneven" and b.delta > 0 else None
        out[k] = config_record(xdrop, torch, ctx, dev, b, per, 2, sample, peak_16, peak_32, tuned_ctx=tc)
        if tc is not None:
            out[k]["tune_table"] = os.path.relpath(tune_table, ROOT)
    if tuned_ctx is not None:
        xdrop.xd_destroy(tuned_ctx)
    return out


# ----------------------------------------------------------------------------- serving

SERVE_MAX_PAIRS = 10_000


class RequestMix:
    """Requests of log-uniform size in [1, 10,000] pairs, half DNA long-read pairs (X drawn
    from {10, 20, 50}) and half protein pairs (BLOSUM62, X = 49), each a contiguous pair
    range of a resident pool (zero-copy views; the library copies at submit)."""

    def __init__(self, dna, prot, seed):
        self.dna, self.prot = dna, prot
        self.rng = np.random.default_rng(seed)

    def next(self):
        rng = self.rng
        pool = self.dna if rng.random() < 0.5 else self.prot
        size = min(pool.n_pairs, int(np.exp(rng.uniform(0.0, np.log(SERVE_MAX_PAIRS + 1)))))
        size = max(1, size)
        a = int(rng.integers(0, pool.n_pairs - size + 1))
        b = pool.pair_range(a, a + size)
        if pool is self.dna:
            b = b.with_params(X=int(rng.choice([10, 20, 50])))
        b.meta["first_seq"] = 2 * a          # the range's sequences in the pool: 2a, 2a + 1, ...
        return b


def serve_run(xdrop, ctx, mix, rate_rps, duration, max_requests=None, submit=None):
    """Open-loop Poisson arrivals at rate_rps for `duration` seconds (rate_rps = inf: all
    at once).  Latency = completion time - scheduled arrival time.  Returns a summary.
    submit(b) -> ticket sends one request (default: the batch with its sequences)."""
    if submit is None:
        submit = lambda b: xdrop.xd_submit_batch(ctx, xdrop.BatchArgs.from_host(b))  # noqa: E731
    import threading
    rng = np.random.default_rng(99)
    arrivals, t = [], 0.0
    while True:
        if np.isinf(rate_rps):
            if len(arrivals) >= (max_requests or 200):
                break
        else:
            t += rng.exponential(1.0 / rate_rps)
            if t > duration or (max_requests and len(arrivals) >= max_requests):
                break
        arrivals.append(t if not np.isinf(rate_rps) else 0.0)
    # requests are drawn when they are sent (zero-copy views of the pools), so that runs of
    # many minutes hold only the outstanding ones
    n_req = len(arrivals)
    req_pairs = [0] * n_req
    outstanding = []          # (ticket, k, out)
    lock = threading.Lock()
    done_at = [None] * n_req
    cells = [0.0] * n_req
    submitted = threading.Event()
    errors = []

    def poller():
        while True:
            with lock:
                cur = list(outstanding)
            if not cur and submitted.is_set():
                return
            finished = []
            for item in cur:
                tk, k, out = item
                try:
                    rc = xdrop.xd_poll(ctx, tk, out, 0)
                except Exception as e:   # reported below
                    errors.append(e)
                    rc = xdrop.XD_OK
                if rc == xdrop.XD_OK:
                    done_at[k] = time.perf_counter()
                    cells[k] = float(out["left"]["cells"].sum() + out["right"]["cells"].sum())
                    finished.append(item)
            if finished:
                with lock:
                    for item in finished:
                        outstanding.remove(item)
            else:
                time.sleep(50e-6)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    start = [0.0] * n_req
    sub_begin = [0.0] * n_req
    sub_end = [0.0] * n_req
    for k, at in enumerate(arrivals):
        b = mix.next()
        req_pairs[k] = b.n_pairs
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        start[k] = t0 + at
        sub_begin[k] = time.perf_counter()
        while True:
            try:
                tk = submit(b)
                break
            except xdrop.XdError as e:
                if e.status != xdrop.XD_ENOMEM:
                    raise
                time.sleep(200e-6)          # admission refused: retry when memory frees up
        sub_end[k] = time.perf_counter()
        out = np.zeros(b.n_pairs, dtype=xdrop.RESULT_DTYPE)
        with lock:
            outstanding.append((tk, k, out))
    submitted.set()
    th.join()
    if errors:
        raise errors[0]
    t_end = max(done_at)
    lat = np.array([(d - s) * 1e3 for d, s in zip(done_at, start)])
    span = t_end - t0
    pairs = sum(req_pairs)
    wait = np.array([(b_ - s_) * 1e3 for b_, s_ in zip(sub_begin, start)])
    sub = np.array([(e_ - b_) * 1e3 for e_, b_ in zip(sub_end, sub_begin)])
    run = np.array([(d - e_) * 1e3 for d, e_ in zip(done_at, sub_end)])
    pct = lambda a, q: float(np.percentile(a, q))  # noqa: E731
    return {"requests": n_req, "pairs": pairs, "span_s": span,
            "pairs_per_s": pairs / span, "gcups": sum(cells) / span / 1e9,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": float(lat.mean()),
            "breakdown_ms": {"arrival_to_submit_p50": pct(wait, 50), "arrival_to_submit_p99": pct(wait, 99),
                             "submit_call_p50": pct(sub, 50), "submit_call_p99": pct(sub, 99),
                             "submitted_to_done_p50": pct(run, 50), "submitted_to_done_p99": pct(run, 99)}}


def serving_bench(xdrop, device, dna_pool, seconds, loads, inflight,
                  mode_names=("continuous", "per_batch", "continuous_resident")):
    """Continuous batching against one launch per request, at fractions of the peak."""
    prot_pool = synth.protein(n_pairs=200_000)
    mean_pairs = SERVE_MAX_PAIRS / np.log(SERVE_MAX_PAIRS + 1) - 0.5   # E[floor(exp(U(0, ln(N+1))))]
    res = {"duration_s_per_load": seconds, "request_pairs": f"log-uniform [1, {SERVE_MAX_PAIRS}]",
           "mix": "50% DNA long-read (X in {10, 20, 50}), 50% protein (BLOSUM62, X = 49)",
           "arrivals": "Poisson, open loop; latency from scheduled arrival to completion"}
    modes = {"continuous": dict(max_inflight=inflight, batching=1),
             "per_batch": dict(max_inflight=1, batching=-1),
             "continuous_resident": dict(max_inflight=inflight, batching=1)}
    res["continuous_resident_note"] = ("the pools' reads added once to the resident sequence store; "
                                       "each request sends only its seed tuples")
    for name in list(modes):
        if name not in mode_names:
            del modes[name]
    for name, kw in modes.items():
        ctx = xdrop.xd_create(device, **kw)
        try:
            submit = None
            if name == "continuous_resident":
                handles = {id(p): xdrop.xd_store_add(ctx, p.alphabet, p.codes, p.offsets, p.lengths)
                           for p in (dna_pool, prot_pool)}
                pools = {"dna": dna_pool, "protein": prot_pool}

                def submit(b, ctx=ctx, handles=handles, pools=pools):
                    h = handles[id(pools[b.alphabet])]
                    pr = b.pairs.copy()
                    base = b.meta["first_seq"]
                    pr[:, 0] = h[base + b.pairs[:, 0]]
                    pr[:, 1] = h[base + b.pairs[:, 1]]
                    return xdrop.xd_submit_pairs(ctx, b.alphabet, pr, b.match, b.mismatch, b.gap, b.matrix,
                                                 b.X, b.delta)
            # warm-up (pinned buffers, scratch), then the saturated peak
            serve_run(xdrop, ctx, RequestMix(dna_pool, prot_pool, 1), float("inf"), 0, max_requests=60,
                      submit=submit)
            peak = serve_run(xdrop, ctx, RequestMix(dna_pool, prot_pool, 2), float("inf"), 0,
                             max_requests=240, submit=submit)
            if "peak_pairs_per_s" not in res:   # the loads are fractions of the first mode's peak
                res["peak_pairs_per_s"] = peak["pairs_per_s"]
                res["peak_gcups"] = peak["gcups"]
                res["peak_mode"] = name
            out = {"saturated": peak, "loads": []}
            for ld in loads:
                rate_pairs = ld * res["peak_pairs_per_s"]
                rate_rps = rate_pairs / mean_pairs
                r = serve_run(xdrop, ctx, RequestMix(dna_pool, prot_pool, 3), rate_rps, seconds, submit=submit)
                r["load"] = ld
                r["offered_pairs_per_s"] = rate_pairs
                out["loads"].append(r)
            st = xdrop.xd_get_stats(ctx)
            out["launches"] = st["host_launches"]
            out["requests_launched"] = st["host_requests"]
            out["launches_with_several_parameter_sets"] = st["mixed_launches"]
            res[name] = out
        finally:
            xdrop.xd_destroy(ctx)
    return res


def run_reference(a, rank, world):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    if rank != 0:
        return
    b = make_batch(a, 0)
    threads = os.cpu_count() or 1
    per_step = max(200, a.cpu_pairs // 4)
    for _ in range(a.warmup):
        cpu_oracle(b, max(200, per_step // 8), threads)
    cells = secs = 0.0
    n_pairs = 0
    for s in range(a.steps):
        c, dt, n = cpu_oracle(b, per_step, threads)
        cells += c
        secs += dt
        n_pairs += n
    v = cells / secs / 1e9
    sample = f"{min(per_step, b.n_pairs)} seeded-random pairs of the workload per step"
    line = {"metric": "GCUPS", "value": v, "unit": "GCUPS", "impl": "reference", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": secs / a.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": workload_config(a, b),
            "pairs_per_s": n_pairs / secs,
            "cpu_baseline": {"value": v, "unit": "GCUPS", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)

    import torch
    from paper_2304_08662_gb300 import xdrop
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    b = make_batch(a, rank)
    cells_paper = paper_cells(b)
    ctx = xdrop.xd_create(local, tune_table=a.tune_table, max_inflight=a.slots)
    try:
        if a.autotune:
            tuned_ms = xdrop.xd_autotune(ctx, xdrop.BatchArgs.from_host(b), a.autotune)
            print(json.dumps({"autotune": a.autotune, "best_ms": tuned_ms}), file=sys.stderr, flush=True)
        codes = torch.from_numpy(b.codes).to(dev)
        offs = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
        lens = torch.from_numpy(b.lengths.view(np.int32)).to(dev)
        pairs = torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)
        args = xdrop.BatchArgs(b.alphabet, codes, offs, lens, pairs, b.match, b.mismatch, b.gap,
                               b.matrix, b.X, b.delta)
        out = torch.zeros(b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream(dev)
        bpl = max(1, a.batches_per_launch)
        for _ in range(max(3, a.warmup)):
            xdrop.xd_run_device(ctx, args, out, stream.cuda_stream)
        torch.cuda.synchronize(dev)
        if xdrop.xd_device_status(ctx) != 0:
            raise RuntimeError("device validation failed")
        res = out.cpu().numpy().view(xdrop.RESULT_DTYPE).copy()
        cells = float(res["left"]["cells"].sum() + res["right"]["cells"].sum())
        # the timed steps: launches of bpl batches each (the last one may hold fewer)
        launch_sizes = [min(bpl, a.steps - k) for k in range(0, a.steps, bpl)]
        out_many = None
        if bpl > 1:
            xdrop.xd_reserve(ctx, bpl * b.codes.size, bpl * b.n_seqs, bpl * b.n_pairs, int(b.lengths.max()))
            out_many = torch.zeros(bpl * b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
            for _ in range(max(1, -(-max(3, a.warmup) // bpl))):
                xdrop.xd_run_device_many(ctx, [args] * bpl, out_many, stream.cuda_stream)
            torch.cuda.synchronize(dev)
            if xdrop.xd_device_status(ctx) != 0:
                raise RuntimeError("device validation failed")
        else:
            xdrop.xd_reserve(ctx, b.codes.size, b.n_seqs, b.n_pairs, int(b.lengths.max()))

        # ---- timed region: device-resident inputs
        xdrop.xd_set_timing(ctx, True)
        clocks = Clocks(local)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        if bpl > 1:
            for k in launch_sizes:
                xdrop.xd_run_device_many(ctx, [args] * k, out_many, stream.cuda_stream)
        else:
            for _ in range(a.steps):
                xdrop.xd_run_device(ctx, args, out, stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1) / a.steps
        tim = xdrop.xd_get_timing(ctx)
        xdrop.xd_set_timing(ctx, False)
        if bpl > 1:
            # every batch of the last launch gave the single-batch results
            got = out_many.cpu().numpy().view(xdrop.RESULT_DTYPE)
            for k in range(launch_sizes[-1]):
                if not np.array_equal(got[k * b.n_pairs:(k + 1) * b.n_pairs], res):
                    raise RuntimeError(f"batch {k} of a shared launch differs from its single-batch run")
        # whole job: every rank's cells over the slowest rank's time (the ranks' batches are
        # seeded differently, so their cell counts differ)
        (job_cells, job_paper, job_pairs), (ms,) = job_totals(dist, dev, [cells, cells_paper, b.n_pairs], [ms])
        value = job_cells / (ms * 1e-3) / 1e9

        if a.trace:
            # outside the timed region: one more batch with the per-side timeline recorded
            xdrop.xd_set_trace(ctx, True)
            xdrop.xd_run_device(ctx, args, out, stream.cuda_stream)
            torch.cuda.synchronize(dev)
            save_trace(a.trace, xdrop.xd_get_trace(ctx))
            xdrop.xd_set_trace(ctx, False)

        # ---- roofline of the dominant alignment tier
        nb = max(1, tim["batches"])
        tier_ms = [x / nb for x in tim["tier_ms"]]
        top = int(np.argmax(tier_ms))
        top_cells = tim["tier_cells"][top] / nb
        achieved = ALG_OPS_PER_CELL * top_cells / (tier_ms[top] * 1e-3) / 1e12 if tier_ms[top] > 0 else 0.0
        props = torch.cuda.get_device_properties(dev)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except (OSError, ValueError):
            pass
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        packed = packed_scores(b)
        width = 2 if packed else 1    # 16-bit lanes per ALU lane
        peak32 = props.multi_processor_count * ALU_LANES_PER_SM * sm_max * 1e6 / 1e12
        peak16 = 2 * peak32
        peak = width * peak32
        # measured in this run: the ALU pipe's issue rate (max, or max on 16x2) and the tiers'
        # own cell update
        alu_meas = width * xdrop.xd_probe(ctx, "max_16x2" if packed else "max") / 1e12
        cell_probe = xdrop.xd_probe(ctx, ("cell_dna" if b.alphabet == "dna" else "cell_prot") +
                                    ("16" if packed else ""))
        tier_names = ["first register launch (fused persistent grid of levels 0-2, or level 0)",
                      "later register levels and band tier", "generic tier"]
        tuned_env = any(k.startswith("XD_") for k in os.environ)
        per_cell = None if tuned_env else DOMINANT_KERNEL_TRAFFIC_PER_CELL.get((workload_config(a, b)["workload"], bpl))
        traffic = per_cell * top_cells if per_cell else None   # bytes per launch
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                    "frac": achieved / peak if peak else None, "traffic": traffic,
                    "traffic_basis": ("dram__bytes_read.sum + dram__bytes_write.sum per computed cell of the same "
                                      "kernel build (ncu, 40,000 pairs) x the launch's cells") if traffic else None,
                    "achieved_hbm_gbs": traffic / (tier_ms[top] * 1e-3) / 1e9 if traffic else None,
                    "kernel": tier_names[top], "ops_per_cell": ALG_OPS_PER_CELL,
                    "peak_basis": f"{props.multi_processor_count} SMs x {ALU_LANES_PER_SM} integer ALU-pipe "
                                  f"lanes x {width} ({'16-bit halves' if packed else '32-bit'}) x "
                                  f"{sm_max:.0f} MHz (max SM clock)",
                    "op_width_bits": 16 if packed else 32,
                    "kernel_ms": tier_ms[top],
                    "measured_alu_peak": alu_meas, "frac_of_measured_alu": achieved / alu_meas,
                    "cell_probe_gcups": cell_probe / 1e9,
                    "frac_of_cell_probe": top_cells / (tier_ms[top] * 1e-3) / cell_probe}
        if clk.get("sm_mhz"):
            roofline["frac_at_sampled_clock"] = achieved / (peak * clk["sm_mhz"] / sm_max)

        # ---- end to end through host buffers
        e2e = None
        if not a.no_e2e:
            hargs = xdrop.BatchArgs.from_host(b)
            hout = np.zeros(b.n_pairs, dtype=xdrop.RESULT_DTYPE)
            # batches in flight: the next batches' host staging and upload overlap the
            # current launch (every copy stays inside the timed region), and batches that
            # wait together leave in one merged launch
            in_flight = max(1, a.e2e_inflight)

            def e2e_pass(n):
                pending = []
                for _ in range(n):
                    pending.append(xdrop.xd_submit_batch(ctx, hargs))
                    if len(pending) == in_flight:
                        if xdrop.xd_poll(ctx, pending.pop(0), hout, -1) != xdrop.XD_OK:
                            raise RuntimeError("e2e batch failed")
                for t in pending:
                    if xdrop.xd_poll(ctx, t, hout, -1) != xdrop.XD_OK:
                        raise RuntimeError("e2e batch failed")

            # warm-up: the same pattern twice, so that every launch slot has grown its device
            # buffers (and the pinned staging cache its buffers) for the merged launches
            for _ in range(2):
                e2e_pass(2 * in_flight)
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            e2e_pass(a.steps)
            e2e_s = (time.perf_counter() - t0) / a.steps
            _, (e2e_s,) = job_totals(dist, dev, [0], [e2e_s])
            assert np.array_equal(hout, res), "host and device entry points disagree"
            # what crosses to the device: the residues as packed while they are staged (2-bit
            # DNA, 16 per word; 5-bit protein, 6 per word), the sequence table and the tuples
            per_word = 16 if b.alphabet == "dna" else 6
            h2d = int(4 * -(-b.codes.size // per_word) + b.offsets.nbytes + b.lengths.nbytes + b.pairs.nbytes)
            e2e = {"value": job_cells / e2e_s / 1e9, "unit": "GCUPS", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": int(hout.nbytes), "ms_per_step": e2e_s * 1e3,
                   "in_flight": in_flight, "slots": a.slots or 3}

        serving = None
        if rank == 0 and a.serve > 0 and a.workload == "dna_longread":
            loads = [float(x) for x in a.serve_loads.split(",") if x]
            serving = serving_bench(xdrop, local, b, a.serve, loads, a.serve_inflight,
                                    tuple(m for m in a.serve_modes.split(",") if m))

        cpu = None
        if rank == 0 and not a.no_cpu:
            cpu = cpu_baseline(b, a.cpu_pairs, os.cpu_count() or 1)

        configs = None
        if rank == 0 and not a.no_configs and a.workload == "dna_longread" and a.pairs is None and a.x is None:
            table = a.configs_tune_table if a.configs_tune_table and os.path.exists(a.configs_tune_table) else None
            configs = configs_bench(xdrop, torch, ctx, dev, bpl, peak16, peak32, b, tune_table=table)

        if rank == 0:
            line = {"metric": "GCUPS", "value": value, "unit": "GCUPS", "n_gpus": world,
                    "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": "int16" if packed_scores(b) else "int32", "data": "synthetic",
                    "config": workload_config(a, b),
                    "pairs_per_s": job_pairs / (ms * 1e-3),
                    "paper_gcups": job_paper / (ms * 1e-3) / 1e9,
                    "cells_per_step": cells,
                    "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                    "gpu_launches": int(tim["launches"]),
                    "stages_ms": {"pack": tim["pack_ms"] / nb, "units": tim["units_ms"] / nb,
                                  "order": tim["order_ms"] / nb, "tiers": tier_ms,
                                  "totals": tim["totals_ms"] / nb},
                    "tier_units": [u / nb for u in tim["tier_units"]],
                    "tier_cells": [c_ / nb for c_ in tim["tier_cells"]],
                    "discarded_cells_per_step": tim["discarded_cells"] / nb,
                    "escalations_per_step": tim["escalations"] / nb,
                    "window_shifts_per_step": tim["window_shifts"] / nb,
                    "register_window_fill": (tim["register_band_cells"] / tim["register_slot_cells"]
                                             if tim["register_slot_cells"] else None),
                    "serving": serving,
                    "configs": configs,
                    "clocks": clk}
            print(json.dumps(line), flush=True)
    finally:
        xdrop.xd_destroy(ctx)
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
