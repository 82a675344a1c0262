"""Benchmark of batched X-Drop seed extension on GB300.

A step is one pass of the whole hot path over one batch: pack the residue codes, build
the work units (left and right extension per pair), order them by cost, run the
alignment tiers, and form the pair totals.  The default workload is the DNA long-read
batch: 100,000 dovetail pairs, lengths lognormal (median 8 kbp) in [1, 30] kbp, 8-18%
error, 10% unrelated, k = 17, +1/-1/-1, X = 20, unrestricted.

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
INT32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dna_longread", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--x", type=int, default=None, help="X (default: the workload's)")
    ap.add_argument("--delta", type=int, default=0)
    ap.add_argument("--pairs", type=int, default=None, help="pairs (default: the workload's full size)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-pairs", type=int, default=8000, help="oracle sample size")
    return ap.parse_args()


def make_batch(a, rank):
    gen = synth.WORKLOADS[a.workload]
    kw = {}
    if a.pairs is not None:
        kw["n_pairs"] = a.pairs
    if a.workload == "uneven":
        kw["delta"] = a.delta
    b = gen(**kw) if rank == 0 else gen(seed=1000 + rank, **kw)
    if a.x is not None:
        b = b.with_params(X=a.x)
    if a.delta and a.workload != "uneven":
        b = b.with_params(delta=a.delta)
    return b


def workload_config(a, b):
    return {"workload": f"{a.workload}_{b.n_pairs}_x{b.X}" + (f"_delta{b.delta}" if b.delta else ""),
            "pairs": b.n_pairs, "residues": int(b.codes.size), "X": b.X, "delta_b": b.delta,
            "alphabet": b.alphabet, "scoring": ("BLOSUM62" if b.alphabet == "protein" else
                                                f"{b.match}/{b.mismatch}/{b.gap}"),
            "l2": "inputs larger than L2 (codes %.2f GB)" % (b.codes.size / 1e9),
            "parallelism": "replicas (one batch per GPU)"}


def paper_cells(b):
    p = b.pairs.astype(np.int64)
    return float((b.lengths[p[:, 0]].astype(np.float64) * b.lengths[p[:, 1]]).sum())


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


def run_reference(a, rank, world):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    if rank != 0:
        return
    b = make_batch(a, 0)
    threads = os.cpu_count() or 1
    for _ in range(a.warmup):
        cpu_oracle(b, max(200, a.cpu_pairs // 8), threads)
    cells = secs = 0.0
    n_pairs = 0
    for s in range(a.steps):
        c, dt, n = cpu_oracle(b, a.cpu_pairs, threads)
        cells += c
        secs += dt
        n_pairs += n
    v = cells / secs / 1e9
    sample = f"{a.cpu_pairs} seeded-random pairs of the workload per step"
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
    ctx = xdrop.xd_create(local)
    try:
        codes = torch.from_numpy(b.codes).to(dev)
        offs = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
        lens = torch.from_numpy(b.lengths.view(np.int32)).to(dev)
        pairs = torch.from_numpy(np.ascontiguousarray(b.pairs).view(np.int32)).to(dev)
        args = xdrop.BatchArgs(b.alphabet, codes, offs, lens, pairs, b.match, b.mismatch, b.gap,
                               b.matrix, b.X, b.delta)
        out = torch.zeros(b.n_pairs * xdrop.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        xdrop.xd_reserve(ctx, b.codes.size, b.n_seqs, b.n_pairs, int(b.lengths.max()))
        stream = torch.cuda.current_stream(dev)
        for _ in range(max(3, a.warmup)):
            xdrop.xd_run_device(ctx, args, out, stream.cuda_stream)
        torch.cuda.synchronize(dev)
        if xdrop.xd_device_status(ctx) != 0:
            raise RuntimeError("device validation failed")
        res = out.cpu().numpy().view(xdrop.RESULT_DTYPE)
        cells = float(res["left"]["cells"].sum() + res["right"]["cells"].sum())

        # ---- timed region: device-resident inputs
        xdrop.xd_set_timing(ctx, True)
        clocks = Clocks(local)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
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
        if dist:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        value = cells * world / (ms * 1e-3) / 1e9

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
        peak = props.multi_processor_count * INT32_LANES_PER_SM * sm_max * 1e6 / 1e12
        tier_names = ["narrow (thread per side)", "wide (warp per side)", "generic (warp per side, global ring)"]
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                    "frac": achieved / peak if peak else None, "traffic": None,
                    "kernel": tier_names[top],
                    "ops_per_cell": ALG_OPS_PER_CELL,
                    "peak_basis": f"{props.multi_processor_count} SMs x {INT32_LANES_PER_SM} INT32 lanes x "
                                  f"{sm_max:.0f} MHz (max SM clock)",
                    "kernel_ms": tier_ms[top]}
        if clk.get("sm_mhz"):
            roofline["frac_at_sampled_clock"] = achieved / (peak * clk["sm_mhz"] / sm_max)

        # ---- end to end through host buffers
        e2e = None
        if not a.no_e2e:
            hargs = xdrop.BatchArgs.from_host(b)
            hout = np.zeros(b.n_pairs, dtype=xdrop.RESULT_DTYPE)
            t = xdrop.xd_submit_batch(ctx, hargs)
            xdrop.xd_poll(ctx, t, hout, -1)
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            for _ in range(a.steps):
                t = xdrop.xd_submit_batch(ctx, hargs)
                if xdrop.xd_poll(ctx, t, hout, -1) != xdrop.XD_OK:
                    raise RuntimeError("e2e batch failed")
            e2e_s = (time.perf_counter() - t0) / a.steps
            if dist:
                tt = torch.tensor([e2e_s], device=dev)
                dist.all_reduce(tt, op=dist.ReduceOp.MAX)
                e2e_s = float(tt.item())
            assert np.array_equal(hout, res), "host and device entry points disagree"
            h2d = int(b.codes.nbytes + b.offsets.nbytes + b.lengths.nbytes + b.pairs.nbytes)
            e2e = {"value": cells * world / e2e_s / 1e9, "unit": "GCUPS", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": int(hout.nbytes), "ms_per_step": e2e_s * 1e3}

        cpu = None
        if rank == 0 and not a.no_cpu:
            threads = os.cpu_count() or 1
            c, dt, n = cpu_oracle(b, a.cpu_pairs, threads)
            cpu = {"value": c / dt / 1e9, "unit": "GCUPS", "cores": threads, "kind": "oracle",
                   "sample": f"{n} seeded-random pairs of the same workload ({c:.3g} cells, {dt:.1f} s)"}

        if rank == 0:
            line = {"metric": "GCUPS", "value": value, "unit": "GCUPS", "n_gpus": world,
                    "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": "int32", "data": "synthetic", "config": workload_config(a, b),
                    "pairs_per_s": b.n_pairs * world / (ms * 1e-3),
                    "paper_gcups": cells_paper * world / (ms * 1e-3) / 1e9,
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
                    "clocks": clk}
            print(json.dumps(line), flush=True)
    finally:
        xdrop.xd_destroy(ctx)
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
