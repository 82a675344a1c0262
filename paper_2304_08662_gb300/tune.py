"""Writes the tuning table of this GPU.

The batching scheme of Sec. 4.2 distributes comparisons over the compute units by their
estimated cost; on this GPU the matching choice is the launch configuration of a class of
batches (register-level chain, queue chunk, band-tier warps per side, role mix of the
persistent grid).  This command runs ``xd_autotune`` on seeded synthetic samples of the
workload shapes and merges each winner into one text table, which
``xd_create(tune_table=...)`` loads.  Entries are keyed by alphabet, X, longest side, size
and memory-restricted window (Sec. 3.3), so the uneven batch gets one entry per delta_b.

    python -m paper_2304_08662_gb300.tune --out paper_2304_08662_gb300/tuning/gb300.txt \\
        --workload uneven --delta 256,1024,4096

Every candidate must reproduce the first candidate's results bit for bit (the library
checks this and fails otherwise), so a table changes speed, never results.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

from . import xdrop  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True, help="table to create or merge into")
    ap.add_argument("--workload", default="uneven", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--pairs", type=int, default=None, help="sample size (default: the workload's)")
    ap.add_argument("--x", default=None, help="comma-separated X values (default: the workload's)")
    ap.add_argument("--delta", default=None, help="comma-separated delta_b values (default: the workload's)")
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    kw = {} if a.pairs is None else {"n_pairs": a.pairs}
    base = synth.WORKLOADS[a.workload](**kw)
    xs = [int(v) for v in a.x.split(",")] if a.x else [base.X]
    deltas = [int(v) for v in a.delta.split(",")] if a.delta else [base.delta]
    ctx = xdrop.xd_create(a.device)
    try:
        for X in xs:
            for d in deltas:
                b = base.with_params(X=X, delta=d)
                t0 = time.perf_counter()
                ms = xdrop.xd_autotune(ctx, xdrop.BatchArgs.from_host(b), a.out)
                print(json.dumps({"workload": a.workload, "pairs": b.n_pairs, "X": X, "delta_b": d,
                                  "best_ms": round(ms, 3), "tuning_s": round(time.perf_counter() - t0, 1)}),
                      flush=True)
    finally:
        xdrop.xd_destroy(ctx)


if __name__ == "__main__":
    main()
