"""Rewrites the 'scores' lines of regression_x_nonmonotone.txt from the oracle alone."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    path = os.path.join(HERE, "regression_x_nonmonotone.txt")
    lines = open(path).read().splitlines()
    sim = oracle.sim_table("dna", 1, -1)
    lut = {c: i for i, c in enumerate("ACGT")}
    out, h = [], None
    for ln in lines:
        if ln.startswith("H "):
            h = [lut[c] for c in ln[2:]]
        elif ln.startswith("V "):
            v = [lut[c] for c in ln[2:]]
        elif ln.startswith("scores"):
            ln = "scores " + " ".join(str(oracle.extend(h, v, sim, -1, X)["score"]) for X in range(5))
        out.append(ln)
    open(path, "w").write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
