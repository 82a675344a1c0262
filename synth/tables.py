"""Scoring tables and residue frequencies used as *inputs* by the workload generators.

These are data, not alignment arithmetic: both the oracle and the CUDA library receive
them as plain arrays through their own interfaces.

* BLOSUM62 (Henikoff & Henikoff 1992), the substitution matrix the paper uses for its
  protein runs together with a linear gap score of -2 and X = 49 (Sec. 5.3, "PASTIS").
  Residue order is the conventional A R N D C Q E G H I L K M F P S T W Y V, and the
  code of a residue is its index in that order (0..19).
* Background amino-acid frequencies of Robinson & Robinson (1991), a published
  approximation used to draw synthetic protein residues.  Nothing in the alignment
  results depends on their exact values, because both sides read identical codes.
"""
import numpy as np

AMINO_ACIDS = "ARNDCQEGHILKMFPSTWYV"
DNA_BASES = "ACGT"

_BLOSUM62_ROWS = """
 4 -1 -2 -2  0 -1 -1  0 -2 -1 -1 -1 -1 -2 -1  1  0 -3 -2  0
-1  5  0 -2 -3  1  0 -2  0 -3 -2  2 -1 -3 -2 -1 -1 -3 -2 -3
-2  0  6  1 -3  0  0  0  1 -3 -3  0 -2 -3 -2  1  0 -4 -2 -3
-2 -2  1  6 -3  0  2 -1 -1 -3 -4 -1 -3 -3 -1  0 -1 -4 -3 -3
 0 -3 -3 -3  9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1
-1  1  0  0 -3  5  2 -2  0 -3 -2  1  0 -3 -1  0 -1 -2 -1 -2
-1  0  0  2 -4  2  5 -2  0 -3 -3  1 -2 -3 -1  0 -1 -3 -2 -2
 0 -2  0 -1 -3 -2 -2  6 -2 -4 -4 -2 -3 -3 -2  0 -2 -2 -3 -3
-2  0  1 -1 -3  0  0 -2  8 -3 -3 -1 -2 -1 -2 -1 -2 -2  2 -3
-1 -3 -3 -3 -1 -3 -3 -4 -3  4  2 -3  1  0 -3 -2 -1 -3 -1  3
-1 -2 -3 -4 -1 -2 -3 -4 -3  2  4 -2  2  0 -3 -2 -1 -2 -1  1
-1  2  0 -1 -3  1  1 -2 -1 -3 -2  5 -1 -3 -1  0 -1 -3 -2 -2
-1 -1 -2 -3 -1  0 -2 -3 -2  1  2 -1  5  0 -2 -1 -1 -1 -1  1
-2 -3 -3 -3 -2 -3 -3 -3 -1  0  0 -3  0  6 -4 -2 -2  1  3 -1
-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4  7 -1 -1 -4 -3 -2
 1 -1  1  0 -1  0  0  0 -1 -2 -2  0 -1 -2 -1  4  1 -3 -2 -2
 0 -1  0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1  1  5 -2 -2  0
-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1  1 -4 -3 -2 11  2 -3
-2 -2 -2 -3 -2 -1 -2 -3  2 -1 -1 -2 -1  3 -3 -2 -2  2  7 -1
 0 -3 -3 -3 -1 -2 -2 -3 -3  3  1 -2  1 -1 -2 -2  0 -3 -1  4
"""

BLOSUM62 = np.array([[int(x) for x in row.split()] for row in _BLOSUM62_ROWS.strip().splitlines()],
                    dtype=np.int8)
BLOSUM62.setflags(write=False)

# Robinson & Robinson (1991) background frequencies, same residue order as above.
_RR_FREQ = {
    "A": 0.07805, "R": 0.05129, "N": 0.04487, "D": 0.05364, "C": 0.01925,
    "Q": 0.04264, "E": 0.06295, "G": 0.07377, "H": 0.02199, "I": 0.05142,
    "L": 0.09019, "K": 0.05744, "M": 0.02243, "F": 0.03856, "P": 0.05203,
    "S": 0.07120, "T": 0.05841, "W": 0.01330, "Y": 0.03216, "V": 0.06441,
}
BACKGROUND = np.array([_RR_FREQ[a] for a in AMINO_ACIDS], dtype=np.float64)
BACKGROUND = BACKGROUND / BACKGROUND.sum()
BACKGROUND.setflags(write=False)


def karlin_altschul_lambda(matrix=BLOSUM62, freqs=BACKGROUND):
    """Positive root of sum_ab p_a p_b exp(lambda * s_ab) = 1 (Karlin-Altschul), by bisection.

    Used only to shape the synthetic substitution model P(b|a) ~ p_b exp(lambda s_ab).
    """
    s = np.asarray(matrix, dtype=np.float64)
    pp = np.outer(freqs, freqs)

    def f(lam):
        return float((pp * np.exp(lam * s)).sum()) - 1.0

    lo, hi = 1e-6, 2.0
    assert f(lo) < 0.0 < f(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def substitution_model(matrix=BLOSUM62, freqs=BACKGROUND):
    """Row-stochastic 20x20 matrix Q[a, b] = P(b | a, substitution), b != a.

    P(b|a) is proportional to p_b * exp(lambda * s_ab) over b != a (a changed residue is
    always a different residue, so the per-site identity of a homolog equals one minus
    its substitution rate before indels).
    """
    lam = karlin_altschul_lambda(matrix, freqs)
    w = freqs[None, :] * np.exp(lam * np.asarray(matrix, dtype=np.float64))
    np.fill_diagonal(w, 0.0)
    return w / w.sum(axis=1, keepdims=True)
