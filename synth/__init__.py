"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the bench.

Holds input generators and input tables only (no alignment arithmetic)."""
from .tables import BLOSUM62, BACKGROUND, AMINO_ACIDS, DNA_BASES
from .workloads import (Batch, DNA, PROTEIN, X_INF, dna_tiny, dna_longread, protein, uneven,
                        from_strings, WORKLOADS)
