"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Input generation only: nothing here computes any part of the alignment method.
"""

from .blosum62 import ALPHABET, STANDARD, blosum62, decode, encode  # noqa: F401
from .generate import (  # noqa: F401
    ALPHABET_SIZE, BACKGROUND, CODE_W, LONG_QUERY_LENGTHS, PAPER_QUERY_LENGTHS, Database,
    Workload, batched, database_from_lengths, draw_residues, from_sequences, long_subject,
    make_database, make_queries, paper_shaped, plain, plant_saturating, poisson_arrivals,
    sample_indices, serving_queries,
)
