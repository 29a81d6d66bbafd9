"""CPU oracle for the parallel sparse-blossom decoder.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import it; the product path never does.
It shares no code with the CUDA path (see sb_oracle.c for what it computes).
"""

from .oracle import OracleGraph, OResult  # noqa: F401
from .schedule import alg3  # noqa: F401
