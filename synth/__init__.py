"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only builds input data: the phenomenological rotated-surface-code
detector multigraph (one physical edge per elementary fault, each with its own
probability and integer weight), the circuit-level detector graph of the same
code's syndrome-extraction circuit, and syndromes sampled from them.  It contains no step of the decoding method itself (no edge merging,
no distances, no matching).
"""

from .surface import (  # noqa: F401
    PhysGraph,
    rotated_surface_code,
    sample_shots,
    mixed_batch,
    weight_of_p,
    pack_defects,
    unpack_defects,
)
from .circuit import rotated_surface_code_circuit  # noqa: F401
