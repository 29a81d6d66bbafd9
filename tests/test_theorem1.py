"""Theorem 1: the hierarchical (parallel) execution equals global sparse blossom.

The oracle runs both modes on the same shots; they must agree bit-exactly on the
matching weight and observable mask, every run must end with primal == dual,
dual feasibility and tight matched edges, and no inherited configuration may be
touched by a processing cluster of its own or a lower level (SI Lemma 'Unique
touching of inherited matching configurations').
"""

import numpy as np
import pytest

from oracle import OracleGraph
from synth import rotated_surface_code, sample_shots, unpack_defects

CASES = [
    ("d5 p=0.005", dict(d=5, p=0.005), 3000),
    ("d11 p~U[.002,.006]", dict(d=11, p_range=(0.002, 0.006), p_seed=1), 600),
    ("d9 p=0.003", dict(d=9, p=0.003), 800),
    ("d7 p=0.04 (blossoms)", dict(d=7, p=0.04), 400),
    ("d13 p=0.01", dict(d=13, p=0.01), 120),
    ("d21 p=0.003", dict(d=21, p=0.003), 25),
]


@pytest.mark.parametrize("name,kw,shots", CASES, ids=[c[0] for c in CASES])
def test_global_equals_hierarchical(name, kw, shots):
    d = kw.pop("d")
    g = rotated_surface_code(d, d, **kw)
    og = OracleGraph.from_phys(g)
    syn, true_obs = sample_shots(g, shots, 17)
    implodes = 0
    for s in range(shots):
        det = unpack_defects(syn[s], g.num_detectors)
        a = og.decode(det, "global")
        b = og.decode(det, "hier")
        assert a.status == 0 and b.status == 0
        assert (a.weight, a.obs) == (b.weight, b.obs), (s, det.tolist())
        for r in (a, b):
            assert r.dual_feasible and r.tight and r.dual_sum == r.primal_internal
        assert b.touch_violations == 0
        implodes += a.events_implode
    if "blossoms" in name:
        assert implodes > 0
