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
    kw = dict(kw)
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


# Alternative schedules: custom level-1 diameters (one, two and three edges of
# the largest weight) and other (q, phi_min).  Theorem 1 holds for any
# admissible schedule, so every candidate must reproduce global sparse blossom.
SCHEDULES = [
    ("d1=2 edges", dict(d1=2)),
    ("d1=3 edges", dict(d1=3)),
    ("d1=2 edges, wide b1", dict(d1=2, b1_factor=3)),
    ("q=1/2, phi_min=1/10", dict(q=(1, 2), phi_min=(1, 10))),
    ("q=1/50, phi_min=1/1000", dict(q=(1, 50), phi_min=(1, 1000))),
]


def schedule_kw(g, spec):
    """Oracle-graph keyword arguments for a schedule spec on graph g."""
    wmax_internal = 2 * int(g.w.max())
    kw = {k: v for k, v in spec.items() if k in ("q", "phi_min")}
    if "d1" in spec:
        kw["d1"] = spec["d1"] * wmax_internal + 1
        if "b1_factor" in spec:
            kw["b1"] = spec["b1_factor"] * kw["d1"]
    return kw


@pytest.mark.parametrize("sname,spec", SCHEDULES, ids=[s[0] for s in SCHEDULES])
@pytest.mark.parametrize("name,kw,shots", [CASES[0], CASES[1], CASES[3]], ids=[CASES[i][0] for i in (0, 1, 3)])
def test_alternative_schedules_equal_global(sname, spec, name, kw, shots):
    kw = dict(kw)
    d = kw.pop("d")
    g = rotated_surface_code(d, d, **kw)
    og = OracleGraph.from_phys(g, **schedule_kw(g, spec))
    ref = OracleGraph.from_phys(g)
    syn, _ = sample_shots(g, min(shots, 400), 23)
    for s in range(syn.shape[0]):
        det = unpack_defects(syn[s], g.num_detectors)
        a = ref.decode(det, "global")
        b = og.decode(det, "hier")
        assert b.status == 0 and (a.weight, a.obs) == (b.weight, b.obs), (sname, s, det.tolist())
        assert b.dual_feasible and b.tight and b.dual_sum == b.primal_internal
        assert b.touch_violations == 0
