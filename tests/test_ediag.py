"""Pins of the oracle's parallel event count E_ideal (Methods, "Numerical
evaluation") against things other than itself: hand-worked examples on a path
graph (tests/golden/ediag_line50.json, each derivation written out there), the
single-cluster special case, which must reduce to the plain event count of one
global sparse-blossom run, and invariants of the critical-path recursion."""

import json
import math
import os

import numpy as np
import pytest

from oracle import OracleGraph
from synth import rotated_surface_code, sample_shots, unpack_defects

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ediag_line50.json")


def line50(w0):
    n = 50
    u = list(range(49)) + [0, 49]
    v = list(range(1, 50)) + [-1, -1]
    w = [5] * 49 + [w0, 5]
    return n, u, v, w, [0] * 51


def golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_worked_examples(case):
    og = OracleGraph(*line50(case["w0"]))
    assert int(og.dk[0]) == 11 and int(og.bk[0]) == 23
    for mode in ("hier", "global"):
        r = og.diag(case["defects"], mode)
        exp = case[mode]
        got = {k: r[k] for k in exp}
        assert got == exp, (mode, got, exp)
        assert r["status"] == 0


CASES = [(7, 0.01, 300, 1), (9, 0.005, 200, 2), (5, 0.03, 300, 3), (11, 0.003, 150, 4)]


@pytest.mark.parametrize("d,p,shots,seed", CASES)
def test_single_cluster_is_the_global_run(d, p, shots, seed):
    """With one level whose link radius and diameter exceed every distance, all
    detection events form one level-1 cluster run from an empty state: its
    E_ideal is its whole event count, equal to global sparse blossom's."""
    pg = rotated_surface_code(d, d, p)
    og = OracleGraph.from_phys(pg)
    og.dk = np.asarray([1 << 60], np.int64)
    og.bk = np.asarray([1 << 60], np.int64)
    syn, _ = sample_shots(pg, shots, seed)
    for row in syn:
        dets = unpack_defects(row, pg.num_detectors)
        h = og.diag(dets, "hier")
        g = og.diag(dets, "global")
        assert h["clusters_above_l1"] == 0
        assert h["l1_clusters"] == (1 if len(dets) else 0)
        for k in ("weight", "obs", "e_ideal", "t_ideal", "events"):
            assert h[k] == g[k], (k, h, g)


@pytest.mark.parametrize("d,p,shots,seed", CASES)
def test_recursion_invariants(d, p, shots, seed):
    pg = rotated_surface_code(d, d, p)
    og = OracleGraph.from_phys(pg)
    syn, _ = sample_shots(pg, shots, seed + 100)
    for row in syn:
        dets = unpack_defects(row, pg.num_detectors)
        k = len(dets)
        h = og.diag(dets, "hier")
        g = og.diag(dets, "global")
        r = og.decode(dets, "hier")
        assert h["weight"] == g["weight"]
        if k == 0:
            assert h["e_ideal"] == g["e_ideal"] == 0 and h["t_ideal"] == 0
            continue
        # every augmentation retires at most two unmatched events
        assert g["events"] >= math.ceil(k / 2) and g["e_ideal"] == g["events"]
        # the critical path holds at least one event and at most all of them
        assert 1 <= h["e_ideal"] <= h["events"]
        # its stopping time is the latest stopping time of any cluster
        assert h["t_ideal"] == r.stop_time
        # level-1 clusters alone run fully in parallel: their critical path is
        # one cluster's event count, at least one per cluster
        if h["clusters_above_l1"] == 0:
            assert h["e_ideal"] <= h["events"] - h["l1_clusters"] + 1
