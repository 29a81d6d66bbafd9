"""Pins of the oracle's sliding-window decoding (windows of W detector layers
every C layers, commit region = first C layers) against things other than
itself: one window over the whole history is global sparse blossom; the
committed edges of all windows form a correction of the whole history's
syndrome (every detector's committed degree has the parity of its syndrome
bit); with W >= C the plan covers every layer once in the commit regions."""

import numpy as np
import pytest

from oracle import OracleGraph
from oracle.window import sliding_window_decode, window_graph, windows
from synth import rotated_surface_code, rotated_surface_code_circuit, sample_shots, unpack_defects


def test_window_plan_tiles_the_layers():
    for L in (1, 2, 7, 24, 25, 100):
        for W, C in ((1, 1), (4, 2), (10, 5), (10, 10), (30, 7)):
            plan = windows(L, W, C)
            assert plan[-1][2] and plan[-1][0] + plan[-1][1] == L
            commits = []
            for a, nl, last in plan:
                commits.extend(range(a, a + (nl if last else C)))
            assert commits == list(range(L))


def test_window_graph_is_the_induced_subgraph():
    g = rotated_surface_code(5, 12, 0.01)
    n, u, v, w, o, emap = window_graph(g, 4, 5)
    lo, hi = 4 * g.nz, 9 * g.nz
    assert n == hi - lo
    inside = [(a, b) for a, b in zip(g.u, g.v) if lo <= a < hi and (b < 0 or lo <= b < hi)]
    assert len(inside) == u.shape[0]
    assert np.array_equal(g.u[emap] - lo, u)
    assert np.array_equal(np.where(g.v[emap] >= 0, g.v[emap] - lo, -1), v)
    assert np.array_equal(g.w[emap], w) and np.array_equal(g.obs[emap], o)
    # a window of the rotated code over layers [a, a + L) is the code's own graph
    # with L - 1 noisy rounds, apart from the perfect last round: same counts of
    # space edges per layer (d*d) and time edges between its layers (nz each)
    assert u.shape[0] == 5 * 25 + 4 * g.nz
    # the first and last layers are cut off from the layers beyond them
    assert not np.any((g.u[emap] < lo) | (g.u[emap] >= hi))


@pytest.mark.parametrize("d,R,p,shots", [(5, 10, 0.01, 80), (7, 7, 0.005, 60)])
def test_single_window_is_global(d, R, p, shots):
    g = rotated_surface_code(d, R, p)
    syn, _ = sample_shots(g, shots, 4)
    obs, st = sliding_window_decode(g, syn, 10 * R, 5 * R)
    W_, O, S = OracleGraph.from_phys(g).decode_bitmaps(syn, "global")
    assert np.array_equal(st, S) and np.array_equal(obs, O)


@pytest.mark.parametrize("d,R,p,W,C,shots,circuit", [(5, 24, 0.01, 10, 5, 60, False), (5, 20, 0.03, 8, 3, 50, False),
                                                      (7, 21, 0.005, 14, 7, 30, False), (5, 16, 0.02, 6, 6, 40, False),
                                                      (5, 20, 0.003, 10, 5, 40, True), (5, 15, 0.006, 6, 3, 30, True)])
def test_committed_edges_correct_the_history(d, R, p, W, C, shots, circuit):
    g = rotated_surface_code_circuit(d, R, p) if circuit else rotated_surface_code(d, R, p)
    syn, _ = sample_shots(g, shots, 8)
    obs, st, edges = sliding_window_decode(g, syn, W, C, return_edges=True)
    assert not st.any()
    for s in range(shots):
        deg = np.zeros(g.num_detectors, np.int64)
        for u, v in edges[s]:
            deg[u] += 1
            if v >= 0:
                deg[v] += 1
        want = np.zeros(g.num_detectors, np.int64)
        want[unpack_defects(syn[s], g.num_detectors)] = 1
        assert np.array_equal(deg & 1, want), s
