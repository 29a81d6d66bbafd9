"""GPU parallel-event-count diagnostics and global mode (qec_decode_batch_ex)
against the oracle, bit-exact per shot.  Needs a GB300."""

import json
import os

import numpy as np
import pytest

from oracle import OracleGraph
from synth import mixed_batch, rotated_surface_code, sample_shots, unpack_defects

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ediag_line50.json")
FIELDS = ("e_ideal", "t_ideal", "events", "l1_clusters", "l1_defects", "defects")
COL = {"e_ideal": 0, "t_ideal": 1, "events": 2, "l1_clusters": 3, "l1_defects": 4, "top_events": 5,
       "bands": 6, "defects": 7}


@pytest.fixture(scope="module")
def qd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_12262_gb300 import build
    build.build()
    import paper_2609_12262_gb300 as q
    q.lib()
    return q


def run(q, graphs, syn, mode, gid=None, offs=None):
    import torch
    t_syn = torch.from_numpy(np.ascontiguousarray(syn).view(np.int32).reshape(-1)).cuda()
    t_gid = torch.from_numpy(np.asarray(gid, np.int32)).cuda() if gid is not None else None
    t_off = torch.from_numpy(np.asarray(offs, np.int64)).cuda() if offs is not None else None
    o, w, s, dg = q.decode_batch_ex(graphs, t_syn, t_gid, t_off, mode=mode)
    torch.cuda.synchronize()
    return w.cpu().numpy(), q.to_uint64(o), s.cpu().numpy(), dg.cpu().numpy()


def test_worked_examples_on_gpu(qd):
    from synth import pack_defects
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        n = 50
        u = list(range(49)) + [0, 49]
        v = list(range(1, 50)) + [-1, -1]
        w = [5] * 49 + [c["w0"], 5]
        g = qd.Graph(n, u, v, w, [0] * 51)
        row = pack_defects(c["defects"], n)[None, :]
        for mode in ("hier", "global"):
            W, O, S, D = run(qd, [g], row, mode)
            exp = c[mode]
            got = {"weight": int(W[0]), "e_ideal": int(D[0, 0]), "t_ideal": int(D[0, 1]), "events": int(D[0, 2])}
            assert S[0] == 0 and got == exp, (c["name"], mode, got, exp)


CASES = [
    ("d5_p005", dict(d=5, p=0.005), 2000, 21),
    ("d9_p005", dict(d=9, p=0.005), 800, 22),
    ("d11_nonuniform", dict(d=11, p_range=(0.002, 0.006), p_seed=1), 500, 23),
    ("d13_p003", dict(d=13, p=0.003), 300, 24),
    ("d7_p02", dict(d=7, p=0.02), 300, 25),
    ("d17_p005", dict(d=17, p=0.005), 60, 26),
]


@pytest.mark.parametrize("label,kw,shots,seed", CASES, ids=[c[0] for c in CASES])
def test_diag_and_global_mode_match_oracle(qd, label, kw, shots, seed):
    d = kw.pop("d")
    pg = rotated_surface_code(d, d, **kw)
    kw["d"] = d
    og = OracleGraph.from_phys(pg)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, shots, seed)
    for mode in ("hier", "global"):
        W, O, S, D = run(qd, [g], syn, mode)
        for i in range(shots):
            r = og.diag(unpack_defects(syn[i], pg.num_detectors), mode)
            # the GPU runs everything above level 1 as one cluster; at these
            # sizes b_2 exceeds the graph's diameter, so the oracle agrees
            assert r["clusters_above_l1"] <= 1, (label, i)
            got = (int(W[i]), int(O[i]), int(S[i])) + tuple(int(D[i, COL[f]]) for f in FIELDS)
            exp = (r["weight"], r["obs"], r["status"]) + tuple(int(r[f]) for f in FIELDS)
            assert got == exp, (label, mode, i, got, exp)
        if mode == "hier":
            # top-level events + level-1 events add up to all events
            assert np.all(D[:, COL["top_events"]] <= D[:, COL["events"]])


def test_diag_in_a_mixed_batch(qd):
    graphs, gid, offs, syn = mixed_batch([5, 9, 13], 300, 0.004, 31)
    qg = [qd.Graph.from_phys(g) for g in graphs]
    W, O, S, D = run(qd, qg, syn, "hier", gid, offs)
    ogs = [OracleGraph.from_phys(g) for g in graphs]
    for i in range(gid.shape[0]):
        gi = int(gid[i])
        row = syn[offs[i]:offs[i] + graphs[gi].words]
        r = ogs[gi].diag(unpack_defects(row, graphs[gi].num_detectors), "hier")
        got = (int(W[i]), int(O[i]), int(S[i]), int(D[i, 0]), int(D[i, 1]), int(D[i, 2]))
        assert got == (r["weight"], r["obs"], r["status"], r["e_ideal"], r["t_ideal"], r["events"]), i


def test_plain_batch_unchanged_by_diag(qd):
    """qec_decode_batch and qec_decode_batch_ex (hierarchical) give the same results."""
    import torch
    pg = rotated_surface_code(11, 11, 0.003)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, 2000, 41)
    t_syn = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    o1, w1, s1 = qd.decode_batch([g], t_syn)
    o2, w2, s2, _ = qd.decode_batch_ex([g], t_syn, mode="hier")
    o3, w3, s3, dg = qd.decode_batch_ex([g], t_syn, mode="global", diag=False)
    torch.cuda.synchronize()
    assert dg is None
    for a, b in ((o1, o2), (w1, w2), (s1, s2), (o1, o3), (w1, w3), (s1, s3)):
        assert torch.equal(a, b)


@pytest.mark.parametrize("d,p,shots,check", [(49, 0.001, 256, 3), (33, 0.001, 256, 4), (49, 0.0001, 256, 8)])
def test_event_study_sizes_sampled(qd, d, p, shots, check):
    """The event study's sizes, run as one batch; the first shots are checked
    against the oracle field by field, all shots for hier = global (Theorem 1)."""
    pg = rotated_surface_code(d, d, p)
    og = OracleGraph.from_phys(pg)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, shots, d * 10 + 3)
    out = {m: run(qd, [g], syn, m) for m in ("hier", "global")}
    (hw, ho, hs, hd), (gw, go, gs, gd) = out["hier"], out["global"]
    assert np.array_equal(hw, gw) and np.array_equal(ho, go) and not hs.any() and not gs.any()
    for i in range(check):
        dets = unpack_defects(syn[i], pg.num_detectors)
        for mode, (W, O, S, D) in out.items():
            r = og.diag(dets, mode)
            assert r["clusters_above_l1"] <= 1
            got = (int(W[i]), int(O[i]), int(S[i])) + tuple(int(D[i, COL[f]]) for f in FIELDS)
            exp = (r["weight"], r["obs"], r["status"]) + tuple(int(r[f]) for f in FIELDS)
            assert got == exp, (d, p, mode, i, got, exp)


SCHED = [("d1=2 edges", dict(d1=2)), ("d1=3 edges", dict(d1=3)), ("d1=2 edges, wide b1", dict(d1=2, b1_factor=3)),
         ("q=1/2, phi_min=1/10", dict(q=(1, 2), phi_min=(1, 10)))]


@pytest.mark.parametrize("sname,spec", SCHED, ids=[s[0] for s in SCHED])
def test_custom_schedule_matches_oracle(qd, sname, spec):
    """Alternative cluster schedules: the GPU under a custom schedule equals the
    oracle under the same schedule (results and parallel event counts) and the
    global run (Theorem 1)."""
    from tests.test_theorem1 import schedule_kw
    for pg, shots, seed in ((rotated_surface_code(9, 9, 0.005), 600, 51),
                            (rotated_surface_code(11, 11, p_range=(0.002, 0.006), p_seed=1), 300, 52),
                            (rotated_surface_code(7, 7, 0.02), 300, 53)):
        kw = schedule_kw(pg, spec)
        og = OracleGraph.from_phys(pg, **kw)
        g = qd.Graph.from_phys(pg, q=kw.get("q"), phi_min=kw.get("phi_min"), d1=kw.get("d1", 0),
                               b1=kw.get("b1", 0))
        assert int(g.info.d_k[0]) == int(og.dk[0]) and int(g.info.b_k[0]) == int(og.bk[0])
        syn, _ = sample_shots(pg, shots, seed)
        W, O, S, D = run(qd, [g], syn, "hier")
        gw, go, gs, _ = run(qd, [g], syn, "global")
        assert np.array_equal(W, gw) and np.array_equal(O, go)
        multi = 0
        for i in range(shots):
            r = og.diag(unpack_defects(syn[i], pg.num_detectors), "hier")
            # results on every shot
            assert (int(W[i]), int(O[i]), int(S[i])) == (r["weight"], r["obs"], r["status"]), (sname, i)
            if r["clusters_above_l1"] > 1:
                multi += 1
                continue
            got = tuple(int(D[i, COL[f]]) for f in FIELDS)
            exp = tuple(int(r[f]) for f in FIELDS)
            assert got == exp, (sname, i, got, exp)
        # these graphs are connected and b_2 exceeds their diameter, so every
        # event above level 1 forms one processing cluster and the parallel
        # event count is compared on every shot
        assert multi == 0, (sname, multi)
        assert g.info.upper_single_cluster == 1


def test_distance_bound_and_single_upper_cluster(qd):
    """qec_graph_info.distance_bound is an upper bound of the largest distance
    between connected detectors, at most twice it (scipy Dijkstra from every
    detector); upper_single_cluster holds for the rotated codes and not for a
    graph of two components."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra
    from synth import rotated_surface_code_circuit
    for pg in (rotated_surface_code(5, 5, 0.005), rotated_surface_code(9, 9, 0.003),
               rotated_surface_code(7, 7, p_range=(0.001, 0.02), p_seed=4), rotated_surface_code_circuit(5, 5, 0.003)):
        g = qd.Graph.from_phys(pg)
        u, v, w, _ = g.merged_edges()
        m = v >= 0
        n = pg.num_detectors
        A = coo_matrix((w[m].astype(float), (u[m], v[m])), shape=(n, n)).tocsr()
        D = dijkstra(A, directed=False)
        diam = D[np.isfinite(D)].max()
        assert diam <= g.info.distance_bound <= 2 * diam
        assert g.info.components == 1 and g.info.upper_single_cluster == 1
    # two disjoint paths: two components
    g = qd.Graph(8, [0, 1, 2, 4, 5, 6, 0, 4], [1, 2, 3, 5, 6, 7, -1, -1], [3] * 8, [0] * 8)
    assert g.info.components == 2 and g.info.upper_single_cluster == 0
