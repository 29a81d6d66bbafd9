"""GPU path vs the CPU oracle, bit-exact on every shot (weight, observable mask,
status), through the C ABI.  Needs a GB300."""

import numpy as np
import pytest

from synth import rotated_surface_code, sample_shots, mixed_batch, pack_defects, unpack_defects
from tests.oracle_pool import oracle_decode

pytestmark = pytest.mark.gpu


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


def gpu_decode(q, graphs, syn_rows, gid=None, plain=False):
    """syn_rows: [S, words] (single graph) or (flat syn, offsets)."""
    import torch
    if isinstance(graphs, list) and gid is not None:
        flat, offs = syn_rows
        t_syn = torch.from_numpy(flat.view(np.int32)).cuda()
        t_gid = torch.from_numpy(np.asarray(gid, np.int32)).cuda()
        t_off = torch.from_numpy(np.asarray(offs, np.int64)).cuda()
        o, w, s = q.decode_batch(graphs, t_syn, t_gid, t_off)
    else:
        g = graphs[0] if isinstance(graphs, list) else graphs
        t_syn = torch.from_numpy(np.ascontiguousarray(syn_rows).view(np.int32).reshape(-1)).cuda()
        if plain:
            o, w, s = q.decode_plain(g, t_syn)
        else:
            o, w, s = q.decode_batch([g], t_syn)
    torch.cuda.synchronize()
    return w.cpu().numpy(), q.to_uint64(o), s.cpu().numpy()


def assert_same(gpu, ref, label):
    gw, go, gs = gpu
    rw, ro, rs = ref
    bad = np.nonzero((gw != rw) | (go != ro) | (gs != rs))[0]
    assert bad.size == 0, "%s: %d mismatches, first %s: gpu (w=%d obs=%d st=%d) oracle (w=%d obs=%d st=%d)" % (
        label, bad.size, bad[:5].tolist(), gw[bad[0]], go[bad[0]], gs[bad[0]], rw[bad[0]], ro[bad[0]], rs[bad[0]])


CASES = [
    ("d5_p005", dict(d=5, p=0.005), 10000, 0),
    ("d11_nonuniform", dict(d=11, p_range=(0.002, 0.006), p_seed=1), 4000, 1),
    ("d9_p003", dict(d=9, p=0.003), 3000, 2),
    ("d21_p003", dict(d=21, p=0.003), 300, 3),
    ("d7_p04_blossoms", dict(d=7, p=0.04), 2000, 4),
    ("d11_p02", dict(d=11, p=0.02), 600, 5),
    ("d3_p10_dense", dict(d=3, p=0.10), 2000, 6),
    # weights spread enough that level-1 neighbourhoods need the bounded search
    ("d9_wide_nonuniform", dict(d=9, p_range=(0.001, 0.02), p_seed=3), 2000, 9),
    ("d7_wider_nonuniform", dict(d=7, p_range=(0.0005, 0.05), p_seed=3), 2000, 10),
]


@pytest.mark.parametrize("name,kw,shots,seed", CASES, ids=[c[0] for c in CASES])
def test_batch_matches_oracle(qd, name, kw, shots, seed):
    kw = dict(kw)
    d = kw.pop("d")
    pg = rotated_surface_code(d, d, **kw)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, shots, seed)
    gpu = gpu_decode(qd, g, syn)
    ref = oracle_decode([pg], np.zeros(shots, np.int32), list(syn))
    assert np.all(ref[2] == 0)
    assert_same(gpu, ref, name)
    # deterministic: a second run is identical
    gpu2 = gpu_decode(qd, g, syn)
    assert_same(gpu2, gpu, name + " rerun")


def test_plain_matches_batch(qd):
    pg = rotated_surface_code(5, 5, 0.005)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, 2000, 9)
    a = gpu_decode(qd, g, syn, plain=True)
    b = gpu_decode(qd, g, syn)
    assert_same(a, b, "plain vs batch")
    ref = oracle_decode([pg], np.zeros(2000, np.int32), list(syn))
    assert_same(a, ref, "plain vs oracle")


def test_mixed_distance_batch(qd):
    ds = [7, 9, 11, 13, 15, 17, 19, 21]
    graphs, gid, offs, syn = mixed_batch(ds, 120, 0.003, seed=11)
    gg = [qd.Graph.from_phys(pg) for pg in graphs]
    gpu = gpu_decode(qd, gg, (syn, offs), gid=gid)
    rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in range(gid.shape[0])]
    ref = oracle_decode(graphs, gid, rows)
    assert_same(gpu, ref, "mixed")


def test_edge_cases(qd):
    pg = rotated_surface_code(5, 5, 0.005)
    g = qd.Graph.from_phys(pg)
    n = pg.num_detectors
    rows = [pack_defects([], n), pack_defects([0], n), pack_defects([n - 1], n),
            pack_defects(list(range(n)), n), pack_defects(list(range(0, n, 2)), n),
            pack_defects([0, 1], n), pack_defects([3, 40], n)]
    # padding bits beyond n are ignored
    r = pack_defects([5], n)
    r[-1] |= np.uint32(1 << 31)
    rows.append(r)
    syn = np.stack(rows)
    gpu = gpu_decode(qd, g, syn)
    masked = np.stack(rows[:-1] + [pack_defects([5], n)])
    ref = oracle_decode([pg], np.zeros(len(rows), np.int32), list(masked))
    assert_same(gpu, ref, "edge cases")
    assert gpu[0][0] == 0 and gpu[1][0] == 0 and gpu[2][0] == 0


def test_internal_observables_and_no_boundary(qd):
    """Random small graphs with observables on detector-detector edges (canonical
    path tracing) and components without a boundary (NO_SOLUTION)."""
    rng = np.random.default_rng(5)
    for trial in range(6):
        n = int(rng.integers(6, 14))
        u, v = [], []
        for x in range(n - 1):
            u.append(x); v.append(x + 1)
        for _ in range(n):
            a, b = int(rng.integers(0, n)), int(rng.integers(-1, n))
            if a != b:
                u.append(a); v.append(b)
        if trial % 2 == 0:
            u.append(0); v.append(-1)
        w = rng.integers(1, 12, size=len(u)).astype(np.int32)
        o = (rng.random(len(u)) < 0.4).astype(np.uint64)

        class PG:
            pass
        pg = PG()
        pg.num_detectors, pg.u, pg.v, pg.w, pg.obs = n, np.array(u, np.int32), np.array(v, np.int32), w, o
        g = qd.Graph(n, pg.u, pg.v, w, o)
        syn = np.stack([pack_defects([x for x in range(n) if (s >> x) & 1], n) for s in range(min(1 << n, 600))])
        gpu = gpu_decode(qd, g, syn)
        ref = oracle_decode([pg], np.zeros(syn.shape[0], np.int32), list(syn), workers=1)
        assert_same(gpu, ref, "random graph %d" % trial)


@pytest.mark.parametrize("band", [1, 3])
def test_band_width_does_not_change_results(qd, band):
    pg = rotated_surface_code(11, 11, 0.01)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, 500, 21)
    qd.set_tuning(band_factor=band)
    try:
        a = gpu_decode(qd, g, syn)
    finally:
        qd.set_tuning(band_factor=1)
    ref = oracle_decode([pg], np.zeros(500, np.int32), list(syn))
    assert_same(a, ref, "band %d" % band)


def test_autotuner_candidates_agree_and_match_oracle(qd):
    """Every launch shape / slab size the autotuner tries returns identical
    results (it raises otherwise); the chosen one matches the oracle."""
    import torch
    from paper_2609_12262_gb300 import autotune
    graphs, gid, offs, syn = mixed_batch([7, 11, 15, 21], 200, 0.003, seed=31)
    gg = [qd.Graph.from_phys(pg) for pg in graphs]
    t_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    t_gid = torch.from_numpy(gid.astype(np.int32)).cuda()
    t_off = torch.from_numpy(offs.astype(np.int64)).cuda()
    best, results = autotune.tune(gg, t_syn, t_gid, t_off, reps=1, budget_s=30.0, save=False)
    assert len(results) >= 4
    autotune.apply(best)
    try:
        gpu = gpu_decode(qd, gg, (syn, offs), gid=gid)
    finally:
        qd.set_tuning(warps_per_block=-1, blocks_per_sm=-1, band_factor=-1, kcap=-1)
    rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in range(gid.shape[0])]
    assert_same(gpu, oracle_decode(graphs, gid, rows), "autotuned")


def test_dense_graphs_overflow_the_lane_local_search(qd):
    """High-degree random graphs with narrow weights: many events have more
    vertices within b_1 than one lane holds, which sends them through the
    warp-wide flooder; observables on internal edges exercise path tracing."""
    rng = np.random.default_rng(3)
    for trial in range(3):
        n = 120
        u, v = [], []
        for x in range(n - 1):
            u.append(x); v.append(x + 1)
        for _ in range(n * 8):
            a, b = int(rng.integers(0, n)), int(rng.integers(-1, n))
            if a != b:
                u.append(a); v.append(b)
        w = rng.integers(3, 9, size=len(u)).astype(np.int32)
        o = (rng.random(len(u)) < 0.3).astype(np.uint64)

        class PG:
            pass
        pg = PG()
        pg.num_detectors, pg.u, pg.v, pg.w, pg.obs = n, np.array(u, np.int32), np.array(v, np.int32), w, o
        g = qd.Graph(n, pg.u, pg.v, w, o)
        rows = [pack_defects(sorted(set(rng.integers(0, n, size=int(rng.integers(0, 30))).tolist())), n)
                for _ in range(300)]
        syn = np.stack(rows)
        gpu = gpu_decode(qd, g, syn)
        ref = oracle_decode([pg], np.zeros(syn.shape[0], np.int32), list(syn), workers=1)
        assert_same(gpu, ref, "dense graph %d" % trial)


@pytest.mark.parametrize("d,p,shots", [(25, 0.005, 6), (31, 0.003, 4), (41, 0.001, 3), (51, 0.001, 2)])
def test_large_windows_match_oracle(qd, d, p, shots):
    """Full-size single windows of the scaling study (hundreds of detection
    events per window) against the oracle, in the main batched path."""
    pg = rotated_surface_code(d, d, p)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, shots, 1000 + d)
    gpu = gpu_decode(qd, g, syn)
    ref = oracle_decode([pg], np.zeros(shots, np.int32), list(syn), chunk=1)
    assert_same(gpu, ref, "d%d p%g" % (d, p))


@pytest.mark.parametrize("d,p,shots", [(41, 0.003, 4), (41, 0.005, 4), (51, 0.003, 3), (51, 0.005, 3)])
def test_large_windows_at_higher_rates(qd, d, p, shots):
    """The scaling study's largest windows at p = 0.003 and 0.005, where the
    top-level cluster is largest (500 - 2,000 detection events per window)."""
    pg = rotated_surface_code(d, d, p)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, shots, 2000 + d + int(p * 1e4))
    gpu = gpu_decode(qd, g, syn)
    ref = oracle_decode([pg], np.zeros(shots, np.int32), list(syn), chunk=1)
    assert np.all(ref[2] == 0)
    assert_same(gpu, ref, "d%d p%g" % (d, p))


def test_overflow_pass_decodes_shots_beyond_the_main_slab(qd):
    """With a small main-pass slab (kcap events), shots with more detection
    events than kcap fail in the main pass and are decoded by the overflow pass
    (room for 4 kcap events); shots beyond that end with QEC_SHOT_CAPACITY."""
    pg = rotated_surface_code(15, 15, 0.008)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, 400, 61)
    K = np.unpackbits(syn.view(np.uint8), axis=1).sum(axis=1)
    ref = oracle_decode([pg], np.zeros(400, np.int32), list(syn))
    try:
        qd.set_tuning(kcap=40)
        gpu = gpu_decode(qd, g, syn)
        # overflow slabs hold 4 x 40 = 160 events: every shot here fits there
        assert K.max() <= 160 and np.count_nonzero(K > 40) >= 50
        assert_same(gpu, ref, "overflow pass")
        qd.set_tuning(kcap=16)
        small = gpu_decode(qd, g, syn)
    finally:
        qd.set_tuning(kcap=-1)
    over = K > 64
    assert np.count_nonzero(over) >= 50
    assert np.all(small[2][over] == qd.SHOT_CAPACITY)
    ok = ~over
    assert_same(tuple(x[ok] for x in small), tuple(x[ok] for x in ref), "overflow pass, small slabs")
