"""Multi-warp teams (a whole thread block decoding one shot, the latency path
for large windows) against the CPU oracle, bit-exact on every shot (weight,
observable mask, status), and against the one-warp-per-shot path for the
parallel-event-count diagnostics.  Needs a GB300."""

import numpy as np
import pytest

from synth import mixed_batch, pack_defects, rotated_surface_code, sample_shots
from tests.oracle_pool import oracle_decode
from tests.test_gpu_parity import assert_same, gpu_decode

pytestmark = pytest.mark.gpu

TEAMS = [4, 16]


@pytest.fixture(scope="module")
def qd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_12262_gb300 import build
    build.build()
    import paper_2609_12262_gb300 as q
    q.lib()
    yield q
    q.set_tuning(team_warps=-1, kcap=-1, team_split_events=-1)


def with_team(q, team, fn, *a, split=1, **kw):
    """Run fn with team_warps = team; split = 1 sends every shot to the whole
    team (the default threshold would give small shots to one warp)."""
    q.set_tuning(team_warps=team, team_split_events=split)
    try:
        return fn(*a, **kw)
    finally:
        q.set_tuning(team_warps=-1, team_split_events=-1)


CASES = [
    ("d5_p005", dict(d=5, p=0.005), 1500, 0),
    ("d7_p04_blossoms", dict(d=7, p=0.04), 400, 4),
    ("d11_p02", dict(d=11, p=0.02), 200, 5),
    ("d9_wide_nonuniform", dict(d=9, p_range=(0.001, 0.02), p_seed=3), 400, 9),
    ("d21_p003", dict(d=21, p=0.003), 150, 3),
]


@pytest.mark.parametrize("team", TEAMS)
@pytest.mark.parametrize("name,kw,shots,seed", CASES, ids=[c[0] for c in CASES])
def test_team_matches_oracle(qd, team, name, kw, shots, seed):
    kw = dict(kw)
    d = kw.pop("d")
    pg = rotated_surface_code(d, d, **kw)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, shots, seed)
    gpu = with_team(qd, team, gpu_decode, qd, g, syn)
    ref = oracle_decode([pg], np.zeros(shots, np.int32), list(syn))
    assert_same(gpu, ref, "%s team %d" % (name, team))


@pytest.mark.parametrize("team", TEAMS)
def test_team_random_graphs_internal_observables(qd, team):
    """Observables on detector-detector edges (team-parallel canonical path
    walks), components without a boundary (NO_SOLUTION), dense graphs whose
    level-1 neighbourhoods go through the team-wide flooder."""
    rng = np.random.default_rng(11 + team)
    for trial in range(4):
        n = int(rng.integers(8, 14)) if trial < 2 else 90
        extra = n if trial < 2 else 6 * n
        u, v = [], []
        for x in range(n - 1):
            u.append(x); v.append(x + 1)
        for _ in range(extra):
            a, b = int(rng.integers(0, n)), int(rng.integers(-1, n))
            if a != b:
                u.append(a); v.append(b)
        if trial % 2 == 0:
            u.append(0); v.append(-1)
        w = rng.integers(1 if trial < 2 else 3, 12 if trial < 2 else 9, size=len(u)).astype(np.int32)
        o = (rng.random(len(u)) < 0.35).astype(np.uint64)

        class PG:
            pass
        pg = PG()
        pg.num_detectors, pg.u, pg.v, pg.w, pg.obs = n, np.array(u, np.int32), np.array(v, np.int32), w, o
        g = qd.Graph(n, pg.u, pg.v, w, o)
        if trial < 2:
            rows = [pack_defects([x for x in range(n) if (s >> x) & 1], n) for s in range(min(1 << n, 300))]
        else:
            rows = [pack_defects(sorted(set(rng.integers(0, n, size=int(rng.integers(0, 26))).tolist())), n)
                    for _ in range(150)]
        syn = np.stack(rows)
        gpu = with_team(qd, team, gpu_decode, qd, g, syn)
        ref = oracle_decode([pg], np.zeros(syn.shape[0], np.int32), list(syn), workers=1)
        assert_same(gpu, ref, "random graph %d team %d" % (trial, team))


@pytest.mark.parametrize("team", TEAMS)
def test_team_global_mode_and_diagnostics_equal_the_warp_path(qd, team):
    import torch
    pg = rotated_surface_code(13, 13, 0.005)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, 200, 71)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    for mode in ("hier", "global"):
        ref = [x.cpu() for x in qd.decode_batch_ex([g], t, mode=mode)]
        got = [x.cpu() for x in with_team(qd, team, qd.decode_batch_ex, [g], t, mode=mode)]
        for a, b in zip(ref, got):
            assert torch.equal(a, b), (mode, team)


def test_team_mixed_batch_and_overflow_pass(qd):
    graphs, gid, offs, syn = mixed_batch([7, 11, 15], 60, 0.006, seed=13)
    gg = [qd.Graph.from_phys(pg) for pg in graphs]
    rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in range(gid.shape[0])]
    ref = oracle_decode(graphs, gid, rows)
    gpu = with_team(qd, 4, gpu_decode, qd, gg, (syn, offs), gid=gid)
    assert_same(gpu, ref, "mixed, team 4")
    # small main-pass slabs: the larger shots are decoded by the overflow pass
    qd.set_tuning(kcap=24)
    try:
        gpu = with_team(qd, 16, gpu_decode, qd, gg, (syn, offs), gid=gid)
    finally:
        qd.set_tuning(kcap=-1)
    K = np.array([np.unpackbits(np.asarray(r, np.uint32).view(np.uint8)).sum() for r in rows])
    assert np.count_nonzero(K > 24) >= 20 and K.max() <= 96
    assert_same(gpu, ref, "mixed, team 16, overflow pass")


@pytest.mark.parametrize("d,p,shots", [(25, 0.005, 4), (41, 0.003, 2), (51, 0.003, 2), (51, 0.005, 1)])
def test_team_large_windows(qd, d, p, shots):
    """Large single windows decoded one at a time: a batch with fewer shots
    than SMs picks a 16-warp team automatically."""
    import torch
    pg = rotated_surface_code(d, d, p)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, shots, 3000 + d + int(p * 1e4))
    ref = oracle_decode([pg], np.zeros(shots, np.int32), list(syn), chunk=1)
    assert np.all(ref[2] == 0)
    qd.set_tuning(team_warps=-1)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    outs = []
    for s in range(shots):
        o, w, st = qd.decode_batch([g], t[s * pg.words:(s + 1) * pg.words], num_shots=1)
        outs.append((w, o, st))
    torch.cuda.synchronize()
    gpu = (np.concatenate([x[0].cpu().numpy() for x in outs]), np.concatenate([qd.to_uint64(x[1]) for x in outs]),
           np.concatenate([x[2].cpu().numpy() for x in outs]))
    assert_same(gpu, ref, "d%d p%g single windows" % (d, p))


@pytest.mark.parametrize("team", [1, 16])
def test_team_sliding_windows(qd, team):
    """Sliding-window decoding (committed paths and carries) with one warp and
    with a 16-warp block per stream window, against the oracle's windows."""
    import torch
    from oracle.window import sliding_window_decode
    from paper_2609_12262_gb300.window import SlidingWindow
    from synth import rotated_surface_code_circuit
    for g, W, C, S in ((rotated_surface_code(7, 28, 0.006), 14, 7, 60),
                       (rotated_surface_code_circuit(5, 15, 0.004), 6, 3, 40)):
        syn, _ = sample_shots(g, S, 29)
        dec = SlidingWindow(qd.Graph.from_phys(g), g.nz, W, C)
        t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
        obs, st = with_team(qd, team, dec.decode, t, S)
        torch.cuda.synchronize()
        ro, rs = sliding_window_decode(g, syn, W, C)
        assert not rs.any()
        assert np.array_equal(qd.to_uint64(obs), ro) and np.array_equal(st.cpu().numpy(), rs), team


def test_team_split_threshold(qd):
    """A 16-warp block hands shots below the split threshold to its first warp:
    results equal the oracle whatever the threshold, and the shots on either
    side of it are both present in the batch."""
    graphs, gid, offs, syn = mixed_batch([9, 17, 25], 40, 0.004, seed=17)
    gg = [qd.Graph.from_phys(pg) for pg in graphs]
    rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in range(gid.shape[0])]
    K = np.array([np.unpackbits(np.asarray(r, np.uint32).view(np.uint8)).sum() for r in rows])
    assert np.count_nonzero(K < 40) >= 20 and np.count_nonzero(K >= 40) >= 20
    ref = oracle_decode(graphs, gid, rows)
    for split in (1, 40, 100000):
        gpu = with_team(qd, 16, gpu_decode, qd, gg, (syn, offs), gid=gid, split=split)
        assert_same(gpu, ref, "split %d" % split)


def test_automatic_team_on_a_batch_of_large_windows(qd):
    """More d = 41 windows than SMs: the automatic choice (4-warp blocks for
    graphs of at least 32,768 detectors) gives the same results as one warp and
    as 16 warps per window, and the oracle's on a sample."""
    import torch
    pg = rotated_surface_code(41, 41, 0.003)
    g = qd.Graph.from_phys(pg)
    n = 200
    syn, _ = sample_shots(pg, n, 4141)
    K = np.unpackbits(syn.view(np.uint8), axis=1).sum(axis=1)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    qd.set_tuning(kcap=int(K.max()) + 64)
    try:
        outs = {}
        for team in (-1, 1, 16):
            qd.set_tuning(team_warps=team)
            o, w, st = qd.decode_batch([g], t, num_shots=n)
            torch.cuda.synchronize()
            outs[team] = (w.cpu().numpy(), qd.to_uint64(o), st.cpu().numpy())
    finally:
        qd.set_tuning(team_warps=-1, kcap=-1)
    for team in (1, 16):
        for a, b in zip(outs[-1], outs[team]):
            assert np.array_equal(a, b), team
    assert not outs[-1][2].any()
    ref = oracle_decode([pg], np.zeros(2, np.int32), list(syn[:2]), chunk=1)
    assert_same(tuple(x[:2] for x in outs[-1]), ref, "d41 automatic team, first windows")


def test_team_autotuner_picks_a_size_without_changing_results(qd):
    """autotune.tune_team decodes the batch with every team size, requires the
    same results and applies the fastest."""
    import torch
    from paper_2609_12262_gb300 import autotune
    pg = rotated_surface_code(25, 25, 0.003)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, 300, 2525)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    try:
        best, totals = autotune.tune_team([g], t, num_shots=300, reps=1)
        assert best in (1, 4, 16) and sorted(tm for _, tm in totals) == [1, 4, 16]
        assert qd.get_tuning()["team_warps"] == best
        o, w, st = qd.decode_batch([g], t, num_shots=300)
        torch.cuda.synchronize()
    finally:
        qd.set_tuning(team_warps=-1)
    ref = oracle_decode([pg], np.zeros(40, np.int32), list(syn[:40]))
    assert_same((w.cpu().numpy()[:40], qd.to_uint64(o)[:40], st.cpu().numpy()[:40]), ref, "tuned team, d25")
