"""Pins of the oracle against things other than itself.

* Exhaustive minimum-weight embedded matching (MWEM, paper "Decoding task")
  over every edge subset of small multigraphs, for every syndrome at once.
* Subset DP over pairings of the detection events, with scipy Dijkstra
  distances on a two-sheet graph that tracks the observable parity.
* networkx Edmonds on the complete graph of detection events plus boundary twins.
* The correction the oracle traces reproduces the syndrome and its weight.
"""

import itertools

import networkx as nx
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import dijkstra

from oracle import OracleGraph
from synth import rotated_surface_code, sample_shots, unpack_defects

INF = np.iinfo(np.int64).max // 4


def brute_force_mwem(n, u, v, w, obs):
    """Return best[syn] (min weight, INF if none) and classes[syn] (obs values at the min)."""
    m = len(u)
    syn = np.zeros(1, np.int64)
    wt = np.zeros(1, np.int64)
    ob = np.zeros(1, np.int64)
    for i in range(m):
        mask = (1 << int(u[i])) | ((1 << int(v[i])) if v[i] >= 0 else 0)
        syn = np.concatenate([syn, syn ^ mask])
        wt = np.concatenate([wt, wt + int(w[i])])
        ob = np.concatenate([ob, ob ^ int(obs[i])])
    best = np.full(1 << n, INF, np.int64)
    np.minimum.at(best, syn, wt)
    hit = wt == best[syn]
    classes = {}
    for s, o in zip(syn[hit].tolist(), ob[hit].tolist()):
        classes.setdefault(s, set()).add(o)
    return best, classes


def random_graph(rng, n, m, wmax=9, with_obs=True):
    u, v, w, o = [], [], [], []
    # a spanning path so every detector reaches the boundary through something
    for x in range(n - 1):
        u.append(x); v.append(x + 1)
    while len(u) < m:
        a = int(rng.integers(0, n))
        b = int(rng.integers(-1, n))
        if b == a:
            continue
        u.append(a); v.append(b)
    u.append(int(rng.integers(0, n))); v.append(-1)
    w = rng.integers(1, wmax + 1, size=len(u)).astype(np.int32)
    o = (rng.random(len(u)) < 0.3).astype(np.uint64) if with_obs else np.zeros(len(u), np.uint64)
    return np.array(u, np.int32), np.array(v, np.int32), w, o


def check_against_brute_force(n, u, v, w, o, modes=("global", "hier")):
    best, classes = brute_force_mwem(n, u, v, w, o)
    og = OracleGraph(n, u, v, w, o)
    mu, mv, mw, mo = og.merged_edges()
    checked_obs = 0
    for s in range(1 << n):
        det = [x for x in range(n) if (s >> x) & 1]
        for mode in modes:
            r, corr = og.decode(det, mode, correction=True)
            if best[s] >= INF:
                assert r.status != 0
                continue
            assert r.status == 0, (s, mode, r.as_dict())
            assert r.weight == best[s], (s, mode, r.weight, best[s])
            assert r.dual_feasible and r.tight and r.dual_sum == r.primal_internal
            # correction reproduces the syndrome, weighs W, carries obs
            par = np.zeros(n, np.int64)
            sel = np.nonzero(corr)[0]
            for e in sel:
                par[mu[e]] ^= 1
                if mv[e] >= 0:
                    par[mv[e]] ^= 1
            assert np.nonzero(par)[0].tolist() == det
            assert int(mw[sel].sum()) == 2 * r.weight
            oo = 0
            for e in sel:
                oo ^= int(mo[e])
            assert oo == r.obs
            if len(classes[s]) == 1:
                assert r.obs == next(iter(classes[s])), (s, mode)
                checked_obs += 1
    return checked_obs


def test_brute_force_surface_d3():
    g = rotated_surface_code(3, 1, p_range=(0.002, 0.02), p_seed=5)
    assert g.num_edges == 22
    n = check_against_brute_force(g.num_detectors, g.u, g.v, g.w, g.obs)
    assert n > 50


def test_brute_force_surface_d3_uniform_ties():
    g = rotated_surface_code(3, 1, 0.01)
    check_against_brute_force(g.num_detectors, g.u, g.v, g.w, g.obs)


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_random_graphs(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(5, 9))
    u, v, w, o = random_graph(rng, n, int(rng.integers(n + 4, 16)))
    check_against_brute_force(n, u, v, w, o)


def test_no_boundary_odd_component():
    # a triangle with no boundary edge: odd event sets have no embedded matching
    u = np.array([0, 1, 2], np.int32); v = np.array([1, 2, 0], np.int32)
    w = np.array([3, 4, 5], np.int32); o = np.zeros(3, np.uint64)
    og = OracleGraph(3, u, v, w, o)
    assert og.decode([0], "global").status == 1
    r = og.decode([0, 2], "global")
    assert r.status == 0 and r.weight == 5
    r = og.decode([], "global")
    assert r.status == 0 and r.weight == 0 and r.obs == 0


# ---------------------------------------------------------------------------
# subset DP with parity-tracking distances (scipy Dijkstra)
# ---------------------------------------------------------------------------

def two_sheet_distances(g, defects):
    """dist[a][b][pi], bd[a][pi] over the physical multigraph (min over parallel copies)."""
    n = g.num_detectors
    best = {}
    bbest = {}
    for a, b, w, o in zip(g.u.tolist(), g.v.tolist(), g.w.tolist(), g.obs.tolist()):
        if b < 0:
            key = (a, o & 1)
            bbest[key] = min(bbest.get(key, 1 << 60), w)
        else:
            key = (min(a, b), max(a, b), o & 1)
            best[key] = min(best.get(key, 1 << 60), w)
    rows, cols, vals = [], [], []
    for (a, b, par), w in best.items():
        for pi in (0, 1):
            rows += [a + n * pi, b + n * pi]
            cols += [b + n * (pi ^ par), a + n * (pi ^ par)]
            vals += [w, w]
    M = coo_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n)).tocsr()
    dist = dijkstra(M, indices=list(defects))
    k = len(defects)
    D = np.full((k, k, 2), np.inf)
    BD = np.full((k, 2), np.inf)
    for i in range(k):
        for j in range(k):
            for pi in (0, 1):
                D[i, j, pi] = dist[i, defects[j] + n * pi]
        for (x, par), w in bbest.items():
            for pi in (0, 1):
                BD[i, pi ^ par] = min(BD[i, pi ^ par], dist[i, x + n * pi] + w)
    return D, BD


def dp_min_weight(D, BD):
    k = D.shape[0]
    full = (1 << k) - 1
    memo = {0: (0.0, np.inf)}

    def f(S):
        if S in memo:
            return memo[S]
        i = (S & -S).bit_length() - 1
        rest = S & ~(1 << i)
        out = [np.inf, np.inf]
        sub = f(rest)
        for pi in (0, 1):
            for q in (0, 1):
                out[pi ^ q] = min(out[pi ^ q], sub[pi] + BD[i, q])
        j_bits = rest
        while j_bits:
            j = (j_bits & -j_bits).bit_length() - 1
            j_bits &= j_bits - 1
            sub = f(rest & ~(1 << j))
            for pi in (0, 1):
                for q in (0, 1):
                    out[pi ^ q] = min(out[pi ^ q], sub[pi] + D[i, j, q])
        memo[S] = tuple(out)
        return memo[S]

    return f(full)


@pytest.mark.parametrize("d,p,seed", [(5, 0.02, 1), (7, 0.01, 2), (9, 0.006, 3)])
def test_subset_dp(d, p, seed):
    g = rotated_surface_code(d, d, p)
    og = OracleGraph.from_phys(g)
    syn, _ = sample_shots(g, 400, seed)
    done = unique = 0
    for s in range(400):
        det = unpack_defects(syn[s], g.num_detectors)
        if not (1 <= len(det) <= 11):
            continue
        D, BD = two_sheet_distances(g, det)
        w0, w1 = dp_min_weight(D, BD)
        wstar = min(w0, w1)
        for mode in ("global", "hier"):
            r = og.decode(det, mode)
            assert r.status == 0
            assert r.weight == wstar
            if w0 != w1:
                assert r.obs == (0 if w0 < w1 else 1)
        unique += int(w0 != w1)
        done += 1
        if done >= 40:
            break
    assert done >= 20 and unique >= 10


@pytest.mark.parametrize("d,p,seed", [(11, 0.01, 4), (15, 0.004, 5)])
def test_networkx_edmonds(d, p, seed):
    g = rotated_surface_code(d, d, p)
    og = OracleGraph.from_phys(g)
    syn, _ = sample_shots(g, 8, seed)
    for s in range(4):
        det = unpack_defects(syn[s], g.num_detectors)
        D, BD = two_sheet_distances(g, det)
        Dm = D.min(axis=2)
        Bm = BD.min(axis=1)
        k = len(det)
        G = nx.Graph()
        for i, j in itertools.combinations(range(k), 2):
            G.add_edge(i, j, weight=float(Dm[i, j]))
            G.add_edge(k + i, k + j, weight=0.0)
        for i in range(k):
            G.add_edge(i, k + i, weight=float(Bm[i]))
        M = nx.min_weight_matching(G)
        wstar = sum(G[a][b]["weight"] for a, b in M)
        r = og.decode(det, "hier")
        assert r.status == 0 and r.weight == wstar
