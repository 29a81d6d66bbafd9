"""Algorithm 3 (parameter schedule) and Algorithm 1 (processing clusters) pins."""

from fractions import Fraction

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import dijkstra

from oracle import OracleGraph, alg3
from oracle.schedule import admissible, big_phi, phibar
from synth import rotated_surface_code, sample_shots, unpack_defects

Q, PMIN = Fraction(1, 10), Fraction(1, 100)


@pytest.mark.parametrize("wmax", [164, 170, 186, 198, 222, 2, 17])
def test_alg3_closed_form_level1(wmax):
    """phi_1 = 1 makes the binding constraint b > 2 d_1, so b_1 = 2 d_1 + 1,
    phi_2 = 1 - 3 d_1 / (4 d_1 + 1) and d_2 = 3 d_1 + 4 b_1 + 2 w_max
    (Algorithm 3 evaluated by hand at k = 1)."""
    d, b, phi = alg3(wmax, levels=2)
    d1 = wmax + 1
    assert d[0] == d1
    assert b[0] == 2 * d1 + 1
    assert phi[1] == Fraction(d1 + 1, 4 * d1 + 1)
    assert d[1] == 11 * d1 + 4 + 2 * wmax


@pytest.mark.parametrize("wmax", [164, 170, 186, 198, 222])
def test_alg3_invariants(wmax):
    """SI 'Analysis of the finite-size parameter schedule': b_k >= d_k,
    phi_k > 2 d_k / b_k, phi_k >= phibar_k >= phi_min, minimality of b_k."""
    d, b, phi = alg3(wmax, levels=4)
    for k in range(4):
        assert b[k] >= d[k]
        assert phi[k] > Fraction(2 * d[k], b[k])
        assert phi[k] >= phibar(k + 1, Q, PMIN) >= PMIN
        nxt = big_phi(phi[k], d[k], b[k])
        assert nxt >= phibar(k + 2, Q, PMIN)
        assert not admissible(phi[k], d[k], b[k] - 1, phibar(k + 2, Q, PMIN))
        if k + 1 < 4:
            assert d[k + 1] == 3 * d[k] + 4 * b[k] + 2 * wmax
    # monotone
    assert all(d[i] < d[i + 1] for i in range(3)) and all(b[i] < b[i + 1] for i in range(3))


def phys_distances(g):
    n = g.num_detectors
    best, bnd = {}, np.full(n, np.inf)
    for a, b, w in zip(g.u.tolist(), g.v.tolist(), g.w.tolist()):
        if b < 0:
            bnd[a] = min(bnd[a], 2 * w)
        else:
            key = (min(a, b), max(a, b))
            best[key] = min(best.get(key, 1 << 60), 2 * w)
    r = [k[0] for k in best] + [k[1] for k in best]
    c = [k[1] for k in best] + [k[0] for k in best]
    v = list(best.values()) * 2
    M = coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    return M, bnd


@pytest.mark.parametrize("d,p,seed", [(7, 0.01, 1), (11, 0.003, 2), (11, None, 3), (15, 0.005, 4)])
def test_alg1_clusters_satisfy_definition(d, p, seed):
    """Every level-k processing cluster C in the residual set D_k is a
    (d_k, b_k)_V-cluster (diam <= d_k, separated from D_k minus C by more than b_k)
    and meets the parity condition (Methods, Def. 'Hierarchy of processing
    clusters'; SI Def. 'Isolation and clustering of a vertex set')."""
    g = (rotated_surface_code(d, d, p) if p else
         rotated_surface_code(d, d, p_range=(0.002, 0.006), p_seed=seed))
    og = OracleGraph.from_phys(g)
    M, bnd = phys_distances(g)
    syn, _ = sample_shots(g, 60, seed)
    for s in range(60):
        det = unpack_defects(syn[s], g.num_detectors)
        if len(det) == 0:
            continue
        st, lev, cl = og.cluster(det)
        assert st == 0
        dist = dijkstra(M, indices=det)
        DD = dist[:, det]
        BD = (dist + bnd[None, :]).min(axis=1)
        resid = np.ones(len(det), bool)
        for k in range(1, lev.max() + 1):
            dk, bk = og.dk[k - 1], og.bk[k - 1]
            for c in np.unique(cl[lev == k]):
                mem = cl == c
                assert DD[np.ix_(mem, mem)].max() <= dk
                others = resid & ~mem
                if others.any():
                    assert DD[np.ix_(mem, others)].min() > bk
                contact = (2 * BD[mem] <= bk).any()
                assert contact or mem.sum() % 2 == 0
            # no residual component that the definition accepts was left behind
            resid_next = resid & (lev != k)
            resid = resid_next
