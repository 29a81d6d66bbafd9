"""The circuit-level detector graph generator (synth/circuit.py) pinned against
things other than its own backward propagation:

* forward Pauli-frame simulation of single faults through the circuit (written
  here independently) gives the same detectors and observable;
* the fewest faults flipping the logical without any detector (the circuit
  distance) is d with the chosen CNOT orders, and smaller when the X-ancilla
  order puts its hook along the logical operator;
* measurement noise alone gives exactly the time edges (one per check and
  round) and the final data-measurement edges; preparation noise alone gives
  the phenomenological graph's first-layer space edges (data qubits) and the
  time edges (Z ancillas), each with the preparation flip probability;
* decoding circuit-level syndromes: hierarchical == global (Theorem 1)."""

from collections import deque

import numpy as np
import pytest

import synth.circuit as sc
from oracle import OracleGraph
from synth import rotated_surface_code, rotated_surface_code_circuit, sample_shots, unpack_defects


def forward_effect(d, R, ops, nq, zc, start, xs, zs):
    """Detectors and observable flipped by X on xs and Z on zs inserted before
    ops[start], by forward frame simulation of the rest of the circuit."""
    x = np.zeros(nq, np.uint8)
    z = np.zeros(nq, np.uint8)
    x[list(xs)] = 1
    z[list(zs)] = 1
    nz = len(zc)
    flipped_z = {}
    flipped_data = set()
    for op in ops[start:]:
        if op[0] == "CX":
            c, t = op[1], op[2]
            x[t] ^= x[c]
            z[c] ^= z[t]
        elif op[0] == "H":
            q = op[1]
            x[q], z[q] = z[q], x[q]
        elif op[0] == "P":
            x[op[1]] = 0
            z[op[1]] = 0
        elif op[0] == "M" and x[op[1]]:
            key = op[2]
            if key[0] == "z":
                flipped_z[(key[1], key[2])] = 1
            elif key[0] == "data":
                flipped_data.add(key[1])
    # detector layer t (t < R) = m_t xor m_{t-1}; layer R = data parity xor m_{R-1}
    dets = set()
    for k in range(nz):
        prev = 0
        for t in range(R):
            cur = flipped_z.get((t, k), 0)
            if cur ^ prev:
                dets.add(t * nz + k)
            prev = cur
        data = sum(1 for q in zc[k].values() if q in flipped_data) & 1
        if data ^ prev:
            dets.add(R * nz + k)
    obs = sum(1 for q in flipped_data if q % d == 0) & 1
    return frozenset(dets), obs


@pytest.mark.parametrize("d", [3, 5])
def test_backward_sensitivity_matches_forward_simulation(d):
    R = d
    ops, nq, zc, xc, zanc, xanc = sc._circuit(d, R)
    key_effect = sc._key_effect_fn(d, R, zc)
    rng = np.random.default_rng(d)
    picks = set(rng.choice(len(ops), size=min(len(ops), 150), replace=False).tolist())
    seen = {}

    def visit(i, op, FX, FZ):
        if i in picks:
            seen[i] = ([FX[q] for q in range(nq)], [FZ[q] for q in range(nq)])

    sc.backward_sensitivity(ops, nq, key_effect, visit)
    checked = 0
    for i in sorted(picks):
        FX, FZ = seen[i]
        for q in rng.choice(nq, size=3, replace=False):
            q = int(q)
            assert FX[q] == forward_effect(d, R, ops, nq, zc, i + 1, {q}, set()), (i, q, "X")
            assert FZ[q] == forward_effect(d, R, ops, nq, zc, i + 1, set(), {q}), (i, q, "Z")
            checked += 1
    assert checked > 100


def circuit_distance(g):
    """Fewest edges whose detector degrees are all even and whose observables XOR to 1."""
    n = g.num_detectors
    adj = [[] for _ in range(n)]
    bnd = [[] for _ in range(n)]
    for u, v, o in zip(g.u, g.v, g.obs):
        if v < 0:
            bnd[u].append(int(o))
        else:
            adj[u].append((int(v), int(o)))
            adj[v].append((int(u), int(o)))
    best = 10 ** 9
    for s in range(n):
        for o1 in set(bnd[s]):
            dist = {(s, o1): 1}
            dq = deque([(s, o1)])
            while dq:
                x, par = dq.popleft()
                dx = dist[(x, par)]
                if dx >= best:
                    continue
                for o2 in bnd[x]:
                    if par ^ o2:
                        best = min(best, dx + 1)
                for y, o in adj[x]:
                    st = (y, par ^ o)
                    if st not in dist:
                        dist[st] = dx + 1
                        dq.append(st)
    return best


@pytest.mark.parametrize("d", [3, 5, 7])
@pytest.mark.parametrize("noise", ["uniform", "physical"])
def test_circuit_distance_is_d(d, noise):
    assert circuit_distance(rotated_surface_code_circuit(d, d, 0.001, noise)) == d


def test_hook_along_the_logical_halves_the_distance(monkeypatch):
    monkeypatch.setattr(sc, "XORDER", ("NW", "NE", "SW", "SE"))
    assert circuit_distance(sc.rotated_surface_code_circuit(7, 7, 0.001)) < 7


def test_measurement_noise_alone_gives_time_edges():
    d, R, p = 5, 6, 0.002
    g = rotated_surface_code_circuit(d, R, p, p_cx=0, p_1q=0, p_idle=0, p_prep=0)
    nz = g.nz
    time_edges = {(t * nz + k, (t + 1) * nz + k) for t in range(R) for k in range(nz)}
    got = {(int(u), int(v)) for u, v in zip(g.u, g.v)}
    assert time_edges <= got
    for (u, v), pe in zip(zip(g.u, g.v), g.p):
        if (int(u), int(v)) in time_edges:
            assert pe == pytest.approx(p)
        else:   # final data-measurement flips: edges inside the last layer
            assert u // nz == R and (v < 0 or v // nz == R)


def test_preparation_noise_alone():
    d, R, p = 5, 4, 0.003
    g = rotated_surface_code_circuit(d, R, p, p_cx=0, p_1q=0, p_idle=0, p_meas=0)
    nz = g.nz
    ph = rotated_surface_code(d, R, 0.01)
    first = [(int(u), int(v), int(o)) for u, v, o, k in zip(ph.u, ph.v, ph.obs, ph.kind)
             if k == 0 and u < nz]
    want = {}
    for e in first:   # each data qubit prepared flipped with probability p; parallel copies combine
        q = want.get(e, 0.0)
        want[e] = q * (1 - p) + p * (1 - q)
    for t in range(R):   # a flipped Z-ancilla preparation flips that round's measurement
        for k in range(nz):
            want[(t * nz + k, (t + 1) * nz + k, 0)] = p
    got = {(int(u), int(v), int(o)): float(pe) for u, v, o, pe in zip(g.u, g.v, g.obs, g.p)}
    assert set(got) == set(want)
    for e in want:
        assert got[e] == pytest.approx(want[e])


@pytest.mark.parametrize("d,p,shots", [(3, 0.005, 300), (5, 0.003, 150)])
def test_theorem1_on_circuit_level_graphs(d, p, shots):
    g = rotated_surface_code_circuit(d, d, p)
    og = OracleGraph.from_phys(g)
    syn, _ = sample_shots(g, shots, 9)
    for s in range(shots):
        det = unpack_defects(syn[s], g.num_detectors)
        a = og.decode(det, "global")
        b = og.decode(det, "hier")
        assert a.status == 0 and b.status == 0
        assert (a.weight, a.obs) == (b.weight, b.obs)
        assert b.dual_feasible and b.tight and b.touch_violations == 0
