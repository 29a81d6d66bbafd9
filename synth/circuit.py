"""Circuit-level detector graphs for the rotated surface code (Z-basis memory).

The paper evaluates on circuit-level detector error models (Methods, noise
models with uniform and physically motivated rates).  This module builds one
from scratch for the same code: the syndrome-extraction circuit, every single
fault of a noise model, and where each fault's Pauli ends up.

Circuit (d x d data qubits, one ancilla per stabiliser, layout and check
types as in surface.py: plaquette (i, j) is Z-type when i + j is even):

* round t = 0 .. R-1: reset all ancillas; H on X ancillas; four CNOT layers;
  H on X ancillas; measure all ancillas.  Z ancilla: CNOT data -> ancilla,
  data order NW, NE, SW, SE; X ancilla: CNOT ancilla -> data, order NW, SW,
  NE, SE (each CNOT layer touches every qubit at most once, and a fault on an
  ancilla part-way through propagates to two data qubits lying across the
  logical operator of its own type, so the circuit distance stays d).
* data qubits start in |0> and are measured in Z after the last round.

Detectors (Z checks only; X errors are decoded): layer 0 is each Z ancilla's
first measurement (deterministic), layer t in 1..R-1 compares rounds t-1 and t,
layer R compares round R-1 with the parity of the final data measurements on
the check's support.  Observable: the parity of the final data measurements in
column j = 0 (Z on the left column is the logical Z).

Noise (uniform depolarising, parameter p): after every CNOT a two-qubit
depolarising channel (one of the 15 non-identity Paulis, each p/15); after
every reset and every H a one-qubit depolarising channel (X, Y or Z, p/3 each);
every qubit idle in a CNOT layer gets the same one-qubit channel; every
measurement result flips with probability p; every data qubit gets a one-qubit
channel before the first round.  Each channel is written exactly as a product
of independent Pauli channels (probabilities chosen so that the product equals
the depolarising channel), so every elementary fault below is independent.
Each fault is propagated through the rest of the circuit (Pauli frame); its X
part flips Z-basis measurements, hence detectors and the observable.  Faults with the same (detectors, observable)
symptom merge into one mechanism with the XOR-combined probability.  Every
mechanism flips one or two detectors for this circuit (checked); it becomes a
boundary edge or an edge of the returned PhysGraph, with integer weight
round(16 ln((1 - p_e) / p_e)).
"""

from __future__ import annotations

import math
from collections import defaultdict

import numpy as np

from .surface import PhysGraph, weight_of_p


def _checks(d: int):
    """Z and X checks as lists of (ancilla id, corner dict) in row-major order;
    corner dict maps 'NW','NE','SW','SE' to data qubit index (missing corners
    absent)."""
    z, x = [], []
    for i in range(-1, d):
        for j in range(-1, d):
            corners = {}
            for name, (a, b) in (("NW", (i, j)), ("NE", (i, j + 1)), ("SW", (i + 1, j)), ("SE", (i + 1, j + 1))):
                if 0 <= a < d and 0 <= b < d:
                    corners[name] = a * d + b
            interior = 0 <= i <= d - 2 and 0 <= j <= d - 2
            if (i + j) % 2 == 0:
                if interior or ((i == -1 or i == d - 1) and 0 <= j <= d - 2):
                    z.append(corners)
            else:
                if interior or ((j == -1 or j == d - 1) and 0 <= i <= d - 2):
                    x.append(corners)
    return z, x


ZORDER = ("NW", "NE", "SW", "SE")
XORDER = ("NW", "SW", "NE", "SE")


def _circuit(d: int, rounds: int):
    """The circuit as a list of operations:
    ('R', q) reset, ('H', q), ('CX', c, t), ('M', q, key) measure, ('IDLE', q),
    ('TICK',) between layers.  Returns (ops, nq, zchecks, xchecks, zanc, xanc)."""
    zc, xc = _checks(d)
    nd = d * d
    zanc = [nd + k for k in range(len(zc))]
    xanc = [nd + len(zc) + k for k in range(len(xc))]
    nq = nd + len(zc) + len(xc)
    ops = []
    for t in range(rounds):
        for q in zanc + xanc:
            ops.append(("R", q))
        for q in xanc:
            ops.append(("H", q))
        ops.append(("TICK",))
        for layer in range(4):
            busy = set()
            for k, c in enumerate(zc):
                name = ZORDER[layer]
                if name in c:
                    ops.append(("CX", c[name], zanc[k]))
                    busy.update((c[name], zanc[k]))
            for k, c in enumerate(xc):
                name = XORDER[layer]
                if name in c:
                    ops.append(("CX", xanc[k], c[name]))
                    busy.update((c[name], xanc[k]))
            for q in range(nq):
                if q not in busy:
                    ops.append(("IDLE", q))
            ops.append(("TICK",))
        for q in xanc:
            ops.append(("H", q))
        for k, q in enumerate(zanc):
            ops.append(("M", q, ("z", t, k)))
        for k, q in enumerate(xanc):
            ops.append(("M", q, ("x", t, k)))
        ops.append(("TICK",))
    for q in range(nd):
        ops.append(("M", q, ("data", q)))
    return ops, nq, zc, xc, zanc, xanc


def _key_effect_fn(d: int, R: int, zc):
    nz = len(zc)
    members = [[] for _ in range(d * d)]
    for k, c in enumerate(zc):
        for q in c.values():
            members[q].append(k)

    def key_effect(key):
        """(detectors, observable) flipped when measurement `key` flips."""
        if key[0] == "z":
            _, t, k = key
            # layer t compares round t with round t-1 (layer 0: round 0 alone);
            # round t also enters layer t+1 (layer R: the final data parities)
            return frozenset((t * nz + k, (t + 1) * nz + k)), 0
        if key[0] == "data":
            q = key[1]
            return frozenset(R * nz + k for k in members[q]), int(q % d == 0)
        return frozenset(), 0
    return key_effect


def backward_sensitivity(ops, nq, key_effect, visit):
    """Walk the circuit backwards keeping, for every qubit, the (detectors,
    observable) flipped by an X (FX) or Z (FZ) error inserted at the current
    point; before stepping back over ops[i], call visit(i, op, FX, FZ) with the
    sensitivity of the point just after ops[i].  Stepping back applies the
    inverse of each operation's action on an error frame: a CNOT copies X from
    control to target and Z from target to control, H exchanges X and Z, a reset
    absorbs every error, a Z measurement reports an X error and keeps it."""
    empty = (frozenset(), 0)
    FX = [empty] * nq
    FZ = [empty] * nq
    for i in range(len(ops) - 1, -1, -1):
        op = ops[i]
        visit(i, op, FX, FZ)
        kind = op[0]
        if kind == "CX":
            c, t = op[1], op[2]
            FX[c] = (FX[c][0] ^ FX[t][0], FX[c][1] ^ FX[t][1])
            FZ[t] = (FZ[t][0] ^ FZ[c][0], FZ[t][1] ^ FZ[c][1])
        elif kind == "H":
            q = op[1]
            FX[q], FZ[q] = FZ[q], FX[q]
        elif kind == "R":
            FX[op[1]] = empty
            FZ[op[1]] = empty
        elif kind == "M":
            e = key_effect(op[2])
            FX[op[1]] = (FX[op[1]][0] ^ e[0], FX[op[1]][1] ^ e[1])
    return FX, FZ


def rotated_surface_code_circuit(d: int, rounds: int | None = None, p: float = 0.001, *, p_cx=None,
                                 p_1q=None, p_idle=None, p_meas=None, p_data=None) -> PhysGraph:
    """Circuit-level detector graph of a d-round (default) Z-basis memory
    experiment (see the module docstring).  Every noise component has rate p
    unless given: p_cx (two-qubit channel after a CNOT), p_1q (after reset and
    H), p_idle (idle qubit in a CNOT layer), p_meas (measurement flip), p_data
    (data qubits before the first round)."""
    if d < 3 or d % 2 == 0:
        raise ValueError("d must be odd and >= 3")
    R = d if rounds is None else int(rounds)
    rate = {k: (p if v is None else float(v)) for k, v in
            (("cx", p_cx), ("1q", p_1q), ("idle", p_idle), ("meas", p_meas), ("data", p_data))}
    ops, nq, zc, xc, zanc, xanc = _circuit(d, R)
    nz = len(zc)
    nd = d * d
    key_effect = _key_effect_fn(d, R, zc)
    mech = defaultdict(float)

    def add(prob, eff):
        if prob <= 0 or (not eff[0] and not eff[1]):
            return
        q0 = mech[eff]
        mech[eff] = q0 * (1 - prob) + prob * (1 - q0)

    def one_qubit(F, G, q, prob):
        # depolarising(prob) = independent X, Y and Z channels of probability
        # r each with (1 - 2r)^2 = 1 - 4 prob / 3 (every non-identity Pauli
        # anticommutes with two of the three)
        r = (1.0 - math.sqrt(max(0.0, 1.0 - 4.0 * prob / 3.0))) / 2.0
        add(r, F[q])
        add(r, (F[q][0] ^ G[q][0], F[q][1] ^ G[q][1]))
        add(r, G[q])

    def visit(i, op, FX, FZ):
        kind = op[0]
        if kind in ("R", "H"):
            one_qubit(FX, FZ, op[1], rate["1q"])
        elif kind == "IDLE":
            one_qubit(FX, FZ, op[1], rate["idle"])
        elif kind == "CX":
            c, t = op[1], op[2]
            # two-qubit depolarising = 15 independent Pauli channels of probability
            # r with (1 - 2r)^8 = 1 - 16 p / 15 (each anticommutes with 8 of 15)
            r = (1.0 - max(0.0, 1.0 - 16.0 * rate["cx"] / 15.0) ** 0.125) / 2.0
            for a in range(4):
                for b in range(4):
                    if a == 0 and b == 0:
                        continue
                    det, ob = frozenset(), 0
                    for q, pc in ((c, a), (t, b)):
                        if pc in (1, 2):
                            det, ob = det ^ FX[q][0], ob ^ FX[q][1]
                        if pc in (2, 3):
                            det, ob = det ^ FZ[q][0], ob ^ FZ[q][1]
                    add(r, (det, ob))
        elif kind == "M" and op[2][0] in ("z", "data"):
            add(rate["meas"], key_effect(op[2]))

    FX, FZ = backward_sensitivity(ops, nq, key_effect, visit)
    for q in range(nd):                # data qubits before the first round
        one_qubit(FX, FZ, q, rate["data"])
    us, vs, obs, pe, kind = [], [], [], [], []
    for (det, ob), prob in sorted(mech.items(), key=lambda kv: (sorted(kv[0][0]), kv[0][1])):
        det = sorted(det)
        if len(det) == 0:
            raise ValueError("a single fault flips the observable without any detector")
        if len(det) > 2:
            raise ValueError("a single fault flips %d detectors" % len(det))
        us.append(det[0])
        vs.append(det[1] if len(det) == 2 else -1)
        obs.append(ob)
        pe.append(prob)
        kind.append(0 if len(det) == 2 and det[0] // nz == det[1] // nz else 1)
    pe = np.asarray(pe, np.float64)
    n_det = nz * (R + 1)
    words = ((n_det + 31) // 32 + 3) // 4 * 4
    return PhysGraph(d=d, rounds=R, num_detectors=n_det, nz=nz,
                     u=np.asarray(us, np.int32), v=np.asarray(vs, np.int32),
                     w=np.asarray([weight_of_p(float(x)) for x in pe], np.int32),
                     obs=np.asarray(obs, np.uint64), p=pe, kind=np.asarray(kind, np.int8), words=words)
