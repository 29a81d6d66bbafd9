"""Circuit-level detector graphs for the rotated surface code (Z-basis memory).

The paper evaluates on circuit-level noise (Methods, "Numerical evaluation"):
memory experiments of d rounds under two i.i.d. noise models with parameter p.
This module builds the detector graph of such an experiment from scratch: the
syndrome-extraction circuit, every single fault of the noise model, and where
each fault's Pauli ends up.  (The paper's experiments use X-basis memory; this
is the Z-basis one, its mirror image under exchanging X and Z.)

Circuit (d x d data qubits, one ancilla per stabiliser, layout and check types
as in surface.py: plaquette (i, j) is Z-type when i + j is even), in time steps:

* step 0: prepare the data qubits in |0>;
* each round t = 0 .. R-1: prepare all ancillas in |0>; H on X ancillas; four
  CNOT steps; H on X ancillas; measure all ancillas in Z.  Z ancilla: CNOT
  data -> ancilla, data order NW, NE, SW, SE; X ancilla: CNOT ancilla -> data,
  order NW, SW, NE, SE (every step touches each qubit at most once; a fault on
  an ancilla part-way through spreads to two data qubits lying across the
  logical of its own type, so the circuit distance stays d);
* finally every data qubit is measured in Z.
Every qubit not acted on in a step idles in it.

Noise models (the paper's two):
* "uniform": a preparation is flipped with probability p; after every one-qubit
  gate and every idle, X, Y or Z with p/3 each; after every CNOT, one of the 15
  non-identity two-qubit Paulis with p/15 each; a measurement result flips with
  probability p.
* "physical": preparation and measurement flips and CNOT noise as above; after
  every non-idle one-qubit gate X, Y or Z with p/30 each; idles are noiseless.
Each depolarising channel is written exactly as a product of independent Pauli
channels (probabilities chosen so that the product equals the channel), so
every elementary fault below is independent.

Detectors (Z checks only; X errors are decoded): layer 0 is each Z ancilla's
first measurement (deterministic), layer t in 1..R-1 compares rounds t-1 and t,
layer R compares round R-1 with the parity of the final data measurements on
the check's support.  Observable: the parity of the final data measurements in
column j = 0 (Z on the left column is the logical Z).  Each fault's X part flips
Z-basis measurements, hence detectors and the observable; faults with the same
(detectors, observable) symptom merge into one mechanism with the XOR-combined
probability.  Every mechanism flips one or two detectors for this circuit
(checked) and becomes a boundary edge or an edge of the returned PhysGraph,
with integer weight round(16 ln((1 - p_e) / p_e)).
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
    """The circuit as a list of operations in time steps: ('P', q) prepare |0>,
    ('H', q), ('CX', c, t), ('M', q, key) measure in Z, ('IDLE', q) for every
    qubit a step does not act on.  Returns (ops, nq, zchecks, xchecks, zanc, xanc)."""
    zc, xc = _checks(d)
    nd = d * d
    zanc = [nd + k for k in range(len(zc))]
    xanc = [nd + len(zc) + k for k in range(len(xc))]
    nq = nd + len(zc) + len(xc)
    ops = []

    def step(acts):
        busy = set()
        for op in acts:
            ops.append(op)
            busy.update(q for q in op[1:] if isinstance(q, int))
        for q in range(nq):
            if q not in busy:
                ops.append(("IDLE", q))

    step([("P", q) for q in range(nd)])
    for t in range(rounds):
        step([("P", q) for q in zanc + xanc])
        step([("H", q) for q in xanc])
        for layer in range(4):
            acts = []
            for k, c in enumerate(zc):
                if ZORDER[layer] in c:
                    acts.append(("CX", c[ZORDER[layer]], zanc[k]))
            for k, c in enumerate(xc):
                if XORDER[layer] in c:
                    acts.append(("CX", xanc[k], c[XORDER[layer]]))
            step(acts)
        step([("H", q) for q in xanc])
        step([("M", q, ("z", t, k)) for k, q in enumerate(zanc)] +
             [("M", q, ("x", t, k)) for k, q in enumerate(xanc)])
    ops.extend(("M", q, ("data", q)) for q in range(nd))
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
    control to target and Z from target to control, H exchanges X and Z, a
    preparation absorbs every earlier error, a Z measurement reports an X error
    and keeps it."""
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
        elif kind == "P":
            FX[op[1]] = empty
            FZ[op[1]] = empty
        elif kind == "M":
            e = key_effect(op[2])
            FX[op[1]] = (FX[op[1]][0] ^ e[0], FX[op[1]][1] ^ e[1])
    return FX, FZ


def rotated_surface_code_circuit(d: int, rounds: int | None = None, p: float = 0.001, noise: str = "uniform",
                                 *, p_cx=None, p_1q=None, p_idle=None, p_meas=None, p_prep=None) -> PhysGraph:
    """Circuit-level detector graph of a d-round (default) Z-basis memory
    experiment under the paper's "uniform" or "physical" noise model with
    parameter p (see the module docstring).  Keyword rates override single
    components: p_cx (two-qubit depolarising after a CNOT), p_1q (one-qubit
    depolarising after H), p_idle (after an idle), p_meas (measurement flip),
    p_prep (preparation flip)."""
    if d < 3 or d % 2 == 0:
        raise ValueError("d must be odd and >= 3")
    if noise not in ("uniform", "physical"):
        raise ValueError("noise must be 'uniform' or 'physical'")
    R = d if rounds is None else int(rounds)
    base = {"cx": p, "1q": p if noise == "uniform" else p / 10, "idle": p if noise == "uniform" else 0.0,
            "meas": p, "prep": p}
    rate = {k: (base[k] if v is None else float(v)) for k, v in
            (("cx", p_cx), ("1q", p_1q), ("idle", p_idle), ("meas", p_meas), ("prep", p_prep))}
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
        if kind == "P":
            add(rate["prep"], FX[op[1]])   # the prepared |0> flipped: an X error
        elif kind == "H":
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

    backward_sensitivity(ops, nq, key_effect, visit)
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
