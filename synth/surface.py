"""Rotated surface code under phenomenological noise: detector multigraph + syndromes.

Construction (the "Decoding task" paragraph of the paper defines the detector
graph: one vertex per detector, an edge per fault that flips two detectors, and
an edge to its own boundary vertex per fault that flips one detector):

* Data qubits sit on a d x d grid (row i, column j).  Plaquette (i, j) has the
  data qubits (i, j), (i+1, j), (i, j+1), (i+1, j+1) at its corners for
  i, j in [-1, d-1]; a plaquette is Z-type when (i + j) is even.  Z checks are
  the interior Z plaquettes plus the weight-2 Z plaquettes on the top and bottom
  sides (rows -1 and d-1); the left and right sides carry X checks only.  That
  gives (d*d - 1) / 2 Z checks.
* Only X errors are decoded (they flip Z checks).  Layer t (0..R) holds one
  physical space edge per data qubit (an X error before measurement round t);
  a qubit in one Z check gives a boundary edge (v = -1).  Rounds 0..R-1 are
  noisy and round R is perfect, so a time edge joins check c in layers t and
  t+1 for t < R (a flipped measurement).
* Detector index = t * nZ + c, with Z checks numbered in row-major plaquette
  order.  Syndrome bit i of a shot is detector i, LSB-first in uint32 words;
  rows are padded to a multiple of 4 words (16 bytes).
* The logical cut is the left column (j = 0): Z on it is a logical operator,
  so an edge carries observable bit 0 exactly when its data qubit is in column 0.
* Integer weight of an edge with probability p is round(16 ln((1-p)/p)) with
  halves rounded away from zero (the paper's weights are -ln q scaled to
  integers; the decoder doubles them internally so all events fall at integer
  times).

Physical edges are listed layer by layer: the d*d space edges of layer t in
row-major data-qubit order, then the nZ time edges from layer t to t+1.
Parallel physical edges (two left-column or right-column qubits in the same
check) are kept; merging them is the decoder's job.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def weight_of_p(p: float) -> int:
    """round(16 * ln((1-p)/p)), halves away from zero, as an int."""
    x = 16.0 * math.log((1.0 - p) / p)
    return int(math.floor(x + 0.5)) if x >= 0 else -int(math.floor(-x + 0.5))


@dataclass
class PhysGraph:
    d: int
    rounds: int
    num_detectors: int
    nz: int
    u: np.ndarray          # int32 [m]
    v: np.ndarray          # int32 [m], -1 = boundary
    w: np.ndarray          # int32 [m], original integer weights (> 0)
    obs: np.ndarray        # uint64 [m]
    p: np.ndarray          # float64 [m]
    kind: np.ndarray       # int8 [m]: 0 space, 1 time
    words: int = field(default=0)   # padded uint32 words per shot

    @property
    def num_edges(self) -> int:
        return int(self.u.shape[0])


def _z_checks(d: int):
    """Z checks as a list of tuples of data-qubit (i, j) pairs, row-major."""
    checks = []
    for i in range(-1, d):
        for j in range(-1, d):
            if (i + j) % 2 != 0:
                continue
            corners = [(a, b) for a in (i, i + 1) for b in (j, j + 1)
                       if 0 <= a < d and 0 <= b < d]
            interior = 0 <= i <= d - 2 and 0 <= j <= d - 2
            top_bottom = (i == -1 or i == d - 1) and 0 <= j <= d - 2
            if interior or top_bottom:
                checks.append(tuple(corners))
    return checks


def rotated_surface_code(d: int, rounds: int | None = None, p=0.003,
                         p_seed: int | None = None,
                         p_range: tuple[float, float] | None = None) -> PhysGraph:
    """Build the phenomenological detector multigraph.

    p        -- uniform physical error rate for every edge, or
    p_range  -- (lo, hi): each physical edge draws p ~ U[lo, hi] i.i.d. from
                numpy Philox(key=p_seed).
    """
    if d < 3 or d % 2 == 0:
        raise ValueError("d must be odd and >= 3")
    R = d if rounds is None else int(rounds)
    checks = _z_checks(d)
    nz = len(checks)
    assert nz == (d * d - 1) // 2
    member = {}
    for c, qs in enumerate(checks):
        for q in qs:
            member.setdefault(q, []).append(c)
    us, vs, obs, kind = [], [], [], []
    for t in range(R + 1):
        base = t * nz
        for i in range(d):
            for j in range(d):
                cs = member.get((i, j), [])
                assert 1 <= len(cs) <= 2
                if len(cs) == 2:
                    us.append(base + cs[0]); vs.append(base + cs[1])
                else:
                    us.append(base + cs[0]); vs.append(-1)
                obs.append(1 if j == 0 else 0)
                kind.append(0)
        if t < R:
            for c in range(nz):
                us.append(base + c); vs.append(base + nz + c)
                obs.append(0); kind.append(1)
    m = len(us)
    if p_range is not None:
        rng = np.random.Generator(np.random.Philox(key=int(p_seed or 0)))
        pe = rng.uniform(p_range[0], p_range[1], size=m)
    else:
        pe = np.full(m, float(p))
    wt = np.array([weight_of_p(float(x)) for x in pe], dtype=np.int32)
    n_det = nz * (R + 1)
    words = (n_det + 31) // 32
    words = (words + 3) // 4 * 4
    return PhysGraph(d=d, rounds=R, num_detectors=n_det, nz=nz,
                     u=np.asarray(us, np.int32), v=np.asarray(vs, np.int32),
                     w=wt, obs=np.asarray(obs, np.uint64), p=pe,
                     kind=np.asarray(kind, np.int8), words=words)


def _sample_flips(rng, pe: np.ndarray, shots: int):
    """Return (row, col) indices of flipped physical edges, i.i.d. Bernoulli(pe)."""
    m = pe.shape[0]
    uniform = bool(np.all(pe == pe[0]))
    if uniform:
        p = float(pe[0])
        rows_all, cols_all = [], []
        pending = np.arange(shots)
        M = int(m * p + 10 * math.sqrt(m * p + 1) + 16)
        while pending.size:
            gaps = rng.geometric(p, size=(pending.size, M))
            pos = np.cumsum(gaps, axis=1) - 1
            done = pos[:, -1] >= m
            ok = pending[done]
            pd = pos[done]
            r, c = np.nonzero(pd < m)
            rows_all.append(ok[r]); cols_all.append(pd[r, c])
            pending = pending[~done]
            M *= 2
        return (np.concatenate(rows_all) if rows_all else np.zeros(0, np.int64),
                np.concatenate(cols_all) if cols_all else np.zeros(0, np.int64))
    flips = rng.random((shots, m)) < pe[None, :]
    r, c = np.nonzero(flips)
    return r, c


def sample_shots(g: PhysGraph, shots: int, seed: int, chunk: int | None = None):
    """Sample `shots` syndromes.

    Returns (syndromes uint32 [shots, g.words], true_obs uint64 [shots]).
    Chunk c of the shots draws from numpy Philox(key=seed, counter=c), so the
    output depends only on (seed, shots, chunk).  The default chunk is 8192
    shots, fewer for graphs above 8192 detectors (2^26 / detectors, at least 64)
    so one chunk's per-detector counters stay near 512 MB.
    """
    n = g.num_detectors
    if chunk is None:
        chunk = max(64, min(8192, (1 << 26) // max(n, 1)))
    out = np.zeros((shots, g.words), dtype=np.uint32)
    true_obs = np.zeros(shots, dtype=np.uint64)
    for c0 in range(0, shots, chunk):
        s = min(chunk, shots - c0)
        rng = np.random.Generator(np.random.Philox(key=int(seed), counter=c0 // chunk))
        r, e = _sample_flips(rng, g.p, s)
        cnt = np.zeros(s * n, dtype=np.int64)
        np.add.at(cnt, r * n + g.u[e], 1)
        bd = g.v[e] >= 0
        np.add.at(cnt, r[bd] * n + g.v[e][bd], 1)
        bits = (cnt.reshape(s, n) & 1).astype(np.uint8)
        packed = np.packbits(bits, axis=1, bitorder="little")
        buf = np.zeros((s, g.words * 4), dtype=np.uint8)
        buf[:, :packed.shape[1]] = packed
        out[c0:c0 + s] = buf.view(np.uint32)
        ob = np.zeros(s, dtype=np.uint64)
        sel = g.obs[e] != 0
        np.bitwise_xor.at(ob, r[sel], g.obs[e][sel])
        true_obs[c0:c0 + s] = ob
    return out, true_obs


def unpack_defects(row: np.ndarray, n: int) -> np.ndarray:
    """Sorted detector indices of the set bits of one syndrome row."""
    bits = np.unpackbits(row.view(np.uint8), bitorder="little")[:n]
    return np.nonzero(bits)[0].astype(np.int32)


def pack_defects(defects, n: int) -> np.ndarray:
    """Inverse of unpack_defects: a padded uint32 row with the given bits set."""
    words = ((n + 31) // 32 + 3) // 4 * 4
    bits = np.zeros(words * 32, dtype=np.uint8)
    for x in defects:
        bits[int(x)] ^= 1
    return np.packbits(bits, bitorder="little").view(np.uint32).copy()


def mixed_batch(ds, shots_per_d: int, p: float, seed: int):
    """Mixed-distance batch (d rounds each), shot order shuffled by a seeded permutation.

    Returns (graphs, graph_of_shot int32 [S], syn_offset_words int64 [S],
    syndromes uint32 [sum words]).
    """
    graphs = [rotated_surface_code(d, d, p) for d in ds]
    per = []
    for gi, g in enumerate(graphs):
        syn, _ = sample_shots(g, shots_per_d, seed * 1000 + gi)
        per.append(syn)
    S = shots_per_d * len(graphs)
    gid = np.repeat(np.arange(len(graphs), dtype=np.int32), shots_per_d)
    rng = np.random.Generator(np.random.Philox(key=int(seed) + 7))
    perm = rng.permutation(S)
    gid = gid[perm]
    local = np.tile(np.arange(shots_per_d), len(graphs))[perm]
    words = np.array([g.words for g in graphs], dtype=np.int64)
    wps = words[gid]
    offs = np.zeros(S, dtype=np.int64)
    np.cumsum(wps[:-1], out=offs[1:])
    syn = np.zeros(int(wps.sum()), dtype=np.uint32)
    for gi in range(len(graphs)):
        sel = np.nonzero(gid == gi)[0]
        w = int(words[gi])
        idx = offs[sel][:, None] + np.arange(w)[None, :]
        syn[idx] = per[gi][local[sel]]
    return graphs, gid, offs, syn
