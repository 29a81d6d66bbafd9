"""Sliding-window decoding with commit regions, on the CPU oracle.

TEST INFRASTRUCTURE ONLY (part of the oracle): only tests/ may use it.

A long syndrome history is decoded in overlapping windows, one after another
(the paper's introduction contrasts this sliding-window use, where the time per
syndrome round sets the throughput, with parallel windows).  Reading used here:

* Window k covers the detector layers [kC, kC + W) of the stream (W layers,
  stride C <= W); the last window reaches the end of the stream.  Its graph is
  the induced subgraph of the stream graph on those layers.
* Its syndrome is the stream syndrome on those layers, XOR the detectors
  flipped by corrections already committed (the carry).
* Its correction (the oracle's canonical matching paths, reading 10 of the
  semantics) is committed on every edge that touches the commit region, which
  is the first C layers of the window, or every layer for the last window.
  The committed observable accumulates; a committed edge whose other endpoint
  lies outside the commit region flips that detector for the next window.

Every detector lies in exactly one commit region, so the committed edges of all
windows together form a correction of the whole stream's syndrome.
"""

from __future__ import annotations

import numpy as np

from .oracle import OracleGraph


def window_graph(g, first_layer: int, num_layers: int):
    """The oracle's window graph: detector layers [first_layer, first_layer +
    num_layers) of a stream graph g (physical edge lists u, v, w, obs and nz
    detectors per layer, as built by the input generator).  Every physical edge
    whose detector endpoints all lie in those layers is kept (a boundary edge
    counts when its one detector does), in the stream's order, with detectors
    renumbered from 0; edges that leave the window are dropped.  Returns
    (num_detectors, u, v, w, obs, edge_map) with edge_map the stream index of
    every kept edge."""
    nz = g.nz
    lo = first_layer * nz
    hi = min(g.num_detectors, (first_layer + num_layers) * nz)
    keep = []
    for e in range(g.u.shape[0]):
        a, b = int(g.u[e]), int(g.v[e])
        if lo <= a < hi and (b < 0 or lo <= b < hi):
            keep.append(e)
    keep = np.asarray(keep, np.int64)
    u = g.u[keep].astype(np.int64) - lo
    v = g.v[keep].astype(np.int64)
    v = np.where(v >= 0, v - lo, -1)
    return (hi - lo, u.astype(np.int32), v.astype(np.int32), g.w[keep].astype(np.int32),
            g.obs[keep].astype(np.uint64), keep)


def windows(num_layers: int, W: int, C: int):
    """(first layer, layers, is last) of each window over num_layers layers."""
    if not (1 <= C <= W):
        raise ValueError("need 1 <= C <= W")
    out, a = [], 0
    while True:
        if a + W >= num_layers:
            out.append((a, num_layers - a, True))
            return out
        out.append((a, W, False))
        a += C


def sliding_window_decode(stream, syn: np.ndarray, W: int, C: int, mode: str = "hier",
                          return_edges: bool = False):
    """Decode each stream syndrome row of `syn` (uint32 [S, stream words]) window
    by window.  Returns (obs uint64 [S], status int32 [S]) and, with
    return_edges, per shot the committed edges as (u, v) stream detector pairs
    (v = -1 for a boundary edge)."""
    nz = stream.nz
    layers = stream.num_detectors // nz
    plan = windows(layers, W, C)
    graphs = []
    for a, nl, last in plan:
        n, u, v, w, o, _ = window_graph(stream, a, nl)
        og = OracleGraph(n, u, v, w, o)
        mu, mv, _, mo = og.merged_edges()
        graphs.append((a, nl, last, og, mu, mv, mo))
    S = syn.shape[0]
    obs = np.zeros(S, np.uint64)
    status = np.zeros(S, np.int32)
    edges = []
    for s in range(S):
        bits = np.unpackbits(np.ascontiguousarray(syn[s], np.uint32).view(np.uint8), bitorder="little")
        defects = bits[:stream.num_detectors].astype(np.uint8)
        carry = np.zeros(stream.num_detectors, np.uint8)
        o = 0
        committed = []
        for a, nl, last, og, mu, mv, mo in graphs:
            lo, hi = a * nz, (a + nl) * nz
            commit_hi = hi if last else lo + C * nz
            win = defects[lo:hi] ^ carry[lo:hi]
            r, corr = og.decode(np.nonzero(win)[0], mode, correction=True)
            if r.status != 0:
                status[s] = r.status
                break
            for e in np.nonzero(corr[:mu.shape[0]])[0]:
                u = int(mu[e]) + lo
                v = int(mv[e]) + lo if mv[e] >= 0 else -1
                cu = u < commit_hi
                cv = 0 <= v < commit_hi
                if not (cu or cv):
                    continue
                o ^= int(mo[e])
                committed.append((u, v))
                if v >= 0 and cu != cv:
                    carry[v if cu else u] ^= 1
        obs[s] = o
        edges.append(np.asarray(committed, np.int64).reshape(-1, 2))
    return (obs, status, edges) if return_edges else (obs, status)
