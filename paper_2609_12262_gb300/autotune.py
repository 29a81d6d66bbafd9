"""Autotuner for the batched decoder's launch shape, per-warp slab sizes and
the team split threshold.

tune() times qec_decode_batch on a sample of the caller's own workload for
every candidate (warps per block, resident blocks per SM, flooder band width,
slab capacity), requires every candidate to return exactly the same weights,
observables and statuses as the first one (tuning never changes results), and
stores the fastest in a JSON cache keyed by GPU name and graph set.
tune_split() chooses, for single windows decoded by a 16-warp block, the
detection-event count below which the block's first warp decodes alone.
tune_team() chooses how many warps decode one shot (1, 4 or 16) for the
caller's batch: the automatic rule only sees graph sizes and shot counts,
while the best team size follows the detection events per shot.
"""

from __future__ import annotations

import hashlib
import itertools
import json
import os
import time

import numpy as np

from . import HERE, decode_batch, set_tuning, get_tuning

CACHE = os.path.join(HERE, "_build", "autotune.json")


def _key(graphs) -> str:
    import torch
    name = torch.cuda.get_device_name()
    sig = hashlib.sha1(json.dumps([[g.info.num_detectors, g.info.num_merged_edges, g.info.wmax_internal]
                                   for g in graphs]).encode()).hexdigest()[:16]
    return "%s|%s" % (name, sig)


def load(graphs):
    try:
        with open(CACHE) as f:
            return json.load(f).get(_key(graphs))
    except Exception:
        return None


def _v(x):
    return x if x > 0 else -1   # 0 means "automatic": reset to the default


def apply(cfg):
    set_tuning(warps_per_block=_v(cfg["warps_per_block"]), blocks_per_sm=_v(cfg["blocks_per_sm"]),
               band_factor=_v(cfg["band_factor"]), kcap=_v(cfg["kcap"]))


def candidates(nmax: int):
    kcaps = sorted({max(64, min(1024, nmax // 16)), max(64, min(1024, nmax // 32))})
    for wpb, bps, band, kc in itertools.product([1, 2, 4], [0, 4, 8, 12], [1, 2], kcaps):
        if bps and wpb * bps > 48:
            continue
        yield {"warps_per_block": wpb, "blocks_per_sm": bps, "band_factor": band, "kcap": kc}


def tune(graphs, syn, graph_of_shot, offsets, reps: int = 2, budget_s: float = 60.0, save: bool = True):
    """Return the fastest configuration on the given device tensors (and cache it)."""
    import torch
    S = int(graph_of_shot.shape[0])
    dev = syn.device
    out = (torch.empty(S, dtype=torch.int64, device=dev), torch.empty(S, dtype=torch.int64, device=dev),
           torch.empty(S, dtype=torch.int32, device=dev))
    saved = get_tuning()
    nmax = max(g.info.num_detectors for g in graphs)
    ref = None
    results = []
    t_start = time.time()
    try:
        for cfg in candidates(nmax):
            if time.time() - t_start > budget_s:
                break
            apply(cfg)
            decode_batch(graphs, syn, graph_of_shot, offsets, num_shots=S, out=out)
            torch.cuda.synchronize()
            got = tuple(t.cpu().numpy().copy() for t in out)
            if ref is None:
                ref = got
            elif not all(np.array_equal(a, b) for a, b in zip(got, ref)):
                raise RuntimeError("tuning configuration %r changed the decoding result" % cfg)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                decode_batch(graphs, syn, graph_of_shot, offsets, num_shots=S, out=out)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            results.append((ms, cfg))
    finally:
        set_tuning(**{k: _v(v) for k, v in saved.items()})
    results.sort(key=lambda r: r[0])
    best = dict(results[0][1])
    best["ms"] = results[0][0]
    best["shots"] = S
    best["candidates"] = len(results)
    if save:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        try:
            with open(CACHE) as f:
                db = json.load(f)
        except Exception:
            db = {}
        db[_key(graphs)] = best
        with open(CACHE, "w") as f:
            json.dump(db, f, indent=1)
    return best, results


def tune_split(samples, splits=(1, 24, 48, 64, 96, 128, 192), team: int = 16, reps: int = 2):
    """Choose the team split threshold for single-window decoding: a block of
    `team` warps hands a window with fewer detection events than the threshold
    to its first warp.  `samples` is a list of (Graph, int32 device tensor of
    one or more syndrome rows); every window is decoded alone (one launch per
    window) for every candidate, the results must agree across candidates,
    and the threshold with the smallest total latency is applied and returned
    with the per-candidate totals (ms)."""
    import torch
    saved = get_tuning()
    ref = None
    totals = []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        for sp in splits:
            set_tuning(team_warps=team, team_split_events=sp)
            got, ms = [], 0.0
            for g, rows in samples:
                n = rows.numel() // g.words
                for k in range(n):
                    one = rows[k * g.words:(k + 1) * g.words]
                    decode_batch([g], one, num_shots=1)   # warm
                    for _ in range(reps):
                        a.record()
                        o, w, st = decode_batch([g], one, num_shots=1)
                        b.record()
                        torch.cuda.synchronize()
                        ms += a.elapsed_time(b) / reps
                    got.append((int(w.item()), int(o.item()), int(st.item())))
            if ref is None:
                ref = got
            elif got != ref:
                raise RuntimeError("split threshold %d changed the decoding result" % sp)
            totals.append((ms, sp))
    finally:
        set_tuning(**{k: _v(v) for k, v in saved.items()})
    totals.sort()
    best = totals[0][1]
    set_tuning(team_split_events=best)
    return best, totals


def tune_team(graphs, syn, graph_of_shot=None, offsets=None, num_shots=None, teams=(1, 4, 16), reps: int = 2):
    """Choose the team size (warps per shot) for a batch: the batch is decoded
    with every candidate, the results must agree across candidates, and the
    fastest is applied and returned with the per-candidate times (ms)."""
    import torch
    if num_shots is None:
        num_shots = int(graph_of_shot.shape[0]) if graph_of_shot is not None else int(syn.numel() // graphs[0].words)
    dev = syn.device
    out = (torch.empty(num_shots, dtype=torch.int64, device=dev), torch.empty(num_shots, dtype=torch.int64, device=dev),
           torch.empty(num_shots, dtype=torch.int32, device=dev))
    saved = get_tuning()
    ref = None
    totals = []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        for team in teams:
            set_tuning(team_warps=team)
            decode_batch(graphs, syn, graph_of_shot, offsets, num_shots=num_shots, out=out)   # warm, sizes the workspace
            torch.cuda.synchronize()
            got = tuple(t.cpu().numpy().copy() for t in out)
            if ref is None:
                ref = got
            elif not all(np.array_equal(x, y) for x, y in zip(got, ref)):
                raise RuntimeError("team size %d changed the decoding result" % team)
            a.record()
            for _ in range(reps):
                decode_batch(graphs, syn, graph_of_shot, offsets, num_shots=num_shots, out=out)
            b.record()
            torch.cuda.synchronize()
            totals.append((a.elapsed_time(b) / reps, team))
    finally:
        set_tuning(**{k: _v(v) for k, v in saved.items()})
    totals.sort()
    best = totals[0][1]
    set_tuning(team_warps=best)
    return best, totals
