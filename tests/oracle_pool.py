"""Run the CPU oracle over many shots in a spawn-started process pool (tests only)."""

from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

_G = {}


def _init(phys_list):
    from oracle import OracleGraph
    _G.clear()
    for i, g in enumerate(phys_list):
        _G[i] = OracleGraph.from_phys(g)


def _work(args):
    gi, rows, mode = args
    return _G[gi].decode_bitmaps(rows, mode)


class OraclePool:
    """A spawn-started pool of oracle workers holding the graphs, reused across calls."""

    def __init__(self, phys_list, workers=None):
        self.phys_list = phys_list
        self.n = max(1, workers or (os.cpu_count() or 2))
        ctx = mp.get_context("spawn")
        self.ex = ProcessPoolExecutor(max_workers=self.n, mp_context=ctx, initializer=_init,
                                      initargs=(phys_list,))
        list(self.ex.map(_noop, range(self.n)))   # start every worker

    def decode(self, graph_of_shot, rows_by_shot, mode="hier", chunk=None):
        return oracle_decode(self.phys_list, graph_of_shot, rows_by_shot, mode=mode,
                             chunk=chunk or max(1, len(rows_by_shot) // (4 * self.n)), executor=self.ex)

    def close(self):
        self.ex.shutdown()


def _noop(_):
    return 0


def oracle_decode(phys_list, graph_of_shot, rows_by_shot, mode="hier", workers=None, chunk=256, executor=None):
    """rows_by_shot: list/array of uint32 rows (shot s uses graph phys_list[graph_of_shot[s]]).

    Returns (weight int64, obs uint64, status int32) per shot.
    """
    S = len(rows_by_shot)
    W = np.zeros(S, np.int64)
    O = np.zeros(S, np.uint64)
    st = np.zeros(S, np.int32)
    gos = np.asarray(graph_of_shot)
    tasks, where = [], []
    for gi in range(len(phys_list)):
        idx = np.nonzero(gos == gi)[0]
        for c0 in range(0, idx.size, chunk):
            sel = idx[c0:c0 + chunk]
            rows = np.stack([np.asarray(rows_by_shot[s], np.uint32) for s in sel])
            tasks.append((gi, rows, mode))
            where.append(sel)
    if not tasks:
        return W, O, st
    n = workers or max(1, min(len(tasks), (os.cpu_count() or 2)))
    if executor is not None:
        results = list(executor.map(_work, tasks))
    elif n == 1:
        _init(phys_list)
        results = [_work(t) for t in tasks]
    else:
        ctx = mp.get_context("spawn")
        with ProcessPoolExecutor(max_workers=n, mp_context=ctx, initializer=_init,
                                 initargs=(phys_list,)) as ex:
            results = list(ex.map(_work, tasks))
    for sel, (w, o, s) in zip(where, results):
        W[sel] = w
        O[sel] = o
        st[sel] = s
    return W, O, st
