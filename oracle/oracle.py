"""ctypes wrapper around the C oracle (sb_oracle.c).  Test infrastructure only."""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build
from .schedule import alg3

_lib = None


class OResult(C.Structure):
    _fields_ = [
        ("weight", C.c_longlong),
        ("obs", C.c_uint64),
        ("status", C.c_int),
        ("events_implode", C.c_longlong),
        ("events_collide", C.c_longlong),
        ("events_boundary", C.c_longlong),
        ("dual_sum", C.c_longlong),
        ("primal_internal", C.c_longlong),
        ("dual_feasible", C.c_int),
        ("tight", C.c_int),
        ("touch_violations", C.c_int),
        ("num_levels", C.c_int),
        ("num_clusters", C.c_int),
        ("level1_events", C.c_int),
        ("stop_time", C.c_longlong),
        ("e_ideal", C.c_longlong),
        ("t_ideal", C.c_longlong),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        L.or_graph_build.argtypes = [C.c_int, C.c_int, P(C.c_int), P(C.c_int), P(C.c_int),
                                     P(C.c_uint64), P(C.c_void_p)]
        L.or_graph_build.restype = C.c_int
        L.or_graph_free.argtypes = [C.c_void_p]
        L.or_graph_num_edges.argtypes = [C.c_void_p]
        L.or_graph_wmax.argtypes = [C.c_void_p]
        L.or_graph_wmax.restype = C.c_longlong
        L.or_graph_edges.argtypes = [C.c_void_p, P(C.c_int), P(C.c_int), P(C.c_longlong), P(C.c_uint64)]
        L.or_decode.argtypes = [C.c_void_p, C.c_int, P(C.c_int), C.c_int, C.c_int,
                                P(C.c_longlong), P(C.c_longlong), P(OResult), C.c_void_p]
        L.or_decode_bitmaps.argtypes = [C.c_void_p, C.c_longlong, C.c_int, P(C.c_uint32), C.c_int,
                                        C.c_int, P(C.c_longlong), P(C.c_longlong),
                                        P(C.c_longlong), P(C.c_uint64), P(C.c_int)]
        L.or_geometry.argtypes = [C.c_void_p, C.c_int, P(C.c_int), P(C.c_longlong), P(C.c_uint64),
                                  P(C.c_longlong), P(C.c_int), P(C.c_uint64)]
        L.or_cluster.argtypes = [C.c_void_p, C.c_int, P(C.c_int), C.c_int, P(C.c_longlong),
                                 P(C.c_longlong), P(C.c_int), P(C.c_int)]
        L.or_result_size.restype = C.c_int
        assert L.or_result_size() == C.sizeof(OResult)
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


STATUS = {0: "OK", 1: "NO_SOLUTION", 2: "BUDGET", 3: "INTERNAL", 4: "BADARG"}


class OracleGraph:
    """Merged detector graph held by the oracle."""

    def __init__(self, n, u, v, w, obs, levels: int = 6, q=(1, 10), phi_min=(1, 100), d1=None, b1=None):
        L = lib()
        self.n = int(n)
        u = np.ascontiguousarray(u, np.int32)
        v = np.ascontiguousarray(v, np.int32)
        w = np.ascontiguousarray(w, np.int32)
        obs = np.ascontiguousarray(obs, np.uint64)
        h = C.c_void_p()
        st = L.or_graph_build(self.n, int(u.shape[0]), _p(u, C.c_int), _p(v, C.c_int),
                              _p(w, C.c_int), _p(obs, C.c_uint64), C.byref(h))
        if st != 0:
            raise ValueError("invalid graph (status %d)" % st)
        self._h = h
        self.wmax = int(L.or_graph_wmax(h))
        from fractions import Fraction
        d, b, _ = alg3(self.wmax, Fraction(*q), Fraction(*phi_min), levels=levels, d1=d1, b1=b1)
        cap = 1 << 60   # larger radii than any graph distance behave identically
        self.dk = np.asarray([min(x, cap) for x in d], np.int64)
        self.bk = np.asarray([min(x, cap) for x in b], np.int64)

    @classmethod
    def from_phys(cls, g, **kw):
        return cls(g.num_detectors, g.u, g.v, g.w, g.obs, **kw)

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().or_graph_free(self._h)
                self._h = None
        except Exception:
            pass

    def merged_edges(self):
        L = lib()
        m = L.or_graph_num_edges(self._h)
        u = np.zeros(m, np.int32); v = np.zeros(m, np.int32)
        w = np.zeros(m, np.int64); o = np.zeros(m, np.uint64)
        L.or_graph_edges(self._h, _p(u, C.c_int), _p(v, C.c_int), _p(w, C.c_longlong),
                         _p(o, C.c_uint64))
        return u, v, w, o

    def decode(self, defects, mode: str = "global", correction: bool = False):
        """Decode one shot; with correction=True also return the correction's
        merged-edge indicator (uint8 per merged edge)."""
        L = lib()
        det = np.ascontiguousarray(np.sort(np.asarray(defects, np.int32)), np.int32)
        r = OResult()
        corr = np.zeros(max(1, L.or_graph_num_edges(self._h)), np.uint8) if correction else None
        L.or_decode(self._h, int(det.shape[0]), _p(det, C.c_int), 0 if mode == "global" else 1,
                    int(self.dk.shape[0]), _p(self.dk, C.c_longlong), _p(self.bk, C.c_longlong),
                    C.byref(r), corr.ctypes.data if corr is not None else None)
        return (r, corr) if correction else r

    def diag(self, defects, mode: str = "hier"):
        """Decode one shot and return its result with the parallel-event-count
        diagnostics (Methods, "Numerical evaluation") as a dict."""
        r = self.decode(defects, mode)
        out = {"weight": r.weight, "obs": r.obs, "status": r.status, "e_ideal": r.e_ideal,
               "t_ideal": r.t_ideal, "events": r.events_implode + r.events_collide + r.events_boundary,
               "l1_clusters": 0, "l1_defects": 0, "clusters_above_l1": 0, "defects": len(defects)}
        if mode != "global" and len(defects):
            _, lev, cl = self.cluster(defects)
            out["l1_clusters"] = len(set(cl[lev == 1].tolist()))
            out["l1_defects"] = int(np.count_nonzero(lev == 1))
            out["clusters_above_l1"] = len(set(cl[lev > 1].tolist()))
        return out

    def decode_bitmaps(self, syn: np.ndarray, mode: str = "hier"):
        L = lib()
        syn = np.ascontiguousarray(syn, np.uint32)
        S, words = syn.shape
        W = np.zeros(S, np.int64); O = np.zeros(S, np.uint64); st = np.zeros(S, np.int32)
        L.or_decode_bitmaps(self._h, S, words, _p(syn, C.c_uint32), 0 if mode == "global" else 1,
                            int(self.dk.shape[0]), _p(self.dk, C.c_longlong), _p(self.bk, C.c_longlong),
                            _p(W, C.c_longlong), _p(O, C.c_uint64), _p(st, C.c_int))
        return W, O, st

    def geometry(self, defects):
        L = lib()
        det = np.ascontiguousarray(np.sort(np.asarray(defects, np.int32)), np.int32)
        k = int(det.shape[0])
        D = np.zeros((k, k), np.int64); PO = np.zeros((k, k), np.uint64)
        BD = np.zeros(k, np.int64); BE = np.zeros(k, np.int32); BO = np.zeros(k, np.uint64)
        L.or_geometry(self._h, k, _p(det, C.c_int), _p(D, C.c_longlong), _p(PO, C.c_uint64),
                      _p(BD, C.c_longlong), _p(BE, C.c_int), _p(BO, C.c_uint64))
        return D, PO, BD, BE, BO

    def cluster(self, defects):
        L = lib()
        det = np.ascontiguousarray(np.sort(np.asarray(defects, np.int32)), np.int32)
        k = int(det.shape[0])
        lev = np.zeros(k, np.int32); cl = np.zeros(k, np.int32)
        st = L.or_cluster(self._h, k, _p(det, C.c_int), int(self.dk.shape[0]),
                          _p(self.dk, C.c_longlong), _p(self.bk, C.c_longlong),
                          _p(lev, C.c_int), _p(cl, C.c_int))
        return st, lev, cl
