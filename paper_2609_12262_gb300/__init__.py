"""Python binding of the GB300 parallel sparse-blossom decoder (include/qec.h).

Argument marshalling only: every step of decoding runs in the CUDA kernels of
libqec.so.  PyTorch supplies device memory and streams.  Importing the package
does not need a GPU; calling a decode without the built library raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqec.so")

QEC_OK, QEC_EINVAL, QEC_ENOMEM, QEC_ECUDA, QEC_EAGAIN, QEC_ERANGE = 0, -1, -2, -3, -4, -5
SHOT_OK, SHOT_NO_SOLUTION, SHOT_BUDGET_EXCEEDED, SHOT_CAPACITY, SHOT_INTERNAL = 0, 1, 2, 3, 4
MAX_GRAPHS_PER_BATCH = 32


class QecError(RuntimeError):
    pass


class qec_params(C.Structure):
    _fields_ = [("q_num", C.c_int32), ("q_den", C.c_int32), ("phi_num", C.c_int32), ("phi_den", C.c_int32),
                ("d1", C.c_int32), ("b1", C.c_int32)]


class qec_graph_desc(C.Structure):
    _fields_ = [
        ("num_detectors", C.c_int32), ("num_edges", C.c_int32), ("num_observables", C.c_int32),
        ("u", C.POINTER(C.c_int32)), ("v", C.POINTER(C.c_int32)), ("w", C.POINTER(C.c_int32)),
        ("obs", C.POINTER(C.c_uint64)), ("params", C.POINTER(qec_params)),
    ]


class qec_graph_info(C.Structure):
    _fields_ = [
        ("num_detectors", C.c_int32), ("num_merged_edges", C.c_int32), ("words_per_shot", C.c_int32),
        ("wmax_internal", C.c_int32), ("num_levels", C.c_int32),
        ("d_k", C.c_int64 * 8), ("b_k", C.c_int64 * 8), ("device", C.c_int32),
        ("has_internal_obs", C.c_int32), ("components", C.c_int32), ("upper_single_cluster", C.c_int32),
        ("distance_bound", C.c_int64),
    ]


class qec_tuning(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("band_factor", C.c_int32),
                ("kcap", C.c_int32), ("max_events", C.c_int64), ("team_warps", C.c_int32),
                ("team_min_detectors", C.c_int32), ("team_split_events", C.c_int32)]


class qec_result(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("obs", C.c_uint64), ("weight", C.c_int64), ("status", C.c_int32),
                ("graph_index", C.c_int32), ("t_submit_ns", C.c_int64), ("t_done_ns", C.c_int64)]


_lib = None


def lib():
    """Load libqec.so (raises QecError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise QecError("libqec.so is not built (run paper_2609_12262_gb300.build.build())")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    vp = C.c_void_p
    L.qec_last_error.restype = C.c_char_p
    L.qec_version.restype = C.c_char_p
    L.qec_schedule.argtypes = [C.c_int32, P(qec_params), P(C.c_int64), P(C.c_int64), C.c_int32]
    L.qec_graph_create.argtypes = [P(qec_graph_desc), P(vp)]
    L.qec_graph_create_window.argtypes = [vp, C.c_int32, C.c_int32, P(qec_params), P(vp)]
    L.qec_graph_destroy.argtypes = [vp]
    L.qec_graph_get_info.argtypes = [vp, P(qec_graph_info)]
    L.qec_graph_merged_edges.argtypes = [vp, P(C.c_int32), P(C.c_int32), P(C.c_int32), P(C.c_uint64)]
    L.qec_decode_batch.argtypes = [P(vp), C.c_int32, vp, vp, vp, C.c_int64, vp, vp, vp, vp]
    L.qec_decode_batch_ex.argtypes = [P(vp), C.c_int32, vp, vp, vp, C.c_int64, C.c_int32, vp, vp, vp, vp, vp]
    L.qec_decode_plain.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp]
    L.qec_graph_set_commit_region.argtypes = [vp, vp]
    L.qec_decode_window_batch.argtypes = [P(vp), C.c_int32, vp, vp, vp, C.c_int64, vp, vp, vp, vp]
    L.qec_window_assemble.argtypes = [vp, C.c_int64, C.c_int64, C.c_int32, vp, C.c_int64, C.c_int64, C.c_int32,
                                      vp, C.c_int64, C.c_int64, vp]
    L.qec_decode_batch_static.argtypes = [P(vp), C.c_int32, vp, vp, vp, C.c_int64, vp, vp, vp, vp]
    L.qec_stream_create.argtypes = [C.c_size_t, C.c_int32, P(vp)]
    L.qec_stream_submit.argtypes = [vp, vp, vp, C.c_uint64]
    L.qec_stream_poll.argtypes = [vp, P(qec_result), C.c_int32, P(C.c_int32)]
    L.qec_stream_submit_many.argtypes = [vp, P(vp), C.c_int32, vp, vp, vp, vp, C.c_int32, P(C.c_int32)]
    L.qec_stream_flush.argtypes = [vp]
    L.qec_stream_destroy.argtypes = [vp]
    L.qec_set_tuning.argtypes = [P(qec_tuning)]
    L.qec_get_tuning.argtypes = [P(qec_tuning)]
    _lib = L
    return L


def last_error() -> str:
    return lib().qec_last_error().decode()


def version() -> str:
    return lib().qec_version().decode()


def _check(rc):
    if rc != QEC_OK:
        raise QecError("qec error %d: %s" % (rc, last_error()))
    return rc


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def schedule(wmax_internal: int, q=(1, 10), phi_min=(1, 100), levels: int = 8, d1: int = 0, b1: int = 0):
    """Algorithm 3 via qec_schedule: returns (d_k list, b_k list), internal units
    (d1, b1 > 0: custom level-1 diameter and buffer)."""
    L = lib()
    d = np.zeros(levels, np.int64)
    b = np.zeros(levels, np.int64)
    p = qec_params(q[0], q[1], phi_min[0], phi_min[1], int(d1), int(b1))
    n = L.qec_schedule(int(wmax_internal), C.byref(p), _ptr(d, C.c_int64), _ptr(b, C.c_int64), levels)
    if n < 1:
        raise QecError(last_error())
    return d[:n].tolist(), b[:n].tolist()


class Graph:
    """A detector graph resident on the current CUDA device (qec_graph_create)."""

    def __init__(self, num_detectors, u, v, w, obs, num_observables: int = 1, q=None, phi_min=None,
                 d1: int = 0, b1: int = 0):
        L = lib()
        self._u = np.ascontiguousarray(u, np.int32)
        self._v = np.ascontiguousarray(v, np.int32)
        self._w = np.ascontiguousarray(w, np.int32)
        self._o = np.ascontiguousarray(obs, np.uint64)
        desc = qec_graph_desc()
        desc.num_detectors = int(num_detectors)
        desc.num_edges = int(self._u.shape[0])
        desc.num_observables = int(num_observables)
        desc.u = _ptr(self._u, C.c_int32)
        desc.v = _ptr(self._v, C.c_int32)
        desc.w = _ptr(self._w, C.c_int32)
        desc.obs = _ptr(self._o, C.c_uint64)
        self._params = None
        if q is not None or phi_min is not None or d1 or b1:
            q = q or (1, 10)
            phi_min = phi_min or (1, 100)
            self._params = qec_params(q[0], q[1], phi_min[0], phi_min[1], int(d1), int(b1))
            desc.params = C.pointer(self._params)
        h = C.c_void_p()
        _check(L.qec_graph_create(C.byref(desc), C.byref(h)))
        self._h = h
        info = qec_graph_info()
        _check(L.qec_graph_get_info(h, C.byref(info)))
        self.info = info
        self.num_detectors = info.num_detectors
        self.words = info.words_per_shot

    @classmethod
    def from_phys(cls, g, **kw):
        return cls(g.num_detectors, g.u, g.v, g.w, g.obs, **kw)

    @classmethod
    def window(cls, stream, first_detector: int, num_detectors: int):
        """qec_graph_create_window: the induced subgraph of the Graph `stream` on
        detectors [first_detector, first_detector + num_detectors), renumbered
        from 0, with the stream graph's schedule parameters."""
        h = C.c_void_p()
        _check(lib().qec_graph_create_window(stream.handle, int(first_detector), int(num_detectors), None,
                                             C.byref(h)))
        return cls._wrap(h)

    @classmethod
    def _wrap(cls, h):
        self = cls.__new__(cls)
        self._h = h
        self._params = None
        info = qec_graph_info()
        _check(lib().qec_graph_get_info(h, C.byref(info)))
        self.info = info
        self.num_detectors = info.num_detectors
        self.words = info.words_per_shot
        return self

    def set_commit_region(self, bitmap=None):
        """qec_graph_set_commit_region: uint32 detector bitmap (words_per_shot words) or None."""
        if bitmap is None:
            _check(lib().qec_graph_set_commit_region(self._h, None))
            return
        b = np.ascontiguousarray(bitmap, np.uint32)
        if b.shape[0] < self.words:
            raise QecError("commit bitmap shorter than a syndrome row")
        _check(lib().qec_graph_set_commit_region(self._h, C.c_void_p(b.ctypes.data)))

    @property
    def handle(self):
        return self._h

    def schedule(self):
        n = self.info.num_levels
        return list(self.info.d_k)[:n], list(self.info.b_k)[:n]

    def merged_edges(self):
        m = self.info.num_merged_edges
        u = np.zeros(m, np.int32); v = np.zeros(m, np.int32)
        w = np.zeros(m, np.int32); o = np.zeros(m, np.uint64)
        _check(lib().qec_graph_merged_edges(self._h, _ptr(u, C.c_int32), _ptr(v, C.c_int32),
                                            _ptr(w, C.c_int32), _ptr(o, C.c_uint64)))
        return u, v, w, o

    def close(self):
        if getattr(self, "_h", None):
            lib().qec_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def decode_batch(graphs, syndromes, graph_of_shot=None, syn_offset_words=None, num_shots=None,
                 out=None, stream=None):
    """qec_decode_batch on torch device tensors.

    syndromes: int32 CUDA tensor holding the uint32 syndrome rows (flat or 2-D).
    graph_of_shot: int32 CUDA tensor or None; syn_offset_words: int64 CUDA tensor or None.
    Returns (obs int64 [S] holding the uint64 bits, weight int64 [S], status int32 [S]).
    """
    import torch
    if isinstance(graphs, Graph):
        graphs = [graphs]
    if num_shots is None:
        if graph_of_shot is not None:
            num_shots = int(graph_of_shot.shape[0])
        else:
            num_shots = int(syndromes.numel() // graphs[0].words)
    dev = syndromes.device
    if out is None:
        out = (torch.empty(num_shots, dtype=torch.int64, device=dev),
               torch.empty(num_shots, dtype=torch.int64, device=dev),
               torch.empty(num_shots, dtype=torch.int32, device=dev))
    obs, w, st = out
    arr = (C.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    _check(lib().qec_decode_batch(arr, len(graphs), _dptr(graph_of_shot), _dptr(syn_offset_words),
                                  _dptr(syndromes), int(num_shots), _dptr(obs), _dptr(w), _dptr(st),
                                  _stream_handle(stream)))
    return obs, w, st


MODES = {"hier": 0, "global": 1}
DIAG_FIELDS = ("e_ideal", "t_ideal", "events", "l1_clusters", "l1_defects", "top_events", "bands", "defects")


def decode_batch_ex(graphs, syndromes, graph_of_shot=None, syn_offset_words=None, num_shots=None,
                    mode="hier", diag=True, out=None, stream=None):
    """qec_decode_batch_ex: decode_batch with an execution mode ("hier" or
    "global") and per-shot diagnostics.  Returns (obs, weight, status, diag)
    with diag an int32 CUDA tensor [S, 8] (columns DIAG_FIELDS) or None."""
    import torch
    if isinstance(graphs, Graph):
        graphs = [graphs]
    if num_shots is None:
        num_shots = int(graph_of_shot.shape[0]) if graph_of_shot is not None else \
            int(syndromes.numel() // graphs[0].words)
    dev = syndromes.device
    if out is None:
        out = (torch.empty(num_shots, dtype=torch.int64, device=dev),
               torch.empty(num_shots, dtype=torch.int64, device=dev),
               torch.empty(num_shots, dtype=torch.int32, device=dev))
    obs, w, st = out
    dg = torch.empty((num_shots, len(DIAG_FIELDS)), dtype=torch.int32, device=dev) if diag else None
    arr = (C.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    _check(lib().qec_decode_batch_ex(arr, len(graphs), _dptr(graph_of_shot), _dptr(syn_offset_words),
                                     _dptr(syndromes), int(num_shots), MODES[mode], _dptr(obs), _dptr(w),
                                     _dptr(st), _dptr(dg), _stream_handle(stream)))
    return obs, w, st, dg


def decode_window_batch(graphs, syndromes, commit_obs, carry, status, graph_of_shot=None, syn_offset_words=None,
                        num_shots=None, stream=None):
    """qec_decode_window_batch on torch device tensors: commit_obs (int64 [S],
    XOR-accumulated), carry (int32, laid out like syndromes), status (int32 [S],
    failures only)."""
    if isinstance(graphs, Graph):
        graphs = [graphs]
    if num_shots is None:
        num_shots = int(graph_of_shot.shape[0]) if graph_of_shot is not None else \
            int(syndromes.numel() // graphs[0].words)
    arr = (C.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    _check(lib().qec_decode_window_batch(arr, len(graphs), _dptr(graph_of_shot), _dptr(syn_offset_words),
                                         _dptr(syndromes), int(num_shots), _dptr(commit_obs), _dptr(carry),
                                         _dptr(status), _stream_handle(stream)))


def window_assemble(stream_rows, stream_words, bit_begin, nbits, window_rows, window_words, num_rows,
                    carry_rows=None, carry_words=0, carry_bit_begin=0, carry_bits=0, stream=None):
    """qec_window_assemble on torch device tensors (int32 views of uint32 rows)."""
    _check(lib().qec_window_assemble(_dptr(stream_rows), int(stream_words), int(bit_begin), int(nbits),
                                     _dptr(carry_rows), int(carry_words), int(carry_bit_begin), int(carry_bits),
                                     _dptr(window_rows), int(window_words), int(num_rows), _stream_handle(stream)))


def decode_batch_static(graphs, syndromes, graph_of_shot=None, syn_offset_words=None, num_shots=None,
                        out=None, stream=None):
    """qec_decode_batch_static: decode_batch with scratch in the library's static
    device array (no device allocation inside the call; see include/qec.h for
    its limits).  `out` must be given by callers that cannot allocate."""
    import torch
    if isinstance(graphs, Graph):
        graphs = [graphs]
    if num_shots is None:
        num_shots = int(graph_of_shot.shape[0]) if graph_of_shot is not None else \
            int(syndromes.numel() // graphs[0].words)
    if out is None:
        dev = syndromes.device
        out = (torch.empty(num_shots, dtype=torch.int64, device=dev),
               torch.empty(num_shots, dtype=torch.int64, device=dev),
               torch.empty(num_shots, dtype=torch.int32, device=dev))
    obs, w, st = out
    arr = (C.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    _check(lib().qec_decode_batch_static(arr, len(graphs), _dptr(graph_of_shot), _dptr(syn_offset_words),
                                         _dptr(syndromes), int(num_shots), _dptr(obs), _dptr(w), _dptr(st),
                                         _stream_handle(stream)))
    return obs, w, st


def decode_plain(graph, syndromes, num_shots=None, out=None, stream=None):
    """qec_decode_plain: one kernel launch per shot (the plain GPU path)."""
    import torch
    if num_shots is None:
        num_shots = int(syndromes.numel() // graph.words)
    dev = syndromes.device
    if out is None:
        out = (torch.empty(num_shots, dtype=torch.int64, device=dev),
               torch.empty(num_shots, dtype=torch.int64, device=dev),
               torch.empty(num_shots, dtype=torch.int32, device=dev))
    obs, w, st = out
    _check(lib().qec_decode_plain(graph.handle, _dptr(syndromes), int(num_shots), _dptr(obs), _dptr(w),
                                  _dptr(st), _stream_handle(stream)))
    return obs, w, st


class Stream:
    """qec_stream_*: continuous-batching request loop on the current device."""

    def __init__(self, device_budget_bytes: int = 6 << 30, max_inflight: int = 65536):
        h = C.c_void_p()
        _check(lib().qec_stream_create(int(device_budget_bytes), int(max_inflight), C.byref(h)))
        self._h = h
        self._buf = (qec_result * 65536)()

    def submit(self, graph, syndrome_row: np.ndarray, request_id: int) -> bool:
        """Copy one window in; False when admission is full (QEC_EAGAIN)."""
        row = np.ascontiguousarray(syndrome_row, np.uint32)
        rc = lib().qec_stream_submit(self._h, graph.handle, C.c_void_p(row.ctypes.data), int(request_id))
        if rc == QEC_EAGAIN:
            return False
        _check(rc)
        return True

    def submit_many(self, graphs, graph_of_req, syn_offset_words, syndromes, request_ids) -> int:
        """Submit windows in order until admission is full; returns how many were taken."""
        arr = (C.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
        gi = np.ascontiguousarray(graph_of_req, np.int32)
        of = np.ascontiguousarray(syn_offset_words, np.int64)
        sy = np.ascontiguousarray(syndromes, np.uint32)
        ri = np.ascontiguousarray(request_ids, np.uint64)
        n = C.c_int32(0)
        _check(lib().qec_stream_submit_many(self._h, arr, len(graphs), C.c_void_p(gi.ctypes.data),
                                            C.c_void_p(of.ctypes.data), C.c_void_p(sy.ctypes.data),
                                            C.c_void_p(ri.ctypes.data), int(gi.shape[0]), C.byref(n)))
        return n.value

    def poll(self, max_results: int = 65536):
        """Finished results as a numpy structured array."""
        n = C.c_int32(0)
        m = min(int(max_results), len(self._buf))
        _check(lib().qec_stream_poll(self._h, self._buf, m, C.byref(n)))
        dt = np.dtype([("request_id", "<u8"), ("obs", "<u8"), ("weight", "<i8"), ("status", "<i4"),
                       ("graph_index", "<i4"), ("t_submit_ns", "<i8"), ("t_done_ns", "<i8")])
        if not n.value:
            return np.zeros(0, dt)
        raw = C.string_at(C.addressof(self._buf), n.value * C.sizeof(qec_result))
        return np.frombuffer(raw, dtype=dt).copy()

    def flush(self):
        _check(lib().qec_stream_flush(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().qec_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_tuning(warps_per_block=0, blocks_per_sm=0, band_factor=0, kcap=0, max_events=0, team_warps=0,
               team_min_detectors=0, team_split_events=0):
    """qec_set_tuning: positive sets a knob, 0 keeps it, negative restores its default."""
    t = qec_tuning(int(warps_per_block), int(blocks_per_sm), int(band_factor), int(kcap), int(max_events),
                   int(team_warps), int(team_min_detectors), int(team_split_events))
    _check(lib().qec_set_tuning(C.byref(t)))


def get_tuning() -> dict:
    t = qec_tuning()
    _check(lib().qec_get_tuning(C.byref(t)))
    return {f: getattr(t, f) for f, _ in qec_tuning._fields_}


def release_workspace():
    _check(lib().qec_release_workspace())


def to_uint64(t) -> np.ndarray:
    """int64 tensor holding uint64 bits -> numpy uint64."""
    return t.detach().cpu().numpy().view(np.uint64)
