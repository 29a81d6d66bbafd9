"""C-ABI library: builds for sm_103a, loads, exports every declared symbol, and
its host-only logic (Algorithm 3, input validation) works without a GPU."""

import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2609_12262_gb300 as q
from paper_2609_12262_gb300 import build as qbuild
from oracle import alg3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    qbuild.build()
    return q.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "qec.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qec_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(L, s), s


@pytest.mark.parametrize("wmax", [164, 170, 186, 198, 222, 9, 2])
def test_schedule_matches_oracle(L, wmax):
    d, b = q.schedule(wmax, levels=8)
    od, ob, _ = alg3(wmax, levels=len(d))
    assert len(d) >= 2
    assert d == od and b == ob


def test_schedule_custom_params(L):
    d, b = q.schedule(186, q=(1, 5), phi_min=(1, 20), levels=3)
    from fractions import Fraction
    od, ob, _ = alg3(186, q=Fraction(1, 5), phi_min=Fraction(1, 20), levels=len(d))
    assert d == od and b == ob


@pytest.mark.parametrize("kw", [dict(d1=373), dict(d1=373, b1=800), dict(d1=559, q=(1, 50), phi_min=(1, 1000)),
                                dict(b1=1000), dict(d1=187, b1=375)])
def test_schedule_custom_level1(L, kw):
    from fractions import Fraction
    qq, pm = kw.get("q", (1, 10)), kw.get("phi_min", (1, 100))
    d, b = q.schedule(186, q=qq, phi_min=pm, levels=3, d1=kw.get("d1", 0), b1=kw.get("b1", 0))
    od, ob, _ = alg3(186, Fraction(*qq), Fraction(*pm), levels=len(d), d1=kw.get("d1"), b1=kw.get("b1"))
    assert len(d) >= 2 and d == od and b == ob
    if "d1" in kw:
        assert d[0] == kw["d1"]
    if "b1" in kw:
        assert b[0] == kw["b1"]


@pytest.mark.parametrize("d1,b1", [(373, 746), (373, 372), (187, 300)])
def test_schedule_rejects_inadmissible_level1(L, d1, b1):
    """phi_1 = 1 > 2 d1 / b1 fails for b1 <= 2 d1: both sides refuse the schedule."""
    from fractions import Fraction
    with pytest.raises(q.QecError):
        q.schedule(186, levels=3, d1=d1, b1=b1)
    with pytest.raises(ValueError):
        alg3(186, Fraction(1, 10), Fraction(1, 100), levels=3, d1=d1, b1=b1)


def _desc(n, u, v, w, o, nobs=1):
    arrs = [np.ascontiguousarray(u, np.int32), np.ascontiguousarray(v, np.int32),
            np.ascontiguousarray(w, np.int32), np.ascontiguousarray(o, np.uint64)]
    d = q.qec_graph_desc()
    d.num_detectors, d.num_edges, d.num_observables = n, len(u), nobs
    d.u = arrs[0].ctypes.data_as(C.POINTER(C.c_int32))
    d.v = arrs[1].ctypes.data_as(C.POINTER(C.c_int32))
    d.w = arrs[2].ctypes.data_as(C.POINTER(C.c_int32))
    d.obs = arrs[3].ctypes.data_as(C.POINTER(C.c_uint64))
    return d, arrs


@pytest.mark.parametrize("case,code", [
    (dict(n=3, u=[0, 5], v=[1, -1], w=[2, 2], o=[0, 0]), q.QEC_EINVAL),     # endpoint out of range
    (dict(n=3, u=[0, 1], v=[0, -1], w=[2, 2], o=[0, 0]), q.QEC_EINVAL),     # self loop
    (dict(n=3, u=[0, 1], v=[1, -1], w=[0, 2], o=[0, 0]), q.QEC_EINVAL),     # weight 0
    (dict(n=3, u=[0, 1], v=[1, -1], w=[-3, 2], o=[0, 0]), q.QEC_EINVAL),    # negative weight
    (dict(n=3, u=[0, 1], v=[1, -1], w=[2, 2], o=[0, 2]), q.QEC_EINVAL),     # obs bit 1 with 1 observable
    (dict(n=0, u=[], v=[], w=[], o=[]), q.QEC_ERANGE),                      # no detectors
])
def test_graph_create_rejects(L, case, code):
    d, _keep = _desc(case["n"], case["u"], case["v"], case["w"], case["o"])
    h = C.c_void_p()
    rc = L.qec_graph_create(C.byref(d), C.byref(h))
    assert rc == code and not h.value
    assert len(q.last_error()) > 0


def test_decode_rejects_bad_args(L):
    vp = C.c_void_p
    arr = (vp * 1)(None)
    assert L.qec_decode_batch(arr, 0, None, None, None, 5, None, None, None, None) == q.QEC_EINVAL
    assert L.qec_decode_batch(arr, 1, None, None, None, -1, None, None, None, None) == q.QEC_EINVAL
    assert L.qec_decode_batch(arr, 1, None, None, None, 0, None, None, None, None) == q.QEC_OK
    assert L.qec_decode_batch(arr, 33, None, None, None, 5, None, None, None, None) == q.QEC_EINVAL


def test_window_assemble_validates_before_touching_memory(L):
    """Argument errors are reported before any device access (the pointers
    below are never dereferenced)."""
    fake = C.c_void_p(16)
    rc = L.qec_window_assemble(fake, 8, 0, 300, None, 0, 0, 0, fake, 8, 4, None)   # 300 bits > 8 words
    assert rc == q.QEC_ERANGE
    rc = L.qec_window_assemble(fake, 8, -1, 10, None, 0, 0, 0, fake, 8, 4, None)
    assert rc == q.QEC_EINVAL
    rc = L.qec_window_assemble(fake, 8, 0, 10, fake, 0, 0, 10, fake, 8, 4, None)   # carry rows of 0 words
    assert rc == q.QEC_EINVAL
    rc = L.qec_window_assemble(None, 8, 0, 10, None, 0, 0, 0, fake, 8, 4, None)
    assert rc == q.QEC_EINVAL
    assert L.qec_window_assemble(fake, 8, 0, 10, None, 0, 0, 0, fake, 8, 0, None) == q.QEC_OK   # no rows


def test_static_entry_point_failure_leaves_no_half_set_up_state(L):
    """Without a usable CUDA device the static-scratch entry point fails before
    its one-time set-up (the device is marked set up only after the fill of its
    array has been enqueued), so every later call fails the same way instead of
    decoding against an unfilled array.  Argument errors come first."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    vp = C.c_void_p
    fake = vp(16)
    arr = (vp * 1)(fake)
    assert L.qec_decode_batch_static(arr, 1, None, None, fake, -1, fake, fake, fake, None) == q.QEC_EINVAL
    assert L.qec_decode_batch_static(arr, 1, None, None, fake, (1 << 20) + 1, fake, fake, fake, None) == q.QEC_ERANGE
    assert L.qec_decode_batch_static(arr, 1, None, None, None, 4, fake, fake, fake, None) == q.QEC_EINVAL
    for _ in range(2):
        rc = L.qec_decode_batch_static(arr, 1, None, None, fake, 4, fake, fake, fake, None)
        assert rc == q.QEC_ECUDA
        assert "cudaGetDevice" in q.last_error()


def test_window_graph_validates_on_the_host(L):
    h = C.c_void_p()
    assert L.qec_graph_create_window(None, 0, 4, None, C.byref(h)) == q.QEC_EINVAL and not h.value
    assert L.qec_graph_create_window(C.c_void_p(16), 0, 4, None, None) == q.QEC_EINVAL


def test_tuning_knobs_validate_keep_and_restore(L):
    """qec_set_tuning / qec_get_tuning on the host: a positive value sets a
    knob, zero keeps it, a negative value restores its default; team sizes
    other than 1, 4 and 16 and out-of-range values are refused without
    changing anything."""
    default = q.get_tuning()
    try:
        q.set_tuning(warps_per_block=2, team_warps=4, kcap=700, team_split_events=48)
        t = q.get_tuning()
        assert (t["warps_per_block"], t["team_warps"], t["kcap"], t["team_split_events"]) == (2, 4, 700, 48)
        q.set_tuning(band_factor=2)   # zero keeps the others
        t2 = q.get_tuning()
        assert t2["band_factor"] == 2 and t2["team_warps"] == 4 and t2["kcap"] == 700
        for bad in (dict(team_warps=8), dict(team_warps=2), dict(warps_per_block=33), dict(blocks_per_sm=65),
                    dict(band_factor=65), dict(kcap=(1 << 18) + 1)):
            with pytest.raises(RuntimeError):
                q.set_tuning(**bad)
            assert q.get_tuning() == t2, bad
        q.set_tuning(warps_per_block=-1, team_warps=-1, kcap=-1, team_split_events=-1, band_factor=-1)
        assert q.get_tuning() == default
    finally:
        q.set_tuning(warps_per_block=-1, blocks_per_sm=-1, band_factor=-1, kcap=-1, max_events=-1, team_warps=-1,
                     team_min_detectors=-1, team_split_events=-1)
