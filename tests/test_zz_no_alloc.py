"""qec_decode_batch_static, the entry point that allocates no device memory.

Callers that cannot allocate while running (a real-time decoding loop that
must not stall on the allocator, or an application that reserves all device
memory at start-up) decode through the library's static device scratch.  Its
results must equal those of qec_decode_batch, call after call, since every call
reuses the same scratch.  This file sorts last so that a run stopping at the
first failure has already run every other test.
"""

import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

from synth import mixed_batch, pack_defects, rotated_surface_code, sample_shots

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_12262_gb300 import build
    build.build()
    import paper_2609_12262_gb300 as q
    q.lib()
    return q


def _run(q, fn, graphs, syn, gid, offs, S):
    import torch
    out = (torch.empty(S, dtype=torch.int64, device="cuda"), torch.empty(S, dtype=torch.int64, device="cuda"),
           torch.empty(S, dtype=torch.int32, device="cuda"))
    fn(graphs, syn, gid, offs, num_shots=S, out=out)
    torch.cuda.synchronize()
    return out[1].cpu().numpy(), q.to_uint64(out[0]), out[2].cpu().numpy()


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_static_matches_workspace_decoder_twice(qd):
    import torch
    graphs, gid, offs, syn = mixed_batch([5, 7, 9, 11, 13], 400, 0.004, seed=77)
    gg = [qd.Graph.from_phys(g) for g in graphs]
    t_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    t_gid = torch.from_numpy(gid.astype(np.int32)).cuda()
    t_off = torch.from_numpy(offs.astype(np.int64)).cuda()
    S = gid.shape[0]
    ref = _run(qd, qd.decode_batch, gg, t_syn, t_gid, t_off, S)
    first = _run(qd, qd.decode_batch_static, gg, t_syn, t_gid, t_off, S)
    second = _run(qd, qd.decode_batch_static, gg, t_syn, t_gid, t_off, S)
    assert np.all(ref[2] == 0)
    assert _same(first, ref)
    assert _same(second, ref)


def test_static_single_graph_default_layout(qd):
    import torch
    pg = rotated_surface_code(5, 5, 0.005)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, 3000, 8)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    ref = _run(qd, qd.decode_batch, [g], t, None, None, 3000)
    for _ in range(2):
        assert _same(_run(qd, qd.decode_batch_static, [g], t, None, None, 3000), ref)


def test_static_capacity_and_limits(qd):
    import torch
    pg = rotated_surface_code(7, 7, 0.003)
    g = qd.Graph.from_phys(pg)
    n = pg.num_detectors          # 192 > 128 detection events when every bit is set
    rows = np.stack([pack_defects(list(range(n)), n), pack_defects([3, 4], n), pack_defects([], n)])
    t = torch.from_numpy(rows.view(np.int32).reshape(-1)).cuda()
    ref = _run(qd, qd.decode_batch, [g], t, None, None, 3)
    got = _run(qd, qd.decode_batch_static, [g], t, None, None, 3)
    assert got[2][0] == qd.SHOT_CAPACITY and ref[2][0] == qd.SHOT_OK
    assert _same([x[1:] for x in got], [x[1:] for x in ref])
    # more shots than the static overflow list holds: rejected before any launch
    L = qd.lib()
    arr = (C.c_void_p * 1)(g.handle.value)
    small = torch.zeros(8, dtype=torch.int64, device="cuda")
    rc = L.qec_decode_batch_static(arr, 1, None, None, C.c_void_p(t.data_ptr()), (1 << 20) + 1,
                                   C.c_void_p(small.data_ptr()), C.c_void_p(small.data_ptr()),
                                   C.c_void_p(small.data_ptr()), None)
    assert rc == qd.QEC_ERANGE
    assert "QEC_STATIC_MAX_SHOTS" in qd.last_error()


_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2609_12262_gb300 as q
from synth import mixed_batch
from tests.oracle_pool import oracle_decode
graphs, gid, offs, syn = mixed_batch([5, 9, 13], 300, 0.004, seed=91)
gg = [q.Graph.from_phys(g) for g in graphs]
S = gid.shape[0]
t_syn = torch.from_numpy(syn.view(np.int32)).cuda()
t_gid = torch.from_numpy(gid.astype(np.int32)).cuda()
t_off = torch.from_numpy(offs.astype(np.int64)).cuda()
out = (torch.empty(S, dtype=torch.int64, device="cuda"), torch.empty(S, dtype=torch.int64, device="cuda"),
       torch.empty(S, dtype=torch.int32, device="cuda"))
side = torch.cuda.Stream()
# the first decode of this process goes through the static entry point
q.decode_batch_static(gg, t_syn, t_gid, t_off, num_shots=S, out=out, stream=side)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
res = []
for i in range(3):
    q.decode_batch_static(gg, t_syn, t_gid, t_off, num_shots=S, out=out, stream=side if i % 2 else None)
    torch.cuda.synchronize()
    res.append((out[1].cpu().numpy().copy(), q.to_uint64(out[0]).copy(), out[2].cpu().numpy().copy()))
free1 = torch.cuda.mem_get_info()[0]
rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in range(S)]
ref = oracle_decode(graphs, gid, rows, workers=1)
same = all(all(np.array_equal(a, b) for a, b in zip(r, ref)) for r in res)
print("RESULT", free0 - free1, int(same), int(np.count_nonzero(ref[2])))
"""


def test_static_allocates_nothing_and_matches_oracle_in_a_fresh_process():
    """In a fresh process whose first decode is the static entry point: free
    device memory is unchanged over three more calls (one on a non-default
    stream), and every call equals the oracle shot by shot."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CHILD, root], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT")][-1].split()
    grew, same, bad = int(line[1]), int(line[2]), int(line[3])
    assert grew == 0, "device memory changed by %d bytes" % grew
    assert same == 1 and bad == 0
