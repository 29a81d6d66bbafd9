"""Serving (qec_stream_*): continuous batching returns, for every window, the
same result as decoding it alone, and the same as qec_decode_batch and the
oracle.  Needs a GB300."""

import numpy as np
import pytest

from synth import mixed_batch
from tests.oracle_pool import oracle_decode

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


def _collect(st, n_expected, by_id):
    while len(by_id) < n_expected:
        r = st.poll()
        for x in r:
            by_id[int(x["request_id"])] = (int(x["weight"]), int(x["obs"]), int(x["status"]))
        if not len(r):
            st.flush()


def test_alone_equals_mix_equals_batch_and_oracle(qd):
    import torch
    graphs, gid, offs, syn = mixed_batch([9, 13, 17, 21, 25], 300, 0.003, seed=41)
    gg = [qd.Graph.from_phys(g) for g in graphs]
    S = gid.shape[0]
    st = qd.Stream(device_budget_bytes=4 << 30, max_inflight=4096)
    try:
        # alone: one window in flight at a time
        alone = {}
        for s in range(60):
            assert st.submit(gg[gid[s]], syn[offs[s]:offs[s] + graphs[gid[s]].words], s)
            st.flush()
            _collect(st, s + 1, alone)
        # in the mix: every window submitted as fast as admission allows
        mix = {}
        i = 0
        while i < S:
            k = st.submit_many(gg, gid[i:], offs[i:], syn, np.arange(i, S, dtype=np.uint64) + 100000)
            i += k
            for x in st.poll():
                mix[int(x["request_id"]) - 100000] = (int(x["weight"]), int(x["obs"]), int(x["status"]))
        st.flush()
        for x in st.poll():
            mix[int(x["request_id"]) - 100000] = (int(x["weight"]), int(x["obs"]), int(x["status"]))
    finally:
        st.close()
    assert len(mix) == S
    for s in range(60):
        assert alone[s] == mix[s]
    t_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    o, w, stt = qd.decode_batch(gg, t_syn, torch.from_numpy(gid.astype(np.int32)).cuda(),
                                torch.from_numpy(offs.astype(np.int64)).cuda())
    torch.cuda.synchronize()
    bw, bo, bs = w.cpu().numpy(), qd.to_uint64(o), stt.cpu().numpy()
    for s in range(S):
        assert mix[s] == (int(bw[s]), int(bo[s]), int(bs[s])), s
    rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in range(S)]
    rw, ro, rs = oracle_decode(graphs, gid, rows)
    assert np.array_equal(rw, bw) and np.array_equal(ro, bo) and np.array_equal(rs, bs)


def test_admission_and_errors(qd):
    graphs, gid, offs, syn = mixed_batch([9], 50, 0.003, seed=42)
    g = qd.Graph.from_phys(graphs[0])
    st = qd.Stream(device_budget_bytes=4 << 30, max_inflight=8)
    try:
        taken = st.submit_many([g], gid, offs, syn, np.arange(50, dtype=np.uint64))
        assert 1 <= taken <= 8          # admission bounded by max_inflight
        st.flush()
        r = st.poll()
        assert len(r) == taken and np.all(r["status"] == 0)
        assert np.all(r["t_done_ns"] >= r["t_submit_ns"])
    finally:
        st.close()
    with pytest.raises(qd.QecError):
        qd.Stream(device_budget_bytes=1 << 20, max_inflight=8)   # budget below two slots
