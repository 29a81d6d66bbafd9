"""Decoding recorded into CUDA graphs: a batched decode and a whole
sliding-window decode are captured once and replayed on new syndromes written
into the same input tensor; every replay equals the uncaptured decode and the
oracle, shot by shot.  Needs a GB300."""

import numpy as np
import pytest

from synth import mixed_batch, rotated_surface_code, sample_shots
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


def test_captured_batch_decode_replays(qd):
    import torch
    graphs, gid, offs, syn = mixed_batch([7, 11, 15], 300, 0.004, seed=51)
    _, _, _, syn2 = mixed_batch([7, 11, 15], 300, 0.004, seed=52)   # same layout, other syndromes
    gg = [qd.Graph.from_phys(g) for g in graphs]
    S = gid.shape[0]
    t_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    t_gid = torch.from_numpy(gid.astype(np.int32)).cuda()
    t_off = torch.from_numpy(offs.astype(np.int64)).cuda()
    out = (torch.empty(S, dtype=torch.int64, device="cuda"), torch.empty(S, dtype=torch.int64, device="cuda"),
           torch.empty(S, dtype=torch.int32, device="cuda"))
    qd.decode_batch(gg, t_syn, t_gid, t_off, num_shots=S, out=out)   # sizes the workspace
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        qd.decode_batch(gg, t_syn, t_gid, t_off, num_shots=S, out=out)
    for host in (syn2, syn, syn2):
        t_syn.copy_(torch.from_numpy(host.view(np.int32)))
        for o in out:
            o.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        got = (out[1].cpu().numpy(), qd.to_uint64(out[0]), out[2].cpu().numpy())
        rows = [host[offs[s]:offs[s] + graphs[gid[s]].words] for s in range(S)]
        ref = oracle_decode(graphs, gid, rows)
        assert all(np.array_equal(a, b) for a, b in zip(got, ref))


def test_capture_needs_a_prior_call_of_the_same_shape(qd):
    import torch
    qd.release_workspace()
    pg = rotated_surface_code(9, 9, 0.003)
    g = qd.Graph.from_phys(pg)
    syn, _ = sample_shots(pg, 64, 5)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    out = (torch.empty(64, dtype=torch.int64, device="cuda"), torch.empty(64, dtype=torch.int64, device="cuda"),
           torch.empty(64, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with pytest.raises(qd.QecError):
        with torch.cuda.graph(cg):
            qd.decode_batch([g], t, num_shots=64, out=out)
    torch.cuda.synchronize()
    qd.decode_batch([g], t, num_shots=64, out=out)   # the device is fine afterwards
    torch.cuda.synchronize()
    ref = oracle_decode([pg], np.zeros(64, np.int32), list(syn))
    assert np.array_equal(out[1].cpu().numpy(), ref[0]) and np.array_equal(out[2].cpu().numpy(), ref[2])


def test_captured_sliding_window_decode_replays(qd):
    import torch
    from oracle.window import sliding_window_decode
    from paper_2609_12262_gb300.window import SlidingWindow
    pg = rotated_surface_code(7, 35, 0.005)
    S = 80
    syn, _ = sample_shots(pg, S, 61)
    syn2, _ = sample_shots(pg, S, 62)
    dec = SlidingWindow(qd.Graph.from_phys(pg), pg.nz, 14, 7)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    cg, obs, st = dec.graph(t, S)
    for host in (syn2, syn):
        t.copy_(torch.from_numpy(host.view(np.int32).reshape(-1)))
        cg.replay()
        torch.cuda.synchronize()
        ro, rs = sliding_window_decode(pg, host, 14, 7)
        assert not rs.any()
        assert np.array_equal(qd.to_uint64(obs), ro) and np.array_equal(st.cpu().numpy(), rs)
