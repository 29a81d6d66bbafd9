"""Circuit-level detector graphs (synth/circuit.py) on the GPU: results and
parallel-event-count diagnostics equal the oracle's, bit-exact.  Needs a
GB300."""

import numpy as np
import pytest

from oracle import OracleGraph
from synth import rotated_surface_code_circuit, sample_shots, unpack_defects
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


CASES = [(3, 0.005, "uniform", 4000), (5, 0.003, "uniform", 2000), (7, 0.002, "uniform", 1000),
         (9, 0.001, "uniform", 800), (5, 0.008, "uniform", 800), (13, 0.003, "uniform", 150),
         (5, 0.006, "physical", 2000), (9, 0.002, "physical", 600)]


@pytest.mark.parametrize("d,p,noise,shots", CASES, ids=["%s_d%d_p%g" % (c[2], c[0], c[1]) for c in CASES])
def test_circuit_level_matches_oracle(qd, d, p, noise, shots):
    import torch
    g = rotated_surface_code_circuit(d, d, p, noise)
    qg = qd.Graph.from_phys(g)
    syn, _ = sample_shots(g, shots, 31)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    o, w, s = qd.decode_batch([qg], t)
    torch.cuda.synchronize()
    rw, ro, rs = oracle_decode([g], np.zeros(shots, np.int32), list(syn))
    assert not rs.any()
    gw, go, gs = w.cpu().numpy(), qd.to_uint64(o), s.cpu().numpy()
    bad = np.nonzero((gw != rw) | (go != ro) | (gs != rs))[0]
    assert bad.size == 0, (d, p, bad[:5].tolist())


def test_circuit_level_diagnostics(qd):
    import torch
    g = rotated_surface_code_circuit(7, 7, 0.003)
    qg = qd.Graph.from_phys(g)
    og = OracleGraph.from_phys(g)
    syn, _ = sample_shots(g, 300, 32)
    t = torch.from_numpy(syn.view(np.int32).reshape(-1)).cuda()
    for mode in ("hier", "global"):
        o, w, s, dg = qd.decode_batch_ex([qg], t, mode=mode)
        torch.cuda.synchronize()
        D = dg.cpu().numpy()
        W, O, S = w.cpu().numpy(), qd.to_uint64(o), s.cpu().numpy()
        multi = 0
        for i in range(300):
            r = og.diag(unpack_defects(syn[i], g.num_detectors), mode)
            assert (int(W[i]), int(O[i]), int(S[i])) == (r["weight"], r["obs"], r["status"]), (mode, i)
            if r["clusters_above_l1"] > 1:
                multi += 1
                continue
            got = (int(D[i, 0]), int(D[i, 1]), int(D[i, 2]), int(D[i, 3]), int(D[i, 4]), int(D[i, 7]))
            exp = (r["e_ideal"], r["t_ideal"], r["events"], r["l1_clusters"], r["l1_defects"], r["defects"])
            assert got == exp, (mode, i, got, exp)
        assert multi == 0
    assert qg.info.upper_single_cluster == 1
