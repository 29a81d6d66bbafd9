"""Replica (shot-sharded) multi-GPU path, exercised on CPU with two gloo ranks:
shards cover every shot exactly once, each rank decodes only its own shots, and
the job time is the maximum over ranks.  The per-rank decode here is the CPU
oracle standing in for a GPU (the sharding and timing logic are the subject)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_12262_gb300 import replicas


def test_shard_covers_every_unit_once():
    for n in (0, 1, 7, 1000, 1000001):
        for ws in (1, 2, 3, 8):
            got = [replicas.shard(n, ws, r) for r in range(ws)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(got[i][1] == got[i + 1][0] for i in range(ws - 1))
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world_size, port, out_dir):
    import torch.distributed as dist
    from oracle import OracleGraph
    from synth import rotated_surface_code, sample_shots
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world_size), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    ws, r, _ = replicas.world()
    pg = rotated_surface_code(5, 5, 0.01)
    syn, _ = sample_shots(pg, 64, 5)
    b, e = replicas.shard(syn.shape[0], ws, r)
    og = OracleGraph.from_phys(pg)
    w, o, st = og.decode_bitmaps(syn[b:e], "hier")
    elapsed = 1.0 + r                       # rank r "took" 1 + r seconds
    t_max = replicas.max_over_ranks(elapsed)
    dist.barrier()
    np.savez(os.path.join(out_dir, "rank%d.npz" % r), b=b, e=e, w=w, o=o, st=st, t=t_max)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_time(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    parts = [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(2)]
    assert int(parts[0]["b"]) == 0 and int(parts[0]["e"]) == int(parts[1]["b"]) and int(parts[1]["e"]) == 64
    assert all(float(p["t"]) == 2.0 for p in parts)     # maximum over ranks
    from oracle import OracleGraph
    from synth import rotated_surface_code, sample_shots
    pg = rotated_surface_code(5, 5, 0.01)
    syn, _ = sample_shots(pg, 64, 5)
    w, o, st = OracleGraph.from_phys(pg).decode_bitmaps(syn, "hier")
    assert np.array_equal(np.concatenate([p["w"] for p in parts]), w)
    assert np.array_equal(np.concatenate([p["o"] for p in parts]), o)
