"""World-size-2 gloo test of the multi-rank host path on CPU: disjoint voxel
shards per rank (uids and seeds), each rank's work checked on the oracle,
and the max-over-ranks of the timed region."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as tmp

import oracle
import synth
from paper_2604_24091_gb300 import shard as S


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    base = [synth.VoxelDesc(4, 1, (0.05, 0.0, 0.0), 563.0, 0, 0, seed=0, uid=u) for u in range(3)]
    mine = S.rank_descs(base, rank, lambda uid: synth.splitmix64(77, uid))
    model = synth.default_model()
    events = 0
    for d in mine:
        v = oracle.Voxel(d, model)
        v.step(200)
        events += v.state()["n_events"]
    t = S.max_over_ranks(1.0 + rank, dist)
    out[rank] = ([d.uid for d in mine], [d.seed for d in mine], events, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    (u0, s0, e0, t0), (u1, s1, e1, t1) = out[0], out[1]
    assert u0 == [0, 1, 2] and u1 == [3, 4, 5]
    assert not set(s0) & set(s1)
    assert e0 == e1 == 600
    assert t0 == t1 == 2.0
    assert S.max_over_ranks(3.5) == 3.5
