"""Multi-rank path on CPU: two gloo ranks shard the replica ids and run their share
(the FP64 oracle stands in for the per-rank GPU work); the union equals one process
running every replica, bit for bit, because the noise is keyed by the global replica
id; the timing reduction takes the maximum over ranks."""
import os
import pickle
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

KT = 2.494
PER_RANK = 2
STEPS = 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(ids):
    import oracle
    import synth
    c = synth.make_chain(1, seed=1)
    ff = oracle.ForceField.from_chain(c)
    R = len(ids)
    x0 = np.stack([c.x_unfolded] * R)
    v0 = np.stack([c.velocities(1, KT, 100 + int(i))[0] for i in ids])
    out = oracle.run_baoab(ff, None, x0, v0, [0.0] * R, [0] * R, ids, 77, 0.002, 1.0, KT, STEPS)
    return out["x"]


def _worker(rank, world, port, path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1705_02180_gb300.replicas import max_over_ranks, replica_ids
    ids = replica_ids(rank, world, PER_RANK)
    x = _run(ids)
    parts = [None] * world
    dist.all_gather_object(parts, (ids.tolist(), x))
    slowest = max_over_ranks(0.5 + rank, dist)
    if rank == 0:
        with open(path, "wb") as f:
            pickle.dump((parts, slowest), f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_replicas(tmp_path):
    world = 2
    path = str(tmp_path / "out.pkl")
    mp.start_processes(_worker, args=(world, _free_port(), path), nprocs=world, join=True,
                       start_method="spawn")
    with open(path, "rb") as f:
        parts, slowest = pickle.load(f)
    assert slowest == 1.5
    ids = [i for p in parts for i in p[0]]
    assert ids == list(range(world * PER_RANK))
    x_sharded = np.concatenate([p[1] for p in parts])
    x_single = _run(np.arange(world * PER_RANK))
    assert np.array_equal(x_sharded, x_single)


def test_replica_ids_are_disjoint_ranges():
    from paper_1705_02180_gb300.replicas import replica_ids
    got = [replica_ids(r, 4, 3) for r in range(4)]
    assert np.array_equal(np.concatenate(got), np.arange(12))
    with pytest.raises(ValueError):
        replica_ids(4, 4, 3)
