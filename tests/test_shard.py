"""Multi-GPU sharding logic on the CPU: shard plans cover every (ligand, pocket) pair exactly once,
and a 2-rank gloo gather + merge equals merging everything in one process; the pocket side's
receptor plan covers every receptor once and its 2-rank gather is the union of the ranks' parts."""
import os
import socket

import pytest

from paper_2506_20043_gb300 import shard


@pytest.mark.parametrize("world,n_pockets,n_ligs", [(1, 10, 1), (2, 10, 1), (4, 3, 5), (8, 2, 7), (3, 5, 3)])
def test_plan_covers_every_pair_once(world, n_pockets, n_ligs):
    plan = shard.plan_shards(list(range(100, 100 + n_pockets)), n_ligs, world)
    assert len(plan) == world
    seen = {}
    for r, (pockets, ligs) in enumerate(plan):
        for p in pockets:
            for l in ligs:
                assert (l, p) not in seen
                seen[(l, p)] = r
    assert set(seen) == {(l, p) for l in range(n_ligs) for p in range(100, 100 + n_pockets)}
    # a pocket's maps live on as few ranks as the split allows
    if world <= n_pockets:
        owners = {}
        for r, (pockets, _) in enumerate(plan):
            for p in pockets:
                owners.setdefault(p, set()).add(r)
        assert all(len(v) == 1 for v in owners.values())


@pytest.mark.parametrize("world,n_pockets,n_ligs", [(1, 10, 1), (2, 10, 1), (4, 10, 4), (8, 10, 8), (3, 5, 3),
                                                    (8, 2, 3)])
def test_pair_plan_is_balanced_and_keeps_pair_keys(world, n_pockets, n_ligs):
    pockets = list(range(50, 50 + n_pockets))
    plan = shard.plan_pairs(pockets, n_ligs, world)
    assert len(plan) == world
    flat = [p for part in plan for p in part]
    # every pair once, with the key it has in one unsplit dock (ligand * n_pockets + position)
    assert sorted(flat) == sorted((l, pockets[k], l * n_pockets + k) for l in range(n_ligs) for k in range(n_pockets))
    sizes = [len(part) for part in plan]
    assert max(sizes) - min(sizes) <= 1
    # runs are contiguous in pocket-major order, so a pocket spans consecutive ranks only
    owners = {}
    for r, part in enumerate(plan):
        for _, p, _ in part:
            owners.setdefault(p, set()).add(r)
    for rs in owners.values():
        assert sorted(rs) == list(range(min(rs), max(rs) + 1))


def test_merge_orders_by_score_pocket_chain():
    a = {0: [(-7.0, 3, 1), (-5.0, 3, 4)], 1: [(-2.0, 0, 0)]}
    b = {0: [(-7.0, 1, 9), (-8.0, 2, 2)]}
    m = shard.merge_records([a, b])
    assert m[0] == [(-8.0, 2, 2), (-7.0, 1, 9), (-7.0, 3, 1), (-5.0, 3, 4)]
    assert m[1] == [(-2.0, 0, 0)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, parts, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = shard.gather_merge(parts[rank])
    if rank == 0:
        import json
        with open(out_path, "w") as f:
            json.dump({str(k): v for k, v in res.items()}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_rank_gather_merge(tmp_path):
    torch = pytest.importorskip("torch")
    import json
    import torch.multiprocessing as mp
    parts = [{0: [(-6.0, 0, 3), (-4.5, 1, 0)], 2: [(-1.0, 1, 2)]},
             {0: [(-6.5, 5, 1)], 1: [(-3.0, 4, 4), (-3.5, 5, 0)]}]
    out = str(tmp_path / "merged.json")
    mp.start_processes(_worker, args=(2, _free_port(), parts, out), nprocs=2, join=True, start_method="spawn")
    got = {int(k): [tuple(r) for r in v] for k, v in json.load(open(out)).items()}
    assert got == shard.merge_records(parts)


@pytest.mark.parametrize("n,world", [(0, 2), (1, 4), (7, 2), (16, 8), (5, 1)])
def test_receptor_plan_covers_each_once(n, world):
    plan = shard.plan_receptors(n, world)
    assert len(plan) == world
    flat = sorted(r for part in plan for r in part)
    assert flat == list(range(n))
    assert max(len(p) for p in plan) - min(len(p) for p in plan) <= 1


def _pocket_worker(rank, world, port, parts, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = shard.gather_pockets(parts[rank])
    if rank == 0:
        import json
        with open(out_path, "w") as f:
            json.dump({str(k): v for k, v in res.items()}, f)
    else:
        assert res is None
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_rank_gather_pockets(tmp_path):
    pytest.importorskip("torch")
    import json
    import torch.multiprocessing as mp
    plan = shard.plan_receptors(5, 2)
    parts = [{r: [(12.5 - r, 1.0 * r, 2.0, -3.0, 40 + r), (3.0, 0.0, 0.0, 0.0, 9)] for r in plan[k]} for k in range(2)]
    out = str(tmp_path / "pockets.json")
    mp.start_processes(_pocket_worker, args=(2, _free_port(), parts, out), nprocs=2, join=True, start_method="spawn")
    got = {int(k): [tuple(p) for p in v] for k, v in json.load(open(out)).items()}
    want = {r: parts[r % 2][r] for r in range(5)}
    assert list(got) == list(range(5)) and got == want


def test_pockets_from_clusters_keeps_rank_order():
    import numpy as np

    class _Clusters:                        # the shape of Clusters.read()
        def read(self):
            return {"score": np.array([9.0, 4.0], np.float32),
                    "center": np.array([[1, 2, 3], [4, 5, 6]], np.float32),
                    "size": np.array([30, 12], np.int32), "first": np.array([5, 0], np.int32),
                    "cluster": np.array([1, 0, 0], np.int32)}

    assert shard.pockets_from_clusters(_Clusters()) == [(9.0, 1.0, 2.0, 3.0, 30), (4.0, 4.0, 5.0, 6.0, 12)]
