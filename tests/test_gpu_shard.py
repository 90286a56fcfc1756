"""A job split into shards (as over several GPUs, one process each), docked here one shard after the
other on one GPU with the job's pair keys and merged on the host, equals the unsplit dock exactly:
the same kept poses per pair and the same per-ligand ranking (score, pocket, chain). Also the
top-ranked-pocket cut (max_pockets) at the boundary."""
import numpy as np
import pytest

import oracle as O
import pvsynth as S
from paper_2506_20043_gb300 import shard
from tests import _gpu as G

pytestmark = pytest.mark.gpu

# one team width for every call: it fixes the order of the floating-point sums
FIXED = dict(search_variant=0, warps_per_cta=2)


@pytest.fixture(scope="module")
def job():
    ctx = G.context()
    rec0, boxes0 = S._carved(3000, 5, (6.0, 8.0), 4, 14.0)
    rec = G.receptor32(rec0)
    boxes = [G.box32(b) for b in boxes0]
    ligs = [G.ligand32(S.ligand_centered(S.make_ligand(n, r, 40 + i)))
            for i, (n, r) in enumerate([(12, 2), (16, 3), (20, 4), (14, 3)])]
    Ls = [O.OracleLigand(l) for l in ligs]
    types = sorted(set(np.concatenate([L.xs for L in Ls]).tolist()))
    gs = ctx.build_grids(rec, boxes, types)
    pls = [ctx.ligand(l) for l in ligs]
    return ctx, gs, pls, rec, boxes, types


def _records(r, ligand_ids):
    return shard.records_from_result(r, ligand_ids)


def test_sharded_job_equals_unsharded(job):
    ctx, gs, pls, rec, boxes, types = job
    pockets = [3, 0, 4, 1, 2]                # any pocket order
    kw = dict(chains=32, steps=40, seed=17, top_k=4, **FIXED)
    whole = ctx.dock(gs, pls, pockets, **kw)
    ref = _records(whole, range(len(pls)))
    for world in (2, 3, 4):
        # pockets first, then ligands (plan_shards): each shard docks its ligands x pockets
        parts = []
        for my_pockets, my_ligs in shard.plan_shards(pockets, len(pls), world):
            if not my_pockets or not my_ligs:
                continue
            keys = [li * len(pockets) + pockets.index(p) for li in my_ligs for p in my_pockets]
            r = ctx.dock(gs, [pls[i] for i in my_ligs], my_pockets, pair_keys=keys, **kw)
            parts.append(_records(r, my_ligs))
        assert shard.merge_records(parts) == ref, ("plan_shards", world)
        # balanced contiguous runs of pairs (plan_pairs): each shard is a pair list
        parts = []
        for run in shard.plan_pairs(pockets, len(pls), world):
            ligs_here = sorted({l for l, _, _ in run})
            local = {l: i for i, l in enumerate(ligs_here)}
            r = ctx.dock_pairs(gs, [pls[l] for l in ligs_here], [local[l] for l, _, _ in run], [p for _, p, _ in run],
                               pair_keys=[k for _, _, k in run], **kw)
            parts.append(_records(r, ligs_here))
        assert shard.merge_records(parts) == ref, ("plan_pairs", world)


def test_max_pockets_takes_the_first_pockets_of_the_callers_order(job):
    """max_pockets = 2 over pockets listed [4, 1, 3, 0]: the same result, bit for bit, as docking
    into [4, 1] only (pairs indexed after the cut), and the merged ranking equals the oracle's merge
    (Algorithm 3: by SF, ties by pocket and chain) of the kept poses of those two pockets."""
    ctx, gs, pls, rec, boxes, types = job
    kw = dict(chains=32, steps=40, seed=23, top_k=4, **FIXED)
    cut = ctx.dock(gs, pls[:2], [4, 1, 3, 0], max_pockets=2, **kw)
    direct = ctx.dock(gs, pls[:2], [4, 1], **kw)
    assert cut.n_pairs == 4
    np.testing.assert_array_equal(cut.chain_records()[1], direct.chain_records()[1])
    assert (cut.poses == direct.poses).all()
    assert set(cut.poses["pocket"][cut.poses["pair"] >= 0].tolist()) <= {4, 1}
    for li in range(2):
        results = []
        for k, p in enumerate([4, 1]):
            q = li * 2 + k
            n = int(cut.n_kept[q])
            results.append(O.PairResult(li, p, None, None, 0, cut.poses[q]["chain"][:n],
                                        cut.poses[q]["score"][:n].astype(np.float64), None, None, None))
        flat = cut.poses.reshape(-1)
        got = [(int(flat[i]["pocket"]), int(flat[i]["chain"])) for i in cut.ranking(li)]
        assert got == [(m[1], m[2]) for m in O.merge_pockets(results)]
    # the same cut through the pair list: each ligand's first two distinct pockets in list order
    pl = [0, 1, 0, 0, 1, 1, 0]
    pp = [4, 3, 1, 3, 0, 2, 4]
    r = ctx.dock_pairs(gs, pls[:2], pl, pp, max_pockets=2, **kw)
    assert r.n_pairs == 5                      # (0,4) (1,3) (0,1) (1,0) (0,4) kept; (0,3) (1,2) cut
    assert [int(x) for x in r.poses["pocket"][:, 0]] == [4, 3, 1, 0, 4]
    # the binding's top-pocket helper is the same cut
    top = ctx.dock_top_pockets(gs, pls[:2], [4, 1, 3, 0], max_pockets=2, **kw)
    assert (top.poses == direct.poses).all()
