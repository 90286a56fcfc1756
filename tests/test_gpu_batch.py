"""GPU parity of batched docking over uneven ligands and several receptors (the uneven-batch and
screening shapes): ligands of 10-60 atoms and 0-15 torsions mixed in one persistent launch, and
receptors appended into one grid set docked through an explicit pair list.

Checked against the FP64 oracle: every chain best is what the oracle scores for that pose, the
per-pair selection equals the oracle's selection of the GPU's chain bests, the random starts equal
the oracle's, and results are bitwise identical across launch shapes.
"""
import numpy as np
import pytest

import oracle as O
import pvsynth as S
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _uneven(n_ligs=12, seed=5):
    rng = np.random.default_rng(seed)
    ligs = []
    for i in range(n_ligs):
        n = int(rng.integers(10, 61))
        k = int(rng.integers(0, 16))
        ligs.append(G.ligand32(S.ligand_centered(S.make_ligand(n, k, 1000 + i))))
    ligs[0] = G.ligand32(S.ligand_centered(S.make_ligand(60, 15, 77)))    # the largest shape
    ligs[1] = G.ligand32(S.ligand_centered(S.make_ligand(10, 0, 78)))     # a rigid one
    return ligs


def _coords(ctx, r, pls, Ls, pair_lig):
    """Per pair: the GPU's and the oracle's atom coordinates of every chain best."""
    pots, _ = r.chain_records()
    out = []
    for q in range(r.n_pairs):
        L = Ls[pair_lig[q]]
        p = pots[q, :, :L.n_pot]
        out.append((G.pose_coords(ctx, pls[pair_lig[q]], p), np.stack([L.fk(x) for x in p.astype(np.float64)])))
    return out


def _lazy_grids(rec_of_box, boxes, coords, pair_box):
    """Oracle maps filled at the cells that either side's coordinates touch."""
    ogs = []
    for b in range(len(boxes)):
        xyz = np.concatenate([np.concatenate([g, o]).reshape(-1, 3) for q, (g, o) in enumerate(coords) if pair_box[q] == b])
        rec = rec_of_box(b)
        ogs.append(O.OracleGrid.lazy(rec, boxes[b], list(range(11)), O.xs_type_receptor(rec), xyz, threads=G.threads()))
    return ogs


def _check_pairs(r, Ls, ogs, coords, pair_lig, pair_box, sites):
    """Every chain best is what the oracle scores for that pose, and the per-pair selection is the
    oracle's selection of the GPU's chain bests."""
    pots, es = r.chain_records()
    for q in range(r.n_pairs):
        L, og = Ls[pair_lig[q]], ogs[pair_box[q]]
        xyz_gpu, xyz_ref = coords[q]
        G.check_pose_scores(L, og, pots[q, :, :L.n_pot], es[q], xyz_gpu, sites[pair_box[q]])
        kept = O.topk(es[q].astype(np.float64), xyz_ref, r.top_k, 1.0)
        assert list(r.poses[q]["chain"][:r.n_kept[q]]) == list(kept), q
    return pots, es


def test_uneven_ligands_in_one_launch():
    ctx = G.context()
    rec0, boxes0 = S._carved(4000, 2, (7.0, 8.0), 11, 16.0)
    rec, boxes = G.receptor32(rec0), [G.box32(b) for b in boxes0]
    ligs = _uneven()
    Ls = [O.OracleLigand(l) for l in ligs]
    gs = ctx.build_grids(rec, boxes, list(range(11)))
    pls = [ctx.ligand(l) for l in ligs]
    chains, steps = 12, 25
    r = ctx.dock(gs, pls, [0, 1], chains=chains, steps=steps, seed=4, top_k=5)
    _, _, st = r.stats()
    assert (st == 0).all()
    pots, es = r.chain_records()
    n_pairs = len(ligs) * 2
    pair_lig = [q // 2 for q in range(n_pairs)]
    pair_box = [q % 2 for q in range(n_pairs)]
    coords = _coords(ctx, r, pls, Ls, pair_lig)
    ogs = _lazy_grids(lambda b: rec, boxes, coords, pair_box)
    sites = [(rec, O.xs_type_receptor(rec), b) for b in boxes]
    _check_pairs(r, Ls, ogs, coords, pair_lig, pair_box, sites)
    # random starts of the largest ligand equal the oracle's
    r0 = ctx.dock(gs, pls, [0, 1], chains=chains, steps=0, seed=4, top_k=5)
    p0, _ = r0.chain_records()
    for c in range(chains):
        ref = O.random_conformation(Ls[0], boxes[1], 4, 1, c)
        np.testing.assert_allclose(p0[1, c, :Ls[0].n_pot], ref, atol=2e-5)
    # bitwise identical across launch shapes (each candidate of the autotuner)
    base_p, base_e = pots, es
    for v, w in ((0, 8), (1, 4), (3, 4)):
        rv = ctx.dock(gs, pls, [0, 1], chains=chains, steps=steps, seed=4, top_k=5, search_variant=v, warps_per_cta=w)
        pv_, ev_ = rv.chain_records()
        np.testing.assert_array_equal(ev_, base_e)
        np.testing.assert_array_equal(pv_, base_p)
    # per-ligand merged ranking covers both pockets' kept poses, best first
    for li in range(len(ligs)):
        rank = r.ranking(li)
        flat = r.poses.reshape(-1)
        assert len(rank) == r.n_kept[2 * li] + r.n_kept[2 * li + 1]
        sc = [flat[i]["score"] for i in rank]
        assert sc == sorted(sc)


def test_uneven_small_ligands_with_half_warp_teams():
    """Ligands of 8-32 atoms and 0-10 torsions (all fit a half-warp team) in one launch with
    half-warp teams: chain bests are what the oracle scores, the selection is the oracle's, and
    the four half-warp register variants agree bitwise."""
    ctx = G.context()
    rec0, boxes0 = S._carved(3000, 2, (6.5, 7.5), 31, 14.0)
    rec, boxes = G.receptor32(rec0), [G.box32(b) for b in boxes0]
    rng = np.random.default_rng(8)
    ligs = [G.ligand32(S.ligand_centered(S.make_ligand(int(rng.integers(8, 33)), int(rng.integers(0, 11)), 500 + i)))
            for i in range(8)]
    ligs[0] = G.ligand32(S.ligand_centered(S.make_ligand(32, 10, 90)))   # the largest that fits
    Ls = [O.OracleLigand(l) for l in ligs]
    gs = ctx.build_grids(rec, boxes, list(range(11)))
    pls = [ctx.ligand(l) for l in ligs]
    chains, steps = 10, 25
    r = ctx.dock(gs, pls, [0, 1], chains=chains, steps=steps, seed=12, top_k=4, search_variant=6, warps_per_cta=4)
    _, _, st = r.stats()
    assert (st == 0).all()
    pots, es = r.chain_records()
    n_pairs = len(ligs) * 2
    pair_lig = [q // 2 for q in range(n_pairs)]
    pair_box = [q % 2 for q in range(n_pairs)]
    coords = _coords(ctx, r, pls, Ls, pair_lig)
    ogs = _lazy_grids(lambda b: rec, boxes, coords, pair_box)
    sites = [(rec, O.xs_type_receptor(rec), b) for b in boxes]
    _check_pairs(r, Ls, ogs, coords, pair_lig, pair_box, sites)
    for v, w in ((4, 8), (5, 4), (7, 4)):
        rv = ctx.dock(gs, pls, [0, 1], chains=chains, steps=steps, seed=12, top_k=4, search_variant=v, warps_per_cta=w)
        pv_, ev_ = rv.chain_records()
        np.testing.assert_array_equal(ev_, es)
        np.testing.assert_array_equal(pv_, pots)


def test_appended_receptors_and_pair_list():
    """Three receptors appended into one grid set; each receptor's two ligands docked into its own
    three pockets through one pair list (the screening shape)."""
    ctx = G.context()
    gs = None
    boxes, recs, Ls, ligs = [], [], [], []
    pair_lig, pair_pocket, pair_box = [], [], []
    for k in range(3):
        rec0, bx0 = S._carved(int(1500 + 700 * k), 3, (6.0, 7.0), 20 + k, 12.0)
        rec, bx = G.receptor32(rec0), [G.box32(b) for b in bx0]
        if gs is None:
            gs = ctx.build_grids(rec, bx, list(range(11)))
            first = 0
        else:
            first = gs.append(rec, bx)
        assert first == 3 * k
        recs.append(rec)
        for j in range(2):
            li = len(ligs)
            ligs.append(G.ligand32(S.ligand_centered(S.make_ligand(30, 6, 300 + li))))
            for p in range(3):
                pair_lig.append(li)
                pair_pocket.append(first + p)
                pair_box.append(len(boxes) + p)
        boxes += bx
    assert gs.n_pockets == 9
    Ls = [O.OracleLigand(l) for l in ligs]
    pls = [ctx.ligand(l) for l in ligs]
    chains = 8
    r = ctx.dock_pairs(gs, pls, pair_lig, pair_pocket, chains=chains, steps=20, seed=2, top_k=4)
    assert r.n_pairs == 18
    coords = _coords(ctx, r, pls, Ls, pair_lig)
    ogs = _lazy_grids(lambda b: recs[b // 3], boxes, coords, pair_box)
    sites = [(recs[b // 3], O.xs_type_receptor(recs[b // 3]), boxes[b]) for b in range(9)]
    _check_pairs(r, Ls, ogs, coords, pair_lig, pair_box, sites)
    flat = r.poses.reshape(-1)
    for li in range(len(ligs)):
        pk = {int(flat[i]["pocket"]) for i in r.ranking(li)}
        assert pk <= {pair_pocket[q] for q in range(18) if pair_lig[q] == li}
    # rescoring uses each pocket's own receptor
    rr = ctx.dock_pairs(gs, pls, pair_lig, pair_pocket, chains=chains, steps=20, seed=2, top_k=4, rescore=True)
    for q in range(18):
        rec = recs[pair_box[q] // 3]
        G.check_rescored(rr, q, Ls[pair_lig[q]], rec, O.xs_type_receptor(rec), r)


def test_mixed_box_sizes_in_one_launch():
    """Boxes of 15, 21.5 and 30 A around two pocket centres (41, 59 and 81 nodes per axis) in one
    grid set and one launch (the box-size sweep): chain bests valid against the oracle, the
    selection and the per-ligand merge equal to the oracle's."""
    ctx = G.context()
    rec0, centres = S._carved(3000, 2, (6.5, 7.5), 41, 14.0)
    rec = G.receptor32(rec0)
    boxes = [G.box32(S.Box(np.array(c.center), np.array([s] * 3))) for c in centres for s in (15.0, 21.5, 30.0)]
    ligs = [G.ligand32(S.ligand_centered(S.make_ligand(22, 5, 71)))]
    Ls = [O.OracleLigand(l) for l in ligs]
    gs = ctx.build_grids(rec, boxes, list(range(11)))
    assert [int(gs.geometry(p, 0)[0][0]) for p in range(6)] == [41, 59, 81, 41, 59, 81]
    pls = [ctx.ligand(l) for l in ligs]
    r = ctx.dock(gs, pls, list(range(6)), chains=12, steps=25, seed=3, top_k=4)
    _, _, st = r.stats()
    assert (st == 0).all()
    pair_lig, pair_box = [0] * 6, list(range(6))
    coords = _coords(ctx, r, pls, Ls, pair_lig)
    ogs = _lazy_grids(lambda b: rec, boxes, coords, pair_box)
    sites = [(rec, O.xs_type_receptor(rec), b) for b in boxes]
    _check_pairs(r, Ls, ogs, coords, pair_lig, pair_box, sites)
    results = [O.PairResult(0, q, None, None, 0, r.poses[q]["chain"][:r.n_kept[q]],
                            r.poses[q]["score"][:r.n_kept[q]].astype(np.float64), None, None, None) for q in range(6)]
    flat = r.poses.reshape(-1)
    got = [(int(flat[i]["pocket"]), int(flat[i]["chain"])) for i in r.ranking(0)]
    assert got == [(m[1], m[2]) for m in O.merge_pockets(results)]
