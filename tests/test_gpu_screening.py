"""Oracle agreement on a seeded 216-pair subset of the screening shape: 24 receptors of 1,500-8,000
atoms (log-uniform) with 3 pockets each (24 A boxes), appended into one grid set, and 3 ligands of
30 atoms / 6 torsions per receptor docked into that receptor's 3 pockets through one pair list.

For every pair: each chain best is what the oracle scores for that pose (coordinates and SF), the
top-k is the oracle's selection of the GPU's chain bests; for every ligand the merged ranking is
the oracle's merge of the GPU's kept poses. Oracle maps are filled at the cells the poses touch.
"""
import os

import numpy as np
import pytest

import oracle as O
import pvsynth as S
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def test_screening_subset_agrees_with_oracle():
    ctx = G.context()
    w = S.screening(seed=3, n_receptors=24, ligands_per_receptor=3, chains=32, steps=60)
    recs = [G.receptor32(r) for r in w.receptors]
    boxes = [[G.box32(b) for b in bx] for bx in w.boxes]
    ligs = [G.ligand32(l) for l in w.ligands]
    Ls = [O.OracleLigand(l) for l in ligs]
    types = sorted(set(np.concatenate([L.xs for L in Ls]).tolist()))
    gs = ctx.build_grids(recs[0], boxes[0], types)
    for r in range(1, len(recs)):
        assert gs.append(recs[r], boxes[r]) == 3 * r
    assert gs.n_pockets == 72
    pair_lig, pair_pocket = [], []
    for r, ids in enumerate(w.ligands_per_receptor):
        for li in ids:
            for p in range(3):
                pair_lig.append(li)
                pair_pocket.append(3 * r + p)
    assert len(pair_lig) == 216
    pls = [ctx.ligand(l) for l in ligs]
    res = ctx.dock_pairs(gs, pls, pair_lig, pair_pocket, chains=w.chains, steps=w.steps, seed=w.seed, top_k=5)
    _, _, st = res.stats()
    assert (st == 0).all()
    pots, es = res.chain_records()
    coords = []
    for q in range(216):
        L, p = Ls[pair_lig[q]], pots[q, :, :Ls[pair_lig[q]].n_pot]
        coords.append((G.pose_coords(ctx, pls[pair_lig[q]], p), np.stack([L.fk(x) for x in p.astype(np.float64)])))
    threads = len(os.sched_getaffinity(0))
    flat = res.poses.reshape(-1)
    for r in range(len(recs)):
        rt = O.xs_type_receptor(recs[r])
        for p in range(3):
            k = 3 * r + p
            qs = [q for q in range(216) if pair_pocket[q] == k]
            xyz = np.concatenate([np.concatenate(coords[q]).reshape(-1, 3) for q in qs])
            lt = sorted(set(np.concatenate([Ls[pair_lig[q]].xs for q in qs]).tolist()))
            og = O.OracleGrid.lazy(recs[r], boxes[r][p], lt, rt, xyz, threads=threads)
            for q in qs:
                L = Ls[pair_lig[q]]
                G.check_pose_scores(L, og, pots[q, :, :L.n_pot], es[q], coords[q][0], (recs[r], rt, boxes[r][p]))
                kept = O.topk(es[q].astype(np.float64), coords[q][1], res.top_k, 1.0)
                assert list(res.poses[q]["chain"][:res.n_kept[q]]) == list(kept), q
    for li in range(len(ligs)):
        results = []
        for q in range(216):
            if pair_lig[q] != li:
                continue
            n = res.n_kept[q]
            results.append(O.PairResult(li, pair_pocket[q], None, None, 0, res.poses[q]["chain"][:n],
                                        res.poses[q]["score"][:n].astype(np.float64), None, None, None))
        merged = O.merge_pockets(results)
        got = [(int(flat[i]["pocket"]), int(flat[i]["chain"])) for i in res.ranking(li)]
        assert got == [(m[1], m[2]) for m in merged], li
