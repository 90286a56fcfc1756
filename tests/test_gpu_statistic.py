"""The search statistic of the parity contract at the headline shape: per ligand, the best SF over
the chains of all its pockets within 0.2 kcal/mol of the FP64 oracle's, and the same top-ranked
pocket (the pocket of that best pose, Algorithm 3's aggregation), on at least 95 % of ligands.

Workload (tests/headline_case.py): the multi-pocket receptor (5,000 atoms, 10 carved pockets, 24 A
boxes at 0.375 A), 20 ligands of 30 heavy atoms and 6 torsions, each docked into all 10 pockets with
256 chains x 300 MC steps per pair in one batched launch. The oracle's results are stored in
tests/golden/headline_search_best.txt, written by tests/golden/make_headline_search.py (FP64 oracle
only; about 25 CPU-minutes). Two oracle runs with different Philox keys, on the file's first five
ligands, show how far two correct searches fall apart at this budget.
"""
import os

import numpy as np
import pytest

from tests import _gpu as G
from tests.headline_case import CHAINS, N_LIGANDS, SEED, STEPS, case

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "headline_search_best.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        rows[(int(v[0]), int(v[1]))] = np.array([float(x) for x in v[2:]])
    return rows


def test_oracle_runs_agree_with_each_other_at_this_budget():
    """The statistic is attainable: two FP64 oracle searches with different random streams already
    meet it on the stored ligands (a budget too small for the search to settle would fail here)."""
    rows = _golden()
    both = [li for li in range(N_LIGANDS) if (SEED + 1, li) in rows]
    assert len(both) >= 5
    for li in both:
        a, b = rows[(SEED, li)], rows[(SEED + 1, li)]
        assert abs(a.min() - b.min()) <= 0.2 and a.argmin() == b.argmin(), (li, a.min(), b.min())


@pytest.mark.gpu
def test_headline_shape_best_score_and_top_pocket_match_oracle():
    ctx = G.context()
    rows = _golden()
    rec, boxes, ligs = case()
    pls = [ctx.ligand(l) for l in ligs]
    types = sorted(set(int(t) for p in pls for t in p.xs_types.tolist()))
    gs = ctx.build_grids(rec, boxes, types)
    r = ctx.dock(gs, pls, list(range(len(boxes))), chains=CHAINS, steps=STEPS, seed=SEED, top_k=9)
    assert r.status_code == 0
    _, es = r.chain_records()
    best = es.min(axis=1).reshape(N_LIGANDS, len(boxes))          # pair = ligand * 10 + pocket
    ok_score, ok_pocket = [], []
    flat = r.poses.reshape(-1)
    for li in range(N_LIGANDS):
        ref = rows[(SEED, li)]
        ok_score.append(abs(best[li].min() - ref.min()) <= 0.2)
        top = flat[r.ranking(li)[0]]
        # the selection re-evaluates the pose, summing e_inter and e_intra separately: the last bits differ
        assert top["score"] == pytest.approx(best[li].min(), abs=1e-5)
        ok_pocket.append(int(top["pocket"]) == int(ref.argmin()))
    ok = np.array(ok_score) & np.array(ok_pocket)
    diff = np.abs(best.min(axis=1) - np.array([rows[(SEED, li)].min() for li in range(N_LIGANDS)]))
    assert ok.mean() >= 0.95, (ok.mean(), np.round(diff, 3), ok_pocket)
