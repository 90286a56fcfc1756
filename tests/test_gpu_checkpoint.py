"""Checkpoint and resume of a dock: a dock of s MC steps saved with DockResult.save_state and
continued by a dock of t > s steps with DockParams.resume_state gives every chain the state, and
every pair the kept poses, of one dock of t steps, bit for bit. Between MC steps a chain carries
only its current and best poses and energies (each local search starts a new L-BFGS history, and
random numbers are drawn by step index, Algorithm 2), plus the neighbour ring of the consistency
check (Eq. 4-5); the checkpoint holds exactly that. A checkpoint of another job is refused."""
import numpy as np
import pytest

import oracle as O
import pvsynth as S
from tests import _gpu as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def site():
    ctx = G.context()
    w = S.tiny()
    rec, box = G.receptor32(w.receptors[0]), G.box32(w.boxes[0][0])
    ligs = [G.ligand32(w.ligands[0]), G.ligand32(S.ligand_centered(S.make_ligand(16, 3, 5)))]
    types = sorted(set().union(*[set(O.OracleLigand(l).xs.tolist()) for l in ligs]))
    gs = ctx.build_grids(rec, [box, box], types)
    return ctx, gs, [ctx.ligand(l) for l in ligs]


def _same(a, b):
    pa, sa = a.chain_records()
    pb, sb = b.chain_records()
    assert np.array_equal(pa, pb) and np.array_equal(sa, sb)
    for x, y in zip(a.fetch(), b.fetch()):
        assert np.array_equal(np.asarray(x).view(np.uint8), np.asarray(y).view(np.uint8))
    for i in range(2):
        assert np.array_equal(a.ranking(i), b.ranking(i))


@pytest.mark.parametrize("mode,focc,resume_mode,spr,variant", [
    ("batched", 0, "batched", 0, 1), ("batched", 4, "batched", 0, 1), ("batched", 0, "batched", 7, 1),
    ("batched", 0, "plain_warp", 0, 1), ("plain", 0, "plain", 0, 1), ("batched", 0, "batched", 0, 5),
    ("batched", 4, "batched", 0, 5)])
def test_resumed_dock_repeats_the_unbroken_one(site, mode, focc, resume_mode, spr, variant):
    """variant 1: a chain per warp; variant 5: a chain per half warp (the flattened chain loop)."""
    ctx, gs, ligs = site
    kw = dict(chains=48, seed=11, focc=focc, search_variant=variant, warps_per_cta=2, map_layout=0)
    if mode == "plain":
        kw = dict(chains=48, seed=11)
    full = ctx.dock(gs, ligs, [0, 1], steps=40, mode=mode, **kw)
    half = ctx.dock(gs, ligs, [0, 1], steps=17, mode=mode, **kw)
    state = half.save_state()
    assert half.status_code == 0 and full.status_code == 0
    more = ctx.dock(gs, ligs, [0, 1], steps=40, mode=resume_mode, resume_state=state, steps_per_round=spr, **kw)
    assert more.status_code == 0 and (more.stats()[2] == 0).all()
    _same(full, more)
    # and again from the resumed dock's own checkpoint
    again = ctx.dock(gs, ligs, [0, 1], steps=55, mode=mode, resume_state=more.save_state(), **kw)
    _same(ctx.dock(gs, ligs, [0, 1], steps=55, mode=mode, **kw), again)


def test_checkpoint_of_another_job_is_refused(site):
    ctx, gs, ligs = site
    from paper_2506_20043_gb300.api import PVError
    kw = dict(chains=16, seed=3, search_variant=1, warps_per_cta=2)
    state = ctx.dock(gs, ligs, [0, 1], steps=10, **kw).save_state()
    with pytest.raises(PVError, match="another job"):
        ctx.dock(gs, ligs, [0, 1], steps=20, resume_state=state, **dict(kw, seed=4))
    with pytest.raises(PVError, match="another job"):
        ctx.dock(gs, ligs, [1, 0], steps=20, resume_state=state, **kw)
    with pytest.raises(PVError, match="another job"):
        ctx.dock(gs, ligs, [0, 1], steps=20, resume_state=state, **dict(kw, temperature=1.0))
    with pytest.raises(PVError, match="another job"):
        ctx.dock(gs, ligs, [0, 1], steps=20, resume_state=state, mode="plain", chains=16, seed=3)
    with pytest.raises(PVError, match="exceed"):
        ctx.dock(gs, ligs, [0, 1], steps=10, resume_state=state, **kw)
    with pytest.raises(PVError, match="resume_bytes"):
        ctx.dock(gs, ligs, [0, 1], steps=20, resume_state=state[:-4], **kw)
    with pytest.raises(PVError, match="not a dock checkpoint"):
        ctx.dock(gs, ligs, [0, 1], steps=20, resume_state=b"\0" * len(state), **kw)
    with pytest.raises(PVError, match="not a dock checkpoint"):
        ctx.dock(gs, ligs, [0, 1], steps=20, resume_state=state[:8], **kw)
    # the context keeps working, and the checkpoint still resumes its own job
    r = ctx.dock(gs, ligs, [0, 1], steps=20, resume_state=state, **kw)
    assert r.status_code == 0 and (r.stats()[2] == 0).all()
