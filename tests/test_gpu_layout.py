"""The cell-packed map layout (pv_grid_set_pack): each cell's eight corner values stored together.
A lookup interpolates the same eight values with the same arithmetic as from the plain maps, so a
dock reading either layout gives the same bits (the plain layout's results are checked against the
oracle in tests/test_gpu_dock.py and tests/test_gpu_score.py); pockets appended after packing are
packed too; the autotuner records which layout it chose; the gather microbenchmark runs on both."""
import numpy as np
import pytest

import pvsynth as S
from tests import _gpu as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def site():
    ctx = G.context()
    rec0, boxes0 = S._carved(3000, 3, (6.0, 8.0), 8, 16.0)
    rec, boxes = G.receptor32(rec0), [G.box32(b) for b in boxes0]
    lig = ctx.ligand(G.ligand32(S.ligand_centered(S.make_ligand(22, 5, 31))))
    small = ctx.ligand(G.ligand32(S.ligand_centered(S.make_ligand(14, 3, 32))))
    types = list(range(11))
    return ctx, rec, boxes, lig, small, types


def test_packed_layout_docks_the_same_bits(site):
    ctx, rec, boxes, lig, small, types = site
    gs = ctx.build_grids(rec, boxes, types)
    from paper_2506_20043_gb300.api import PVError
    with pytest.raises(PVError):
        ctx.dock(gs, [lig], [0], steps=1, map_layout=1)          # no packed copy yet
    plain_bytes = gs.bytes
    gs.pack()
    assert gs.bytes > 8 * plain_bytes * 0.9                      # about 8x the plain maps
    for ligand, shape in ((lig, dict(search_variant=0, warps_per_cta=2)),
                          (small, dict(search_variant=4, warps_per_cta=4)),
                          (lig, dict(mode="plain_warp", search_variant=1, warps_per_cta=4))):
        out = []
        for layout in (0, 1):
            r = ctx.dock(gs, [ligand], [0, 1, 2], chains=48, steps=30, seed=3, map_layout=layout, **shape)
            assert r.map_layout() == layout
            out.append(r)
        np.testing.assert_array_equal(out[0].chain_records()[1], out[1].chain_records()[1])
        np.testing.assert_array_equal(out[0].chain_records()[0], out[1].chain_records()[0])
        assert (out[0].poses == out[1].poses).all()
    # autotuned: either layout, the same bits as the plain run of the chosen shape
    r = ctx.dock(gs, [lig], [0, 1, 2], chains=48, steps=30, seed=3)
    v, w = r.launch_shape()
    ref = ctx.dock(gs, [lig], [0, 1, 2], chains=48, steps=30, seed=3, map_layout=0, search_variant=v, warps_per_cta=w)
    assert r.map_layout() in (0, 1)
    np.testing.assert_array_equal(r.chain_records()[1], ref.chain_records()[1])


def test_pockets_appended_after_packing_are_packed(site):
    ctx, rec, boxes, lig, small, types = site
    gs = ctx.build_grids(rec, boxes[:1], types).pack()
    other0, other_boxes = S._carved(2500, 1, (7.0, 7.0), 9, 15.0)
    first = gs.append(G.receptor32(other0), [G.box32(other_boxes[0])])
    assert first == 1
    a = ctx.dock(gs, [lig], [1], chains=32, steps=20, seed=5, map_layout=1, search_variant=0, warps_per_cta=2)
    b = ctx.dock(gs, [lig], [1], chains=32, steps=20, seed=5, map_layout=0, search_variant=0, warps_per_cta=2)
    np.testing.assert_array_equal(a.chain_records()[1], b.chain_records()[1])


def test_gather_probe_on_both_layouts(site):
    ctx, rec, boxes, lig, small, types = site
    gs = ctx.build_grids(rec, boxes, types)
    from paper_2506_20043_gb300.api import PVError
    with pytest.raises(PVError):
        ctx.measure_gather(gs, 0, n_points=1 << 16, reps=2, layout=1)
    gs.pack()
    for layout in (0, 1):
        ms, pts, gbs = ctx.measure_gather(gs, -1, n_points=1 << 20, reps=3, layout=layout)
        assert ms > 0 and gbs > 0


def test_scoring_reads_the_packed_maps_with_the_same_bits(site):
    """pv_score, pv_score_backward and pv_score_xyz read the cell-packed maps once the set holds
    them: the same energies, gradients and coordinate gradients, bit for bit, as from the plain
    maps (which tests/test_gpu_score.py checks against the oracle)."""
    import torch
    ctx, rec, boxes, lig, small, types = site
    gs = ctx.build_grids(rec, boxes[:2], types)
    poses = torch.tensor(S.random_poses(3000, boxes[1], lig.n_rot, 77), device="cuda")
    xyz = ctx.pose_coords(lig, poses)
    ge = torch.linspace(-1.0, 2.0, poses.shape[0], device="cuda")
    out = []
    for packed in (False, True):
        if packed:
            gs.pack()
        e, g, parts = ctx.score(gs, lig, 1, poses, grad=True, parts=True)
        gp, gx = ctx.score_backward(gs, lig, 1, poses, ge, want_pose=True, want_xyz=True)
        ex, gxx = ctx.score_xyz(gs, lig, 1, xyz, grad=True)
        out.append([t.cpu().numpy() for t in (e, g, parts, gp, gx, ex, gxx)])
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
