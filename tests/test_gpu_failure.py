"""Failure paths of the docking calls, made on the host: bad inputs, a non-finite energy, a step
block whose wait for its predecessor runs out. Each call returns its status and the context keeps
working afterwards (a normal dock follows every failure). No GPU fault is provoked: inputs the
library refuses are refused on the host, and the NaN map and the short wait bound are ordinary
data and parameters the kernels handle."""
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
    rec, box, lig = G.receptor32(w.receptors[0]), G.box32(w.boxes[0][0]), G.ligand32(w.ligands[0])
    L = O.OracleLigand(lig)
    types = sorted(set(L.xs.tolist()))
    gs = ctx.build_grids(rec, [box], types)
    return ctx, rec, box, lig, L, types, gs, ctx.ligand(lig)


def _still_works(ctx, gs, pl):
    r = ctx.dock(gs, [pl], [0], chains=8, steps=5, seed=1)
    assert r.status_code == 0 and r.n_kept[0] >= 1 and (r.stats()[2] == 0).all()


def _ring_ligand():
    """A six-membered ring (1.4 A, planar) with a two-atom chain on it: bonds 0-5 close the ring."""
    ang = np.arange(6) * np.pi / 3
    ring = np.stack([1.4 * np.cos(ang), 1.4 * np.sin(ang), np.zeros(6)], axis=1)
    xyz = np.concatenate([ring, [[2.9, 0.0, 0.0], [3.6, 1.3, 0.0]]])
    bonds = np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 5], [5, 0], [0, 6], [6, 7]], np.int32)
    el = np.array([0, 0, 0, 0, 0, 0, 0, 2], np.uint8)
    z = np.zeros(8, np.uint8)
    return S.Ligand(xyz, el, z, z.copy(), bonds, np.zeros(len(bonds), np.uint8))


def test_bad_ligands_are_refused(site):
    ctx, rec, box, lig, L, types, gs, pl = site
    from paper_2506_20043_gb300.api import PVError
    bad = S.Ligand(lig.xyz.copy(), lig.element, lig.donor, lig.acceptor, lig.bonds, lig.rotatable)
    bad.xyz[3, 1] = np.nan
    with pytest.raises(PVError, match="finite"):
        ctx.ligand(bad)
    # a rotatable bond inside a ring is not a bridge of the bond graph
    ring = _ring_ligand()
    rot = ring.rotatable.copy()
    rot[2] = 1
    with pytest.raises(PVError, match="bridge"):
        ctx.ligand(S.Ligand(ring.xyz, ring.element, ring.donor, ring.acceptor, ring.bonds, rot))
    # the chain bond off the ring is a bridge and may rotate
    rot = ring.rotatable.copy()
    rot[6] = 1
    assert ctx.ligand(S.Ligand(ring.xyz, ring.element, ring.donor, ring.acceptor, ring.bonds, rot)).n_rot == 1
    # two atoms without a bond: no tree
    with pytest.raises(PVError, match="connected"):
        ctx.ligand(S.Ligand(np.array([[0.0, 0, 0], [3.0, 0, 0]]), np.zeros(2, np.uint8), np.zeros(2, np.uint8),
                            np.zeros(2, np.uint8), np.zeros((0, 2), np.int32), np.zeros(0, np.uint8)))
    # 27 rotatable bonds (a zigzag chain of 30 atoms) is one more than the limit
    n = 30
    xyz = np.stack([1.25 * np.arange(n), 0.85 * (np.arange(n) % 2), np.zeros(n)], axis=1)
    bonds = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1).astype(np.int32)
    rot = np.zeros(n - 1, np.uint8)
    rot[1:-1] = 1
    assert rot.sum() == 27
    z = np.zeros(n, np.uint8)
    with pytest.raises(PVError, match="26"):
        ctx.ligand(S.Ligand(xyz, z, z, z.copy(), bonds, rot))
    rot[1] = 0
    assert ctx.ligand(S.Ligand(xyz, z, z, z.copy(), bonds, rot)).n_rot == 26
    _still_works(ctx, gs, pl)


def test_bad_receptors_and_boxes_are_refused(site):
    ctx, rec, box, lig, L, types, gs, pl = site
    from paper_2506_20043_gb300.api import PVError
    bad = S.Receptor(rec.xyz.copy(), rec.element, rec.donor, rec.acceptor)
    bad.xyz[17, 2] = np.inf
    with pytest.raises(PVError, match="finite"):
        ctx.build_grids(bad, [box], types)
    for center, size in (((np.nan, 0.0, 0.0), (20.0, 20.0, 20.0)), ((0.0, 0.0, 0.0), (20.0, np.inf, 20.0)),
                         ((0.0, 0.0, 0.0), (20.0, 0.0, 20.0))):
        with pytest.raises(PVError):
            ctx.build_grids(rec, [S.Box(np.array(center), np.array(size), 0.375)], types)
    _still_works(ctx, gs, pl)


def test_empty_pocket_and_box_outside_the_receptor(site):
    """A box far from every receptor atom (all maps zero: the SF is e_intra plus the out-of-grid
    penalty) and a box straddling the receptor's surface both dock normally; in the empty box the
    kept poses lie inside it (e_inter = 0) and their SF is their e_intra, which the oracle gives."""
    ctx, rec, box, lig, L, types, gs, pl = site
    side = float(np.ptp(rec.xyz[:, 0]))
    far = G.box32(S.Box(np.array([side + 40.0, 0.0, 0.0]), np.array([20.0, 20.0, 20.0]), 0.375))
    edge = G.box32(S.Box(np.array([side / 2, 0.0, 0.0]), np.array([20.0, 20.0, 20.0]), 0.375))
    gs2 = ctx.build_grids(rec, [far, edge], types)
    assert not np.any(gs2.read_map(0, types[0]))
    r = ctx.dock(gs2, [pl], [0, 1], chains=32, steps=40, seed=3)
    assert r.status_code == 0 and (r.stats()[2] == 0).all()
    n = int(r.n_kept[0])
    assert n >= 1
    og = O.OracleGrid(rec, far, types, maps=np.zeros((len(types), int(np.prod(O.grid_geometry(far)[1])))))
    for slot in range(n):
        p = r.poses[0][slot]
        assert abs(float(p["e_inter"])) <= 1e-6
        e, _, parts = L.score(og, r.pots[0, slot, :L.n_pot].astype(np.float64), False)
        assert G.close(p["score"], e) and G.close(p["e_intra"], parts[1])
    assert np.isfinite(r.poses[1]["score"][:int(r.n_kept[1])]).all()
    _still_works(ctx, gs, pl)


def _device_view(ptr, n):
    """A float32 tensor over n floats of device memory at ptr (no copy)."""
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 2}

    return torch.as_tensor(_View(), device="cuda")


def test_non_finite_energy_returns_nan_status(site):
    """One map of a fresh grid set overwritten with NaN (through its device view): every chain of
    the pair meets a NaN energy, the dock returns PV_ERR_NAN with the pair's status NaN, and no
    pose is kept; the context docks normally afterwards."""
    import torch
    ctx, rec, box, lig, L, types, gs, pl = site
    from paper_2506_20043_gb300 import _capi as A
    gs_bad = ctx.build_grids(rec, [box], types)
    dims, _, _, ptr = gs_bad.geometry(0, types[0])
    _device_view(ptr, int(np.prod(dims))).fill_(float("nan"))
    torch.cuda.synchronize()
    r = ctx.dock(gs_bad, [pl], [0], chains=16, steps=10, seed=2)
    assert r.status_code == A.PV_ERR_NAN, r.status_code
    assert (r.stats()[2] == A.PV_ERR_NAN).all()
    assert int(r.n_kept[0]) == 0
    _still_works(ctx, gs, pl)


def test_step_block_wait_bound_skips_and_reports(site):
    """With a wait bound of a nanosecond, the step blocks after the first cannot find their
    predecessor published (64 one-chain CTAs all run block 0 at once; block 1 is taken while they
    run) and are skipped: the dock returns PV_ERR_STATE with that status per pair, the chains keep
    the state of their last completed block, and the context docks normally afterwards."""
    ctx, rec, box, lig, L, types, gs, pl = site
    from paper_2506_20043_gb300 import _capi as A
    r = ctx.dock(gs, [pl], [0], chains=64, steps=100, seed=4, search_variant=0, warps_per_cta=1,
                 block_wait_s=1e-9)
    assert r.status_code == A.PV_ERR_STATE, r.status_code
    assert "waiting" in r.error
    assert (r.stats()[2] == A.PV_ERR_STATE).all()
    full = ctx.dock(gs, [pl], [0], chains=64, steps=100, seed=4, search_variant=0, warps_per_cta=1)
    assert full.status_code == 0
    assert r.stats()[0] < full.stats()[0]          # the skipped blocks did no work
    _still_works(ctx, gs, pl)
    from paper_2506_20043_gb300.api import PVError
    with pytest.raises(PVError):
        ctx.dock(gs, [pl], [0], steps=1, block_wait_s=float("nan"))
