"""GPU parity of the grid cache ("Kernel 1") against the FP64 oracle's direct summation.

Small boxes are compared node by node on every map; the full-size boxes of the tiny (20 A) and
multi-pocket (24 A) workloads are compared on sampled nodes the oracle computes one by one.
Typing of receptor atoms is checked through maps of every XS type.
"""
import numpy as np
import pytest

import oracle as O
import pvsynth as S
from tests import _gpu as G

pytestmark = pytest.mark.gpu
ALL_TYPES = list(range(11))


def _check(ctx, rec, boxes, types, sample=None, seed=0):
    rec32 = G.receptor32(rec)
    gs = ctx.build_grids(rec32, boxes, types)
    rt = O.xs_type_receptor(rec32)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for p, b in enumerate(boxes):
        b32 = G.box32(b)
        origin, dims = O.grid_geometry(b32)
        for t in types:
            gpu = gs.read_map(p, t)
            assert gpu.shape == (dims[2], dims[1], dims[0])
            if sample is None:
                ref = O.OracleGrid(rec32, b32, [t], rec_types=rt, threads=G.threads()).map(t)
                ok = G.close(gpu, ref)
                worst = max(worst, float(np.abs(gpu - ref).max()))
                assert ok.all(), f"pocket {p} type {t}: {np.argwhere(~ok)[:5]}"
            else:
                idx = rng.integers(0, dims, size=(sample, 3))
                ref = np.array([O.grid_node_value(rec32, rt, b32, t, *i) for i in idx])
                got = gpu[idx[:, 2], idx[:, 1], idx[:, 0]]
                assert G.close(got, ref).all(), f"pocket {p} type {t}"
    return gs, worst


def test_small_boxes_all_types_every_node():
    ctx = G.context()
    w = S.tiny()
    rec = w.receptors[0]
    # ragged boxes: node counts 17, 14, 23 per axis (not multiples of the 8-node tile)
    boxes = [S.Box(np.array([0.0, 0.0, 0.0]), np.array([6.0, 4.9, 8.25]), 0.375),
             S.Box(np.array([3.0, -4.0, 2.0]), np.array([3.0, 3.0, 3.0]), 0.5)]
    _check(ctx, rec, boxes, ALL_TYPES)


def test_tiny_workload_box_sampled_nodes():
    ctx = G.context()
    w = S.tiny()
    _check(ctx, w.receptors[0], w.boxes[0], [0, 1, 5, 6, 8], sample=300)


def test_multipocket_boxes_sampled_nodes():
    ctx = G.context()
    w = S.multipocket(chains=1, steps=1)
    gs, _ = _check(ctx, w.receptors[0], w.boxes[0][:3], [0, 3, 8], sample=120, seed=1)
    assert gs.n_pockets == 3
    assert gs.bytes == 3 * 3 * 65 ** 3 * 4


def test_device_resident_receptor_matches_host():
    torch = pytest.importorskip("torch")
    ctx = G.context()
    w = S.tiny()
    rec = w.receptors[0]
    box = [S.Box(np.zeros(3), np.array([5.0, 5.0, 5.0]), 0.375)]
    a = ctx.build_grids(G.receptor32(rec), box, [0, 4])
    drec = S.Receptor(torch.tensor(rec.xyz, dtype=torch.float32, device="cuda"),
                      torch.tensor(rec.element, device="cuda"), torch.tensor(rec.donor, device="cuda"),
                      torch.tensor(rec.acceptor, device="cuda"))
    b = ctx.build_grids(drec, box, [0, 4])
    for t in (0, 4):
        np.testing.assert_array_equal(a.read_map(0, t), b.read_map(0, t))


def test_append_receptor_and_determinism():
    ctx = G.context()
    w = S.tiny()
    rec = G.receptor32(w.receptors[0])
    box = [S.Box(np.zeros(3), np.array([4.0, 4.0, 4.0]), 0.375)]
    gs = ctx.build_grids(rec, box, [0, 6])
    other = S.make_receptor(1500, 3, [(np.zeros(3), 5.0)])
    first = gs.append(G.receptor32(other), box)
    assert first == 1 and gs.n_pockets == 2
    again = ctx.build_grids(G.receptor32(other), box, [0, 6])
    np.testing.assert_array_equal(gs.read_map(1, 6), again.read_map(0, 6))
    np.testing.assert_array_equal(gs.read_map(0, 0), ctx.build_grids(rec, box, [0, 6]).read_map(0, 0))


def test_grid_argument_errors():
    from paper_2506_20043_gb300.api import PVError
    ctx = G.context()
    w = S.tiny()
    with pytest.raises(PVError):
        ctx.build_grids(w.receptors[0], [S.Box(np.zeros(3), np.array([4.0, 4.0, 4.0]), 0.0)], [0])
    with pytest.raises(PVError):
        ctx.build_grids(w.receptors[0], [S.Box(np.zeros(3), np.array([4.0, 4.0, 4.0]), 0.375)], [11])
    gs = ctx.build_grids(w.receptors[0], [S.Box(np.zeros(3), np.array([4.0, 4.0, 4.0]), 0.375)], [0])
    with pytest.raises(PVError):
        gs.read_map(0, 3)


def test_pinned_host_receptor_is_uploaded_before_return():
    """A receptor in page-locked host memory: the call returns only after its upload, so the caller
    may overwrite the arrays at once (here before any synchronisation) without changing the maps."""
    torch = pytest.importorskip("torch")
    ctx = G.context()
    rec = G.receptor32(S.tiny().receptors[0])
    box = [S.Box(np.array([1.0, -2.0, 0.5]), np.array([9.0, 9.0, 9.0]), 0.375)]
    ref = ctx.build_grids(rec, box, [0, 6, 9])
    pin = [torch.tensor(np.asarray(rec.xyz, np.float32)).pin_memory()] + \
          [torch.tensor(np.asarray(a, np.uint8)).pin_memory() for a in (rec.element, rec.donor, rec.acceptor)]
    for _ in range(3):
        fresh = [t.clone().pin_memory() for t in pin]
        gs = ctx.build_grids(S.Receptor(*fresh), box, [0, 6, 9])
        fresh[0].fill_(0.0)
        fresh[1].fill_(3)
        for t in (0, 6, 9):
            np.testing.assert_array_equal(gs.read_map(0, t), ref.read_map(0, t))
