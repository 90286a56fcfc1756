"""The allocation-free grid build (pv_build_grid_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory when they need a grid. Its maps must equal
those of the allocating pv_build_grids within the grid tolerance, on two calls in a row (the
second with a different receptor, box and type set, so anything the first call left in the
shared scratch array would show), and the FP64 oracle's direct sums at sampled nodes; the
receptor may be host or device memory. Named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import pvsynth as S
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _call_noalloc(ctx, rec, box, types, out):
    from paper_2506_20043_gb300 import _capi as A
    keep = []
    r = ctx._receptor(rec, keep)
    b = ctx._boxes([box])
    t = (C.c_uint8 * len(types))(*types)
    st = ctx.lib.pv_build_grid_noalloc(ctx.h, C.byref(r), b, t, len(types), C.c_void_p(out.data_ptr()))
    msg = ctx.lib.pv_last_error(ctx.h)
    return st, (msg.decode() if msg else "")


def test_noalloc_maps_match_pv_build_grids_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2506_20043_gb300 import _capi as A
    ctx = G.context()
    w = S.tiny()
    cases = [
        (G.receptor32(w.receptors[0]), G.box32(w.boxes[0][0]), [0, 1, 5, 6, 8]),
        (G.receptor32(S.make_receptor(1500, 7, [(np.array([2.0, -1.0, 0.5]), 6.0)])),
         G.box32(S.Box(np.array([2.0, -1.0, 0.5]), np.array([14.0, 12.5, 13.0]), 0.375)), [0, 3, 8, 10]),
    ]
    for rec, box, types in cases:
        origin, dims = O.grid_geometry(box)
        nxyz = int(np.prod(dims))
        out = torch.full((len(types), nxyz), float("nan"), dtype=torch.float32, device="cuda")
        st, msg = _call_noalloc(ctx, rec, box, types, out)
        assert st == A.PV_OK, msg
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(len(types), dims[2], dims[1], dims[0])
        ref_set = ctx.build_grids(rec, [box], types)
        for m, t in enumerate(sorted(types)):
            ref = ref_set.read_map(0, t)
            assert G.close(got[m], ref).all(), (t, np.abs(got[m] - ref).max())
        # the oracle's direct sum over every receptor atom at sampled nodes of every map
        rt = O.xs_type_receptor(rec)
        idx = np.random.default_rng(5).integers(0, dims, size=(60, 3))
        for m, t in enumerate(sorted(types)):
            ref = np.array([O.grid_node_value(rec, rt, box, t, *i) for i in idx])
            assert G.close(got[m][idx[:, 2], idx[:, 1], idx[:, 0]], ref).all(), t


def test_noalloc_device_resident_receptor():
    """The receptor given as device arrays (PV_MEM_DEVICE: read in place, nothing uploaded into
    the scratch array): the same maps as from host arrays, twice in a row."""
    torch = pytest.importorskip("torch")
    from paper_2506_20043_gb300 import _capi as A
    ctx = G.context()
    rec = G.receptor32(S.make_receptor(2500, 11, [(np.array([1.0, 2.0, -1.0]), 7.0)]))
    box = G.box32(S.Box(np.array([1.0, 2.0, -1.0]), np.array([16.0, 16.0, 16.0]), 0.375))
    types = [0, 2, 6, 9]
    drec = S.Receptor(torch.tensor(rec.xyz, dtype=torch.float32, device="cuda"),
                      torch.tensor(rec.element, device="cuda"), torch.tensor(rec.donor, device="cuda"),
                      torch.tensor(rec.acceptor, device="cuda"))
    _, dims = O.grid_geometry(box)
    nxyz = int(np.prod(dims))
    outs = []
    for r in (rec, drec, rec):
        out = torch.full((len(types), nxyz), float("nan"), dtype=torch.float32, device="cuda")
        st, msg = _call_noalloc(ctx, r, box, types, out)
        assert st == A.PV_OK, msg
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_2506_20043_gb300 import _capi as A
    ctx = G.context()
    big = S.make_receptor(16385, 3)
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    st, msg = _call_noalloc(ctx, big, S.Box(np.zeros(3), np.array([10.0] * 3), 0.375), [0], out)
    assert st == A.PV_ERR_ARG and "16384" in msg
    rec = S.make_receptor(1000, 4)
    st, msg = _call_noalloc(ctx, rec, S.Box(np.zeros(3), np.array([120.0] * 3), 1.0), [0], out)
    assert st == A.PV_ERR_ARG and "scratch" in msg
    # a non-finite centre or size is refused before any size is derived from it
    for c, sz in (((np.nan, 0.0, 0.0), 10.0), ((0.0, np.inf, 0.0), 10.0), ((0.0, 0.0, 0.0), np.nan)):
        st, msg = _call_noalloc(ctx, rec, S.Box(np.array(c), np.array([sz] * 3), 0.375), [0], out)
        assert st == A.PV_ERR_ARG and "finite" in msg
