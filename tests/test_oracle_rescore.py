"""Pins of the oracle's direct rescoring of selected poses (Algorithm 2, "rescoring"): e_inter
summed over every receptor atom within the 8 A cutoff, with no grid and no box.

Pinned by the grid's definition (a ligand whose atoms all sit on grid nodes has a direct e_inter
equal to the sum of the node values of its atom types), by the cutoff (an atom at 7.9 A counts,
one at 8.1 A does not), by additivity over receptor atoms, and by invariance when ligand and
receptor move rigidly together.
"""
import numpy as np
import pytest

import oracle as O
import pvsynth as S
from tests.test_oracle_grid import _Rec


@pytest.fixture(scope="module")
def site():
    rec = S.make_receptor(1500, 3, [(np.zeros(3), 7.0)])
    lig = S.ligand_centered(S.make_ligand(12, 2, 5))
    return rec, O.xs_type_receptor(rec), O.OracleLigand(lig)


def test_direct_equals_node_values_on_nodes(site):
    rec, rt, L = site
    box = S.Box(np.zeros(3), np.array([16.0] * 3), 0.375)
    origin, dims = O.grid_geometry(box)
    rng = np.random.default_rng(1)
    idx = rng.integers(4, dims - 4, size=(L.n, 3))
    xyz = origin + 0.375 * idx
    want = sum(O.grid_node_value(rec, rt, box, int(L.xs[i]), *idx[i]) for i in range(L.n))
    assert L.direct_inter(rec, rt, xyz) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_cutoff_and_additivity(site):
    _, _, L = site
    xyz = np.zeros((L.n, 3))
    xyz[1:] = 1000.0 + np.arange(L.n - 1)[:, None] * 50.0      # other atoms far from everything
    t0 = int(L.xs[0])
    one = _Rec([[7.9, 0, 0]], [0])
    both = _Rec([[7.9, 0, 0], [0, 8.1, 0]], [0, 0])
    far = _Rec([[0, 8.1, 0]], [0])
    r1, r2, r3 = (O.xs_type_receptor(r) for r in (one, both, far))
    e1 = L.direct_inter(one, r1, xyz)
    assert e1 == pytest.approx(O.pair_energy(t0, int(r1[0]), 7.9)[0], abs=1e-15) and e1 != 0.0
    assert L.direct_inter(far, r3, xyz) == 0.0
    assert L.direct_inter(both, r2, xyz) == pytest.approx(e1, abs=1e-15)
    near = _Rec([[3.4, 0, 0], [-2.9, 1.0, 0]], [1, 2])
    rn = O.xs_type_receptor(near)
    parts = sum(L.direct_inter(_Rec([near.xyz[k]], [near.element[k]]), rn[k:k + 1], xyz) for k in range(2))
    assert L.direct_inter(near, rn, xyz) == pytest.approx(parts, rel=1e-13)


def test_rigid_motion_invariance(site):
    rec, rt, L = site
    pot = S.random_poses(1, S.Box(np.zeros(3), np.array([6.0] * 3)), L.n_rot, 4)[0]
    xyz = L.fk(pot)
    e = L.direct_inter(rec, rt, xyz)
    a = 0.7
    R = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    t = np.array([3.0, -1.0, 2.5])
    moved = _Rec(rec.xyz @ R.T + t, rec.element, rec.donor, rec.acceptor)
    assert L.direct_inter(moved, rt, xyz @ R.T + t) == pytest.approx(e, rel=1e-10, abs=1e-10)
