"""Pins of the oracle's grid cache (Kernel 1) and trilinear interpolation (Eq. 3).

The grid is pinned by single-atom fields (their maximum sits on the atom's node, their value at a
node a known distance away is the closed-form pair energy), by superposition over receptor
atoms, by invariance under a 90-degree rotation of receptor + box, and by the node-count rule.
Interpolation is pinned by exactness at nodes and for affine fields, and by the clamped penalty.
"""
import math

import numpy as np
import pytest

import oracle as O
import pvsynth as S

C_H, C_P, N_P, N_D, N_A, N_DA, O_P, O_D, O_A, O_DA, S_P = range(11)


class _Rec:
    def __init__(self, xyz, element, donor=None, acceptor=None):
        self.xyz = np.asarray(xyz, float).reshape(-1, 3)
        self.element = np.asarray(element, np.uint8)
        self.donor = np.zeros(len(self.element), np.uint8) if donor is None else np.asarray(donor, np.uint8)
        self.acceptor = np.zeros(len(self.element), np.uint8) if acceptor is None else np.asarray(acceptor, np.uint8)
        self.n = len(self.element)


def test_node_count_rule():
    assert O.grid_dims(20.0, 0.375) == 55
    assert O.grid_dims(24.0, 0.375) == 65
    assert O.grid_dims(15.0, 0.375) == 41
    assert O.grid_dims(30.0, 0.375) == 81
    assert O.grid_dims(1.0, 0.5) == 3


def test_single_atom_field_layout_and_values():
    box = S.Box(np.array([1.0, -2.0, 0.5]), np.array([6.0, 5.0, 4.0]), 0.5)
    origin, dims = O.grid_geometry(box)
    assert list(dims) == [13, 11, 9]
    node = (7, 3, 5)  # x, y, z indices
    atom = origin + np.array(node) * 0.5
    rec = _Rec([atom], [0])
    g = O.OracleGrid(rec, box, [C_H, O_A], rec_types=np.array([C_H], np.int32))
    m = g.map(C_H)
    assert m.shape == (9, 11, 13)                     # [z][y][x]
    assert np.unravel_index(np.argmax(m), m.shape) == (5, 3, 7)
    # at the atom's own node: r = 0, d = -3.8, all five terms known in closed form
    d = -3.8
    expect = (-0.0356 * math.exp(-(d / 0.5) ** 2) - 0.00516 * math.exp(-((d - 3) / 2) ** 2)
              + 0.840 * d * d - 0.0351 * 1.0)
    assert m[5, 3, 7] == pytest.approx(expect, rel=1e-13)
    # two nodes along +x (r = 1.0): d = -2.8; O_A probe (radius 1.7) vs C_H: d = -2.6, no hydrophobic
    assert m[5, 3, 9] == pytest.approx(O.pair_energy(C_H, C_H, 1.0)[0], rel=1e-13)
    assert g.map(O_A)[5, 3, 9] == pytest.approx(O.pair_energy(O_A, C_H, 1.0)[0], rel=1e-13)
    # a node beyond the 8 A cutoff of the atom (corner to corner of a 6 A box is ~8.8 A)
    far = (0, 10, 0)
    r = np.linalg.norm(origin + np.array(far) * 0.5 - atom)
    if r >= 8.0:
        assert m[far[2], far[1], far[0]] == 0.0


def test_superposition_over_atoms():
    rng = np.random.default_rng(5)
    box = S.Box(np.zeros(3), np.array([4.0, 4.0, 4.0]), 0.5)
    xyz = rng.uniform(-6, 6, size=(12, 3))
    el = rng.integers(0, 4, size=12)
    don = (rng.random(12) < 0.5) & ((el == 1) | (el == 2))
    acc = (rng.random(12) < 0.5) & ((el == 1) | (el == 2))
    rec = _Rec(xyz, el, don, acc)
    rt = O.xs_type_receptor(rec)
    types = list(range(11))
    full = O.OracleGrid(rec, box, types, rec_types=rt)
    parts = [O.OracleGrid(_Rec(xyz[i:i + 1], el[i:i + 1], don[i:i + 1], acc[i:i + 1]), box, types,
                          rec_types=rt[i:i + 1]) for i in range(12)]
    np.testing.assert_allclose(full.maps, sum(p.maps for p in parts), rtol=1e-12, atol=1e-12)


def test_rotation_of_receptor_and_box():
    # rotating receptor and (cubic, centred) box by 90 degrees about z maps nodes onto nodes
    rng = np.random.default_rng(6)
    box = S.Box(np.zeros(3), np.array([4.0, 4.0, 4.0]), 0.5)
    xyz = rng.uniform(-7, 7, size=(40, 3))
    el = rng.integers(0, 4, size=40)
    rec = _Rec(xyz, el)
    rt = O.xs_type_receptor(rec)
    rot = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float)
    rec2 = _Rec(xyz @ rot.T, el)
    a = O.OracleGrid(rec, box, [C_H, N_D], rec_types=rt).map(C_H)
    b = O.OracleGrid(rec2, box, [C_H, N_D], rec_types=rt).map(C_H)
    # node (x, y) -> (-y, x): b[z, x, n-1-y] == a[z, y, x]
    n = a.shape[2]
    for z in range(0, a.shape[0], 3):
        for y in range(n):
            for x in range(n):
                assert b[z, x, n - 1 - y] == pytest.approx(a[z, y, x], rel=1e-12, abs=1e-12)


def test_node_value_matches_full_build():
    w = S.tiny()
    rec = w.receptors[0]
    rt = O.xs_type_receptor(rec)
    box = S.Box(w.boxes[0][0].center, np.array([3.0, 3.0, 3.0]), 0.375)
    g = O.OracleGrid(rec, box, [C_H, O_A], rec_types=rt)
    for (ix, iy, iz) in [(0, 0, 0), (3, 5, 8), (8, 8, 8)]:
        assert O.grid_node_value(rec, rt, box, C_H, ix, iy, iz) == g.map(C_H)[iz, iy, ix]


def _affine_grid(a, b, box):
    origin, dims = O.grid_geometry(box)
    zz, yy, xx = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    pts = np.stack([xx, yy, zz], -1) * box.spacing + origin
    vals = pts @ a + b
    return O.OracleGrid(None, box, [C_H], maps=vals.reshape(1, -1))


def test_trilinear_exact_for_affine_fields_and_at_nodes():
    box = S.Box(np.array([0.5, 0.0, -1.0]), np.array([5.0, 4.0, 3.0]), 0.5)
    a, b = np.array([0.7, -1.3, 2.1]), 0.25
    g = _affine_grid(a, b, box)
    origin, dims = O.grid_geometry(box)
    rng = np.random.default_rng(7)
    hi = origin + (dims - 1) * box.spacing
    for _ in range(200):
        p = rng.uniform(origin, hi)
        v, grad = g.eval(C_H, p)
        assert v == pytest.approx(p @ a + b, rel=1e-12, abs=1e-12)
        np.testing.assert_allclose(grad, a, rtol=1e-12, atol=1e-12)
    # at nodes interpolation returns the stored value for any field
    rnd = O.OracleGrid(None, box, [C_H], maps=rng.normal(size=(1, int(np.prod(dims)))))
    for _ in range(50):
        idx = rng.integers(0, dims)
        v, _ = rnd.eval(C_H, origin + idx * box.spacing)
        assert v == pytest.approx(rnd.map(C_H)[idx[2], idx[1], idx[0]], rel=1e-13, abs=1e-13)


def test_outside_penalty_and_clamp():
    box = S.Box(np.zeros(3), np.array([4.0, 4.0, 4.0]), 0.5)
    a, b = np.array([1.0, 2.0, -0.5]), 0.0
    g = _affine_grid(a, b, box)
    # 1.5 A beyond the +x face: value at the clamped point plus 10 * 1.5
    p = np.array([3.5, 0.3, -0.7])
    v, grad = g.eval(C_H, p)
    pc = np.array([2.0, 0.3, -0.7])
    assert v == pytest.approx(pc @ a + 10.0 * 1.5, rel=1e-12)
    np.testing.assert_allclose(grad, [10.0, 2.0, -0.5], rtol=1e-12)
    # outside a corner: Euclidean distance to the clamped point
    p = np.array([-3.0, 5.0, 0.0])
    v, grad = g.eval(C_H, p)
    pc = np.array([-2.0, 2.0, 0.0])
    dist = math.sqrt(1 + 9)
    assert v == pytest.approx(pc @ a + 10 * dist, rel=1e-12)
    np.testing.assert_allclose(grad, [10 * -1 / dist, 10 * 3 / dist, -0.5], rtol=1e-12)


def test_trilinear_gradient_matches_fd_inside():
    w = S.tiny()
    rec = w.receptors[0]
    rt = O.xs_type_receptor(rec)
    box = S.Box(w.boxes[0][0].center, np.array([6.0, 6.0, 6.0]), 0.375)
    g = O.OracleGrid(rec, box, [N_A], rec_types=rt)
    origin, dims = O.grid_geometry(box)
    rng = np.random.default_rng(8)
    n = 0
    while n < 100:
        p = rng.uniform(origin + 0.1, origin + (dims - 1) * 0.375 - 0.1)
        frac = (p - origin) / 0.375 % 1.0
        if (np.minimum(frac, 1 - frac) < 1e-4).any():
            continue
        _, grad = g.eval(N_A, p)
        h = 1e-6
        fd = [(g.eval(N_A, p + h * e)[0] - g.eval(N_A, p - h * e)[0]) / (2 * h) for e in np.eye(3)]
        np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-6)
        n += 1


def test_lazy_grid_matches_full_build_at_filled_nodes():
    w = S.tiny()
    rec = w.receptors[0]
    rt = O.xs_type_receptor(rec)
    box = S.Box(w.boxes[0][0].center, np.array([4.0, 4.0, 4.0]), 0.375)
    full = O.OracleGrid(rec, box, [C_H, O_A], rec_types=rt)
    rng = np.random.default_rng(9)
    pts = rng.uniform(-3, 3, size=(40, 3)) + box.center       # some outside: clamped cells
    lazy = O.OracleGrid.lazy(rec, box, [C_H, O_A], rt, pts)
    filled = ~np.isnan(lazy.maps)
    assert filled.any() and (~filled).any()
    np.testing.assert_array_equal(lazy.maps[filled], full.maps[filled])
    for p in pts:
        for t in (C_H, O_A):
            assert lazy.eval(t, p)[0] == full.eval(t, p)[0]
