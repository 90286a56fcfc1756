"""Pins of the oracle's torsion tree, forward kinematics (Eq. 1) and SF = e_inter + e_intra (Eq. 3)
with its analytic gradient.

Kinematics: psi = 0 reproduces the input, bond lengths / angles and rigid fragments are
preserved, 2 pi is the identity, a torsion changes its dihedral by exactly psi (right-handed),
the quaternion convention rotates x towards y about +z. Score: e_intra invariant under rigid
motion, e_inter invariant when receptor and box move together, gradient equal to central
finite differences (FP64), intra pairs of a hand-built chain equal the rule's enumeration.
"""
import math

import numpy as np
import pytest

import oracle as O
import pvsynth as S


def _lig(n=24, n_rot=6, seed=3):
    return S.ligand_centered(S.make_ligand(n, n_rot, seed))


def _identity_pot(L):
    pot = np.zeros(L.n_pot)
    pot[0:3] = L.src.xyz[L.origin]
    pot[3] = 1.0
    return pot


def _random_pot(L, rng):
    pot = np.zeros(L.n_pot)
    pot[0:3] = rng.normal(size=3) * 3
    q = rng.normal(size=4)
    pot[3:7] = q / np.linalg.norm(q)
    pot[7:] = rng.uniform(-math.pi, math.pi, size=L.n_rot)
    return pot


def _dihedral(a, b, c, d):
    b0, b1, b2 = a - b, c - b, d - c
    b1n = b1 / np.linalg.norm(b1)
    v = b0 - np.dot(b0, b1n) * b1n
    w = b2 - np.dot(b2, b1n) * b1n
    return math.atan2(np.dot(np.cross(b1n, v), w), np.dot(v, w))


def test_tree_structure():
    lig = _lig()
    L = O.OracleLigand(lig)
    assert L.n_rot == int(lig.rotatable.sum())
    assert L.n_frag == L.n_rot + 1                   # acyclic: each torsion splits one fragment
    sizes = np.bincount(L.frag_of)
    assert sizes[L.root] == sizes.max()
    assert L.frag_of[L.origin] == L.root
    assert L.origin == np.nonzero(L.frag_of == L.root)[0][0]
    rb = lig.bonds[lig.rotatable.astype(bool)]
    for k in range(L.n_rot):                          # torsion k = k-th rotatable bond
        assert {int(L.tor_p[k]), int(L.tor_c[k])} == {int(rb[k][0]), int(rb[k][1])}


def test_psi_zero_reproduces_input():
    for seed in range(5):
        lig = _lig(seed=seed)
        L = O.OracleLigand(lig)
        np.testing.assert_allclose(L.fk(_identity_pot(L)), lig.xyz, atol=1e-12)


def test_bonds_angles_fragments_preserved():
    rng = np.random.default_rng(0)
    for seed in range(6):
        lig = _lig(n=30, n_rot=8, seed=seed)
        L = O.OracleLigand(lig)
        ref = lig.xyz
        d_ref = np.linalg.norm(ref[:, None] - ref[None], axis=2)
        same = L.frag_of[:, None] == L.frag_of[None]
        nb = [[] for _ in range(L.n)]
        for a, b in lig.bonds:
            nb[a].append(b)
            nb[b].append(a)
        for _ in range(5):
            x = L.fk(_random_pot(L, rng))
            d = np.linalg.norm(x[:, None] - x[None], axis=2)
            for a, b in lig.bonds:
                assert d[a, b] == pytest.approx(d_ref[a, b], abs=1e-10)
            for c in range(L.n):                       # bond angles: 1-3 distances
                for i in nb[c]:
                    for j in nb[c]:
                        if i < j:
                            assert d[i, j] == pytest.approx(d_ref[i, j], abs=1e-10)
            np.testing.assert_allclose(d[same], d_ref[same], atol=1e-10)


def test_full_turn_is_identity_and_dihedral_sign():
    rng = np.random.default_rng(1)
    lig = _lig(n=20, n_rot=4, seed=11)
    L = O.OracleLigand(lig)
    base = _random_pot(L, rng)
    x0 = L.fk(base)
    for k in range(L.n_rot):
        p = base.copy()
        p[7 + k] += 2 * math.pi
        np.testing.assert_allclose(L.fk(p), x0, atol=1e-10)
    nb = [[] for _ in range(L.n)]
    for a, b in lig.bonds:
        nb[a].append(b)
        nb[b].append(a)
    for k in range(L.n_rot):
        pa, ca = int(L.tor_p[k]), int(L.tor_c[k])
        a = [v for v in nb[pa] if v != ca][0]
        d = [v for v in nb[ca] if v != pa][0]
        for delta in (0.3, -1.1, 2.0):
            p = base.copy()
            p[7 + k] += delta
            x1 = L.fk(p)
            before = _dihedral(x0[a], x0[pa], x0[ca], x0[d])
            after = _dihedral(x1[a], x1[pa], x1[ca], x1[d])
            change = (after - before + math.pi) % (2 * math.pi) - math.pi
            # right-handed rotation of the far side about root-side -> far-side axis
            assert change == pytest.approx(delta, abs=1e-9)


def test_quaternion_convention():
    lig = _lig(n=12, n_rot=0, seed=2)
    L = O.OracleLigand(lig)
    pot = _identity_pot(L)
    th = 0.7
    pot[3:7] = [math.cos(th / 2), 0, 0, math.sin(th / 2)]    # rotation by th about +z
    x = L.fk(pot)
    o = lig.xyz[L.origin]
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    np.testing.assert_allclose(x, (lig.xyz - o) @ R.T + o, atol=1e-12)
    # tangent step: rotation vector w applied in the world frame about the origin atom
    w = np.array([0.1, -0.2, 0.3])
    p2 = L.retract(pot, np.concatenate([[0, 0, 0], w]))
    ang = np.linalg.norm(w)
    ax = w / ang
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rw = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
    np.testing.assert_allclose(L.fk(p2), (x - o) @ Rw.T + o, atol=1e-12)


def test_intra_pairs_of_a_chain():
    # linear chain 0-1-2-3-4-5-6, bonds 1-2 and 4-5 rotatable: fragments {0,1} {2,3,4} {5,6}
    n = 7
    xyz = np.zeros((n, 3))
    for i in range(1, n):
        ang = 0.955 * (1 if i % 2 else -1)
        xyz[i] = xyz[i - 1] + 1.5 * np.array([math.cos(ang * (i % 2)), math.sin(ang * (i % 2)), 0.1 * i])
    lig = S.Ligand(xyz, np.zeros(n, np.uint8), np.zeros(n, np.uint8), np.zeros(n, np.uint8),
                   np.array([[i, i + 1] for i in range(n - 1)], np.int32),
                   np.array([0, 1, 0, 0, 1, 0], np.uint8))
    L = O.OracleLigand(lig)
    assert L.n_frag == 3
    assert L.root == L.frag_of[2]                 # the 3-atom fragment is the root
    got = {tuple(p) for p in L.pairs}
    # different fragments and more than three bonds apart
    assert got == {(0, 4), (0, 5), (0, 6), (1, 5), (1, 6), (2, 6)}


def _small_site(seed=0, box_size=9.0):
    rec = S.make_receptor(900, seed, [(np.zeros(3), 5.0)])
    box = S.Box(np.zeros(3), np.array([box_size] * 3), 0.375)
    return rec, box


def test_intra_rigid_invariance_and_inter_moves_with_receptor():
    rec, box = _small_site()
    lig = _lig(n=20, n_rot=5, seed=4)
    L = O.OracleLigand(lig)
    rt = O.xs_type_receptor(rec)
    G = O.OracleGrid(rec, box, L.xs, rec_types=rt)
    rng = np.random.default_rng(2)
    pot = _random_pot(L, rng)
    pot[0:3] = rng.uniform(-3, 3, size=3)
    _, _, parts = L.score(G, pot)
    for _ in range(5):
        p2 = pot.copy()
        p2[0:3] += rng.normal(size=3)
        p2 = L.retract(p2, np.concatenate([[0, 0, 0], rng.normal(size=3), np.zeros(L.n_rot)]))
        assert L.score(G, p2)[2][1] == pytest.approx(parts[1], rel=1e-10, abs=1e-12)
    # receptor + box translated by a whole number of grid steps and rotated by 90 deg about z:
    # the maps of the moved system sample the same field at the moved nodes
    rot = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float)
    shift = np.array([0.375 * 4, -0.375 * 8, 0.375 * 2])
    rec2 = S.Receptor(rec.xyz @ rot.T + shift, rec.element, rec.donor, rec.acceptor)
    box2 = S.Box(box.center @ rot.T + shift, box.size, box.spacing)
    G2 = O.OracleGrid(rec2, box2, L.xs, rec_types=rt)
    qz = np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])
    p2 = pot.copy()
    p2[0:3] = pot[0:3] @ rot.T + shift
    q = pot[3:7]
    p2[3:7] = [qz[0] * q[0] - qz[3] * q[3], qz[0] * q[1] - qz[3] * q[2],
               qz[0] * q[2] + qz[3] * q[1], qz[0] * q[3] + qz[3] * q[0]]
    np.testing.assert_allclose(L.fk(p2), L.fk(pot) @ rot.T + shift, atol=1e-10)
    _, _, parts2 = L.score(G2, p2)
    assert parts2[0] == pytest.approx(parts[0], rel=1e-9, abs=1e-9)
    assert parts2[1] == pytest.approx(parts[1], rel=1e-9, abs=1e-9)


def _fd_ok(L, G, pot, h):
    """True when no atom sits within h*lever of a cell face and no pair near a term kink."""
    x = L.fk(pot)
    frac = (x - G.origin) / G.spacing % 1.0
    if (np.minimum(frac, 1 - frac) < 2e-3).any():
        return False
    return True


def test_gradient_matches_central_differences():
    rec, box = _small_site(seed=1)
    rt = O.xs_type_receptor(rec)
    rng = np.random.default_rng(3)
    checked = 0
    for seed in range(4):
        lig = _lig(n=18 + 4 * seed, n_rot=2 + seed, seed=20 + seed)
        L = O.OracleLigand(lig)
        G = O.OracleGrid(rec, box, L.xs, rec_types=rt)
        for _ in range(10):
            pot = _random_pot(L, rng)
            pot[0:3] = rng.uniform(-4, 4, size=3)
            if not _fd_ok(L, G, pot, 1e-5):
                continue
            e, g, _ = L.score(G, pot)
            h = 1e-6
            fd = np.zeros_like(g)
            for k in range(len(g)):
                s = np.zeros(len(g))
                s[k] = h
                fd[k] = (L.score(G, L.retract(pot, s))[0] - L.score(G, L.retract(pot, -s))[0]) / (2 * h)
            np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-5 * max(1.0, np.abs(fd).max()))
            checked += 1
    assert checked >= 20


def test_score_parts_add_up_and_translation_grad_is_force_sum():
    rec, box = _small_site(seed=2)
    lig = _lig(n=16, n_rot=3, seed=9)
    L = O.OracleLigand(lig)
    G = O.OracleGrid(rec, box, L.xs, rec_types=O.xs_type_receptor(rec))
    pot = _random_pot(L, np.random.default_rng(4))
    pot[0:3] = [1.0, -0.5, 0.2]
    e, g, parts = L.score(G, pot)
    assert e == pytest.approx(parts.sum(), rel=1e-14)
    ea, dx = L.score_atoms(G, L.fk(pot))
    assert ea == pytest.approx(e, rel=1e-13)
    np.testing.assert_allclose(g[0:3], dx.sum(axis=0), rtol=1e-12, atol=1e-12)
