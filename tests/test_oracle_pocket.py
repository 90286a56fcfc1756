"""Pins of the pocket-side oracle (Methods "Pocket Prediction with P2Rank", Eq. 1-2,
Supplementary Algorithm 1) against closed forms, hand-computed values, an independent library
routine (scipy's single-linkage clustering) and invariants."""
import math

import numpy as np
import pytest

import oracle as O


# ---------------------------------------------------------------- Step 1: lattice and SAS --

def test_lattice_unit_and_equal_area_strata():
    n = 997
    d = O.sphere_lattice(n)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    # z is equispaced, so any band z > c holds (1 - c) / 2 of the points up to one point
    for c in (-0.9, -0.3, 0.0, 0.25, 0.8):
        assert abs((d[:, 2] > c).sum() - n * (1 - c) / 2) <= 1.0


def test_lattice_caps_about_random_axes():
    # equal-area in every direction, which pins the azimuth step: a cap of angular radius t
    # about any axis holds (1 - cos t) / 2 of the points (Archimedes' hat-box theorem)
    n = 4000
    d = O.sphere_lattice(n)
    rng = np.random.default_rng(3)
    for _ in range(20):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        t = rng.uniform(0.3, 2.5)
        frac = (d @ ax > math.cos(t)).mean()
        assert abs(frac - (1 - math.cos(t)) / 2) < 0.01


def test_isolated_atom_keeps_every_point():
    keep, pts, margin = O.sas_points([[1.0, -2.0, 0.5]], [1.52], 1.6, 50)
    assert keep.all()
    assert np.allclose(np.linalg.norm(pts - [1.0, -2.0, 0.5], axis=1), 3.12, atol=1e-12)
    assert (margin > 1e299).all()


@pytest.mark.parametrize("d,r0,r1", [(3.0, 1.7, 1.7), (4.1, 1.55, 1.8), (1.2, 1.52, 1.7)])
def test_two_atoms_buried_cap_fraction(d, r0, r1):
    # atom 0's expanded sphere (radius a0) inside atom 1's (a1, centre at distance d) is a cap
    # of half-angle t with cos t = (d^2 + a0^2 - a1^2) / (2 d a0): its share is (1 - cos t) / 2
    probe, n = 1.6, 4000
    a0, a1 = r0 + probe, r1 + probe
    keep, _, margin = O.sas_points([[0, 0, 0], [d, 0, 0]], [r0, r1], probe, n)
    for i, (ai, aj) in enumerate(((a0, a1), (a1, a0))):
        cos_t = (d * d + ai * ai - aj * aj) / (2 * d * ai)
        buried = 1.0 - keep[i * n:(i + 1) * n].mean()
        assert abs(buried - (1 - cos_t) / 2) < 0.01
    assert ((margin >= 0) == (keep == 1)).all()


def test_engulfed_atom_is_fully_buried():
    keep, _, _ = O.sas_points([[0, 0, 0], [0.2, 0, 0]], [3.0, 1.0], 1.4, 64)
    assert keep[:64].all() and not keep[64:].any()


def test_sas_rule_against_kdtree():
    # a point is kept iff no OTHER atom's expanded sphere strictly contains it
    cKDTree = pytest.importorskip("scipy.spatial").cKDTree
    rng = np.random.default_rng(7)
    n, ns, probe = 40, 30, 1.6
    xyz = rng.uniform(-6, 6, size=(n, 3))
    rad = rng.choice([1.7, 1.55, 1.52, 1.8], size=n)
    keep, pts, _ = O.sas_points(xyz, rad, probe, ns)
    tree = cKDTree(xyz)
    for row in range(n * ns):
        i = row // ns
        near = tree.query_ball_point(pts[row], r=rad.max() + probe)
        inside = [j for j in near if j != i and np.linalg.norm(pts[row] - xyz[j]) < rad[j] + probe]
        assert keep[row] == (len(inside) == 0)
    sel = np.array([5, 0, 17], np.int32)
    k2, p2, _ = O.sas_points(xyz, rad, probe, ns, atoms=sel)
    for s, i in enumerate(sel):
        assert (k2[s * ns:(s + 1) * ns] == keep[i * ns:(i + 1) * ns]).all()
        assert np.array_equal(p2[s * ns:(s + 1) * ns], pts[i * ns:(i + 1) * ns])


# --------------------------------------------------------- Step 2: Eq. 1 and protrusion --

def test_features_hand_example():
    # atoms at distances 0, 3, 6, 7, 9.99, 10 and 10.01 from the point at the origin
    xyz = np.array([[0, 0, 0], [3, 0, 0], [0, 6, 0], [0, 0, 7], [9.99, 0, 0], [0, 0, -10.0],
                    [0, -10.01, 0]], float)
    props = np.array([[1, 0], [1, 2], [1, 4], [1, 8], [1, 16], [1, 32], [1, 64]], float)
    f, prot = O.point_features(xyz, props, [[0, 0, 0]])
    # weights 1, 1/2, 0, 0, ...: column 0 = 1.5, column 1 = 0.5 * 2
    assert np.allclose(f[0], [1.5, 1.0], atol=1e-15)
    assert prot[0] == 6                       # d <= 10 counts; 10.01 does not


def test_features_linear_and_rigid_invariant():
    rng = np.random.default_rng(11)
    xyz = rng.uniform(-8, 8, size=(300, 3))
    props = rng.normal(size=(300, 5))
    pts = rng.uniform(-6, 6, size=(50, 3))
    f, prot = O.point_features(xyz, props, pts)
    f2, _ = O.point_features(xyz, 2.0 * props[:, ::-1], pts)
    assert np.allclose(f2, 2.0 * f[:, ::-1], atol=1e-12)
    # rotate and translate atoms and points together
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    t = np.array([3.0, -1.0, 12.0])
    f3, prot3 = O.point_features(xyz @ q.T + t, props, pts @ q.T + t)
    assert np.allclose(f3, f, atol=1e-10)
    # counts agree except for atoms within rounding of the 10 A sphere
    d = np.linalg.norm(pts[:, None] - xyz[None], axis=2)
    assert (np.abs(d - 10.0) > 1e-9).all()
    assert np.array_equal(prot3, prot)
    assert np.array_equal(prot, (d <= 10.0).sum(1))


def test_features_radii_are_parameters():
    f, prot = O.point_features([[2.0, 0, 0]], [[1.0]], [[0, 0, 0]], r_feat=4.0, r_prot=1.5)
    assert abs(f[0, 0] - 0.5) < 1e-15 and prot[0] == 0


# --------------------------------------------- Steps 4-5: clusters, Eq. 2 score, ranking --

def test_single_linkage_matches_scipy():
    hier = pytest.importorskip("scipy.cluster.hierarchy")
    rng = np.random.default_rng(5)
    centres = rng.uniform(-20, 20, size=(6, 3))
    pts = np.concatenate([c + rng.normal(scale=1.6, size=(40, 3)) for c in centres])
    pts = np.concatenate([pts, rng.uniform(-25, 25, size=(60, 3))])
    n = pts.shape[0]
    score = np.ones(n)
    cl = O.cluster_points(pts, score, 0.5, 3.0)
    lab = hier.fcluster(hier.linkage(pts, method="single"), t=3.0, criterion="distance")
    # same partition: two points share a cluster on one side iff on the other
    same_o = cl.root[:, None] == cl.root[None, :]
    same_s = lab[:, None] == lab[None, :]
    assert np.array_equal(same_o, same_s)
    assert cl.size.sum() == n and len(cl.score) == len(np.unique(lab))
    # the root is the lowest index of the cluster
    for r in np.unique(cl.root):
        assert r == np.flatnonzero(cl.root == r).min()


def test_chain_links_at_three_angstrom_inclusive():
    pts = np.array([[0, 0, 0], [3, 0, 0], [6, 0, 0], [9, 0, 0], [12.5, 0, 0]], float)
    cl = O.cluster_points(pts, np.ones(5), 1.0, 3.0)
    # hops of exactly 3 A link (<=); 3.5 A does not; single linkage is transitive along the chain
    assert cl.root.tolist() == [0, 0, 0, 0, 4]
    assert cl.size.tolist() == [4, 1]


def test_threshold_score_center_and_ranking():
    pts = np.array([[0, 0, 0], [2, 0, 0], [20, 0, 0], [21, 1, 0], [40, 0, 0], [50, 0, 0], [60, 0, 0]],
                   float)
    s = np.array([0.5, 0.6, 0.9, 0.2, 0.3, 0.3, np.nan])
    cl = O.cluster_points(pts, s, 0.3)
    # 0.2 and NaN are below the threshold; 0.3 == theta is kept (the algorithm's >=)
    assert cl.root.tolist() == [0, 0, 2, -1, 4, 5, -1]
    # Eq. 2: 0.25 + 0.36 = 0.61, 0.81, 0.09 (twice: the tie goes to the lower index)
    assert np.allclose(cl.score, [0.81, 0.61, 0.09, 0.09], atol=1e-15)
    assert cl.first.tolist() == [2, 0, 4, 5]
    assert cl.size.tolist() == [1, 2, 1, 1]
    assert np.allclose(cl.center[1], [1, 0, 0]) and np.allclose(cl.center[0], [20, 0, 0])
    assert cl.cluster.tolist() == [1, 1, 0, -1, 2, 3, -1]


def test_cluster_degenerate_inputs():
    cl = O.cluster_points(np.zeros((0, 3)), np.zeros(0), 0.0)
    assert len(cl.score) == 0 and cl.root.shape == (0,)
    cl = O.cluster_points(np.zeros((5, 3)), np.full(5, 0.1), 0.5)
    assert len(cl.score) == 0 and (cl.cluster == -1).all()
    cl = O.cluster_points(np.zeros((5, 3)), np.full(5, 1.0), 0.5)
    assert cl.size.tolist() == [5] and abs(cl.score[0] - 5.0) < 1e-15
