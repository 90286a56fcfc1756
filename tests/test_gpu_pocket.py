"""GPU parity of the pocket-side steps (Supplementary Algorithm 1) against the FP64 oracle:
SAS points (Step 1), Eq. 1 feature sums and protrusion counts (Step 2), single-linkage clusters
with Eq. 2 scores, centres and ranking (Steps 4-5), and the pipeline from a receptor to ranked
pocket boxes that the docking consumes.

Inputs: seeded receptors of 1,500-8,000 atoms at 0.05 atoms per cubic A with carved spherical
pockets of radius 6-10 A (the full size is the 8,000-atom, 10-pocket receptor), Bondi radii, a
1.6 A probe, 50-100 lattice points per atom; clustering clouds of Gaussian blobs plus a uniform
background with uniform scores.

Decisions taken in float32 on the GPU and in float64 in the oracle (a point's burial, an atom inside
the protrusion sphere, a hop within the link distance) agree except within rounding of the
boundary: such cases are identified from the oracle's own margins and left out of exact
comparisons.
"""
import numpy as np
import pytest

import oracle as O
import pvsynth as S
from tests import _gpu as G

pytestmark = pytest.mark.gpu

EDGE = 1e-4        # A: decisions this close to a boundary may differ between float32 and float64
COORD_TOL = 1e-4   # A: a lattice point formed in float32 vs float64
PROT_EDGE = 2e-5   # A: |d - 10| below which float32 and float64 may count an atom differently


def _rec32(rec):
    return G.receptor32(rec)


def _radii32(rec):
    return np.asarray(S.vdw_radii(rec), np.float32).astype(np.float64)


def _params(**kw):
    from paper_2506_20043_gb300 import api
    return api.PocketParams(**kw)


def _surface_keys(surf, n_sphere):
    src = surf.sources()
    pts = surf.points().cpu().numpy().astype(np.float64)
    assert (np.diff(src) > 0).all()                      # ordered by (atom, k), no repeats
    return src, pts


def _check_sas(rec, surf, n_sphere, probe=1.6, atoms=None, radii=None):
    radii = _radii32(rec) if radii is None else radii
    keep, opts, margin = O.sas_points(rec.xyz, radii, probe, n_sphere, atoms=atoms)
    src, pts = _surface_keys(surf, n_sphere)
    if atoms is None:
        keys = np.arange(rec.n * n_sphere)
    else:
        keys = (np.asarray(atoms)[:, None] * n_sphere + np.arange(n_sphere)[None, :]).reshape(-1)
        sel = np.isin(src // n_sphere, atoms)
        src, pts = src[sel], pts[sel]
    gpu_keep = np.isin(keys, src)
    differ = gpu_keep != (keep == 1)
    assert (np.abs(margin[differ]) < EDGE).all(), "a burial decision differs away from the boundary"
    # coordinates of the points both sides keep
    row_of = {k: i for i, k in enumerate(keys)}
    both = np.array([row_of[k] for k in src if keep[row_of[k]]], dtype=np.int64)
    gsel = np.array([keep[row_of[k]] == 1 for k in src])
    assert np.abs(pts[gsel] - opts[both]).max(initial=0.0) <= COORD_TOL
    return int(differ.sum()), int(keep.sum())


@pytest.mark.parametrize("n_sphere", [50, 100])
def test_sas_points_parity(n_sphere):
    ctx = G.context()
    site = S.pocket_site(1, 1500, 2)
    rec = _rec32(site.receptor)
    surf = ctx.surface(rec, params=_params(n_sphere=n_sphere))   # Bondi radii built in
    assert surf.n_atoms == rec.n
    differ, kept = _check_sas(rec, surf, n_sphere)
    assert kept > 1000 and differ <= 3


def test_sas_points_full_size_sampled():
    # the 8,000-atom / 10-pocket receptor at 100 points per atom; 300 sampled atoms plus the
    # first and last atom against the oracle
    ctx = G.context()
    site = S.pocket_site(0, 8000, 10)
    rec = _rec32(site.receptor)
    surf = ctx.surface(rec, params=_params(n_sphere=100))
    rng = np.random.default_rng(4)
    atoms = np.unique(np.concatenate([[0, rec.n - 1], rng.choice(rec.n, 300, replace=False)])).astype(np.int32)
    differ, kept = _check_sas(rec, surf, 100, atoms=atoms)
    assert kept > 100 and differ <= 3
    assert surf.n_points > 10000


def test_sas_custom_radii_device_memory():
    torch = pytest.importorskip("torch")
    ctx = G.context()
    site = S.pocket_site(2, 1200, 1)
    rec = _rec32(site.receptor)
    rng = np.random.default_rng(9)
    radii = rng.uniform(1.2, 2.4, size=rec.n).astype(np.float32)
    drec = S.Receptor(torch.tensor(rec.xyz, dtype=torch.float32, device="cuda"),
                      torch.tensor(rec.element, device="cuda"), torch.tensor(rec.donor, device="cuda"),
                      torch.tensor(rec.acceptor, device="cuda"))
    surf = ctx.surface(drec, radius=torch.tensor(radii, device="cuda"), params=_params(n_sphere=64, probe=1.4))
    differ, kept = _check_sas(rec, surf, 64, probe=1.4, radii=radii.astype(np.float64))
    assert kept > 500 and differ <= 3


def test_sas_edge_cases():
    from paper_2506_20043_gb300.api import PVError
    ctx = G.context()
    one = S.Receptor(np.array([[1.0, 2.0, 3.0]]), np.array([2], np.uint8), np.zeros(1, np.uint8), np.zeros(1, np.uint8))
    s = ctx.surface(one, params=_params(n_sphere=37))
    assert s.n_points == 37
    d = np.linalg.norm(s.points().cpu().numpy() - [1, 2, 3], axis=1)
    assert np.allclose(d, 1.52 + 1.6, atol=1e-5)
    s = ctx.surface(one, params=_params(n_sphere=1))
    assert s.n_points == 1
    # a small atom inside a large one has no surface; the large one keeps every point
    two = S.Receptor(np.array([[0.0, 0, 0], [0.2, 0, 0]]), np.array([3, 2], np.uint8), np.zeros(2, np.uint8),
                     np.zeros(2, np.uint8))
    s = ctx.surface(two, radius=np.array([3.0, 1.0], np.float32), params=_params(n_sphere=64, probe=1.4))
    assert s.n_points == 64 and (s.sources() < 64).all()
    bad = S.Receptor(np.zeros((3, 3)), np.array([0, 7, 1], np.uint8), np.zeros(3, np.uint8), np.zeros(3, np.uint8))
    with pytest.raises(PVError, match="ARG"):
        ctx.surface(bad)
    with pytest.raises(PVError, match="ARG"):
        ctx.surface(one, radius=np.array([0.0], np.float32))
    nan = S.Receptor(np.array([[0.0, np.nan, 0.0]]), np.zeros(1, np.uint8), np.zeros(1, np.uint8), np.zeros(1, np.uint8))
    with pytest.raises(PVError, match="ARG"):
        ctx.surface(nan)
    with pytest.raises(PVError, match="ARG"):
        ctx.surface(one, params=_params(n_sphere=2000))


# ------------------------------------------------------------------ Eq. 1 + protrusion --

def _check_features(rec, props, pts, feat, prot, r_feat=6.0, r_prot=10.0):
    ref, _ = O.point_features(rec.xyz, props, pts, r_feat, r_prot)
    # an atom within PROT_EDGE of the protrusion sphere may count on either side (float32 d^2)
    lo = O.point_features(rec.xyz, props[:, :1], pts, r_feat, r_prot - PROT_EDGE)[1]
    hi = O.point_features(rec.xyz, props[:, :1], pts, r_feat, r_prot + PROT_EDGE)[1]
    ok = G.close(feat, ref)
    assert ok.all(), f"{(~ok).sum()} feature sums off; worst {np.abs(feat - ref).max()}"
    assert ((prot >= lo) & (prot <= hi)).all()
    assert (lo == hi).mean() > 0.99


@pytest.mark.parametrize("n_props", [7, 20])
def test_features_at_given_points(n_props):
    ctx = G.context()
    site = S.pocket_site(3, 3000, 3)
    rec = _rec32(site.receptor)
    props = S.atom_properties(rec, 3)
    if n_props > props.shape[1]:
        rng = np.random.default_rng(5)
        props = np.concatenate([props, rng.normal(size=(rec.n, n_props - props.shape[1])).astype(np.float32)], axis=1)
    surf = ctx.surface(rec)
    rng = np.random.default_rng(6)
    lo, hi = rec.xyz.min(0) - 4, rec.xyz.max(0) + 4
    pts = rng.uniform(lo, hi, size=(3001, 3)).astype(np.float32).astype(np.float64)
    feat, prot = surf.features(props, points=pts)
    _check_features(rec, props.astype(np.float64), pts, feat.cpu().numpy(), prot.cpu().numpy())


def test_features_at_surface_points():
    # the surface's own points (the pipeline's call) against the oracle at the oracle's points
    ctx = G.context()
    site = S.pocket_site(4, 2000, 2)
    rec = _rec32(site.receptor)
    props = S.atom_properties(rec, 4).astype(np.float64)
    surf = ctx.surface(rec, params=_params(n_sphere=60))
    feat, prot = surf.features(props)
    src = surf.sources()
    keep, opts, margin = O.sas_points(rec.xyz, _radii32(rec), 1.6, 60)
    both = keep[src] == 1
    ref_pts = opts[src[both]]
    _check_features(rec, props, ref_pts, feat.cpu().numpy()[both], prot.cpu().numpy()[both])


def test_features_full_size_sampled():
    # the bench's configuration (8,000 atoms, 100 points per atom, 7 columns), 1,000 sampled surface
    # points: GPU sums at the GPU's points against the oracle's at its own points of the same keys
    ctx = G.context()
    site = S.pocket_site(0, 8000, 10)
    rec = _rec32(site.receptor)
    props = S.atom_properties(rec, 0).astype(np.float64)
    surf = ctx.surface(rec, params=_params(n_sphere=100))
    feat, prot = surf.features(props)
    src = surf.sources()
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(len(src), 1000, replace=False))
    atoms = np.unique(src[rows] // 100).astype(np.int32)
    keep, opts, _ = O.sas_points(rec.xyz, _radii32(rec), 1.6, 100, atoms=atoms)
    row_of = {int(a) * 100 + k: i * 100 + k for i, a in enumerate(atoms) for k in range(100)}
    orow = np.array([row_of[int(k)] for k in src[rows]])
    both = keep[orow] == 1
    assert both.mean() > 0.99
    _check_features(rec, props, opts[orow[both]], feat.cpu().numpy()[rows[both]], prot.cpu().numpy()[rows[both]])


def test_features_edge_cases():
    torch = pytest.importorskip("torch")
    ctx = G.context()
    site = S.pocket_site(5, 1000, 1)
    rec = _rec32(site.receptor)
    props = S.atom_properties(rec, 5).astype(np.float64)
    surf = ctx.surface(rec)
    # no points; one point far away; a non-finite point
    f, p = surf.features(props, points=np.zeros((0, 3)))
    assert f.shape == (0, 7)
    pts = np.array([[500.0, 0, 0], [np.nan, 0, 0], [0.0, 0.0, 0.0]])
    f, p = surf.features(props, points=pts)
    f, p = f.cpu().numpy(), p.cpu().numpy()
    assert (f[:2] == 0).all() and (p[:2] == 0).all()
    _check_features(rec, props, pts[2:], f[2:], p[2:])
    from paper_2506_20043_gb300.api import PVError
    with pytest.raises(PVError):
        surf.features(np.zeros((rec.n, 0), np.float32), points=pts)


# -------------------------------------------------------------------------- clusters --

def _stable_partition(pts, score, theta, link):
    a = O.cluster_points(pts, score, theta, link - 1e-5)
    b = O.cluster_points(pts, score, theta, link + 1e-5)
    return np.array_equal(a.root, b.root)


def _check_clusters(gpu, ref):
    assert len(gpu["score"]) == len(ref.score)
    assert np.array_equal(gpu["cluster"], ref.cluster)
    assert np.array_equal(gpu["size"], ref.size) and np.array_equal(gpu["first"], ref.first)
    assert np.allclose(gpu["score"], ref.score, rtol=1e-6, atol=1e-6)
    assert np.abs(gpu["center"] - ref.center).max(initial=0.0) <= 1e-4


@pytest.mark.parametrize("seed,n_blobs,per_blob,n_bg", [(0, 20, 500, 5003), (1, 3, 40, 17), (2, 60, 300, 20000)])
def test_cluster_parity(seed, n_blobs, per_blob, n_bg):
    ctx = G.context()
    pts, sc = S.cluster_cloud(seed, n_blobs, per_blob, n_bg)
    p64, s64 = pts.astype(np.float64), sc.astype(np.float64)
    assert _stable_partition(p64, s64, 0.5, 3.0)
    ref = O.cluster_points(p64, s64, 0.5, 3.0)
    gpu = ctx.cluster(pts, sc, _params(threshold=0.5, link=3.0)).read()
    _check_clusters(gpu, ref)


def test_cluster_edge_cases():
    ctx = G.context()
    from paper_2506_20043_gb300.api import PVError
    c = ctx.cluster(np.zeros((0, 3)), np.zeros(0))
    assert c.n_clusters == 0 and c.read()["cluster"].shape == (0,)
    c = ctx.cluster(np.zeros((5, 3)), np.full(5, 0.1))
    assert c.n_clusters == 0 and (c.read()["cluster"] == -1).all()
    r = ctx.cluster(np.zeros((5, 3)), np.ones(5)).read()
    assert r["size"].tolist() == [5] and abs(r["score"][0] - 5.0) < 1e-6
    # threshold inclusive, NaN score excluded, exact 3 A hops link, ties by lowest index
    pts = np.array([[0, 0, 0], [3, 0, 0], [6, 0, 0], [40, 0, 0], [50, 0, 0], [60, 0, 0]], np.float32)
    sc = np.array([0.5, 0.5, np.nan, 0.7, 0.7, 0.2], np.float32)
    r = ctx.cluster(pts, sc, _params(threshold=0.5)).read()
    ref = O.cluster_points(pts.astype(np.float64), sc.astype(np.float64), 0.5, 3.0)
    _check_clusters(r, ref)
    assert r["cluster"].tolist() == [0, 0, -1, 1, 2, -1]
    # a non-finite coordinate is an error on a clustered point only
    bad = pts.copy()
    bad[5, 0] = np.inf
    ctx.cluster(bad, sc)
    sc2 = sc.copy()
    sc2[5] = 1.0
    with pytest.raises(PVError, match="ARG"):
        ctx.cluster(bad, sc2)
    with pytest.raises(PVError, match="ARG"):
        ctx.cluster(pts, sc, _params(link=0.0))


# ------------------------------------------------------------------- batched calls --

def test_batched_calls_equal_single_calls():
    # pv_surface_create_many / pv_cluster_points_many: bit-for-bit the results of one call each,
    # with host and device receptors, default and given radii, an empty point set, and an error in
    # one receptor failing the whole call without leaving the context unusable
    torch = pytest.importorskip("torch")
    from paper_2506_20043_gb300.api import PVError
    ctx = G.context()
    sites = [S.pocket_site(20 + k, n, 2) for k, n in enumerate((900, 1500, 1200))]
    recs = [_rec32(s.receptor) for s in sites]
    drec = S.Receptor(torch.tensor(recs[1].xyz, dtype=torch.float32, device="cuda"),
                      torch.tensor(recs[1].element, device="cuda"), torch.tensor(recs[1].donor, device="cuda"),
                      torch.tensor(recs[1].acceptor, device="cuda"))
    rad2 = np.random.default_rng(3).uniform(1.3, 2.2, size=recs[2].n).astype(np.float32)
    prm = _params(n_sphere=60)
    many = ctx.surfaces([recs[0], drec, recs[2]], radii=[None, None, rad2], params=prm)
    single = [ctx.surface(recs[0], params=prm), ctx.surface(recs[1], params=prm),
              ctx.surface(recs[2], radius=rad2, params=prm)]
    scores = []
    for k, (a, b) in enumerate(zip(many, single)):
        assert a.n_points == b.n_points > 0
        assert np.array_equal(a.sources(), b.sources())
        assert torch.equal(a.points(), b.points())
        props = S.atom_properties(recs[k], k)
        fa, pa = a.features(props)
        fb, pb = b.features(props)
        assert torch.equal(fa, fb) and torch.equal(pa, pb)
        scores.append(S.ligandability(b.points().cpu().numpy(), sites[k], k, noise=0.0))
    cm = ctx.cluster_many([(a, sc) for a, sc in zip(many, scores)] + [(np.zeros((0, 3)), np.zeros(0))])
    assert len(cm) == 4 and cm[3].n_clusters == 0 and cm[3].n_points == 0
    for c, b, sc in zip(cm, single, scores):
        r1, r2 = c.read(), ctx.cluster(b.points(), sc).read()
        assert r1.keys() == r2.keys() and all(np.array_equal(r1[x], r2[x]) for x in r1)
        assert len(r1["score"]) >= 1
    bad = S.Receptor(np.zeros((3, 3)), np.array([0, 7, 1], np.uint8), np.zeros(3, np.uint8), np.zeros(3, np.uint8))
    with pytest.raises(PVError, match="ARG"):
        ctx.surfaces([recs[0], bad], params=prm)
    again = ctx.surfaces([recs[0]], params=prm)
    assert len(again) == 1 and np.array_equal(again[0].sources(), single[0].sources())


# ------------------------------------------------------------------ receptor -> boxes --

def test_pocket_pipeline_matches_oracle_and_docks():
    # Supplementary Algorithm 1 end to end on each side (the score stands in for the classifier),
    # then Algorithm 3's boxes on the ranked centres go to the grid build and the docking
    torch = pytest.importorskip("torch")
    ctx = G.context()
    site = S.pocket_site(6, 5000, 5)
    rec = _rec32(site.receptor)
    surf = ctx.surface(rec, params=_params(n_sphere=80))
    gpts = surf.points()
    gsc = S.ligandability(gpts.cpu().numpy(), site, 6, noise=0.0)
    cl = ctx.cluster(gpts, gsc)
    gpu = cl.read()
    keep, opts, _ = O.sas_points(rec.xyz, _radii32(rec), 1.6, 80)
    opts = opts[keep == 1].astype(np.float32).astype(np.float64)
    osc = S.ligandability(opts, site, 6, noise=0.0).astype(np.float64)
    ref = O.cluster_points(opts, osc, 0.5, 3.0)
    # the largest clusters (the carved pockets) agree; a borderline point can move a stray singleton
    big = ref.size >= 20
    assert big.sum() >= 3
    for c, s in zip(ref.center[big], ref.size[big]):
        j = np.argmin(np.linalg.norm(gpu["center"] - c, axis=1))
        assert np.linalg.norm(gpu["center"][j] - c) < 0.05 and abs(int(gpu["size"][j]) - int(s)) <= 2
    # every top cluster sits in a carved pocket
    for c in gpu["center"][:3]:
        assert (np.linalg.norm(site.centers - c, axis=1) < site.radii).any()
    boxes = cl.boxes(size=20.0, max_pockets=3)
    lig = G.ligand32(S.ligand_centered(S.make_ligand(20, 4, 6)))
    gs = ctx.build_grids(rec, boxes)
    res = ctx.dock(gs, [ctx.ligand(lig)], [0, 1, 2], chains=32, steps=50, seed=6, top_k=3)
    poses, n_kept, _, _ = res.fetch()
    assert (np.asarray(n_kept) > 0).all()
