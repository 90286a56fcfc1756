"""GPU parity of pose scoring (Eq. 3) and its adjoint gradient against the FP64 oracle, plus the
autograd function against central finite differences.

Score+adjoint workload shapes: a 4,000-atom receptor with a 24 A box, a 32-atom ligand with 8
torsions, random poses (uniform translation in the box, uniform quaternion, torsions in
[-pi, pi)). Every pose of a few-thousand batch is compared with the oracle; at the full
65,536-pose size a sample is compared using oracle maps filled at the nodes those poses touch.
"""
import numpy as np
import pytest

import oracle as O
import pvsynth as S
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _site(n_rec=4000, box_size=24.0, n_atoms=32, n_rot=8, seed=0):
    rec = G.receptor32(S.make_receptor(n_rec, seed, [(np.zeros(3), 8.0)]))
    box = G.box32(S.Box(np.zeros(3), np.array([box_size] * 3), 0.375))
    lig = G.ligand32(S.ligand_centered(S.make_ligand(n_atoms, n_rot, seed)))
    return rec, box, lig


def _near_face(xyz, box, tol=2e-4):
    origin, _ = O.grid_geometry(box)
    f = (xyz - origin) / box.spacing % 1.0
    return (np.minimum(f, 1 - f) < tol).any(axis=-1).any(axis=-1)


def _run(ctx, rec, box, lig, poses, lazy=True):
    torch = pytest.importorskip("torch")
    L = O.OracleLigand(lig)
    gs = ctx.build_grids(rec, [box], sorted(set(L.xs.tolist())))
    pl = ctx.ligand(lig)
    assert pl.n_rot == L.n_rot and pl.n_pairs == L.n_pairs and pl.origin == L.origin
    assert (pl.xs_types == L.xs).all()
    p32 = torch.tensor(poses, dtype=torch.float32, device="cuda")
    e, g, parts = ctx.score(gs, pl, 0, p32, grad=True, parts=True)
    poses64 = p32.double().cpu().numpy()
    xyz = np.stack([L.fk(p) for p in poses64])
    rt = O.xs_type_receptor(rec)
    og = O.OracleGrid.lazy(rec, box, L.xs, rt, xyz, threads=G.threads()) if lazy else \
        O.OracleGrid(rec, box, L.xs, rec_types=rt, threads=G.threads())
    ref = [L.score(og, p) for p in poses64]
    return (e.cpu().numpy(), g.cpu().numpy(), parts.cpu().numpy(), np.array([r[0] for r in ref]),
            np.stack([r[1] for r in ref]), np.stack([r[2] for r in ref]), xyz, gs, pl, L, og)


def test_score_and_gradient_match_oracle():
    ctx = G.context()
    rec, box, lig = _site(n_rec=4000, box_size=12.0)
    poses = S.random_poses(3000, box, int(lig.rotatable.sum()), seed=1)
    e, g, parts, er, gr, pr, xyz, *_ = _run(ctx, rec, box, lig, poses, lazy=False)
    assert G.close(e, er).all(), np.abs(e - er).max()
    assert G.close(parts, pr).all()
    face = _near_face(xyz, box)
    ok = np.abs(g - gr) <= G.GRAD_TOL * np.maximum(np.abs(gr), 1.0)
    bad = ~ok.all(axis=1) & ~face
    assert bad.sum() == 0, (np.argwhere(bad)[:5], np.abs(g - gr).max())


def test_full_size_microbench_sampled():
    """The 65,536-pose workload on the GPU; 256 sampled poses checked against the oracle."""
    torch = pytest.importorskip("torch")
    ctx = G.context()
    rec, box, lig, poses = S.score_microbench()
    rec, box, lig = G.receptor32(rec), G.box32(box), G.ligand32(lig)
    L = O.OracleLigand(lig)
    gs = ctx.build_grids(rec, [box], sorted(set(L.xs.tolist())))
    pl = ctx.ligand(lig)
    p32 = torch.tensor(poses, dtype=torch.float32, device="cuda")
    e, g, _ = ctx.score(gs, pl, 0, p32)
    assert torch.isfinite(e).all() and torch.isfinite(g).all()
    idx = np.random.default_rng(0).choice(len(poses), 256, replace=False)
    poses64 = p32[idx].double().cpu().numpy()
    xyz = np.stack([L.fk(p) for p in poses64])
    og = O.OracleGrid.lazy(rec, box, L.xs, O.xs_type_receptor(rec), xyz, threads=G.threads())
    ref = np.array([L.score(og, p, want_grad=False)[0] for p in poses64])
    assert G.close(e.cpu().numpy()[idx], ref).all()


def test_pose_coords_match_oracle_kinematics():
    torch = pytest.importorskip("torch")
    ctx = G.context()
    for n_atoms, n_rot, seed in [(10, 0, 1), (32, 8, 2), (60, 15, 3), (64, 26, 4)]:
        lig = G.ligand32(S.ligand_centered(S.make_ligand(n_atoms, n_rot, seed)))
        L = O.OracleLigand(lig)
        pl = ctx.ligand(lig)
        box = S.Box(np.zeros(3), np.array([10.0] * 3))
        poses = S.random_poses(500, box, L.n_rot, seed)
        p32 = torch.tensor(poses, dtype=torch.float32, device="cuda")
        x = ctx.pose_coords(pl, p32).cpu().numpy()
        ref = np.stack([L.fk(p) for p in p32.double().cpu().numpy()])
        np.testing.assert_allclose(x, ref, atol=2e-4)


def test_autograd_pose_gradient_vs_fd_and_oracle():
    torch = pytest.importorskip("torch")
    from paper_2506_20043_gb300.api import PVScore
    ctx = G.context()
    rec, box, lig = _site(n_rec=3000, box_size=10.0, n_atoms=24, n_rot=5, seed=4)
    L = O.OracleLigand(lig)
    gs = ctx.build_grids(rec, [box], sorted(set(L.xs.tolist())))
    pl = ctx.ligand(lig)
    poses = S.random_poses(64, box, L.n_rot, seed=5)
    poses[:, 3:7] *= np.random.default_rng(6).uniform(0.5, 2.0, size=(64, 1))   # non-unit quaternions
    p = torch.tensor(poses, dtype=torch.float32, device="cuda", requires_grad=True)
    e = PVScore.apply(p, ctx, gs, pl, 0)
    w = torch.linspace(0.5, 1.5, 64, device="cuda")
    (e * w).sum().backward()
    got = p.grad.cpu().numpy() / w.cpu().numpy()[:, None]
    # reference: central differences of the FP64 oracle over the raw POT entries
    p64 = p.detach().double().cpu().numpy()
    og = O.OracleGrid(rec, box, L.xs, rec_types=O.xs_type_receptor(rec), threads=G.threads())
    checked = 0
    for i in range(64):
        if _near_face(L.fk(p64[i])[None], box, tol=1e-3)[0]:
            continue
        h = 1e-6
        fd = np.zeros(L.n_pot)
        for k in range(L.n_pot):
            a, b = p64[i].copy(), p64[i].copy()
            a[k] += h
            b[k] -= h
            fd[k] = (L.score(og, a, False)[0] - L.score(og, b, False)[0]) / (2 * h)
        assert (np.abs(got[i] - fd) <= G.GRAD_TOL * np.maximum(np.abs(fd), 1.0)).all(), (i, got[i], fd)
        checked += 1
    assert checked >= 40
    # FP32 central differences of the GPU score itself (h = 1e-3): compared on components where
    # the field is smooth over +-h (the FP64 oracle's differences at h = 1e-3 and 1e-6 agree),
    # since a step of 1e-3 can carry an atom across a grid-cell face or a term's kink
    compared = 0
    for i in range(16):
        base = p.detach()[i:i + 1].clone()
        for k in range(L.n_pot):
            h3 = []
            for h in (1e-3, 1e-6):
                a, b = p64[i].copy(), p64[i].copy()
                a[k] += h
                b[k] -= h
                h3.append((L.score(og, a, False)[0] - L.score(og, b, False)[0]) / (2 * h))
            if abs(h3[0] - h3[1]) > 1e-3 * max(abs(h3[1]), 1.0):
                continue
            a, b = base.clone(), base.clone()
            a[0, k] += 1e-3
            b[0, k] -= 1e-3
            fd32 = ((ctx.score(gs, pl, 0, a, grad=False)[0] - ctx.score(gs, pl, 0, b, grad=False)[0]) / 2e-3).item()
            assert abs(got[i, k] - fd32) <= 2e-2 * max(abs(fd32), 1.0), (i, k, got[i, k], fd32)
            compared += 1
    assert compared >= 50


def test_coordinate_gradient_matches_oracle():
    torch = pytest.importorskip("torch")
    ctx = G.context()
    rec, box, lig = _site(n_rec=3000, box_size=10.0, n_atoms=20, n_rot=4, seed=7)
    L = O.OracleLigand(lig)
    gs = ctx.build_grids(rec, [box], sorted(set(L.xs.tolist())))
    pl = ctx.ligand(lig)
    poses = S.random_poses(128, box, L.n_rot, seed=8)
    p = torch.tensor(poses, dtype=torch.float32, device="cuda")
    ge = torch.full((128,), 2.0, device="cuda")
    _, gx = ctx.score_backward(gs, pl, 0, p, ge, want_pose=False, want_xyz=True)
    gx = gx.cpu().numpy()
    og = O.OracleGrid(rec, box, L.xs, rec_types=O.xs_type_receptor(rec), threads=G.threads())
    for i, pp in enumerate(p.double().cpu().numpy()):
        x = L.fk(pp)
        if _near_face(x[None], box)[0]:
            continue
        _, dx = L.score_atoms(og, x)
        assert (np.abs(gx[i] - 2 * dx) <= G.GRAD_TOL * np.maximum(np.abs(2 * dx), 1.0)).all()


def test_rigid_and_edge_ligands():
    """Edge cases: a single atom, a rigid ligand (no torsions, no intra pairs), the atom and
    torsion maxima, and a ligand entirely outside its grid (penalty branch)."""
    torch = pytest.importorskip("torch")
    ctx = G.context()
    rec = G.receptor32(S.make_receptor(1500, 2, [(np.zeros(3), 5.0)]))
    box = G.box32(S.Box(np.zeros(3), np.array([8.0] * 3), 0.375))
    single = S.Ligand(np.zeros((1, 3)), np.array([0], np.uint8), np.zeros(1, np.uint8), np.zeros(1, np.uint8),
                      np.zeros((0, 2), np.int32), np.zeros(0, np.uint8))
    ligs = [single, S.ligand_centered(S.make_ligand(12, 0, 9)), S.ligand_centered(S.make_ligand(64, 26, 10))]
    gs = ctx.build_grids(rec, [box], list(range(11)))
    og = O.OracleGrid(rec, box, list(range(11)), rec_types=O.xs_type_receptor(rec), threads=G.threads())
    for lig in ligs:
        lig = G.ligand32(lig)
        L = O.OracleLigand(lig)
        pl = ctx.ligand(lig)
        poses = S.random_poses(40, box, L.n_rot, seed=11)
        poses[:10, 0] += 30.0                                 # far outside the grid
        p = torch.tensor(poses, dtype=torch.float32, device="cuda")
        e, g, _ = ctx.score(gs, pl, 0, p)
        ref = np.array([L.score(og, q)[0] for q in p.double().cpu().numpy()])
        assert G.close(e.cpu().numpy(), ref).all()
    # zero poses is a no-op; wrong ligand type set is rejected
    e, _, _ = ctx.score(gs, pl, 0, torch.zeros((0, 7 + L.n_rot), device="cuda"))
    assert e.shape == (0,)
    from paper_2506_20043_gb300.api import PVError
    gs_c = ctx.build_grids(rec, [box], [0])
    with pytest.raises(PVError):
        ctx.score(gs_c, pl, 0, p)
    with pytest.raises(PVError):
        ctx.score(gs, pl, 5, p)


def test_gather_microbenchmark_runs_and_rejects_bad_arguments():
    """The gather probe (the interpolation step alone) times real launches on a pocket's maps."""
    from paper_2506_20043_gb300.api import PVError
    ctx = G.context()
    rec, box, lig = _site(n_rec=2000, box_size=12.0, n_atoms=12, n_rot=2, seed=5)
    gs = ctx.build_grids(rec, [box], [0, 1, 2])
    ms, pts, gbs = ctx.measure_gather(gs, 0, n_points=1 << 20, reps=3)
    assert ms > 0 and pts > 1e8 and gbs == pytest.approx(32 * pts / 1e9)
    ms_all, _, _ = ctx.measure_gather(gs, -1, n_points=1 << 20, reps=3)   # every pocket of the set
    assert ms_all > 0
    for kw in (dict(pocket=1), dict(pocket=-2), dict(n_points=0), dict(reps=0)):
        with pytest.raises(PVError):
            ctx.measure_gather(gs, **{**dict(pocket=0, n_points=1024, reps=1), **kw})


def test_score_of_coordinates_matches_pose_score_and_oracle():
    """pv_score_xyz: the SF of posed atom coordinates equals pv_score of the pose they come from,
    and the oracle's SF and coordinate gradient at those coordinates (atoms within 2e-4 cells of
    a face excluded from the gradient check: the field's gradient jumps there)."""
    torch = pytest.importorskip("torch")
    ctx = G.context()
    rec, box, lig = _site(n_rec=3000, box_size=12.0, n_atoms=40, n_rot=7, seed=8)
    L = O.OracleLigand(lig)
    gs = ctx.build_grids(rec, [box], sorted(set(L.xs.tolist())))
    pl = ctx.ligand(lig)
    poses = torch.tensor(S.random_poses(400, box, L.n_rot, seed=9), dtype=torch.float32, device="cuda")
    xyz = ctx.pose_coords(pl, poses)
    e_pose, _, _ = ctx.score(gs, pl, 0, poses, grad=False)
    e, g = ctx.score_xyz(gs, pl, 0, xyz)
    assert G.close(e.cpu().numpy(), e_pose.cpu().numpy(), abs_tol=1e-5, rel_tol=1e-6).all()
    x64 = xyz.double().cpu().numpy()
    og = O.OracleGrid.lazy(rec, box, L.xs, O.xs_type_receptor(rec), x64.reshape(-1, 3), threads=G.threads())
    ref = [L.score_atoms(og, x) for x in x64]
    er = np.array([r[0] for r in ref])
    assert G.close(e.cpu().numpy(), er).all(), np.abs(e.cpu().numpy() - er).max()
    gr = np.stack([r[1] for r in ref])
    gg = g.cpu().numpy()
    far = ~_near_face(x64, box)
    d = np.abs(gg[far] - gr[far])
    assert (d <= G.GRAD_TOL * np.maximum(np.abs(gr[far]), 1.0)).all(), d.max()
    # the scaled form (a vector-Jacobian product) is the plain gradient times the scale
    w = torch.linspace(0.25, 2.0, 400, device="cuda")
    _, gw = ctx.score_xyz(gs, pl, 0, xyz, grad_energy=w)
    np.testing.assert_allclose(gw.cpu().numpy(), gg * w.cpu().numpy()[:, None, None], rtol=1e-6, atol=1e-6)


def test_autograd_over_coordinates_vs_fd():
    """PVScoreXYZ backward against FP64 central differences of the oracle over the coordinates."""
    torch = pytest.importorskip("torch")
    from paper_2506_20043_gb300.api import PVScoreXYZ
    ctx = G.context()
    rec, box, lig = _site(n_rec=3000, box_size=10.0, n_atoms=20, n_rot=4, seed=11)
    L = O.OracleLigand(lig)
    gs = ctx.build_grids(rec, [box], sorted(set(L.xs.tolist())))
    pl = ctx.ligand(lig)
    poses = torch.tensor(S.random_poses(32, box, L.n_rot, seed=12), dtype=torch.float32, device="cuda")
    x = ctx.pose_coords(pl, poses).clone().requires_grad_(True)
    e = PVScoreXYZ.apply(x, ctx, gs, pl, 0)
    w = torch.linspace(0.5, 1.5, 32, device="cuda")
    (e * w).sum().backward()
    got = x.grad.cpu().numpy() / w.cpu().numpy()[:, None, None]
    x64 = x.detach().double().cpu().numpy()
    og = O.OracleGrid(rec, box, L.xs, rec_types=O.xs_type_receptor(rec), threads=G.threads())
    checked = 0
    for i in range(32):
        if _near_face(x64[i][None], box, tol=1e-3)[0]:
            continue
        h = 1e-6
        fd = np.zeros_like(x64[i])
        for a in range(L.n):
            for k in range(3):
                p, m = x64[i].copy(), x64[i].copy()
                p[a, k] += h
                m[a, k] -= h
                fd[a, k] = (L.score_atoms(og, p)[0] - L.score_atoms(og, m)[0]) / (2 * h)
        assert (np.abs(got[i] - fd) <= G.GRAD_TOL * np.maximum(np.abs(fd), 1.0)).all(), (i, np.abs(got[i] - fd).max())
        checked += 1
    assert checked >= 16


@pytest.mark.parametrize("rings", ["single", "fused", "linked"])
def test_ring_ligands_score_and_gradient_match_oracle(rings):
    """Ligands with rigid six-membered rings (one, two fused, two linked by a rotatable bond): SF,
    parts and tangent gradient of 1,000 random poses against the oracle."""
    ctx = G.context()
    rec, box, _ = _site(n_rec=4000, box_size=12.0)
    lig = G.ligand32(S.ligand_centered(S.make_ring_ligand(28, 6, 7, rings)))
    poses = S.random_poses(1000, box, int(lig.rotatable.sum()), seed=2)
    e, g, parts, er, gr, pr, xyz, *_ = _run(ctx, rec, box, lig, poses, lazy=False)
    assert G.close(e, er).all(), np.abs(e - er).max()
    assert G.close(parts, pr).all()
    ok = np.abs(g - gr) <= G.GRAD_TOL * np.maximum(np.abs(gr), 1.0)
    bad = ~ok.all(axis=1) & ~_near_face(xyz, box)
    assert bad.sum() == 0, (np.argwhere(bad)[:5], np.abs(g - gr).max())
