"""Shared setup of the GPU parity tests: a library context, synthetic sites and oracle twins."""
import functools
import os

import numpy as np
import pytest

import oracle as O
import pvsynth as S

# Parity tolerance for grid values and per-pose SF (FP32 kernel vs FP64 oracle):
# |gpu - oracle| <= 1e-3 kcal/mol or <= 1e-4 relative.
ABS_TOL, REL_TOL = 1e-3, 1e-4
# Gradient tolerance: |gpu - oracle| <= 1e-3 * max(|oracle|, 1).
GRAD_TOL = 1e-3
# Pose -> atom coordinates (Eq. 1) in FP32 vs FP64, in Angstrom.
COORD_TOL = 2e-4
# The pair terms stop at 8 A without smoothing, so the SF jumps there by one pair's term (about
# 3e-3 kcal/mol for two heavy atoms). Two places meet that edge in FP32 vs FP64:
#  - intra pairs: local optimisation seeks the edge (the step that brings a pair inside the cutoff
#    lowers the SF), and the same pose posed by two FP32 kernels can put the pair a few ulps to
#    either side;
#  - grid nodes: a receptor atom at 8 A from a node, to within rounding, counts on one side only
#    (about 1e-4 of the nodes of a pocket), and an atom interpolating there inherits its jump times
#    the corner's weight.
# A pair or a (node, receptor atom) within CUTOFF_EDGE of 8 A adds its jump to the tolerance.
CUTOFF, CUTOFF_EDGE = 8.0, 1e-4


def close(gpu, ref, abs_tol=ABS_TOL, rel_tol=REL_TOL):
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    return (np.abs(gpu - ref) <= abs_tol) | (np.abs(gpu - ref) <= rel_tol * np.abs(ref))


def threads():
    return len(os.sched_getaffinity(0))


@functools.lru_cache(maxsize=None)
def context():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_20043_gb300 as pv
    pv.build()
    from paper_2506_20043_gb300 import api
    return api.Context(0)


def box32(box):
    """The box as the float32 values the library receives (so both sides use the same grid)."""
    return S.Box(np.asarray(box.center, np.float32).astype(np.float64),
                 np.asarray(box.size, np.float32).astype(np.float64), float(np.float32(box.spacing)))


def receptor32(rec):
    return S.Receptor(np.asarray(rec.xyz, np.float32).astype(np.float64), rec.element, rec.donor, rec.acceptor)


def ligand32(lig):
    import dataclasses
    return dataclasses.replace(lig, xyz=np.asarray(lig.xyz, np.float32).astype(np.float64))


def pose_coords(ctx, pl, pots):
    """The GPU's FP32 atom coordinates [n, atoms, 3] of POTs [n, 7 + n_rot] (input atom order)."""
    import torch
    p = torch.tensor(np.ascontiguousarray(pots, np.float32), device="cuda")
    return ctx.pose_coords(pl, p).cpu().numpy().astype(np.float64)


def check_pose_scores(L, og, pots, es, xyz_gpu, site=None):
    """Scores reported for poses, checked in two steps. (1) The GPU's atom coordinates equal the
    oracle's kinematics of the same POT within COORD_TOL. (2) The reported SF equals the oracle's SF
    at the GPU's own coordinates within ABS_TOL / REL_TOL. Scoring the oracle's coordinates instead
    would add |force| x the FP32 coordinate rounding to the comparison: at a clash, forces of
    hundreds of kcal/mol/A times 1e-5 A of rounding move the SF by a few 1e-3 kcal/mol."""
    pots = np.asarray(pots, np.float64)
    ref_xyz = np.stack([L.fk(p) for p in pots])
    dx = np.abs(xyz_gpu - ref_xyz).max()
    assert dx <= COORD_TOL, dx
    ref = np.array([L.score_atoms(og, x)[0] for x in xyz_gpu])
    diff = np.abs(np.asarray(es, np.float64) - ref)
    ok = close(es, ref)
    for k in np.nonzero(~ok)[0]:        # the cutoff edges, only where the strict test fails
        slack = cutoff_slack(L, xyz_gpu[k]) + (node_cutoff_slack(L, xyz_gpu[k], *site) if site else 0.0)
        ok[k] = diff[k] <= slack + ABS_TOL
    assert ok.all(), (np.nonzero(~ok)[0], diff.max())
    return ref_xyz


def cutoff_slack(L, xyz):
    """Sum of the cutoff jumps of the intra pairs within CUTOFF_EDGE of the cutoff at xyz."""
    if L.n_pairs == 0:
        return 0.0
    i, j = L.pairs[:, 0], L.pairs[:, 1]
    r = np.linalg.norm(xyz[i] - xyz[j], axis=1)
    near = np.nonzero(np.abs(r - CUTOFF) < CUTOFF_EDGE)[0]
    return float(sum(abs(O.pair_energy(int(L.xs[i[k]]), int(L.xs[j[k]]), CUTOFF - 1e-9)[0]) for k in near))


def node_cutoff_slack(L, xyz, rec, rec_types, box):
    """Sum over the ligand atoms' interpolation corners of weight x the cutoff jumps of the receptor
    atoms within CUTOFF_EDGE of 8 A from that node (the grid's cutoff edge)."""
    origin, dims = O.grid_geometry(box)
    sp = float(box.spacing)
    rxyz = np.asarray(rec.xyz, np.float64)
    total = 0.0
    for a in range(L.n):
        g = np.clip((xyz[a] - origin) / sp, 0, dims - 1)
        i = np.minimum(np.floor(g).astype(int), dims - 2)
        f = g - i
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                    node = origin + sp * (i + np.array([dx, dy, dz]))
                    r = np.linalg.norm(rxyz - node, axis=1)
                    for j in np.nonzero(np.abs(r - CUTOFF) < CUTOFF_EDGE)[0]:
                        total += w * abs(O.pair_energy(int(L.xs[a]), int(rec_types[j]), CUTOFF - 1e-9)[0])
    return total


def direct_cutoff_slack(L, xyz, rec, rec_types):
    """Cutoff jumps of the (ligand atom, receptor atom) pairs within CUTOFF_EDGE of 8 A, for
    directly summed e_inter."""
    rxyz = np.asarray(rec.xyz, np.float64)
    total = 0.0
    for a in range(L.n):
        r = np.linalg.norm(rxyz - xyz[a], axis=1)
        for j in np.nonzero(np.abs(r - CUTOFF) < CUTOFF_EDGE)[0]:
            total += abs(O.pair_energy(int(L.xs[a]), int(rec_types[j]), CUTOFF - 1e-9)[0])
    return total


def check_rescored(r, q, L, rec, rec_types, base=None):
    """Pair q of a result docked with rescore: e_inter equals the oracle's direct sum at the
    reported coordinates, score = e_inter + e_intra, affinity from it, poses sorted by score; the
    grid values equal those of the same dock without rescoring (base), chain by chain."""
    n = int(r.n_kept[q])
    poses = r.poses[q]
    for slot in range(n):
        p = poses[slot]
        xyz = r.xyz[q, slot, :L.n].astype(np.float64)
        ref = L.direct_inter(rec, rec_types, xyz)
        d = abs(float(p["e_inter"]) - ref)
        assert close(p["e_inter"], ref) or d <= direct_cutoff_slack(L, xyz, rec, rec_types) + ABS_TOL, (q, slot, d)
        assert float(p["score"]) == pytest.approx(float(p["e_inter"]) + float(p["e_intra"]), abs=2e-6)
        assert close(p["affinity"], O.affinity(ref, L.n_rot))
    sc = poses["score"][:n]
    assert (np.diff(sc) >= 0).all()
    if base is not None:
        assert int(base.n_kept[q]) == n
        by_chain = {int(b["chain"]): b for b in base.poses[q][:n]}
        assert set(by_chain) == {int(c) for c in poses["chain"][:n]}
        for p in poses[:n]:
            b = by_chain[int(p["chain"])]
            assert p["score_grid"] == b["score"] and p["e_inter_grid"] == b["e_inter"]


def oracle_chains_perturbed(L, grid, box, params, unit, n_chains, noise, seed):
    """The oracle's Monte-Carlo chains (its random start, mutation, RILC-BFGS, Metropolis test and
    refinement, step for step as oracle.mc_chains runs them) with every score evaluation's energy
    and gradient multiplied by (1 + noise * N(0, 1)) draws: how far FP64 runs part ways with the
    oracle under perturbations of the size of FP32 rounding. With noise = 0 it reproduces
    mc_chains exactly. Returns the chains' best SF and their score evaluation counts."""
    rng = np.random.default_rng(seed)

    def fg(x):
        e, g, _ = L.score(grid, x, True)
        return e * (1 + noise * rng.standard_normal()), g * (1 + noise * rng.standard_normal(g.shape))

    def bfgs(x):
        xo, f, _, ev = O.bfgs_generic(fg, L.retract, x, 6 + L.n_rot, params)
        return xo, f, ev

    out = np.zeros(n_chains)
    evals = np.zeros(n_chains, np.int64)
    for c in range(n_chains):
        cur = O.random_conformation(L, box, params.seed, unit, c)
        e_cur = fg(cur)[0]
        e_best = e_cur
        n_ev = 1
        for st in range(params.steps):
            cand, e_new, k = bfgs(O.mutate(L, cur, params.amplitude, params.seed, unit, c, st))
            n_ev += k
            u = O.metropolis_uniform(params.seed, unit, c, st)
            if O.metropolis_accept(e_cur, e_new, params.temperature, u):
                cur, e_cur = cand, e_new
                if e_cur < e_best:
                    cur, e_cur, k = bfgs(cur)
                    n_ev += k
                    e_best = e_cur
        out[c] = e_best
        evals[c] = n_ev
    return out, evals
