"""Pins of the oracle's RILC-BFGS (Eq. 6-12), random start / mutation (Eq. 2), MC chain
(Algorithm 2, Eq. 13) and top-k selection.

BFGS: known minimisers of convex quadratics and Rosenbrock; a 1-D case whose line-search trace
follows from Eq. 7-8 by hand; both stopping rules. MC: one-entity mutation with bounded
amplitude, uniform quaternions, counter-based independence of chains, the best score of a
chain never rises with more steps, and a brute-force rigid search on a tiny box that the MC
search must match. Top-k: hand-built candidates with known RMSD relations.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import pvsynth as S

P = O.SearchParams


def _euclid(x, s):
    return x + s


@pytest.mark.parametrize("n", [6, 13, 21])
def test_bfgs_convex_quadratic(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n))
    H = A @ A.T + n * np.eye(n)
    H /= np.linalg.eigvalsh(H).max()          # largest curvature 1: unit step is admissible
    xs = rng.normal(size=n)
    f = lambda x: (0.5 * (x - xs) @ H @ (x - xs), H @ (x - xs))
    x, fv, g, ev = O.bfgs_generic(f, _euclid, np.zeros(n), n, P(max_iter=500, eps=1e-9))
    np.testing.assert_allclose(x, xs, atol=1e-6)
    assert np.linalg.norm(g) <= 1e-9 or fv < 1e-14


def test_bfgs_rosenbrock():
    def f(x):
        a, b = x[0], x[1]
        return (1 - a) ** 2 + 100 * (b - a * a) ** 2, np.array(
            [-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])
    x, fv, g, ev = O.bfgs_generic(f, _euclid, np.array([-1.2, 1.0]), 2,
                                  P(max_iter=2000, eps=1e-8, max_trials=40))
    np.testing.assert_allclose(x, [1.0, 1.0], atol=1e-4)


def test_line_search_trace_by_hand():
    # f = (x - 10)^2 from x = 0: d = -g = 20. lambda = 1 -> x = 20, f = 100 > 100 - 1e-4*400:
    # Armijo fails (Eq. 7 holds), upper bound 1; lambda = 0.5 -> x = 10, f = 0, g = 0:
    # g_new.d = 0 >= 0.1 * (-400): accepted. Then ||g|| = 0 <= eps stops (Eq. 12).
    f = lambda x: ((x[0] - 10) ** 2, np.array([2 * (x[0] - 10)]))
    x, fv, g, ev = O.bfgs_generic(f, _euclid, np.array([0.0]), 1, P(max_iter=10))
    assert x[0] == 10.0 and fv == 0.0 and ev == 3


def test_line_search_expands_on_wolfe_failure():
    # f = 1e-3 x^2 from x = -100: d = 0.2; lambda = 1 -> x = -99.8: Armijo holds, slope still
    # steep (Eq. 8 holds) -> lower bound 1, lambda doubles: 2, 4, ... until Wolfe is satisfied.
    f = lambda x: (1e-3 * x[0] ** 2, np.array([2e-3 * x[0]]))
    x, fv, g, ev = O.bfgs_generic(f, _euclid, np.array([-100.0]), 1, P(max_iter=1))
    # accepted lambda is the first power of two with x_new = -100 + 0.2 lam, g_new*0.2 >= 0.1*g*0.2
    # i.e. 2e-3 * x_new >= 0.1 * (-0.2) -> x_new >= -10 -> lam >= 450 -> the bracket stays
    # open for 9 doublings (lam = 512 after 10 trials: x = 2.4, Armijo holds, Wolfe holds)
    assert x[0] == pytest.approx(-100.0 + 0.2 * 512)
    assert ev == 1 + 10


def test_bfgs_stops_on_non_descent_and_keeps_state():
    f = lambda x: (0.0, np.zeros(3))
    x0 = np.array([1.0, 2.0, 3.0])
    x, fv, g, ev = O.bfgs_generic(f, _euclid, x0, 3, P(max_iter=10))
    np.testing.assert_array_equal(x, x0)
    assert ev == 1


# ------------------------------------------------------------------------------- MC parts --

def _site():
    rec = S.make_receptor(700, 1, [(np.zeros(3), 5.0)])
    box = S.Box(np.zeros(3), np.array([9.0, 9.0, 9.0]), 0.375)
    return rec, box


def test_random_conformation_distribution():
    lig = S.ligand_centered(S.make_ligand(15, 3, 2))
    L = O.OracleLigand(lig)
    box = S.Box(np.array([1.0, 2.0, 3.0]), np.array([6.0, 8.0, 10.0]))
    pots = np.array([O.random_conformation(L, box, 5, 1, c) for c in range(4000)])
    assert ((np.abs(pots[:, :3] - box.center) <= box.size / 2).all())
    np.testing.assert_allclose(np.linalg.norm(pots[:, 3:7], axis=1), 1.0, atol=1e-12)
    assert (np.abs(pots[:, 7:]) <= math.pi).all()
    # uniform rotations: E[q q^T] = I / 4
    np.testing.assert_allclose(pots[:, 3:7].T @ pots[:, 3:7] / len(pots), np.eye(4) / 4, atol=0.02)
    # distinct chains / units / seeds give distinct starts
    assert not np.allclose(O.random_conformation(L, box, 5, 1, 0), O.random_conformation(L, box, 5, 2, 0))
    assert not np.allclose(O.random_conformation(L, box, 5, 1, 0), O.random_conformation(L, box, 6, 1, 0))


def test_mutation_changes_one_entity_within_amplitude():
    lig = S.ligand_centered(S.make_ligand(22, 4, 5))
    L = O.OracleLigand(lig)
    box = S.Box(np.zeros(3), np.array([10.0] * 3))
    base = O.random_conformation(L, box, 0, 0, 0)
    counts = np.zeros(2 + L.n_rot)
    for step in range(3000):
        m = O.mutate(L, base, 2.0, 0, 0, 0, step)
        dt = np.linalg.norm(m[:3] - base[:3])
        dq = abs(np.dot(m[3:7], base[3:7]))
        dpsi = np.nonzero(np.abs(m[7:] - base[7:]) > 0)[0]
        changed = [dt > 0, dq < 1 - 1e-15] + [k in dpsi for k in range(L.n_rot)]
        assert sum(changed) == 1
        ent = int(np.argmax(changed))
        counts[ent] += 1
        if ent == 0:
            assert dt <= 2.0 + 1e-12
        elif ent == 1:
            ang = 2 * math.acos(min(1.0, dq))
            assert ang <= 2.0 / L.rgyr + 1e-9
            np.testing.assert_allclose(m[:3], base[:3])
        else:
            assert -math.pi <= m[7 + ent - 2] < math.pi
    # entity choice uniform over 2 + N_rot (5-sigma)
    p = 1.0 / len(counts)
    assert (np.abs(counts / 3000 - p) < 5 * math.sqrt(p * (1 - p) / 3000)).all()


def test_chains_are_independent_and_prefix_monotone():
    rec, box = _site()
    lig = S.ligand_centered(S.make_ligand(14, 3, 7))
    L = O.OracleLigand(lig)
    G = O.OracleGrid(rec, box, L.xs, rec_types=O.xs_type_receptor(rec))
    p = P(steps=40, seed=3)
    pots, es, ev = O.mc_chains(L, G, box, p, unit=2, n_chains=4)
    pots1, es1, _ = O.mc_chains(L, G, box, p, unit=2, n_chains=1, chain0=2)
    np.testing.assert_array_equal(pots1[0], pots[2])
    assert es1[0] == es[2]
    # a longer run replays the same prefix, so its best can only be lower or equal
    _, es_long, _ = O.mc_chains(L, G, box, P(steps=80, seed=3), unit=2, n_chains=4)
    assert (es_long <= es).all()
    # each chain's reported best is its pose's score
    for c in range(4):
        assert L.score(G, pots[c], want_grad=False)[0] == pytest.approx(es[c], rel=1e-12)


def test_mc_matches_brute_force_rigid_search():
    # rigid 6-atom ligand in a 6 A box; exhaustive start set: translations on a 1 A lattice
    # (216) x 48 random rotations, each locally minimised by the same BFGS. The MC best must
    # reach the best of that exhaustive search within 0.2 kcal/mol.
    rec = S.make_receptor(500, 4, [(np.zeros(3), 4.5)])
    box = S.Box(np.zeros(3), np.array([6.0, 6.0, 6.0]), 0.375)
    lig = S.ligand_centered(S.make_ligand(6, 0, 8))
    L = O.OracleLigand(lig)
    G = O.OracleGrid(rec, box, L.xs, rec_types=O.xs_type_receptor(rec))
    rng = np.random.default_rng(0)
    qs = rng.normal(size=(48, 4))
    qs /= np.linalg.norm(qs, axis=1, keepdims=True)
    best_brute = np.inf
    pp = P(max_iter=30)
    for t in itertools.product(np.arange(-2.5, 2.51, 1.0), repeat=3):
        for q in qs:
            pot = np.concatenate([t, q])
            _, f, _, _ = O.bfgs_pose(L, G, pot, pp)
            best_brute = min(best_brute, f)
    _, es, _ = O.mc_chains(L, G, box, P(steps=150, seed=1), unit=0, n_chains=16)
    assert es.min() <= best_brute + 0.2


# ------------------------------------------------------------------------------------ top-k --

def test_topk_sort_filter_and_ties():
    base = np.zeros((3, 3))
    xyz = np.stack([base, base + 0.5, base + 3.0, base + 0.2, base + 6.0, base + 3.1])
    scores = np.array([-5.0, -6.0, -4.0, -6.0, -1.0, -4.5])
    # order by score (ties by index): 1 (-6), 3 (-6), 0 (-5), 5 (-4.5), 2 (-4), 4 (-1)
    # RMSD of rigid shifts = |shift| * sqrt(3); 1 vs 3: 0.3*sqrt3 = 0.52 < 1 -> drop 3;
    # 0 vs 1: 0.87 < 1 -> drop 0; 5 kept; 2 vs 5: 0.17 -> drop; 4 kept
    kept = O.topk(scores, xyz, k=9, rmsd_min=1.0)
    assert list(kept) == [1, 5, 4]
    assert list(O.topk(scores, xyz, k=2, rmsd_min=1.0)) == [1, 5]
    assert list(O.topk(scores, xyz, k=9, rmsd_min=0.0)) == [1, 3, 0, 5, 2, 4]


def test_merge_orders_by_score_then_pocket_then_chain():
    r0 = O.PairResult(0, 0, None, None, 0, np.array([4, 1]), np.array([-7.0, -5.0]), None, None, None)
    r1 = O.PairResult(0, 1, None, None, 0, np.array([0, 2]), np.array([-7.0, -8.0]), None, None, None)
    assert O.merge_pockets([r1, r0]) == [(-8.0, 1, 2), (-7.0, 0, 4), (-7.0, 1, 0), (-5.0, 0, 1)]


def test_perturbed_chain_replay_reproduces_the_oracle_without_noise():
    """The GPU tests' perturbed replay of the oracle's chains (tests/_gpu.py) follows mc_chains step
    for step: with no noise it gives the same best SF on every chain (an empty box: zero maps)."""
    from tests import _gpu as G
    lig = S.ligand_centered(S.make_ligand(14, 3, 5))
    L = O.OracleLigand(lig)
    box = S.Box(np.array([100.0, 0.0, 0.0]), np.array([16.0, 16.0, 16.0]), 0.375)
    types = sorted(set(L.xs.tolist()))
    og = O.OracleGrid(None, box, types, maps=np.zeros((len(types), int(np.prod(O.grid_geometry(box)[1])))))
    p = O.SearchParams(seed=4, steps=3, max_iter=6)
    _, ref, ref_ev = O.mc_chains(L, og, box, p, unit=2, n_chains=12)
    got, ev = G.oracle_chains_perturbed(L, og, box, p, 2, 12, 0.0, 1)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(ev, ref_ev)
