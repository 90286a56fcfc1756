"""Pins of the oracle's first-order consistency check (Eq. 4-5) and the tangent-space difference it
uses; the check itself is a reading (the paper leaves the neighbourhood and the quantifiers open):
a candidate is worth a local search unless some stored neighbour shows no sign of a stationary
point between the two along any coordinate where they differ.

The difference is pinned as the inverse of the optimiser's retraction (b (+) s - b = s), by the
quaternion double cover and by torsion wrapping; the check by truth tables derived by hand from
Eq. 4 and Eq. 5 on one-coordinate cases; the chain with the check on by the switch's contract
(off = unchanged, on = fewer evaluations, valid results).
"""
import math

import numpy as np
import pytest

import oracle as O
import pvsynth as S


@pytest.fixture(scope="module")
def lig():
    return O.OracleLigand(S.ligand_centered(S.make_ligand(14, 3, 4)))


def _pot(lig, seed):
    return S.random_poses(1, S.Box(np.zeros(3), np.array([8.0] * 3)), lig.n_rot, seed)[0]


@pytest.mark.parametrize("seed", range(6))
def test_delta_inverts_the_retraction(lig, seed):
    rng = np.random.default_rng(seed)
    b = _pot(lig, seed)
    s = rng.normal(size=6 + lig.n_rot)
    s[3:6] *= 2.5 / max(np.linalg.norm(s[3:6]), 1.0)       # rotation angle below pi
    s[6:] = rng.uniform(-3.0, 3.0, lig.n_rot)               # torsion steps inside (-pi, pi)
    a = lig.retract(b, s)
    np.testing.assert_allclose(O.tangent_delta(lig.n_rot, a, b), s, atol=1e-12)
    np.testing.assert_allclose(O.tangent_delta(lig.n_rot, b, a)[:3], -s[:3], atol=1e-12)


def test_delta_double_cover_and_wrap(lig):
    a = _pot(lig, 11)
    b = a.copy()
    b[3:7] = -b[3:7]                                        # the same rotation
    assert np.abs(O.tangent_delta(lig.n_rot, a, b)[3:6]).max() < 1e-12
    b = a.copy()
    b[3:7] *= 3.0                                           # unnormalised: the same rotation
    assert np.abs(O.tangent_delta(lig.n_rot, a, b)[3:6]).max() < 1e-12
    a2, b2 = a.copy(), a.copy()
    a2[7], b2[7] = 3.0, -3.0
    assert O.tangent_delta(lig.n_rot, a2, b2)[6] == pytest.approx(6.0 - 2 * math.pi, abs=1e-12)
    a2[7], b2[7] = -3.0, 3.0
    assert O.tangent_delta(lig.n_rot, a2, b2)[6] == pytest.approx(2 * math.pi - 6.0, abs=1e-12)


def _one_coordinate(lig, dx, g_i, f_i, g_j, f_j, p=0):
    """Candidate and neighbour that differ by dx along tangent coordinate p only (a translation
    or a torsion); gradients g_i, g_j along p, zero elsewhere."""
    n_tan = 6 + lig.n_rot
    b = _pot(lig, 3)
    s = np.zeros(n_tan)
    s[p] = dx
    a = lig.retract(b, s)
    gi = np.zeros(n_tan); gi[p] = g_i
    gj = np.zeros(n_tan); gj[p] = g_j
    return a, f_i, gi, b[None], np.array([f_j]), gj[None]


@pytest.mark.parametrize("p", [0, 2, 6])
@pytest.mark.parametrize("g_i,f_i,g_j,want", [
    (+1.0, 1.0, +1.0, False),   # both slopes ascend towards the candidate, SF rises: no sign change
    (-1.0, 1.0, -1.0, True),    # Eq. 5: secant rises, derivative at the candidate falls
    (-1.0, 1.0, +1.0, True),    # Eq. 4: the derivative changes sign
    (+1.0, -1.0, +1.0, True),   # Eq. 5: secant falls, derivative rises
    (-1.0, -1.0, -1.0, False),  # both descend along +p and the SF falls: no sign change
    (0.0, 1.0, +1.0, True),     # sign 0: Eq. 4 holds (product 0)
])
def test_check_truth_table_one_coordinate(lig, p, g_i, f_i, g_j, want):
    a, fi, gi, nb, fj, gj = _one_coordinate(lig, 0.5, g_i, f_i, g_j, 0.0, p)
    assert O.focc_pass(lig, a, fi, gi, nb, fj, gj) is want


def test_check_needs_evidence_against_every_neighbour(lig):
    a, fi, gi, nb1, f1, g1 = _one_coordinate(lig, 0.5, -1.0, 1.0, +1.0, 0.0)   # evidence (Eq. 4)
    _, _, _, nb2, f2, g2 = _one_coordinate(lig, 0.5, -1.0, 1.0, -1.0, 0.0)     # evidence (Eq. 5)
    assert O.focc_pass(lig, a, fi, gi, np.concatenate([nb1, nb2]), np.concatenate([f1, f2]),
                       np.concatenate([g1, g2]))
    gi2 = gi.copy(); gi2[0] = +1.0
    _, _, _, nb3, f3, g3 = _one_coordinate(lig, 0.5, +1.0, 1.0, +1.0, 0.0)     # no evidence
    assert not O.focc_pass(lig, a, fi, gi2, np.concatenate([nb1, nb3]), np.concatenate([f1, f3]),
                           np.concatenate([g1, g3]))
    assert O.focc_pass(lig, a, fi, gi, np.zeros((0, lig.n_pot)), np.zeros(0), np.zeros((0, 6 + lig.n_rot)))


def test_identical_conformation_has_no_evidence(lig):
    b = _pot(lig, 5)
    g = np.ones(6 + lig.n_rot)
    assert not O.focc_pass(lig, b, 1.0, -g, b[None], np.array([0.0]), g[None])   # no coordinate differs
    # a difference below the threshold carries no sign either
    a = lig.retract(b, np.r_[5e-5, np.zeros(5 + lig.n_rot)])
    assert not O.focc_pass(lig, a, 1.0, -g, b[None], np.array([0.0]), g[None], 1e-4)
    assert O.focc_pass(lig, a, 1.0, -g, b[None], np.array([0.0]), g[None], 1e-5)


def test_chain_with_the_check_off_is_unchanged_and_on_saves_evaluations():
    w = S.tiny()
    lig = O.OracleLigand(w.ligands[0])
    rec, box = w.receptors[0], w.boxes[0][0]
    og = O.OracleGrid(rec, box, lig.xs, rec_types=O.xs_type_receptor(rec))
    base = O.SearchParams(seed=2, steps=40)
    p0, e0, ev0 = O.mc_chains(lig, og, box, base, unit=0, n_chains=8)
    p1, e1, ev1 = O.mc_chains(lig, og, box, O.SearchParams(seed=2, steps=40, focc=0), unit=0, n_chains=8)
    np.testing.assert_array_equal(e0, e1)
    np.testing.assert_array_equal(ev0, ev1)
    p4, e4, ev4 = O.mc_chains(lig, og, box, O.SearchParams(seed=2, steps=40, focc=4), unit=0, n_chains=8)
    assert ev4.sum() < ev0.sum()
    for pot, e in zip(p4, e4):            # every chain best is a scored pose
        assert lig.score(og, pot, False)[0] == pytest.approx(e, abs=1e-9)
