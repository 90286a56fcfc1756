"""Pins of the oracle's random numbers, Vina terms, pair energies and XS typing.

Philox4x32-10 against the published known-answer vectors; every term against its closed form
at points where the definition gives an exact value; typing against the XS rules.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _weights():
    w = {}
    for line in open(os.path.join(GOLD, "vina_weights.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        w[parts[0]] = float(parts[1])
    return w


W = _weights()
C_H, C_P, N_P, N_D, N_A, N_DA, O_P, O_D, O_A, O_DA, S_P = range(11)


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_u01_is_exact_24bit():
    assert O.u01(0) == 0.0
    assert O.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert O.u01(0x100) == 2.0 ** -24
    assert O.u01(0xFF) == 0.0


def test_uniform_stream_is_uniform():
    # 40,000 Metropolis draws, chi-square over 20 bins (99.9 % critical value 43.8 for 19 dof)
    u = np.array([O.metropolis_uniform(7, 3, c, s) for c in range(200) for s in range(200)])
    hist = np.histogram(u, bins=20, range=(0, 1))[0]
    exp = len(u) / 20
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 43.8
    assert 0.0 <= u.min() and u.max() < 1.0


@pytest.mark.parametrize("d,expect", [
    (0.0, [1.0, math.exp(-2.25), 0.0, 1.0, 0.0]),
    (0.5, [math.exp(-1.0), math.exp(-6.25 / 4.0), 0.0, 1.0, 0.0]),
    (-1.0, [math.exp(-4.0), math.exp(-4.0), 1.0, 1.0, 1.0]),
    (1.0, [math.exp(-4.0), math.exp(-1.0), 0.0, 0.5, 0.0]),
    (3.0, [math.exp(-36.0), 1.0, 0.0, 0.0, 0.0]),
    (5.0, [math.exp(-100.0), math.exp(-1.0), 0.0, 0.0, 0.0]),
    (-0.35, [math.exp(-0.49), math.exp(-(3.35 / 2) ** 2), 0.1225, 1.0, 0.5]),
    (1.6, [math.exp(-10.24), math.exp(-0.49), 0.0, 0.0, 0.0]),
    (-2.0, [math.exp(-16.0), math.exp(-6.25), 4.0, 1.0, 1.0]),
])
def test_terms_closed_forms(d, expect):
    np.testing.assert_allclose(O.terms(d), expect, rtol=1e-14, atol=1e-300)


def _radius(t):
    return {0: 1.9, 1: 1.9}.get(t, 1.8 if t <= 5 else (1.7 if t <= 9 else 2.0))


def test_pair_energy_at_contact():
    # d = 0: gauss1 = 1, gauss2 = e^-2.25, hydrophobic = 1 (both C_H), hbond = 0, repulsion = 0
    e, _ = O.pair_energy(C_H, C_H, 3.8)
    assert e == pytest.approx(W["gauss1"] + W["gauss2"] * math.exp(-2.25) + W["hydrophobic"], abs=1e-14)
    # C_P is not hydrophobic
    e, _ = O.pair_energy(C_H, C_P, 3.8)
    assert e == pytest.approx(W["gauss1"] + W["gauss2"] * math.exp(-2.25), abs=1e-14)
    # donor N (1.8) with acceptor O (1.7) at d = -1: repulsion 1, hbond 1
    e, _ = O.pair_energy(N_D, O_A, 2.5)
    assert e == pytest.approx(W["gauss1"] * math.exp(-4) + W["gauss2"] * math.exp(-4) + W["repulsion"]
                              + W["hbond"], abs=1e-14)
    # donor with donor: no hbond
    e2, _ = O.pair_energy(N_D, O_D, 2.5)
    assert e2 == pytest.approx(e - W["hbond"], abs=1e-14)
    # acceptor-donor order does not matter, N_DA pairs with either
    assert O.pair_energy(O_A, N_D, 2.5)[0] == pytest.approx(e, abs=1e-15)
    assert O.pair_energy(N_DA, O_DA, 2.5)[0] == pytest.approx(e, abs=1e-15)
    # S radius 2.0: S-S at r = 4 is d = 0, no hydrophobic, no hbond
    e, _ = O.pair_energy(S_P, S_P, 4.0)
    assert e == pytest.approx(W["gauss1"] + W["gauss2"] * math.exp(-2.25), abs=1e-14)


def test_pair_energy_cutoff_and_symmetry():
    assert O.pair_energy(C_H, C_H, 8.0)[0] == 0.0
    assert O.pair_energy(C_H, C_H, 7.999)[0] != 0.0
    rng = np.random.default_rng(0)
    for _ in range(200):
        ti, tj = rng.integers(0, 11, size=2)
        r = rng.uniform(0.5, 8.5)
        assert O.pair_energy(ti, tj, r)[0] == pytest.approx(O.pair_energy(tj, ti, r)[0], rel=1e-13, abs=1e-15)


def test_pair_energy_derivative_matches_fd():
    rng = np.random.default_rng(1)
    kinks = np.array([0.5, 1.5, -0.7, 0.0])
    n = 0
    while n < 300:
        ti, tj = (int(x) for x in rng.integers(0, 11, size=2))
        r = rng.uniform(1.0, 7.9)
        d = r - _radius(ti) - _radius(tj)
        if np.abs(d - kinks).min() < 1e-3:
            continue
        h = 1e-6
        fd = (O.pair_energy(ti, tj, r + h)[0] - O.pair_energy(ti, tj, r - h)[0]) / (2 * h)
        assert O.pair_energy(ti, tj, r)[1] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        n += 1


def test_xs_typing_ligand():
    class L:  # C0-C1-N2, C1-O3, C4 bonded to C0 only, S5 bonded to C4
        n = 6
        element = np.array([0, 0, 1, 2, 0, 3], np.uint8)
        donor = np.array([0, 0, 1, 0, 0, 0], np.uint8)
        acceptor = np.array([0, 0, 1, 1, 0, 0], np.uint8)
        bonds = np.array([[0, 1], [1, 2], [1, 3], [0, 4], [4, 5]], np.int32)
    t = O.xs_type_ligand(L)
    assert list(t) == [C_H, C_P, N_DA, O_A, C_H, S_P]


def test_xs_typing_receptor():
    class R:
        n = 5
        xyz = np.array([[0, 0, 0], [1.7, 0, 0], [10, 0, 0], [11.8, 0, 0], [20, 0, 0]], float)
        element = np.array([0, 2, 0, 1, 1], np.uint8)
        donor = np.array([0, 1, 0, 0, 0], np.uint8)
        acceptor = np.array([0, 0, 0, 0, 1], np.uint8)
    t = O.xs_type_receptor(R)
    # C within 1.75 A of O is polar; C 1.8 A from N is not; N with no flags is N_P
    assert list(t) == [C_P, O_D, C_H, N_P, N_A]


def test_metropolis_rule():
    T = 1.2
    assert O.metropolis_accept(0.0, -1.0, T, 0.999999)       # improvement: always
    assert O.metropolis_accept(0.0, 0.0, T, 0.999999)        # equal: exp(0) = 1 > u
    # acceptance frequency of a worse candidate equals exp(-dE/T) (binomial 5-sigma)
    rng = np.random.default_rng(3)
    for de in (0.3, 1.0, 2.5):
        u = rng.random(20000)
        acc = np.mean([O.metropolis_accept(0.0, de, T, x) for x in u])
        p = math.exp(-de / T)
        assert abs(acc - p) < 5 * math.sqrt(p * (1 - p) / len(u))


def test_affinity_normalisation():
    assert O.affinity(-10.0, 0) == -10.0
    assert O.affinity(-10.0, 4) == pytest.approx(-10.0 / (1 + 4 * W["nrot"]), rel=1e-15)
