"""The intra-pair schedules of the library's ligand records (host code, no GPU): built by the
library's own ligand builder, decoded, and checked against the oracle's pair list (C-intra: pairs
in different rigid fragments more than three bonds apart).

Each schedule (the warp's 32 lanes, and the half warp's 16 lanes for ligands that fit one) must
hold every oracle pair exactly once, carry the pair's hydrophobic / H-bond flags, have every pair
received by its target atom's lane from its sending lane, let a lane send and receive at most one
pair per round, and use no more rounds than the largest sending or receiving load of a lane (a
proper edge colouring of a bipartite multigraph, Koenig's theorem)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle as O
import pvsynth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_20043_gb300", "csrc")
XS = ["C_H", "C_P", "N_P", "N_D", "N_A", "N_DA", "O_P", "O_D", "O_A", "O_DA", "S_P"]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("sched") / "libsched.so")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-I", cuda_inc,
                           os.path.join(ROOT, "tests", "csrc", "ligand_schedule.cpp"),
                           os.path.join(CSRC, "pv_ligand.cpp"), "-o", out])
    L = C.CDLL(out)
    L.lig_schedule.restype = C.c_int
    return L


def _raw(lib, lig, lanes):
    """The schedule's meta words (rounds x lanes), the device-to-input atom map, the header."""
    xyz = np.ascontiguousarray(lig.xyz, np.float32)
    el, don, acc = (np.ascontiguousarray(a, np.uint8) for a in (lig.element, lig.donor, lig.acceptor))
    bonds = np.ascontiguousarray(lig.bonds, np.int32).reshape(-1, 2)
    rot = np.ascontiguousarray(lig.rotatable, np.uint8)
    words = np.zeros(8192, np.uint32)
    src = np.zeros(64, np.int32)
    info = np.zeros(5, np.int32)
    p = lambda a, t: a.ctypes.data_as(C.POINTER(t))   # noqa: E731
    nr = lib.lig_schedule(len(xyz), p(xyz, C.c_float), p(el, C.c_uint8), p(don, C.c_uint8), p(acc, C.c_uint8),
                          len(bonds), p(bonds, C.c_int32), p(rot, C.c_uint8), lanes, p(words, C.c_uint32),
                          len(words), p(src, C.c_int32), p(info, C.c_int32))
    assert nr >= 0, nr
    return words[:nr * lanes].reshape(nr, lanes), src, info


def _decode(lib, lig, lanes):
    """Rows (round, lane, source input atom, target input atom, hyd, hb) of the pairs sent, rows
    (round, lane, sending lane, receiving input atom) of the pairs received, the header and the
    round count."""
    words, src, info = _raw(lib, lig, lanes)
    words = words.reshape(-1)
    nr = len(words) // lanes
    n = int(info[4])
    sent, recv = [], []
    for r in range(nr):
        for l in range(lanes):
            w = int(words[r * lanes + l])
            if w >> 31:
                s_dev, t_dev = l + lanes * ((w >> 7) & 1), w & 127
                assert s_dev < n and t_dev < n
                sent.append((r, l, int(src[s_dev]), int(src[t_dev]), (w >> 16) & 1, (w >> 17) & 1))
            if (w >> 13) & 1:
                a_dev = l + lanes * ((w >> 14) & 1)
                assert a_dev < n
                recv.append((r, l, (w >> 8) & 31, int(src[a_dev])))
    return np.array(sent, dtype=np.int64).reshape(-1, 6), np.array(recv, dtype=np.int64).reshape(-1, 4), info, nr


CASES = [(n, r, s) for s, (n, r) in enumerate([(5, 0), (8, 2), (12, 3), (16, 4), (20, 4), (24, 6), (30, 6), (32, 8),
                                               (32, 10), (31, 9), (40, 8), (48, 12), (60, 15), (64, 20)])]


@pytest.mark.parametrize("n_atoms,n_rot,seed", CASES + [(int(n), int(r), 100 + i) for i, (n, r) in enumerate(
    zip(np.random.default_rng(4).integers(6, 33, 24), np.random.default_rng(5).integers(0, 11, 24)))])
def test_schedules_hold_every_oracle_pair_once(lib, n_atoms, n_rot, seed):
    _check_schedules(lib, S.ligand_centered(S.make_ligand(n_atoms, n_rot, seed)), n_atoms)


RING_CASES = [(n, r, s, k) for s, (n, r, k) in enumerate([(8, 1, "single"), (16, 3, "single"), (30, 6, "single"),
                                                          (12, 1, "fused"), (24, 4, "fused"), (40, 8, "fused"),
                                                          (14, 2, "linked"), (30, 6, "linked"), (60, 12, "linked")])]


@pytest.mark.parametrize("n_atoms,n_rot,seed,rings", RING_CASES)
def test_schedules_of_ring_ligands(lib, n_atoms, n_rot, seed, rings):
    """Ligands with rigid rings: pairs inside a ring are excluded (one rigid fragment), and the
    'more than three bonds apart' rule counts bonds along the shorter way round a ring."""
    _check_schedules(lib, S.ligand_centered(S.make_ring_ligand(n_atoms, n_rot, seed, rings)), n_atoms)


def _check_schedules(lib, lig, n_atoms):
    L = O.OracleLigand(lig)
    ref = {(min(int(a), int(b)), max(int(a), int(b))) for a, b in L.pairs}
    assert len(ref) == L.n_pairs
    xs = [XS[t] for t in L.xs]
    donor = {t for t in XS if t.endswith("_D") or t.endswith("_DA")}
    acceptor = {t for t in XS if t.endswith("_A") or t.endswith("_DA")}
    _, _, info, _ = _decode(lib, lig, 32)
    widths = [32] + ([16] if info[2] else [])
    # a half-warp team holds up to 32 atoms (two per lane) and 16 tangent coordinates
    assert bool(info[2]) == (n_atoms <= 32 and 6 + L.n_rot <= 16)
    for lanes in widths:
        rows, recv, info, n_rounds = _decode(lib, lig, lanes)
        got = [(min(s, t), max(s, t)) for _, _, s, t, _, _ in rows]
        assert len(got) == len(set(got)) == len(ref), lanes
        assert set(got) == ref, lanes
        for rnd, lane, s, t, hyd, hb in rows:
            assert s != t and s >= 0 and t >= 0
            assert hyd == int(xs[s] == "C_H" and xs[t] == "C_H")
            assert hb == int((xs[s] in donor and xs[t] in acceptor) or (xs[s] in acceptor and xs[t] in donor))
        assert n_rounds == (info[0] if lanes == 32 else info[1])
        # every pair sent is received once, by the lane of its target atom, from its sending lane;
        # a lane sends at most one pair and receives at most one per round
        want = sorted((rnd, lane, t) for rnd, lane, s, t, _, _ in rows)
        got_recv = sorted((rnd, sl, a) for rnd, l, sl, a in recv)
        assert want == got_recv, lanes
        assert len({(rnd, l) for rnd, l, _, _ in recv}) == len(recv)
        if len(rows):
            src_load = np.bincount(rows[:, 1], minlength=lanes).max()
            tgt_load = np.bincount(recv[:, 1], minlength=lanes).max()
            assert n_rounds == max(src_load, tgt_load), lanes


def _bank_cost(words, lanes):
    """Shared-memory wavefronts of the partner gathers: per round and quarter-warp, the largest
    number of distinct partner positions (float4, 16-byte bank groups) sharing a residue mod 8;
    and the lower bound per quarter-warp: its round count, or its largest load on one residue."""
    cost, load = 0, np.zeros((lanes // 8, 8), np.int64)
    for r in range(words.shape[0]):
        for q in range(0, lanes, 8):
            part = {int(w) & 127 for w in words[r, q:q + 8]}
            cost += max(np.bincount([a & 7 for a in part], minlength=8))
            for w in words[r, q:q + 8]:
                if int(w) >> 31:
                    load[q // 8, int(w) & 7] += 1
    return cost, int(sum(max(words.shape[0], load[q].max()) for q in range(lanes // 8)))


@pytest.mark.parametrize("n_atoms,n_rot,seed,rings,at_bound", [
    (30, 6, 0, None, True), (30, 6, 1, None, True), (30, 6, 2, None, True), (24, 6, 5, None, True),
    (31, 9, 9, None, True), (30, 6, 2, "single", True), (40, 8, 5, "fused", True), (48, 12, 11, None, False),
    (64, 20, 13, None, False), (60, 12, 8, "linked", False)])
def test_schedule_partner_gathers_spread_over_bank_groups(lib, n_atoms, n_rot, seed, rings, at_bound):
    """Empty slots read a dummy atom (64-71) of a residue that no partner of their quarter-warp has,
    and the rounds are arranged so that a quarter-warp's partners fall into distinct bank groups:
    ligands of the bench's size reach the lower bound, larger ones stay within 40 % of it."""
    lig = S.make_ring_ligand(n_atoms, n_rot, seed, rings) if rings else S.make_ligand(n_atoms, n_rot, seed)
    _, _, info, _ = _decode(lib, S.ligand_centered(lig), 32)
    for lanes in [32] + ([16] if info[2] else []):
        words, _, _ = _raw(lib, S.ligand_centered(lig), lanes)
        for r in range(words.shape[0]):
            for q in range(0, lanes, 8):
                w = [int(x) for x in words[r, q:q + 8]]
                used = {x & 7 for x in w if x >> 31}
                for x in w:
                    if not x >> 31:
                        assert 64 <= (x & 127) < 72 and (x & 7) not in used
        cost, bound = _bank_cost(words, lanes)
        assert bound <= cost
        assert cost == bound if at_bound else cost <= 1.4 * bound, (lanes, cost, bound)
