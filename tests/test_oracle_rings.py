"""Oracle pins on ligands with rigid rings (six-membered, single, fused and linked): the torsion
tree, the intra pair set and the kinematics, checked against graph facts computed independently
(networkx shortest paths and bridges) and against invariants of rigid motion."""
import networkx as nx
import numpy as np
import pytest

import oracle as O
import pvsynth as S


def _graph(lig):
    g = nx.Graph()
    g.add_nodes_from(range(lig.n))
    g.add_edges_from(map(tuple, lig.bonds.tolist()))
    return g


@pytest.mark.parametrize("rings", ["single", "fused", "linked"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ring_fragments_and_intra_pairs(rings, seed):
    lig = S.ligand_centered(S.make_ring_ligand(28, 6, seed, rings))
    L = O.OracleLigand(lig)
    g = _graph(lig)
    # rigid fragments: components of the graph without its rotatable bonds
    h = g.copy()
    h.remove_edges_from(tuple(b) for b, r in zip(lig.bonds.tolist(), lig.rotatable) if r)
    comps = list(nx.connected_components(h))
    assert L.n_frag == len(comps)
    for c in comps:
        assert len({int(L.frag_of[i]) for i in c}) == 1
    # every ring lies inside one fragment, and no ring bond rotates
    for cyc in nx.cycle_basis(g):
        assert len({int(L.frag_of[i]) for i in cyc}) == 1
    bridges = {tuple(sorted(e)) for e in nx.bridges(g)}
    for (a, b), r in zip(lig.bonds.tolist(), lig.rotatable):
        if r:
            assert tuple(sorted((a, b))) in bridges
    # intra pairs: different fragments and shortest path longer than three bonds
    d = dict(nx.all_pairs_shortest_path_length(g))
    want = {(i, j) for i in range(lig.n) for j in range(i + 1, lig.n)
            if L.frag_of[i] != L.frag_of[j] and d[i][j] > 3}
    got = {(int(a), int(b)) for a, b in L.pairs}
    assert got == want


@pytest.mark.parametrize("rings", ["single", "fused", "linked"])
def test_ring_kinematics_keep_every_bond_and_the_ring_planar(rings):
    lig = S.ligand_centered(S.make_ring_ligand(30, 6, 4, rings))
    L = O.OracleLigand(lig)
    b = lig.bonds
    ref_len = np.linalg.norm(lig.xyz[b[:, 0]] - lig.xyz[b[:, 1]], axis=1)
    rings_idx = [c for c in nx.cycle_basis(_graph(lig))]
    box = S.Box(np.zeros(3), np.array([20.0, 20.0, 20.0]))
    for pot in S.random_poses(50, box, L.n_rot, 3):
        x = L.fk(pot)
        np.testing.assert_allclose(np.linalg.norm(x[b[:, 0]] - x[b[:, 1]], axis=1), ref_len, atol=1e-10)
        for c in rings_idx:
            p = x[c] - x[c].mean(axis=0)
            assert np.linalg.svd(p, compute_uv=False)[-1] < 1e-9      # six atoms in one plane


def test_rotatable_ring_bond_is_refused():
    lig = S.make_ring_ligand(10, 0, 1, "single")
    rot = lig.rotatable.copy()
    rot[2] = 1                                   # a bond of the hexagon
    with pytest.raises(ValueError):
        O.OracleLigand(S.Ligand(lig.xyz, lig.element, lig.donor, lig.acceptor, lig.bonds, rot))
