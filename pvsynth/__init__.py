"""Seeded synthetic docking inputs: receptors with carved pockets, torsion-tree ligands (acyclic, or
built around rigid six-membered rings), poses.

This module only *generates inputs*. It holds none of the docking arithmetic: no atom typing,
no scoring terms, no kinematics, no search. Both the FP64 oracle (``oracle/``) and the CUDA
path (``paper_2506_20043_gb300``) consume what it produces; neither is imported here.

Shapes follow the paper's workloads: drug-like ligands stratified by rotatable bonds
(<= 5 / 6-10 / > 10, Results "rotatable bonds" figure) and heavy atoms (<= 15 / 15-25 / > 25),
search boxes of 15-30 A centred on pocket centres (Methods, "Parameters"), 20 A for the
screening set.

Conventions shared with both consumers (input format only):
  * elements: 0 = C, 1 = N, 2 = O, 3 = S
  * ``donor`` / ``acceptor``: 0/1 flags, only ever set on N and O
  * ``bonds``: int32 [nb, 2] atom index pairs; ``rotatable``: uint8 [nb]
  * POT pose vector (Eq. 1): x, y, z, qw, qx, qy, qz, psi_1 .. psi_Nrot
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

ELEM_C, ELEM_N, ELEM_O, ELEM_S = 0, 1, 2, 3
ELEMENT_NAMES = ("C", "N", "O", "S")

RECEPTOR_ELEMENT_P = (0.62, 0.17, 0.19, 0.02)   # C / N / O / S
LIGAND_ELEMENT_P = (0.70, 0.15, 0.15)           # C / N / O
HBOND_FLAG_P = 0.30                             # per N/O, donor and acceptor drawn independently
DENSITY = 0.05                                  # heavy atoms per cubic Angstrom
BOND_LENGTH = 1.5
BOND_ANGLE = math.radians(109.5)
MAX_VALENCE = {ELEM_C: 4, ELEM_N: 3, ELEM_O: 2}


@dataclasses.dataclass
class Receptor:
    xyz: np.ndarray        # float64 [n, 3]
    element: np.ndarray    # uint8 [n]
    donor: np.ndarray      # uint8 [n]
    acceptor: np.ndarray   # uint8 [n]

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


@dataclasses.dataclass
class Ligand:
    xyz: np.ndarray        # float64 [n, 3], the input conformer (psi = 0)
    element: np.ndarray    # uint8 [n]
    donor: np.ndarray      # uint8 [n]
    acceptor: np.ndarray   # uint8 [n]
    bonds: np.ndarray      # int32 [nb, 2]
    rotatable: np.ndarray  # uint8 [nb]

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_rot(self) -> int:
        return int(self.rotatable.sum())


@dataclasses.dataclass
class Box:
    center: np.ndarray     # float64 [3]
    size: np.ndarray       # float64 [3]
    spacing: float = 0.375


def _hbond_flags(rng: np.random.Generator, element: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    polar = (element == ELEM_N) | (element == ELEM_O)
    donor = (polar & (rng.random(element.shape[0]) < HBOND_FLAG_P)).astype(np.uint8)
    acceptor = (polar & (rng.random(element.shape[0]) < HBOND_FLAG_P)).astype(np.uint8)
    return donor, acceptor


def receptor_side(n_atoms: int, density: float = DENSITY) -> float:
    """Edge of the cube that holds ``n_atoms`` at ``density`` atoms per cubic Angstrom."""
    return (n_atoms / density) ** (1.0 / 3.0)


def place_pockets(n: int, radius_range: Tuple[float, float], side: float, seed: int,
                  margin: float = 6.0) -> Tuple[np.ndarray, np.ndarray]:
    """Pocket centres (uniform in the cube shrunk by ``margin``) whose spheres do not overlap.

    Falls back to allowing touching spheres, then any placement, if the cube is too small.
    """
    rng = np.random.default_rng([seed, 0x9E37])
    radii = rng.uniform(radius_range[0], radius_range[1], size=n)
    half = side / 2.0 - margin
    centers = np.zeros((n, 3))
    for gap in (2.0, 0.0, -1e9):
        ok = True
        for i in range(n):
            for _ in range(20000):
                c = rng.uniform(-half, half, size=3)
                if all(np.linalg.norm(c - centers[j]) >= radii[i] + radii[j] + gap for j in range(i)):
                    centers[i] = c
                    break
            else:
                ok = False
                break
        if ok:
            return centers, radii
    raise RuntimeError("pocket placement failed")


def make_receptor(n_atoms: int, seed: int, pockets: Sequence[Tuple[Sequence[float], float]] = (),
                  density: float = DENSITY, side: float | None = None) -> Receptor:
    """``n_atoms`` heavy atoms uniform in a cube centred on the origin, none inside a pocket sphere.

    The cube edge keeps ``density`` for ``n_atoms`` atoms; atoms that fall inside a carved pocket
    are redrawn, so the final count is exactly ``n_atoms``.
    """
    rng = np.random.default_rng([seed, 0x5EC])
    side = receptor_side(n_atoms, density) if side is None else side
    pc = np.array([p[0] for p in pockets], dtype=np.float64).reshape(-1, 3)
    pr = np.array([p[1] for p in pockets], dtype=np.float64)
    out = np.zeros((0, 3))
    while out.shape[0] < n_atoms:
        cand = rng.uniform(-side / 2, side / 2, size=(2 * n_atoms, 3))
        if pc.shape[0]:
            d = np.linalg.norm(cand[:, None, :] - pc[None, :, :], axis=2)
            cand = cand[(d >= pr[None, :]).all(axis=1)]
        out = np.concatenate([out, cand])
    xyz = out[:n_atoms].copy()
    element = rng.choice(4, size=n_atoms, p=RECEPTOR_ELEMENT_P).astype(np.uint8)
    donor, acceptor = _hbond_flags(rng, element)
    return Receptor(xyz, element, donor, acceptor)


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v)


def _perp(v: np.ndarray) -> np.ndarray:
    a = np.array([1.0, 0.0, 0.0]) if abs(v[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    return _unit(np.cross(v, a))


def _graph_dist(nbrs: List[List[int]], src: int) -> np.ndarray:
    dist = np.full(len(nbrs), 10**6, dtype=np.int64)
    dist[src] = 0
    frontier = [src]
    while frontier:
        nxt = []
        for a in frontier:
            for b in nbrs[a]:
                if dist[b] > dist[a] + 1:
                    dist[b] = dist[a] + 1
                    nxt.append(b)
        frontier = nxt
    return dist


def make_ligand(n_atoms: int, n_rot: int, seed: int) -> Ligand:
    """Random acyclic heavy-atom tree grown atom by atom.

    1.5 A bonds, 109.5 degree bond angles, random dihedrals; valence <= 4 (C 4, N 3, O 2).
    A placement is rejected if it brings an atom two bonds away closer than 2.3 A or one
    three or more bonds away closer than 2.5 A. ``n_rot`` rotatable bonds are drawn among the
    non-terminal bonds (both ends with degree >= 2) and capped at their number.
    """
    if n_atoms < 1:
        raise ValueError("n_atoms must be >= 1")
    rng = np.random.default_rng([seed, 0x11A])
    for _attempt in range(1000):
        element = rng.choice(3, size=n_atoms, p=LIGAND_ELEMENT_P).astype(np.uint8)
        element[0] = ELEM_C
        xyz = np.zeros((n_atoms, 3))
        nbrs: List[List[int]] = [[] for _ in range(n_atoms)]
        bonds: List[Tuple[int, int]] = []
        ok = True
        for k in range(1, n_atoms):
            placed = False
            for _try in range(200):
                free = [a for a in range(k) if len(nbrs[a]) < MAX_VALENCE[int(element[a])]]
                if not free:
                    break
                p = int(rng.choice(free))
                if not nbrs[p]:
                    pos = xyz[p] + BOND_LENGTH * _unit(rng.normal(size=3))
                else:
                    g = nbrs[p][0]
                    u = _unit(xyz[g] - xyz[p])
                    w = _perp(u)
                    phi = rng.uniform(-math.pi, math.pi)
                    w = w * math.cos(phi) + np.cross(u, w) * math.sin(phi)
                    pos = xyz[p] + BOND_LENGTH * (math.cos(BOND_ANGLE) * u + math.sin(BOND_ANGLE) * w)
                dist_p = _graph_dist(nbrs[:k] + [[]], p)[:k]
                d = np.linalg.norm(xyz[:k] - pos, axis=1)
                two = (dist_p == 1)      # new atom would be two bonds from these
                far = (dist_p >= 2)      # three or more bonds
                if (d[two] < 2.3).any() or (d[far] < 2.5).any():
                    continue
                xyz[k] = pos
                nbrs[p].append(k)
                nbrs[k].append(p)
                bonds.append((p, k))
                placed = True
                break
            if not placed:
                ok = False
                break
        if not ok:
            continue
        bonds_a = np.array(bonds, dtype=np.int32).reshape(-1, 2)
        deg = np.array([len(x) for x in nbrs])
        nonterminal = [i for i, (a, b) in enumerate(bonds) if deg[a] >= 2 and deg[b] >= 2]
        k_rot = min(n_rot, len(nonterminal))
        rot = np.zeros(len(bonds), dtype=np.uint8)
        if k_rot:
            rot[rng.choice(nonterminal, size=k_rot, replace=False)] = 1
        donor, acceptor = _hbond_flags(rng, element)
        return Ligand(xyz, element, donor, acceptor, bonds_a, rot)
    raise RuntimeError("ligand growth failed")


RING_BOND = 1.40                                # aromatic six-membered ring: side = circumradius


def make_ring_ligand(n_atoms: int, n_rot: int, seed: int, rings: str = "single") -> Ligand:
    """Heavy-atom ligand built around rigid six-membered rings (planar hexagons, 1.40 A bonds):
    ``rings`` = "single" (one ring), "fused" (two rings sharing a bond, naphthalene-like) or
    "linked" (two rings joined by a 1.5 A single bond, biphenyl-like). Ring atoms are C, or N with
    probability 0.15, and take at most one substituent, placed on the outward bisector in the ring
    plane; the remaining atoms grow as trees (as in ``make_ligand``: 1.5 A bonds, 109.5 degree angles,
    random dihedrals, the same clash rejection). Ring bonds are never rotatable (they are not
    bridges); ``n_rot`` rotatable bonds are drawn among the bridges whose two atoms both have degree
    >= 2 (the ring-ring link included) and capped at their number."""
    if rings not in ("single", "fused", "linked"):
        raise ValueError("rings must be single, fused or linked")
    rng = np.random.default_rng([seed, 0x21C])
    n_ring = 6 if rings == "single" else (10 if rings == "fused" else 12)
    if n_atoms < n_ring:
        raise ValueError(f"a {rings} ring scaffold needs at least {n_ring} atoms")
    for _attempt in range(1000):
        u = _unit(rng.normal(size=3))
        v = _perp(u)
        ang = np.arange(6) * (math.pi / 3.0)
        hexagon = lambda c, a0: c + RING_BOND * (np.cos(ang + a0)[:, None] * u + np.sin(ang + a0)[:, None] * v)  # noqa: E731
        xyz = [*hexagon(np.zeros(3), 0.0)]
        bonds: List[Tuple[int, int]] = [(k, (k + 1) % 6) for k in range(6)]
        ring_bonds = set(range(6))
        if rings == "fused":
            # the second hexagon shares atoms 0 and 1; its centre is the first's reflected across them
            c2 = xyz[0] + xyz[1]
            second = hexagon(c2, math.pi)            # vertex k = c2 - (vertex k of the first ring)
            # so second[0] is atom 1 and second[1] is atom 0; add the four others
            idx = {0: 1, 1: 0}
            for k in (2, 3, 4, 5):
                idx[k] = len(xyz)
                xyz.append(second[k])
            for k in range(6):
                a, b = idx[k], idx[(k + 1) % 6]
                if {a, b} != {0, 1}:
                    ring_bonds.add(len(bonds))
                    bonds.append((a, b))
        elif rings == "linked":
            out = _unit(xyz[3])                        # radial direction of atom 3
            c2 = xyz[3] + (BOND_LENGTH + RING_BOND) * out
            second = hexagon(c2, 0.0)                  # its vertex 0 faces atom 3
            base = len(xyz)
            xyz.extend(second)
            for k in range(6):
                ring_bonds.add(len(bonds))
                bonds.append((base + k, base + (k + 1) % 6))
            bonds.append((3, base))                    # the link: a bridge
        xyz = np.array(xyz)
        n0 = len(xyz)
        element = np.zeros(n_atoms, np.uint8)
        element[:n0] = np.where(rng.random(n0) < 0.15, ELEM_N, ELEM_C)
        element[0] = ELEM_C
        element[n0:] = rng.choice(3, size=n_atoms - n0, p=LIGAND_ELEMENT_P)
        nbrs: List[List[int]] = [[] for _ in range(n_atoms)]
        for a, b in bonds:
            nbrs[a].append(b)
            nbrs[b].append(a)
        in_ring = np.zeros(n_atoms, bool)
        for bi in ring_bonds:
            in_ring[list(bonds[bi])] = True
        xyz = np.concatenate([xyz, np.zeros((n_atoms - n0, 3))])
        ok = True
        for k in range(n0, n_atoms):
            placed = False
            for _try in range(200):
                free = [a for a in range(k) if len(nbrs[a]) < (3 if in_ring[a] else MAX_VALENCE[int(element[a])])]
                if not free:
                    break
                p = int(rng.choice(free))
                if in_ring[p]:
                    w = -sum(_unit(xyz[q] - xyz[p]) for q in nbrs[p] if in_ring[q])
                    pos = xyz[p] + BOND_LENGTH * _unit(w)
                elif not nbrs[p]:
                    pos = xyz[p] + BOND_LENGTH * _unit(rng.normal(size=3))
                else:
                    g = nbrs[p][0]
                    uu = _unit(xyz[g] - xyz[p])
                    ww = _perp(uu)
                    phi = rng.uniform(-math.pi, math.pi)
                    ww = ww * math.cos(phi) + np.cross(uu, ww) * math.sin(phi)
                    pos = xyz[p] + BOND_LENGTH * (math.cos(BOND_ANGLE) * uu + math.sin(BOND_ANGLE) * ww)
                dist_p = _graph_dist(nbrs[:k] + [[]], p)[:k]
                d = np.linalg.norm(xyz[:k] - pos, axis=1)
                if (d[dist_p == 1] < 2.3).any() or (d[dist_p >= 2] < 2.5).any():
                    continue
                xyz[k] = pos
                nbrs[p].append(k)
                nbrs[k].append(p)
                bonds.append((p, k))
                placed = True
                break
            if not placed:
                ok = False
                break
        if not ok:
            continue
        deg = np.array([len(x) for x in nbrs])
        cand = [i for i, (a, b) in enumerate(bonds) if i not in ring_bonds and deg[a] >= 2 and deg[b] >= 2]
        k_rot = min(n_rot, len(cand))
        rot = np.zeros(len(bonds), dtype=np.uint8)
        if k_rot:
            rot[rng.choice(cand, size=k_rot, replace=False)] = 1
        donor, acceptor = _hbond_flags(rng, element)
        return Ligand(xyz, element, donor, acceptor, np.array(bonds, dtype=np.int32).reshape(-1, 2), rot)
    raise RuntimeError("ring ligand growth failed")


def ligand_centered(lig: Ligand) -> Ligand:
    """Copy of ``lig`` with its coordinates shifted to the centroid (placement is arbitrary)."""
    return dataclasses.replace(lig, xyz=lig.xyz - lig.xyz.mean(axis=0))


def random_poses(n: int, box: Box, n_rot: int, seed: int) -> np.ndarray:
    """``n`` POT vectors (Eq. 1): translation uniform in the box, uniform random unit quaternion
    (Shoemake's subgroup method), torsions uniform in [-pi, pi). float64 [n, 7 + n_rot]."""
    rng = np.random.default_rng([seed, 0x905E])
    c = np.asarray(box.center, dtype=np.float64)
    s = np.asarray(box.size, dtype=np.float64)
    t = c + (rng.random((n, 3)) - 0.5) * s
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    q = np.stack([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2), np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3), np.sqrt(u1) * np.cos(2 * np.pi * u3)], axis=1)
    psi = rng.uniform(-np.pi, np.pi, size=(n, n_rot))
    return np.concatenate([t, q, psi], axis=1)


# --------------------------------------------------------------------------------------------
# Workloads. Each returns plain data; sizes follow the five benchmark configurations.
# --------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    receptors: List[Receptor]
    boxes: List[List[Box]]           # per receptor, one box per pocket
    ligands: List[Ligand]
    chains: int
    steps: int
    top_k: int
    seed: int = 0
    ligands_per_receptor: List[List[int]] | None = None   # screening: ligand subsets


def _carved(n_atoms: int, n_pockets: int, radius_range: Tuple[float, float], seed: int,
            box: float) -> Tuple[Receptor, List[Box]]:
    side = receptor_side(n_atoms)
    if n_pockets == 1 and radius_range[0] == radius_range[1]:
        centers, radii = np.zeros((1, 3)), np.array([radius_range[0]])
    else:
        centers, radii = place_pockets(n_pockets, radius_range, side, seed,
                                       margin=min(6.0, side / 4))
    rec = make_receptor(n_atoms, seed, list(zip(centers, radii)))
    boxes = [Box(np.array(c), np.array([box, box, box])) for c in centers]
    return rec, boxes


def tiny(seed: int = 0) -> Workload:
    """2,000-atom receptor, one 8 A pocket at the centre, 20 A box; 20-atom ligand with
    4 torsions; 8 chains x 1,000 MC steps."""
    rec, boxes = _carved(2000, 1, (8.0, 8.0), seed, 20.0)
    lig = ligand_centered(make_ligand(20, 4, seed))
    return Workload("tiny", [rec], [boxes], [lig], chains=8, steps=1000, top_k=9, seed=seed)


def score_microbench(seed: int = 0) -> Tuple[Receptor, Box, Ligand, np.ndarray]:
    """4,000-atom receptor, one 24 A box on an 8 A pocket; 32-atom ligand with 8 torsions;
    65,536 random poses."""
    rec, boxes = _carved(4000, 1, (8.0, 8.0), seed, 24.0)
    lig = ligand_centered(make_ligand(32, 8, seed))
    poses = random_poses(65536, boxes[0], lig.n_rot, seed)
    return rec, boxes[0], lig, poses


def multipocket(seed: int = 0, chains: int = 1000, steps: int = 2000) -> Workload:
    """5,000-atom receptor, 10 pockets of radius 6-10 A with 24 A boxes; 30-atom ligand with
    6 torsions; 1,000 chains x 2,000 steps per pocket; top-9 per pocket."""
    rec, boxes = _carved(5000, 10, (6.0, 10.0), seed, 24.0)
    lig = ligand_centered(make_ligand(30, 6, seed))
    return Workload("multipocket", [rec], [boxes], [lig], chains=chains, steps=steps, top_k=9,
                    seed=seed)


def uneven(seed: int = 0, n_ligands: int = 512, chains: int = 64, steps: int = 1000) -> Workload:
    """6,000-atom receptor with 5 pockets; ``n_ligands`` ligands of 10-60 heavy atoms and
    0-15 torsions (capped at the non-terminal bond count); 64 chains x 1,000 steps per pair."""
    rec, boxes = _carved(6000, 5, (6.0, 10.0), seed, 24.0)
    rng = np.random.default_rng([seed, 0x0E7])
    ligs = [ligand_centered(make_ligand(int(rng.integers(10, 61)), int(rng.integers(0, 16)),
                                        seed * 100003 + i)) for i in range(n_ligands)]
    return Workload("uneven", [rec], [boxes], ligs, chains=chains, steps=steps, top_k=9, seed=seed)


def screening(seed: int = 0, n_receptors: int = 256, ligands_per_receptor: int = 100,
              chains: int = 32, steps: int = 1000) -> Workload:
    """``n_receptors`` receptors of 1,500-8,000 atoms (log-uniform), 3 pockets each with 24 A
    boxes; ``ligands_per_receptor`` 30-atom / 6-torsion ligands per receptor."""
    rng = np.random.default_rng([seed, 0x5C2])
    recs, boxes, ligs, subsets = [], [], [], []
    for r in range(n_receptors):
        n_at = int(round(math.exp(rng.uniform(math.log(1500), math.log(8000)))))
        rec, bx = _carved(n_at, 3, (6.0, 10.0), seed * 7919 + r, 24.0)
        recs.append(rec)
        boxes.append(bx)
        ids = []
        for j in range(ligands_per_receptor):
            ids.append(len(ligs))
            ligs.append(ligand_centered(make_ligand(30, 6, (seed * 7919 + r) * 1000 + j)))
        subsets.append(ids)
    return Workload("screening", recs, boxes, ligs, chains=chains, steps=steps, top_k=9, seed=seed,
                    ligands_per_receptor=subsets)


def box_sweep(seed: int = 0, sizes: Sequence[float] = tuple(range(15, 31)), n_pockets: int = 5,
              chains: int = 256, steps: int = 1000) -> Workload:
    """5,000-atom receptor with ``n_pockets`` pockets (radius 6-10 A, listed in rank order), each
    docked in boxes of every edge in ``sizes`` (15-30 A by 1 A by default) centred on the pocket;
    one 30-atom / 6-torsion ligand. Boxes are pocket-major: box i = pocket i // len(sizes), size
    sizes[i % len(sizes)]."""
    rec, centres = _carved(5000, n_pockets, (6.0, 10.0), seed, 24.0)
    boxes = [Box(np.array(b.center), np.array([float(s)] * 3)) for b in centres for s in sizes]
    lig = ligand_centered(make_ligand(30, 6, seed))
    return Workload("box_sweep", [rec], [boxes], [lig], chains=chains, steps=steps, top_k=9, seed=seed)


# ------------------------------------------------------------------ pocket-side inputs --
# Inputs of the pocket prediction (Supplementary Algorithm 1). The Random Forest score of
# Step 3 is replaced by a synthetic ligandability that is high inside the carved pockets.

# Bondi (J. Phys. Chem. 68, 441, 1964) van der Waals radii by element: C, N, O, S.
VDW_RADIUS = (1.70, 1.55, 1.52, 1.80)
PROPERTY_NAMES = ("is_C", "is_N", "is_O", "is_S", "donor", "acceptor", "charge")


def vdw_radii(rec: Receptor) -> np.ndarray:
    return np.asarray(VDW_RADIUS, dtype=np.float64)[rec.element]


def atom_properties(rec: Receptor, seed: int) -> np.ndarray:
    """float32 [n, 7] per-atom property columns (PROPERTY_NAMES): element one-hot, the donor and
    acceptor flags, and a synthetic partial charge uniform in [-0.5, 0.5]."""
    rng = np.random.default_rng([seed, 0x9C0])
    out = np.zeros((rec.n, len(PROPERTY_NAMES)), dtype=np.float32)
    out[np.arange(rec.n), rec.element] = 1.0
    out[:, 4] = rec.donor
    out[:, 5] = rec.acceptor
    out[:, 6] = rng.uniform(-0.5, 0.5, size=rec.n)
    return out


@dataclasses.dataclass
class PocketSite:
    receptor: Receptor
    centers: np.ndarray     # [P, 3] carved pocket centres
    radii: np.ndarray       # [P]


def pocket_site(seed: int = 0, n_atoms: int = 8000, n_pockets: int = 10,
                radius_range: Tuple[float, float] = (6.0, 10.0)) -> PocketSite:
    """A receptor of ``n_atoms`` atoms (0.05 per cubic A) with ``n_pockets`` carved spherical pockets."""
    side = receptor_side(n_atoms)
    centers, radii = place_pockets(n_pockets, radius_range, side, seed, margin=min(6.0, side / 4))
    rec = make_receptor(n_atoms, seed, list(zip(centers, radii)))
    return PocketSite(rec, centers, radii)


def ligandability(points, site: PocketSite, seed: int, noise: float = 0.1) -> np.ndarray:
    """Synthetic stand-in for the classifier score of each point, float32 in [0, 1]: 1 inside a
    carved pocket sphere, falling off over about 2 A outside it, mixed with uniform noise."""
    p = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    rng = np.random.default_rng([seed, 0x5C0])
    if p.shape[0] == 0:
        return np.zeros(0, dtype=np.float32)
    d = np.linalg.norm(p[:, None, :] - site.centers[None, :, :], axis=2) - site.radii[None, :]
    base = np.exp(-(np.maximum(d, 0.0) / 2.0) ** 2).max(axis=1)
    return ((1.0 - noise) * base + noise * rng.random(p.shape[0])).astype(np.float32)


def cluster_cloud(seed: int = 0, n_blobs: int = 20, per_blob: int = 500, n_background: int = 5000,
                  extent: float = 60.0, spread: float = 2.0) -> Tuple[np.ndarray, np.ndarray]:
    """Points for clustering: ``n_blobs`` Gaussian blobs (sd ``spread`` A) and a uniform background
    in a cube of edge ``extent``, with uniform scores in [0, 1]. float32 [n, 3], float32 [n]."""
    rng = np.random.default_rng([seed, 0xC1C])
    centres = rng.uniform(-extent / 2, extent / 2, size=(n_blobs, 3))
    blobs = (centres[:, None, :] + rng.normal(scale=spread, size=(n_blobs, per_blob, 3))).reshape(-1, 3)
    bg = rng.uniform(-extent / 2, extent / 2, size=(n_background, 3))
    pts = np.concatenate([blobs, bg])[rng.permutation(n_blobs * per_blob + n_background)]
    return pts.astype(np.float32), rng.random(pts.shape[0]).astype(np.float32)
