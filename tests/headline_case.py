"""Inputs of the search statistic at the headline shape (shared by tests/test_gpu_statistic.py and
the script that writes its expected values, tests/golden/make_headline_search.py): the multi-pocket
receptor (5,000 atoms, 10 carved pockets, 24 A boxes at 0.375 A) and 20 ligands of 30 heavy atoms
and 6 torsions, with coordinates rounded to float32 as the library receives them."""
import numpy as np

import pvsynth as S

CHAINS, STEPS, N_LIGANDS, SEED = 256, 300, 20, 0


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def case():
    w = S.multipocket(seed=0)
    r = w.receptors[0]
    rec = S.Receptor(_f32(r.xyz), r.element, r.donor, r.acceptor)
    boxes = [S.Box(_f32(b.center), _f32(b.size), float(np.float32(b.spacing))) for b in w.boxes[0]]
    ligs = []
    for i in range(N_LIGANDS):
        l = S.ligand_centered(S.make_ligand(30, 6, 1000 + i))
        ligs.append(S.Ligand(_f32(l.xyz), l.element, l.donor, l.acceptor, l.bonds, l.rotatable))
    return rec, boxes, ligs
