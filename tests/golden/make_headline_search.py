"""Writes headline_search_best.txt: the FP64 oracle's search results at the benchmark's headline
shape, the expected values of tests/test_gpu_statistic.py.

The search is stochastic (Monte-Carlo chains with RILC-BFGS, Supplementary Algorithm 2), so the GPU
is compared with the oracle statistically: per ligand, its best SF over the chains of all its
pockets and the pocket of that best pose (Algorithm 3's top-ranked pocket). Workload: the
multi-pocket receptor (5,000 atoms, 10 carved pockets with 24 A boxes at 0.375 A), 20 ligands of
30 heavy atoms and 6 torsions (seeds 1000-1019), every ligand docked into every pocket, 256 chains x
300 MC steps per pair, Philox key 0, pair index = ligand * 10 + pocket. A second oracle run with key
1 on the first five ligands records how far two oracle runs fall apart at this budget.

Only ``oracle/`` computes here; run from the repository root:
    python tests/golden/make_headline_search.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from tests.headline_case import CHAINS, STEPS, N_LIGANDS, SEED, case  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "headline_search_best.txt")


def main():
    threads = len(os.sched_getaffinity(0))
    rec, boxes, ligs = case()
    Ls = [O.OracleLigand(l) for l in ligs]
    types = sorted(set(np.concatenate([L.xs for L in Ls]).tolist()))
    rt = O.xs_type_receptor(rec)
    t0 = time.time()
    grids = [O.OracleGrid(rec, b, types, rec_types=rt, threads=threads) for b in boxes]
    print(f"grids {time.time() - t0:.1f} s", flush=True)
    rows = []
    for key, n_lig in ((SEED, N_LIGANDS), (SEED + 1, 5)):
        for li in range(n_lig):
            t0 = time.time()
            best = []
            for k, (g, b) in enumerate(zip(grids, boxes)):
                _, es, _ = O.mc_chains(Ls[li], g, b, O.SearchParams(seed=key, steps=STEPS),
                                       unit=li * len(boxes) + k, n_chains=CHAINS, threads=threads)
                best.append(float(es.min()))
            rows.append((key, li, best))
            print(f"key {key} ligand {li}: best {min(best):.4f} pocket {int(np.argmin(best))} "
                  f"({time.time() - t0:.0f} s)", flush=True)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle (oracle/pv_oracle.c) search results at the headline shape, written by\n"
                "# tests/golden/make_headline_search.py (see its docstring for the workload).\n"
                f"# chains {CHAINS}, MC steps {STEPS}, pockets {len(boxes)}, ligands {N_LIGANDS}\n"
                "# columns: philox key, ligand, best SF (kcal/mol) of each pocket's chains, pockets 0..9\n")
        for key, li, best in rows:
            f.write(f"{key} {li} " + " ".join(f"{v:.6f}" for v in best) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
