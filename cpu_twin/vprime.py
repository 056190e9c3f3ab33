"""Vertices in V' per best-move round, on the CPU twin.

The paper plots |V'| per best-move iteration for two vertex-subset rules,
neighbours of vertices that moved and neighbours of the clusters they left
(Sec. 3.2.2).  This prints the same quantity for level 0's coarsening call on
seeded R-MAT and Chung-Lu graphs, for the plain synchronous rounds and with
the symmetry-breaking coin, as a percentage of the level's vertices.

    python cpu_twin/vprime.py [scale]
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import cpu_twin as T  # noqa: E402
from paper_2108_01731_gb300 import inputs as I  # noqa: E402


def main():
    scale = int(sys.argv[1]) if len(sys.argv) > 1 else 20
    base = I.BASE_SEED
    graphs = [("R-MAT 2^%d" % scale, I.to_numpy(I.rmat(scale, 16 << scale, seed=base + 4))),
              ("Chung-Lu 2^%d" % scale,
               I.to_numpy(I.chung_lu(1 << scale, 2.1, 32, seed=base + 2)))]
    rules = [("neighbours of vertices", T.VSET_NBR_VERTICES),
             ("neighbours of clusters", T.VSET_NBR_CLUSTERS)]
    print("| graph | schedule | V' rule | |V'| per round of level 0, % of n |")
    print("|---|---|---|---|")
    for gname, g in graphs:
        for coin in (False, True):
            for rname, vset in rules:
                _, tr = T.cluster_trace(g["off"], g["nbr"], g["w"], 1, 1, mode=T.NODEW_DEGREE,
                                        vset=vset, coin=coin, seed=0)
                lvl0 = tr[(tr[:, 0] == 0) & (tr[:, 1] == 0)]
                cells = " ".join("%.1f" % (100.0 * r[3] / g["n"]) for r in lvl0)
                print("| %s | %s | %s | %s |" % (gname, "coin" if coin else "synchronous",
                                                 rname, cells))


if __name__ == "__main__":
    main()
