"""Schedule options of the method compared on the CPU twin.

The paper weighs its options by running time and objective (Sec. 4): the
synchronous against the asynchronous setting, the three vertex subsets V'
(Sec. 3.2.2), and refinement (Sec. 3.2.3).  The twin runs the library's
deterministic schedules, so the seeded symmetry-breaking coin stands in for
the asynchronous setting.  For each option this prints the modularity
(CC / 2m), the entries scanned and the twin's wall time on all host cores.

    python cpu_twin/schedules.py [scale]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import cpu_twin as T  # noqa: E402
from paper_2108_01731_gb300 import inputs as I  # noqa: E402

OPTIONS = [
    ("synchronous, V' = neighbours of moved vertices, refinement", dict()),
    ("synchronous, V' = all vertices", dict(vset=T.VSET_ALL)),
    ("synchronous, V' = neighbours of clusters", dict(vset=T.VSET_NBR_CLUSTERS)),
    ("synchronous, no refinement", dict(refine=False)),
    ("coin, V' = neighbours of moved vertices, refinement", dict(coin=True)),
    ("coin, V' = all vertices", dict(coin=True, vset=T.VSET_ALL)),
    ("coin, V' = neighbours of clusters", dict(coin=True, vset=T.VSET_NBR_CLUSTERS)),
    ("coin, no refinement", dict(coin=True, refine=False)),
]


def main():
    scale = int(sys.argv[1]) if len(sys.argv) > 1 else 20
    base = I.BASE_SEED
    graphs = [
        ("R-MAT 2^%d, %d edges" % (scale, 16 << scale),
         I.to_numpy(I.rmat(scale, 16 << scale, seed=base + 4))),
        ("Chung-Lu 2^%d, beta 2.1, degree 32" % scale,
         I.to_numpy(I.chung_lu(1 << scale, 2.1, 32, seed=base + 2))),
    ]
    print("| graph | schedule | modularity | clusters | entries scanned | rounds | seconds |")
    print("|---|---|---:|---:|---:|---:|---:|")
    for gname, g in graphs:
        for oname, kw in OPTIONS:
            t = time.perf_counter()
            lab, num, den, st, nt = T.cluster(g["off"], g["nbr"], g["w"], 1, 1,
                                              mode=T.NODEW_DEGREE, seed=0, **kw)
            secs = time.perf_counter() - t
            print("| %s | %s | %.4f | %d | %d | %d | %.1f |"
                  % (gname, oname, num / den / den,  # q = 1, so den = 2m and CC / 2m
                     len(np.unique(lab)), st[2], st[1], secs),
                  flush=True)
    print("\nhost threads: %d" % nt)


if __name__ == "__main__":
    main()
