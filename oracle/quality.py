"""Objective of the synchronous schedule, with and without the symmetry-
breaking coin, against the sequential method.

Test infrastructure (oracle only): runs the synchronous Parallel-CC
(Algorithm 1, Sec. 3.2.1; the GPU library gives the same labels bit for bit),
the same with the coin of LCC_SCHED_COIN (three seeds) and Sequential-CC
(Sec. 3.1, Algorithm 2; three seeds) on small seeded graphs of the benchmark
families, and prints their objectives (modularity CC / 2m in modularity
mode) and cluster counts.

    python oracle/quality.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2108_01731_gb300 import inputs as I  # noqa: E402


def cases():
    base = I.BASE_SEED
    return [
        ("planted partition 100x100, lambda 1/100, 20 rounds",
         I.to_numpy(I.sbm([100] * 100, 0.05, 0.0005, seed=base + 1)), O.NODEW_UNIT, 1, 100, 20),
        ("Chung-Lu 2^15, beta 2.1, degree 32, modularity",
         I.to_numpy(I.chung_lu(1 << 15, 2.1, 32, seed=base + 2)), O.NODEW_DEGREE, 1, 1, 10),
        ("R-MAT 2^15, 2^19 edges, modularity",
         I.to_numpy(I.rmat(15, 1 << 19, seed=base + 4)), O.NODEW_DEGREE, 1, 1, 10),
    ]


def main():
    print("| graph | synchronous | with the coin (seeds 0, 1, 2) | Sequential-CC (seeds 0, 1, 2) |")
    print("|---|---:|---:|---:|")
    for name, g, mode, p, q, it in cases():
        sl, snum, sden, _ = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, num_iter=it)
        coin = [O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, num_iter=it, coin=True,
                          seed=s) for s in range(3)]
        seq = [O.sequential_cc(g["off"], g["nbr"], g["w"], p, q, mode=mode, seed=s)
               for s in range(3)]
        scale = (sden // q) if mode == O.NODEW_DEGREE else 1  # modularity: CC / 2m

        def cell(runs):
            return " / ".join("%.4g (%d)" % (r[1] / r[2] / scale, len(np.unique(r[0])))
                              for r in runs)
        print("| %s | %.4g (%d) | %s | %s |" % (name, snum / sden / scale, len(np.unique(sl)),
                                              cell(coin), cell(seq)))
    print("\nobjective (clusters); modularity-mode rows give CC / 2m")


if __name__ == "__main__":
    main()
