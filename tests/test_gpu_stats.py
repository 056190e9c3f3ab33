"""lcc_stats.bytes_contract_min against the sizes the oracle gives for the
same run: one contraction (max_levels = 2) reads the input level's offsets,
neighbours, weights and labels once and writes the coarse offsets,
neighbours, int64 weights and node weights once."""
import numpy as np
import pytest

import oracle as O
from paper_2108_01731_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("weighted", [False, True])
def test_contraction_minimum_bytes(weighted):
    import torch
    torch.cuda.set_device(0)
    from paper_2108_01731_gb300 import lcc as L
    L.load()
    g = I.to_numpy(I.hub_graph(20000, 5, 3, 7000, seed=2, w_lo=1, w_hi=4) if weighted
                   else I.chung_lu(30000, 2.1, 12, seed=4))
    n, nnz = g["n"], g["nnz"]
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
    _, _, st = L.lcc_cluster(G, 1, 1, L.LCC_NODEW_DEGREE, L.schedule(max_levels=2))
    G.free()
    k, two_m = O.weighted_degrees(g["off"], g["w"])
    lab, moved, _ = O.best_moves(g["off"], g["nbr"], g["w"], k, 1, two_m,
                                 np.arange(n, dtype=np.int32), 10)
    assert moved and st["levels"] == 2
    _, off2, nbr2, _, _ = O.compress(g["off"], g["nbr"], g["w"], k, lab)
    n2, nnz2 = len(off2) - 1, len(nbr2)
    wb = 4 if weighted else 0
    want = (n + 1) * 8 + nnz * (4 + wb) + n * 4 + (n2 + 1) * 8 + nnz2 * (4 + 8) + n2 * 8
    assert st["bytes_contract_min"] == want
