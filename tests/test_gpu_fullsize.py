"""Parity at the full sizes of the benchmark configurations.

* R-MAT, 2^26 vertices, 2^31 entries (the benchmark workload): the first
  best-move round of every vertex on the GPU, compared with the oracle on a
  sample of vertices (random ones plus the highest-degree hubs), and the
  invariants of a whole run.
* Chung-Lu, 2^20 vertices, ~32M entries: three synchronous rounds, the
  compression of their labels and a two-level run, element by element.
* kNN similarity graph, 10^6 points (signed fixed-point weights): two rounds
  element by element and sampled first rounds for the three resolutions.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_01731_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def L():
    import torch
    torch.cuda.set_device(0)
    from paper_2108_01731_gb300 import lcc
    lcc.load()
    return lcc


def sample_rows(g_dev, verts):
    """Compact CSR of the rows of `verts` (device graph -> host arrays)."""
    import torch
    off = g_dev["off"]
    vt = torch.as_tensor(verts, dtype=torch.int64, device=off.device)
    beg, end = off[vt], off[vt + 1]
    deg = end - beg
    off_l = torch.zeros(len(verts) + 1, dtype=torch.int64, device=off.device)
    off_l[1:] = torch.cumsum(deg, 0)
    rel = torch.arange(int(off_l[-1]), device=off.device) - torch.repeat_interleave(off_l[:-1], deg)
    idx = torch.repeat_interleave(beg, deg) + rel
    nbr = g_dev["nbr"][idx].cpu().numpy()
    w = g_dev["w"][idx].cpu().numpy() if g_dev["w"] is not None else None
    return off_l.cpu().numpy(), nbr, w


def test_rmat_2e26_first_round_sampled(L):
    import torch
    g = I.rmat(26, 1 << 30, seed=I.BASE_SEED + 4, device="cuda")
    n = g["n"]
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
    labels = np.arange(n, dtype=np.int32)
    D = L.lcc_desired(G, 1, 1, L.LCC_NODEW_DEGREE, labels)
    off = g["off"].cpu().numpy()
    k, two_m = O.weighted_degrees(off, g["w"].cpu().numpy())
    deg = np.diff(off)
    rng = np.random.default_rng(26)
    verts = np.unique(np.concatenate([rng.integers(0, n, 3000), np.argsort(deg)[-40:]]))
    off_l, nbr_l, w_l = sample_rows(g, verts)
    want = O.desired_list(n, verts, off_l, nbr_l, w_l, k, 1, two_m, labels, k)
    assert np.array_equal(D[verts], want)
    assert (D != labels).sum() > 0
    del g, D
    torch.cuda.empty_cache()  # the generator's tensors; the library keeps its copy
    # a whole run: canonical labels and a consistent exact objective
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    _, obj, st = L.lcc_cluster(G, 1, 1, L.LCC_NODEW_DEGREE, None, labels_out=out)
    lab = out.cpu().numpy()
    assert np.all(lab <= np.arange(n)) and np.all(lab[lab] == lab)
    assert st["num_clusters"] == int((lab == np.arange(n)).sum())
    num, den = L.lcc_objective(G, 1, 1, L.LCC_NODEW_DEGREE, lab)
    assert num == st["obj_num"] and den == st["obj_den"] == two_m
    G.free()


def test_chung_lu_2e20_rounds_compress_and_levels(L):
    g = I.to_numpy(I.chung_lu(1 << 20, 2.1, 32, seed=I.BASE_SEED + 2))
    n = g["n"]
    G = L.lcc_load_csr(g["off"], g["nbr"])
    k, two_m = O.weighted_degrees(g["off"], None)
    L0 = np.arange(n, dtype=np.int32)
    got, moved, rounds = L.lcc_best_moves(G, 1, 1, L.LCC_NODEW_DEGREE, 3, 1, L0)
    want, wmoved, wrounds = O.best_moves(g["off"], g["nbr"], None, k, 1, two_m, L0, 3)
    assert rounds == wrounds and np.array_equal(got, want)
    mp, C = L.lcc_compress(G, L.LCC_NODEW_DEGREE, got)
    off2, nbr2, w2, k2 = L.lcc_graph_export(C)
    wmp, woff, wnbr, ww, wk = O.compress(g["off"], g["nbr"], None, k, want)
    assert np.array_equal(mp, wmp) and np.array_equal(off2, woff)
    assert np.array_equal(nbr2, wnbr) and np.array_equal(w2, ww) and np.array_equal(k2, wk)
    C.free()
    sched = L.schedule(num_iter=3, max_levels=2)
    lab, obj, st = L.lcc_cluster(G, 1, 1, L.LCC_NODEW_DEGREE, sched)
    wl, num, den, _ = O.cluster(g["off"], g["nbr"], None, 1, 1, mode=O.NODEW_DEGREE,
                                num_iter=3, max_levels=2)
    assert np.array_equal(lab, wl) and st["obj_num"] == num and st["obj_den"] == den
    G.free()


def test_knn_1e6_signed_weights(L):
    import torch
    g = I.knn(1_000_000, 64, 1000, 0.1, 32, seed=I.BASE_SEED + 3, device="cuda")
    n = g["n"]
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
    off = g["off"].cpu().numpy()
    nbr = g["nbr"].cpu().numpy()
    w = g["w"].cpu().numpy()
    rng = np.random.default_rng(3)
    verts = np.sort(rng.choice(n, 4000, replace=False))
    off_l, nbr_l, w_l = sample_rows(g, verts)
    del g
    torch.cuda.empty_cache()
    assert w.min() < 65536 and w.max() <= 65536
    k = np.ones(n, np.int64)
    L0 = np.arange(n, dtype=np.int32)
    p, q = 16384, 25  # lambda = 0.01 on the 2^16 weight scale
    got, _, rounds = L.lcc_best_moves(G, p, q, L.LCC_NODEW_UNIT, 2, 1, L0)
    want, _, wrounds = O.best_moves(off, nbr, w, k, p, q, L0, 2)
    assert rounds == wrounds and np.array_equal(got, want)
    for p, q in [(32768, 5), (32768, 1)]:  # lambda = 0.1, 0.5
        D = L.lcc_desired(G, p, q, L.LCC_NODEW_UNIT, L0)
        wantd = O.desired_list(n, verts, off_l, nbr_l, w_l, k, p, q, L0, k)
        assert np.array_equal(D[verts], wantd)
    G.free()
