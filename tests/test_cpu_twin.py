"""The OpenMP CPU twin against the oracle (CPU only).

The twin is the multi-core CPU baseline the benchmark times beside the GPU.
It runs the same synchronous schedule, so every output is compared with the
oracle's bit for bit: labels, the exact objective, levels, rounds and
scanned entries of whole runs, labels after single Best-Moves calls from
arbitrary labellings (every V' rule, isolation into empty cluster ids),
coarse graphs of Compress and the desired clusters of a full round, at
several thread counts (integer sums make the result independent of them).
"""
import numpy as np
import pytest

import cpu_twin as T
import oracle as O
from paper_2108_01731_gb300 import inputs as I


def graphs():
    return {
        "sbm": I.to_numpy(I.sbm([60] * 30, 0.2, 0.01, seed=1)),
        "hubs": I.to_numpy(I.hub_graph(20000, 5, 3, 7000, seed=2)),
        "hubs_w": I.to_numpy(I.hub_graph(12000, 7, 2, 9000, seed=3, w_lo=-5, w_hi=9)),
        "cl": I.to_numpy(I.chung_lu(30000, 2.1, 12, seed=4)),
        "rmat": I.to_numpy(I.rmat(14, 120000, seed=5)),
        "signed": I.to_numpy(I.random_signed_graph(300, 0.1, -4, 6, seed=6)),
    }


GRAPHS = graphs()

CASES = [
    ("sbm", O.NODEW_UNIT, 1, 50, {}),
    ("sbm", O.NODEW_UNIT, 1, 50, {"refine": False}),
    ("sbm", O.NODEW_UNIT, 1, 50, {"vset": O.VSET_ALL, "num_iter": 5}),
    ("hubs", O.NODEW_DEGREE, 1, 1, {}),
    ("hubs_w", O.NODEW_UNIT, 1, 8, {}),
    ("hubs_w", O.NODEW_CUSTOM, 2, 9, {"vset": O.VSET_NBR_CLUSTERS}),
    ("cl", O.NODEW_DEGREE, 1, 1, {}),
    ("cl", O.NODEW_UNIT, 1, 100, {"max_levels": 2}),
    ("rmat", O.NODEW_DEGREE, 1, 1, {}),
    ("rmat", O.NODEW_DEGREE, 1 << 40, 3, {}),
    ("signed", O.NODEW_UNIT, 1, 10, {"num_iter": 20}),
]


def custom_k(g, seed):
    return np.random.default_rng(seed).integers(0, 7, g["n"]).astype(np.int64)


def degrees(g):
    w = g["w"] if g["w"] is not None else np.ones(g["nnz"], np.int64)
    k = np.zeros(g["n"], np.int64)
    np.add.at(k, np.repeat(np.arange(g["n"]), np.diff(g["off"])), w.astype(np.int64))
    return k


@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%d-%d/%d-%s" % (
    c[0], c[1], c[2], c[3], "-".join("%s%s" % kv for kv in sorted(c[4].items()))))
def test_twin_cluster_matches_oracle(case, threads):
    name, mode, p, q, kw = case
    g = GRAPHS[name]
    k = custom_k(g, 9) if mode == O.NODEW_CUSTOM else None
    sched = dict(num_iter=kw.get("num_iter", 10), max_levels=kw.get("max_levels", 64),
                 refine=kw.get("refine", True), vset=kw.get("vset", O.VSET_NBR_VERTICES))
    wl, num, den, wst = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, k=k, **sched)
    lab, tnum, tden, tst, used = T.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, k=k,
                                           threads=threads, **sched)
    assert used == threads
    assert np.array_equal(lab, wl)
    assert (tnum, tden) == (num, den)
    assert tst == wst


def test_twin_results_do_not_depend_on_thread_count():
    g = GRAPHS["rmat"]
    ref = T.cluster(g["off"], g["nbr"], g["w"], 1, 1, mode=T.NODEW_DEGREE, threads=1)
    for nt in (2, 3, 8):
        got = T.cluster(g["off"], g["nbr"], g["w"], 1, 1, mode=T.NODEW_DEGREE, threads=nt)
        assert np.array_equal(got[0], ref[0]) and got[1:4] == ref[1:4]


@pytest.mark.parametrize("vset", [O.VSET_ALL, O.VSET_NBR_VERTICES, O.VSET_NBR_CLUSTERS])
@pytest.mark.parametrize("name", ["hubs_w", "signed", "cl"])
def test_twin_best_moves_from_arbitrary_labels(name, vset):
    """Labels drawn from a small id range leave most ids empty, so vertices
    may isolate themselves (cluster id v empty and not adjacent)."""
    g = GRAPHS[name]
    rng = np.random.default_rng(31)
    L0 = rng.integers(0, max(2, g["n"] // 7), g["n"]).astype(np.int32)
    k = custom_k(g, 5)
    for p, q in [(1, 3), (2, 1)]:
        want, wmoved, wrounds = O.best_moves(g["off"], g["nbr"], g["w"], k, p, q, L0, 6, vset)
        got, moved, rounds = T.best_moves(g["off"], g["nbr"], g["w"], k, p, q, L0, 6, vset,
                                          threads=4)
        assert np.array_equal(got, want) and moved == wmoved and rounds == wrounds


@pytest.mark.parametrize("name", ["hubs_w", "rmat", "signed"])
def test_twin_compress_matches_oracle(name):
    g = GRAPHS[name]
    rng = np.random.default_rng(17)
    k = degrees(g) if name != "hubs_w" else custom_k(g, 2)
    for span in (3, g["n"] // 5, g["n"]):
        L = rng.integers(0, span, g["n"]).astype(np.int32)
        want = O.compress(g["off"], g["nbr"], g["w"], k, L)
        got = T.compress(g["off"], g["nbr"], g["w"], k, L, threads=4)
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
    # coarse weights are int64 and pass through a second Compress
    mp, off2, nbr2, w2, k2 = want
    L2 = rng.integers(0, max(1, len(k2) // 3), len(k2)).astype(np.int32)
    want2 = O.compress(off2, nbr2, w2, k2, L2)
    got2 = T.compress(off2, nbr2, w2, k2, L2, threads=3)
    for a, b in zip(got2, want2):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["hubs", "rmat", "hubs_w"])
def test_twin_first_round_matches_oracle(name):
    g = GRAPHS[name]
    k = degrees(g) if name != "hubs_w" else np.ones(g["n"], np.int64)
    q = int(k.sum()) if name != "hubs_w" else 4
    n = g["n"]
    L0 = np.arange(n, dtype=np.int32)
    want = O.desired(g["off"], g["nbr"], g["w"], k, 1, q, L0, k)
    D, ent, secs, used = T.first_round(g["off"], g["nbr"], g["w"], k, 1, q, threads=4)
    assert np.array_equal(D, want)
    assert ent == g["nnz"] and secs >= 0 and used == 4
    if name != "hubs_w":  # modularity weights derived inside the twin
        D2 = T.first_round(g["off"], g["nbr"], g["w"], None, 1, 1, threads=3)[0]
        assert np.array_equal(D2, want)


def test_twin_edge_cases():
    # no vertices
    lab, num, den, st, _ = T.cluster(np.zeros(1, np.int64), np.zeros(0, np.int32), None, 1, 2)
    assert len(lab) == 0 and num == 0 and st == O.cluster(np.zeros(1, np.int64),
                                                          np.zeros(0, np.int32), None, 1, 2)[3]
    # vertices without edges stay singletons
    off = np.zeros(6, np.int64)
    lab, num, _, st, _ = T.cluster(off, np.zeros(0, np.int32), None, 1, 2)
    assert np.array_equal(lab, np.arange(5)) and num == 0
    # K2 oscillates for num_iter rounds, then singletons with CC = 0
    off = np.array([0, 1, 2], np.int64)
    nbr = np.array([1, 0], np.int32)
    for it in (1, 4, 7):
        got = T.cluster(off, nbr, None, 1, 2, num_iter=it)
        want = O.cluster(off, nbr, None, 1, 2, num_iter=it)
        assert np.array_equal(got[0], want[0]) and got[1:4] == want[1:4]
        assert np.array_equal(got[0], [0, 1]) and got[3][1] == it
    # gains that could leave __int128 are refused, not wrapped
    g = GRAPHS["sbm"]
    with pytest.raises(ValueError, match="status 5"):
        T.cluster(g["off"], g["nbr"], None, (1 << 62), 1, mode=T.NODEW_CUSTOM,
                  k=np.full(g["n"], 1 << 40, np.int64))
    # modularity needs non-negative degrees
    h = GRAPHS["signed"]
    with pytest.raises(ValueError, match="status 1"):
        T.cluster(h["off"], h["nbr"], h["w"], 1, 1, mode=T.NODEW_DEGREE)


COIN_CASES = [
    ("sbm", O.NODEW_UNIT, 1, 50, {"num_iter": 20}),
    ("hubs_w", O.NODEW_CUSTOM, 2, 9, {"vset": O.VSET_NBR_CLUSTERS}),
    ("cl", O.NODEW_DEGREE, 1, 1, {}),
    ("rmat", O.NODEW_DEGREE, 1, 1, {}),
    ("signed", O.NODEW_UNIT, 1, 10, {"vset": O.VSET_ALL, "num_iter": 30}),
]


@pytest.mark.parametrize("threads", [1, 6])
@pytest.mark.parametrize("case", COIN_CASES, ids=lambda c: "%s-%d-%d/%d" % c[:4])
def test_twin_coin_schedule_matches_oracle(case, threads):
    """The symmetry-breaking coin: same held-back vertices, rounds and labels
    as the oracle for every seed and thread count."""
    name, mode, p, q, kw = case
    g = GRAPHS[name]
    k = custom_k(g, 9) if mode == O.NODEW_CUSTOM else None
    sched = dict(num_iter=kw.get("num_iter", 10), vset=kw.get("vset", O.VSET_NBR_VERTICES))
    for seed in (0, 12345, (1 << 64) - 3):
        wl, num, den, wst = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, k=k,
                                      coin=True, seed=seed, **sched)
        lab, tnum, tden, tst, _ = T.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, k=k,
                                            coin=True, seed=seed, threads=threads, **sched)
        assert np.array_equal(lab, wl) and (tnum, tden) == (num, den) and tst == wst


@pytest.mark.parametrize("vset", [O.VSET_ALL, O.VSET_NBR_VERTICES, O.VSET_NBR_CLUSTERS])
def test_twin_coin_best_moves_matches_oracle(vset):
    g = GRAPHS["hubs_w"]
    rng = np.random.default_rng(4)
    L0 = rng.integers(0, g["n"] // 5, g["n"]).astype(np.int32)
    k = custom_k(g, 6)
    for it in (1, 3, 40):
        want = O.best_moves(g["off"], g["nbr"], g["w"], k, 1, 3, L0, it, vset, coin=True, seed=9)
        got = T.best_moves(g["off"], g["nbr"], g["w"], k, 1, 3, L0, it, vset, coin=True, seed=9,
                           threads=4)
        assert np.array_equal(got[0], want[0]) and got[1:] == want[1:]


@pytest.mark.parametrize("coin", [False, True])
def test_twin_round_trace(coin):
    """Per-round records: one per round; entries sum to the scanned total;
    each call's first round evaluates every vertex of its level; level 0's
    coarsening rounds and moves agree with the oracle's Best-Moves; the same
    records at every thread count."""
    g = GRAPHS["cl"]
    res, tr = T.cluster_trace(g["off"], g["nbr"], g["w"], 1, 1, mode=T.NODEW_DEGREE, coin=coin,
                              seed=5, threads=4)
    lab, num, den, st, _ = res
    assert len(tr) == st[1] and int(tr[:, 4].sum()) == st[2]
    firsts = tr[tr[:, 2] == 0]
    assert firsts[0, 3] == g["n"] and (firsts[:, 3] > 0).all()
    if not coin:
        assert (tr[:, 6] == 0).all()
    lvl0 = tr[(tr[:, 0] == 0) & (tr[:, 1] == 0)]
    k, two_m = O.weighted_degrees(g["off"], g["w"])
    L0 = np.arange(g["n"], dtype=np.int32)
    prev = L0
    for r in range(1, len(lvl0) + 1):
        Lr, _, rounds = O.best_moves(g["off"], g["nbr"], g["w"], k, 1, two_m, L0, r,
                                     coin=coin, seed=5)
        assert rounds == r
        moved = int((Lr != prev).sum())
        assert moved == lvl0[r - 1, 5], r  # moves of round r (row r - 1)
        prev = Lr
    again = T.cluster_trace(g["off"], g["nbr"], g["w"], 1, 1, mode=T.NODEW_DEGREE, coin=coin,
                            seed=5, threads=1)[1]
    assert np.array_equal(again, tr)


def test_exact_range_bound_equals_the_oracles():
    """Custom node weights summing to 2^32: p = 2^61 puts p * (sum k)^2 at
    exactly 2^125 and both the twin and the oracle refuse; p = 2^61 - 1 is
    accepted by both with the same result."""
    import torch
    import oracle as O
    from paper_2108_01731_gb300 import inputs as I
    g = I.to_numpy(I.pairs_to_csr(torch.tensor([0, 1, 2, 0]), torch.tensor([1, 2, 3, 3]), 5))
    k = np.full(5, 1 << 30, np.int64)
    k[4] = 0
    with pytest.raises(Exception):
        T.cluster(g["off"], g["nbr"], None, 1 << 61, 1, mode=T.NODEW_CUSTOM, k=k)
    with pytest.raises(OverflowError):
        O.cluster(g["off"], g["nbr"], None, 1 << 61, 1, mode=O.NODEW_CUSTOM, k=k)
    p = (1 << 61) - 1
    a = T.cluster(g["off"], g["nbr"], None, p, 1, mode=T.NODEW_CUSTOM, k=k)
    b = O.cluster(g["off"], g["nbr"], None, p, 1, mode=O.NODEW_CUSTOM, k=k)
    assert np.array_equal(a[0], b[0]) and a[1:4] == b[1:4]
