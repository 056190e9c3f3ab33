"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Labels, desired clusters, coarse graphs and exact objectives are compared
element by element (bit-exact: every quantity is an integer).  Graph sizes
span several work tiles of every degree bucket, including rows above the
shared-memory limit (global-table hubs), with ragged tails.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_01731_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    torch.cuda.set_device(0)
    from paper_2108_01731_gb300 import lcc
    lcc.load()
    return lcc


def graphs():
    return {
        "sbm": I.to_numpy(I.sbm([60] * 30, 0.2, 0.01, seed=1)),
        "hubs": I.to_numpy(I.hub_graph(20000, 5, 3, 7000, seed=2)),
        "hubs_w": I.to_numpy(I.hub_graph(12000, 7, 2, 9000, seed=3, w_lo=-5, w_hi=9)),
        "cl": I.to_numpy(I.chung_lu(30000, 2.1, 12, seed=4)),
        "rmat": I.to_numpy(I.rmat(14, 120000, seed=5)),
        "signed": I.to_numpy(I.random_signed_graph(300, 0.1, -4, 6, seed=6)),
        "giant": I.to_numpy(I.hub_graph(150000, 5, 0,
                                        [1300, 1700, 2000, 3000, 5000, 12000, 25000, 50000,
                                         100000, 140000],
                                        seed=7, w_lo=1, w_hi=3)),
    }


GRAPHS = graphs()


def node_weights(g, mode, seed):
    if mode == O.NODEW_CUSTOM:
        return np.random.default_rng(seed).integers(0, 7, g["n"]).astype(np.int64)
    if mode == O.NODEW_UNIT:
        return np.ones(g["n"], np.int64)
    w = g["w"] if g["w"] is not None else np.ones(g["nnz"], np.int64)
    k = np.zeros(g["n"], np.int64)
    np.add.at(k, np.repeat(np.arange(g["n"]), np.diff(g["off"])), w.astype(np.int64))
    return k


def lam(mode, g, p, q):
    """(p, q) as the library takes them -> (p, q_eff) as the oracle's
    per-level functions take them (modularity: q * 2m)."""
    if mode == O.NODEW_DEGREE:
        return p, q * int(node_weights(g, mode, 0).sum())
    return p, q


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("mode", [O.NODEW_UNIT, O.NODEW_DEGREE, O.NODEW_CUSTOM])
def test_desired_matches_oracle(L, name, mode):
    g = GRAPHS[name]
    if mode == O.NODEW_DEGREE and g["w"] is not None and g["w"].min() < 0:
        pytest.skip("modularity needs non-negative degrees")
    n = g["n"]
    k = node_weights(g, mode, 11)
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k if mode == O.NODEW_CUSTOM else None)
    rng = np.random.default_rng(7)
    for trial, (p, q) in enumerate([(1, 50), (3, 7), (1 << 50, 7)]):
        if trial == 0:
            Lb = np.arange(n, dtype=np.int32)
        else:
            Lb = I.random_labels(n, max(2, n // (30 * trial)), seed=100 + trial).numpy()
        fr = (rng.random(n) < 0.7).astype(np.uint8) if trial == 1 else None
        got = L.lcc_desired(G, p, q, mode, Lb, fr)
        K = np.zeros(n, np.int64)
        np.add.at(K, Lb, k)
        pe, qe = lam(mode, g, p, q)
        want = O.desired(g["off"], g["nbr"], g["w"], k, pe, qe, Lb, K)
        if fr is not None:
            want = np.where(fr.astype(bool), want, Lb)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (name, mode, trial, bad[:10], got[bad[:10]], want[bad[:10]])
    G.free()


@pytest.mark.parametrize("vset", [O.VSET_ALL, O.VSET_NBR_VERTICES, O.VSET_NBR_CLUSTERS])
@pytest.mark.parametrize("name", ["sbm", "hubs", "rmat", "giant"])
def test_best_moves_rounds_match_oracle(L, name, vset):
    g = GRAPHS[name]
    n = g["n"]
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
    k = np.ones(n, np.int64)
    L0 = np.arange(n, dtype=np.int32)
    for r in (1, 2, 3, 6):
        got, moved, rounds = L.lcc_best_moves(G, 1, 40, O.NODEW_UNIT, r, vset, L0)
        want, wmoved, wrounds = O.best_moves(g["off"], g["nbr"], g["w"], k, 1, 40, L0, r,
                                            vset=vset)
        assert rounds == wrounds and moved == wmoved
        assert np.array_equal(got, want), (name, vset, r)
    G.free()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_compress_matches_oracle(L, name):
    g = GRAPHS[name]
    n = g["n"]
    k = node_weights(g, O.NODEW_CUSTOM, 3)
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k)
    for nc in (max(2, n // 50), max(2, n // 3)):
        Lb = I.random_labels(n, nc, seed=nc).numpy()
        mp, C = L.lcc_compress(G, O.NODEW_CUSTOM, Lb)
        off2, nbr2, w2, k2 = L.lcc_graph_export(C)
        wmp, woff, wnbr, ww, wk = O.compress(g["off"], g["nbr"], g["w"], k, Lb)
        assert np.array_equal(mp, wmp)
        assert np.array_equal(off2, woff)
        assert np.array_equal(nbr2, wnbr)
        assert np.array_equal(w2, ww)
        assert np.array_equal(k2, wk)
        C.free()
    G.free()


def test_compress_long_runs_of_equal_keys(L):
    """Compress sums parallel edges (Sec. 3.1): two 200-vertex cliques joined
    by a complete bipartite graph, labelled as the two cliques, give one run
    of 40,000 equal keys per direction, which crosses many warp chunks and
    sort tiles of the reduction; a chain of cliques gives uneven runs."""
    import torch
    a = torch.arange(200)
    pairs = [torch.combinations(a).T, torch.combinations(a + 200).T,
             torch.stack([a.repeat_interleave(200), (a + 200).repeat(200)])]
    # a chain of 12 cliques of 5..60 vertices, consecutive ones joined by one edge
    base = 400
    sizes = [5 + 5 * i for i in range(12)]
    starts = []
    for s_ in sizes:
        starts.append(base)
        pairs.append(torch.combinations(torch.arange(base, base + s_)).T)
        base += s_
    pairs.append(torch.tensor([[starts[i], starts[i + 1]] for i in range(11)]).T)
    e = torch.cat(pairs, 1)
    n = base
    g = I.to_numpy(I.pairs_to_csr(e[0], e[1], n,
                                  w=((e[0] * 2654435761 + e[1]) % 7 + 1).to(torch.int32)))
    w = g["w"]
    src = np.repeat(np.arange(n), np.diff(g["off"]))
    labels = np.zeros(n, np.int32)
    labels[200:400] = 200
    for st_, s_ in zip(starts, sizes):
        labels[st_:st_ + s_] = st_
    k = np.ones(n, np.int64)
    G = L.lcc_load_csr(g["off"], g["nbr"], w, node_w=k)
    mp, C = L.lcc_compress(G, O.NODEW_CUSTOM, labels)
    off2, nbr2, w2, k2 = L.lcc_graph_export(C)
    wmp, woff, wnbr, ww, wk = O.compress(g["off"], g["nbr"], w, k, labels)
    assert np.array_equal(mp, wmp) and np.array_equal(off2, woff)
    assert np.array_equal(nbr2, wnbr) and np.array_equal(w2, ww) and np.array_equal(k2, wk)
    assert off2[1] - off2[0] == 1 and w2[0] == int(w[(src < 200) & (g["nbr"] >= 200)].sum())
    C.free()
    G.free()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_objective_matches_oracle(L, name):
    g = GRAPHS[name]
    n = g["n"]
    k = node_weights(g, O.NODEW_CUSTOM, 5)
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k)
    for nc in (1, 7, n // 10, n):
        Lb = (np.arange(n, dtype=np.int32) if nc == n
              else I.random_labels(n, nc, seed=nc + 1).numpy())
        num, den = L.lcc_objective(G, 3, 11, O.NODEW_CUSTOM, Lb)
        assert den == 11
        assert num == O.objective_num(g["off"], g["nbr"], g["w"], k, 3, 11, Lb)
    G.free()


CLUSTER_CASES = [
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
    ("giant", O.NODEW_DEGREE, 1, 1, {}),
    ("giant", O.NODEW_UNIT, 1, 4, {"vset": O.VSET_ALL}),
]


@pytest.mark.parametrize("case", CLUSTER_CASES, ids=lambda c: "%s-%d-%d/%d-%s" % (
    c[0], c[1], c[2], c[3], "-".join("%s%s" % kv for kv in sorted(c[4].items()))))
def test_cluster_matches_oracle(L, case):
    check_cluster_case(L, case)


TRACE_CASES = [("sbm", O.NODEW_UNIT, 1, 50, O.VSET_NBR_VERTICES, False),
               ("hubs", O.NODEW_DEGREE, 1, 1, O.VSET_NBR_VERTICES, False),
               ("rmat", O.NODEW_DEGREE, 1, 1, O.VSET_NBR_CLUSTERS, False),
               ("cl", O.NODEW_DEGREE, 1, 1, O.VSET_ALL, False),
               ("signed", O.NODEW_UNIT, 1, 9, O.VSET_NBR_VERTICES, False),
               ("rmat", O.NODEW_DEGREE, 1, 1, O.VSET_NBR_VERTICES, True),
               ("hubs_w", O.NODEW_UNIT, 1, 9, O.VSET_NBR_CLUSTERS, True)]


@pytest.mark.parametrize("case", TRACE_CASES, ids=lambda c: "%s-%d-%s" % (c[0], c[4], c[5]))
def test_round_trace_matches_oracle(L, case):
    """Per-round |V'|, scanned entries, moves and held-back vertices (the
    paper's plot of |V'| per round) equal the oracle's record, round by round
    over the whole multi-level run; the pull rounds of the neighbour rule
    report the same V' as marking."""
    name, mode, p, q, vset, coin = case
    g = GRAPHS[name]
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
    sched = L.schedule(vset=vset, coin=coin, seed=3)
    labels, obj, st, rows = L.lcc_cluster_trace(G, p, q, mode, sched)
    wl, num, den, ws, wtr = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, vset=vset,
                                      coin=coin, seed=3, trace=True)
    assert np.array_equal(labels, wl) and st["obj_num"] == num
    assert np.array_equal(rows, wtr)
    assert rows[:, 4].sum() == st["edges_scanned"] and len(rows) == st["rounds_total"]
    G.free()


def test_gather_layout_matches_oracle(L, monkeypatch):
    """The degree-ordered storage of the packed label words (forced here on
    graphs far below the size that gets it by default) moves words only:
    labels, objective and every counter stay the oracle's."""
    monkeypatch.setenv("LCC_LAYOUT_MIN_BYTES", "0")
    for case in CLUSTER_CASES:
        check_cluster_case(L, case)
    g = GRAPHS["rmat"]
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
    k, two_m = O.weighted_degrees(g["off"], g["w"])
    L0 = np.arange(g["n"], dtype=np.int32)
    got, _, rounds = L.lcc_best_moves(G, 1, 1, L.LCC_NODEW_DEGREE, 4, 1, L0)
    want, _, wrounds = O.best_moves(g["off"], g["nbr"], g["w"], k, 1, two_m, L0, 4)
    assert rounds == wrounds and np.array_equal(got, want)
    G.free()


def test_tuning_routes_without_changing_results(L, tmp_path):
    """Every tuning -- the degree routing (rows of 33..warp_max entries in the
    warp kernels, longer rows up to 1024 in the block kernel) crossed with the
    small rows in one resident launch or in one launch per bucket -- gives
    the oracle's labels, objective and scanned entries, alone and in a batch;
    the autotuner picks one of them, and its cache file is read back on the
    next call."""
    before = L.lcc_get_tuning(0)
    try:
        for name, mode, p, q in [("hubs", O.NODEW_DEGREE, 1, 1), ("rmat", O.NODEW_DEGREE, 1, 1),
                                 ("signed", O.NODEW_UNIT, 1, 10)]:
            g = GRAPHS[name]
            G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
            wl, num, _, wst = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode)
            for fs, pf, pg in ((0, 0, 0), (1, 0, 1), (0, 1, 1), (1, 1, 0)):
                for wm in (32, 64, 128, 256):
                    L.lcc_set_tuning(0, wm, fs, pf, pg)
                    labels, _, st = L.lcc_cluster(G, p, q, mode, None)
                    assert np.array_equal(labels, wl), (name, wm, fs, pf, pg)
                    assert st["obj_num"] == num and st["edges_scanned"] == wst[2]
            G.free()
        graphs = [GRAPHS[x] for x in ("sbm", "rmat", "cl")]
        Gs = [L.lcc_load_csr(g["off"], g["nbr"], g["w"]) for g in graphs]
        for fs in (0, 1):
            L.lcc_set_tuning(0, 256, fs, fs, 1 - fs)
            labs, _ = L.lcc_cluster_batch(Gs, [1] * 3, [1] * 3, [O.NODEW_DEGREE] * 3)
            for g, lab in zip(graphs, labs):
                wl, *_ = O.cluster(g["off"], g["nbr"], g["w"], 1, 1, mode=O.NODEW_DEGREE)
                assert np.array_equal(lab, wl), fs
        for G in Gs:
            G.free()
        g = GRAPHS["rmat"]
        G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
        path = tmp_path / "tuning.txt"
        t = L.lcc_autotune(G, 1, 1, O.NODEW_DEGREE, str(path))
        assert t["warp_max"] in (32, 64, 128, 256) and t["fuse_small"] in (0, 1)
        assert t["prefetch"] in (0, 1) and t["pregather"] in (0, 1)
        assert t["part_min"] in (0, 1024, 4096, 8192, 16384)
        assert L.lcc_get_tuning(0) == t
        assert path.read_text().strip().endswith(
            " %d %d %d %d %d" % (t["warp_max"], t["fuse_small"], t["prefetch"], t["pregather"],
                                 t["part_min"]))
        L.lcc_set_tuning(0, 32 if t["warp_max"] != 32 else 256, 1 - t["fuse_small"],
                         1 - t["prefetch"], 1 - t["pregather"], 1024 if t["part_min"] != 1024 else 0)
        assert L.lcc_autotune(G, 1, 1, O.NODEW_DEGREE, str(path)) == t
        assert L.lcc_get_tuning(0) == t
        G.free()
        for bad in ((0, 1), (48, 1), (512, 1), (256, 2), (256, 1, 2), (256, 1, 0, 2),
                    (256, 1, 0, 1, 1), (256, 1, 0, 1, 2048)):
            with pytest.raises(L.LccError):
                L.lcc_set_tuning(0, *bad)
    finally:
        L.lcc_set_tuning(0, before["warp_max"], before["fuse_small"], before["prefetch"],
                         before["pregather"], before["part_min"])


def test_partitioned_long_rows_match_oracle(L, monkeypatch):
    """Rows longer than part_min entries split by cluster hash into parts of
    at most about 1024 entries, each merged in one block's shared memory, for
    every part_min from 1024 to 16384 and with the path off; the "giant" graph's hubs of 1,300 to
    140,000 draws, a signed-weight graph with rows of 8,000 to 32,000 entries
    and the hub and R-MAT graphs, alone and in a batch.  Then with the parts'
    tables cut to 64 slots, so that nearly every part overflows and its row
    takes the global-table fallback.  Labels, objective and scanned entries
    are the oracle's every time."""
    before = L.lcc_get_tuning(0)
    graphs = dict(GRAPHS)
    graphs["giant_w"] = I.to_numpy(I.hub_graph(60000, 6, 0, [9000, 20000, 30000, 45000],
                                               seed=8, w_lo=-5, w_hi=9))
    cases = [("giant", O.NODEW_DEGREE, 1, 1, {}),
             ("giant", O.NODEW_UNIT, 1, 40, {"vset": O.VSET_NBR_VERTICES}),
             ("giant_w", O.NODEW_CUSTOM, 2, 9, {"vset": O.VSET_NBR_CLUSTERS}),
             ("giant_w", O.NODEW_UNIT, 1, 8, {}),
             ("giant", O.NODEW_DEGREE, 1, 1, {"coin": True, "seed": 11}),
             ("hubs", O.NODEW_DEGREE, 1, 1, {}),
             ("rmat", O.NODEW_DEGREE, 1, 1, {"vset": O.VSET_ALL})]
    want = {}
    for i, (name, mode, p, q, kw) in enumerate(cases):
        g = graphs[name]
        k = node_weights(g, O.NODEW_CUSTOM, 9) if mode == O.NODEW_CUSTOM else None
        wl, num, _, wst = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, k=k, **kw)
        want[i] = (wl, num, wst[2])

    def run_all(tag):
        for i, (name, mode, p, q, kw) in enumerate(cases):
            g = graphs[name]
            k = node_weights(g, O.NODEW_CUSTOM, 9) if mode == O.NODEW_CUSTOM else None
            G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k)
            sched = L.schedule(**kw) if kw else None
            labels, _, st = L.lcc_cluster(G, p, q, mode, sched)
            G.free()
            wl, num, scanned = want[i]
            assert np.array_equal(labels, wl), (tag, name, mode, kw)
            assert st["obj_num"] == num and st["edges_scanned"] == scanned, (tag, name, mode, kw)
        batch = [graphs[x] for x in ("giant", "giant_w", "giant")]
        Gs = [L.lcc_load_csr(g["off"], g["nbr"], g["w"]) for g in batch]
        labs, _ = L.lcc_cluster_batch(Gs, [1, 1, 1], [1, 8, 1],
                                      [O.NODEW_DEGREE, O.NODEW_UNIT, O.NODEW_DEGREE])
        for G in Gs:
            G.free()
        assert np.array_equal(labs[0], want[0][0]) and np.array_equal(labs[2], want[0][0]), tag
        assert np.array_equal(labs[1], want[3][0]), tag

    try:
        for pm in (8192, 1024, 4096, 16384, 0):
            L.lcc_set_tuning(0, 256, 1, 0, 1, pm)
            run_all(pm)
        L.lcc_set_tuning(0, 256, 1, 0, 1, 1024)
        monkeypatch.setenv("LCC_PART_TABLE_SLOTS", "64")
        run_all("64 slots")
    finally:
        L.lcc_set_tuning(0, before["warp_max"], before["fuse_small"], before["prefetch"],
                         before["pregather"], before["part_min"])


def check_cluster_case(L, case):
    name, mode, p, q, kw = case
    g = GRAPHS[name]
    k = node_weights(g, O.NODEW_CUSTOM, 9) if mode == O.NODEW_CUSTOM else None
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k)
    sched = L.schedule(num_iter=kw.get("num_iter", 10), max_levels=kw.get("max_levels", 64),
                       refine=kw.get("refine", True), vset=kw.get("vset", 1))
    labels, obj, st = L.lcc_cluster(G, p, q, mode, sched)
    wl, num, den, wst = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, k=k,
                                  num_iter=kw.get("num_iter", 10),
                                  max_levels=kw.get("max_levels", 64),
                                  refine=kw.get("refine", True), vset=kw.get("vset", 1))
    assert np.array_equal(labels, wl)
    assert st["obj_num"] == num and st["obj_den"] == den
    assert abs(obj - num / den) <= 1e-12 * max(1.0, abs(num / den))
    assert st["levels"] == wst[0] and st["rounds_total"] == wst[1]
    assert st["edges_scanned"] == wst[2]
    assert st["num_clusters"] == len(np.unique(wl))
    G.free()


COIN_CASES = [
    ("sbm", O.NODEW_UNIT, 1, 50, {"num_iter": 20}),
    ("hubs", O.NODEW_DEGREE, 1, 1, {}),
    ("hubs_w", O.NODEW_CUSTOM, 2, 9, {"vset": O.VSET_NBR_CLUSTERS}),
    ("cl", O.NODEW_DEGREE, 1, 1, {}),
    ("rmat", O.NODEW_DEGREE, 1, 1, {}),
    ("signed", O.NODEW_UNIT, 1, 10, {"vset": O.VSET_ALL, "num_iter": 30}),
    ("giant", O.NODEW_DEGREE, 1, 1, {}),
]


@pytest.mark.parametrize("case", COIN_CASES, ids=lambda c: "%s-%d-%d/%d" % c[:4])
def test_coin_schedule_matches_oracle(L, case):
    """LCC_SCHED_COIN: the same held-back vertices in every round as the
    oracle (labels, objective, levels, rounds and scanned entries), for
    several seeds, through every degree bucket and V' rule."""
    name, mode, p, q, kw = case
    g = GRAPHS[name]
    k = node_weights(g, O.NODEW_CUSTOM, 9) if mode == O.NODEW_CUSTOM else None
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k)
    ni, vset = kw.get("num_iter", 10), kw.get("vset", O.VSET_NBR_VERTICES)
    for seed in (0, 977, (1 << 64) - 5):
        sched = L.schedule(num_iter=ni, vset=vset, coin=True, seed=seed)
        labels, obj, st = L.lcc_cluster(G, p, q, mode, sched)
        wl, num, den, wst = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, k=k,
                                      num_iter=ni, vset=vset, coin=True, seed=seed)
        assert np.array_equal(labels, wl), (name, seed)
        assert st["obj_num"] == num and st["obj_den"] == den
        assert (st["levels"], st["rounds_total"], st["edges_scanned"]) == wst
    G.free()


def test_coin_batch_equals_single(L):
    """Jobs of one batch draw their own coins (keys by vertex, round, depth
    and phase of each job): the batch gives every graph its single-run result."""
    names = ["sbm", "hubs", "cl", "rmat"]
    modes = [O.NODEW_UNIT, O.NODEW_DEGREE, O.NODEW_DEGREE, O.NODEW_DEGREE]
    ps, qs = [1, 1, 1, 1], [50, 1, 1, 1]
    sched = L.schedule(num_iter=15, coin=True, seed=31)
    Gs = [L.lcc_load_csr(GRAPHS[n]["off"], GRAPHS[n]["nbr"], GRAPHS[n]["w"]) for n in names]
    outs, objs = L.lcc_cluster_batch(Gs, ps, qs, modes, sched)
    for i, G in enumerate(Gs):
        lab, obj, _ = L.lcc_cluster(G, ps[i], qs[i], modes[i], sched)
        assert np.array_equal(outs[i], lab), names[i]
        assert objs[i] == obj
        g = GRAPHS[names[i]]
        wl = O.cluster(g["off"], g["nbr"], g["w"], ps[i], qs[i], mode=modes[i], num_iter=15,
                       coin=True, seed=31)[0]
        assert np.array_equal(lab, wl), names[i]
    for G in Gs:
        G.free()


def test_pull_and_mark_frontiers_agree(L):
    """V' = neighbours of the movers (Sec. 3.2.2), found by marking them or by
    evaluating every vertex with an edge and keeping the labels of those with
    no moved neighbour: same labels, rounds and scanned entries as the oracle
    either way, and the second way does run (it processes more entries)."""
    extra = 0
    for name, mode, p, q, kw in CLUSTER_CASES:
        if kw.get("vset", 1) != O.VSET_NBR_VERTICES:
            continue
        g = GRAPHS[name]
        k = node_weights(g, O.NODEW_CUSTOM, 9) if mode == O.NODEW_CUSTOM else None
        G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k)
        wl, num, den, wst = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=mode, k=k,
                                      num_iter=kw.get("num_iter", 10),
                                      max_levels=kw.get("max_levels", 64),
                                      refine=kw.get("refine", True))
        for mark_only in (True, False):
            sched = L.schedule(num_iter=kw.get("num_iter", 10),
                               max_levels=kw.get("max_levels", 64),
                               refine=kw.get("refine", True), mark_only=mark_only)
            labels, _, st = L.lcc_cluster(G, p, q, mode, sched)
            assert np.array_equal(labels, wl), (name, mark_only)
            assert st["obj_num"] == num and st["rounds_total"] == wst[1]
            assert st["edges_scanned"] == wst[2], (name, mark_only)
            processed = sum(st["bucket_entries"])
            if mark_only:
                assert processed == st["edges_scanned"]
            else:
                assert processed >= st["edges_scanned"]
                extra += processed - st["edges_scanned"]
        G.free()
    assert extra > 0


def test_device_labels_and_device_csr(L):
    import torch
    g = GRAPHS["hubs"]
    dev = {k: torch.from_numpy(g[k]).cuda() for k in ("off", "nbr")}
    G = L.lcc_load_csr(dev["off"], dev["nbr"])
    out = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    L.lcc_cluster(G, 1, 1, O.NODEW_DEGREE, None, labels_out=out)
    wl, *_ = O.cluster(g["off"], g["nbr"], None, 1, 1, mode=O.NODEW_DEGREE)
    assert np.array_equal(out.cpu().numpy(), wl)
    G.free()


# ------------------------------------------------------------ edge cases --

def csr(n, edges):
    import torch
    if not edges:
        return {"off": np.zeros(n + 1, np.int64), "nbr": np.zeros(0, np.int32), "w": None,
                "n": n, "nnz": 0}
    a = torch.tensor([min(e) for e in edges])
    b = torch.tensor([max(e) for e in edges])
    return I.to_numpy(I.pairs_to_csr(a, b, n))


@pytest.mark.parametrize("n,edges", [
    (0, []), (1, []), (5, []), (2, [(0, 1)]), (3, [(0, 1), (1, 2)]),
    (7, [(0, 1), (1, 2), (0, 2), (4, 5)]),
])
def test_degenerate_graphs(L, n, edges):
    g = csr(n, edges)
    G = L.lcc_load_csr(g["off"], g["nbr"])
    for p, q, mode in [(1, 3, O.NODEW_UNIT), (1, 1, O.NODEW_DEGREE)]:
        if mode == O.NODEW_DEGREE and not edges:
            with pytest.raises(L.LccError):
                L.lcc_cluster(G, p, q, mode)
            continue
        labels, obj, st = L.lcc_cluster(G, p, q, mode)
        if n == 0:
            assert len(labels) == 0
            continue
        wl, num, den, _ = O.cluster(g["off"], g["nbr"], None, p, q, mode=mode)
        assert np.array_equal(labels, wl) and st["obj_num"] == num
    G.free()


def test_isolated_edge_oscillation_and_cliques_closed_form(L):
    g = csr(2, [(0, 1)])
    G = L.lcc_load_csr(g["off"], g["nbr"])
    labels, obj, st = L.lcc_cluster(G, 1, 3, O.NODEW_UNIT, L.schedule(num_iter=7))
    assert list(labels) == [0, 1] and st["obj_num"] == 0 and st["rounds_total"] == 7
    G.free()
    r, s, p, q = 40, 6, 1, 3
    perm = np.random.default_rng(0).permutation(r * s)
    edges = [(perm[c * s + i], perm[c * s + j]) for c in range(r) for i in range(s)
             for j in range(i + 1, s)]
    g = csr(r * s, edges)
    G = L.lcc_load_csr(g["off"], g["nbr"])
    labels, obj, st = L.lcc_cluster(G, p, q, O.NODEW_UNIT)
    for c in range(r):
        mem = sorted(perm[c * s:(c + 1) * s])
        assert all(labels[v] == mem[0] for v in mem)
    assert st["obj_num"] == r * s * (s - 1) * (q - p)
    G.free()


def test_input_validation(L):
    g = csr(4, [(0, 1), (1, 2), (2, 3)])
    off, nbr = g["off"], g["nbr"]
    bad = nbr.copy()
    bad[0] = 7
    with pytest.raises(L.LccError) as e:
        L.lcc_load_csr(off, bad)
    assert e.value.status == L.LCC_ERR_INVALID
    bad = nbr.copy()
    bad[0] = 0  # vertex 0 -> 0
    with pytest.raises(L.LccError) as e:
        L.lcc_load_csr(off, bad)
    assert e.value.status in (L.LCC_ERR_SELF_LOOP, L.LCC_ERR_NOT_SYMMETRIC)
    w = np.ones(len(nbr), np.int32)
    w[0] = 2
    with pytest.raises(L.LccError) as e:
        L.lcc_load_csr(off, nbr, w)
    assert e.value.status == L.LCC_ERR_NOT_SYMMETRIC
    off2 = off.copy()
    off2[2] = off2[3] + 1
    with pytest.raises(L.LccError) as e:
        L.lcc_load_csr(off2, nbr)
    assert e.value.status == L.LCC_ERR_INVALID
    G = L.lcc_load_csr(off, nbr)
    with pytest.raises(L.LccError):
        L.lcc_cluster(G, 0, 1)
    with pytest.raises(L.LccError):
        L.lcc_desired(G, 1, 2, 0, np.array([0, 1, 2, 9], np.int32))
    G.free()


def test_exact_range_guard(L):
    """The 128-bit gains stay exact only while q * sum|w| and p * (sum k)^2
    are below 2^125; past that the library refuses with LCC_ERR_OVERFLOW
    instead of returning wrapped scores, exactly where the oracle refuses.

    Custom node weights: one vertex of weight 2^40 and the rest of weight 1,
    q = 2^62.  The largest accepted p has p * (sum k)^2 just below 2^125, and
    the unit-weight vertices still merge (lambda = p / q is about 2^-17), so
    the accepted run moves vertices with gains near 2^66 and is compared
    with the oracle; p + 1 is refused by both.  In modularity mode, int32
    weights near 2^31 and a resolution numerator at the limit do the same."""
    g = GRAPHS["signed"]
    n = g["n"]
    k = np.ones(n, np.int64)
    k[n // 2] = 1 << 40
    kt = int(k.sum())
    q = 1 << 62
    pmax = ((1 << 125) - 1) // (kt * kt)
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k)
    Lb = np.arange(n, dtype=np.int32)
    for fn in (lambda p: L.lcc_cluster(G, p, q, O.NODEW_CUSTOM),
               lambda p: L.lcc_desired(G, p, q, O.NODEW_CUSTOM, Lb),
               lambda p: L.lcc_objective(G, p, q, O.NODEW_CUSTOM, Lb)):
        with pytest.raises(L.LccError) as e:
            fn(pmax + 1)
        assert e.value.status == L.LCC_ERR_OVERFLOW
    with pytest.raises(OverflowError):
        O.cluster(g["off"], g["nbr"], g["w"], pmax + 1, q, mode=O.NODEW_CUSTOM, k=k)
    labels, obj, st = L.lcc_cluster(G, pmax, q, O.NODEW_CUSTOM)
    wl, num, den, ws = O.cluster(g["off"], g["nbr"], g["w"], pmax, q, mode=O.NODEW_CUSTOM, k=k)
    assert np.array_equal(labels, wl) and st["obj_num"] == num and st["obj_den"] == den
    assert (st["levels"], st["rounds_total"], st["edges_scanned"]) == ws
    assert len(np.unique(labels)) < n // 2  # the unit-weight vertices merged
    G.free()
    # modularity mode: heavy int32 weights, gamma = p / 1 at the limit
    rng = np.random.default_rng(5)
    h = GRAPHS["hubs_w"]
    off, nbr = h["off"], h["nbr"]
    src = np.repeat(np.arange(h["n"]), np.diff(off))
    a, b = np.minimum(src, nbr), np.maximum(src, nbr)
    # one weight per undirected edge, the same in both directions
    key = a.astype(np.int64) * h["n"] + b
    uniq, inv = np.unique(key, return_inverse=True)
    w = rng.integers(1 << 29, (1 << 31) - 1, len(uniq)).astype(np.int64)[inv].astype(np.int32)
    two_m = int(w.astype(np.int64).sum())
    pmax = ((1 << 125) - 1) // (two_m * two_m)
    assert 1 < pmax < (1 << 62)
    G = L.lcc_load_csr(off, nbr, w)
    with pytest.raises(L.LccError) as e:
        L.lcc_cluster(G, pmax + 1, 1, O.NODEW_DEGREE)
    assert e.value.status == L.LCC_ERR_OVERFLOW
    with pytest.raises(OverflowError):
        O.cluster(off, nbr, w, pmax + 1, 1, mode=O.NODEW_DEGREE)
    labels, obj, st = L.lcc_cluster(G, pmax, 1, O.NODEW_DEGREE, L.schedule(num_iter=4))
    wl, num, den, ws = O.cluster(off, nbr, w, pmax, 1, mode=O.NODEW_DEGREE, num_iter=4)
    assert np.array_equal(labels, wl) and st["obj_num"] == num and st["obj_den"] == den
    assert (st["levels"], st["rounds_total"], st["edges_scanned"]) == ws
    G.free()


# --------------------------------------------------- batching and serving --

@pytest.mark.parametrize("force_layout", [False, True])
def test_batch_equals_single(L, monkeypatch, force_layout):
    """A batch gives every graph its single-run labels and objective.  The
    coarse levels of a batch share one entry array, so every job but the
    first indexes it from a nonzero offset; forcing the degree-ordered
    layout (taken by the levels whose entries start at 0) mixes levels with
    and without it in one contraction."""
    if force_layout:
        monkeypatch.setenv("LCC_LAYOUT_MIN_BYTES", "0")
    names = ["sbm", "hubs", "cl", "rmat", "signed", "hubs_w"]
    modes = [O.NODEW_UNIT, O.NODEW_DEGREE, O.NODEW_DEGREE, O.NODEW_DEGREE, O.NODEW_UNIT,
             O.NODEW_UNIT]
    ps = [1, 1, 1, 1, 1, 1]
    qs = [50, 1, 1, 1, 10, 8]
    Gs = [L.lcc_load_csr(GRAPHS[n]["off"], GRAPHS[n]["nbr"], GRAPHS[n]["w"]) for n in names]
    outs, objs = L.lcc_cluster_batch(Gs, ps, qs, modes)
    for i, G in enumerate(Gs):
        lab, obj, _ = L.lcc_cluster(G, ps[i], qs[i], modes[i])
        assert np.array_equal(outs[i], lab), names[i]
        assert objs[i] == obj
    for G in Gs:
        G.free()


def test_server_results_match_single_runs(L):
    import time
    graphs = [I.to_numpy(I.serving_graph(i)) for i in range(12)]
    srv = L.Server(hbm_budget_bytes=8 << 30, max_slots=5)
    tickets = []
    for i, g in enumerate(graphs):
        tickets.append(srv.submit(g["off"], g["nbr"], None, 1, 1, O.NODEW_DEGREE))
        if i % 3 == 2:
            time.sleep(0.01)  # later jobs arrive while earlier ones run
    srv.wait_idle(600000)
    for t, g in zip(tickets, graphs):
        res = srv.poll(t)
        assert res is not None
        labels, obj, lat = res
        wl, num, den, _ = O.cluster(g["off"], g["nbr"], None, 1, 1, mode=O.NODEW_DEGREE)
        assert np.array_equal(labels, wl)
        assert abs(obj - num / den) <= 1e-12 * max(1.0, abs(num / den))
        assert lat > 0
    c = srv.counters()
    assert c["done"] == len(graphs) and c["peak_jobs"] <= 5
    srv.close()


def test_server_isolates_failing_jobs(L):
    """Bad jobs mixed into a stream fail alone: an asymmetric CSR and a CSR
    with a self loop are refused when admitted, and a job whose fault
    injection raises an error inside an engine tick fails with that error;
    every other job of the stream, including those that ran in the same
    ticks, returns the oracle's labels."""
    import time
    good = [I.to_numpy(I.serving_graph(i)) for i in range(20, 29)]
    asym = dict(good[0])
    asym["nbr"] = good[0]["nbr"].copy()
    r0 = slice(asym["off"][0], asym["off"][1])
    asym["nbr"][r0] = (asym["nbr"][r0] + 1) % asym["n"]  # row 0 points elsewhere
    asym["nbr"][r0] = np.where(asym["nbr"][r0] == 0, 1, asym["nbr"][r0])
    loop = dict(good[1])
    loop["nbr"] = good[1]["nbr"].copy()
    loop["nbr"][loop["off"][3]] = 3
    srv = L.Server(hbm_budget_bytes=8 << 30, max_slots=6)
    tickets, kinds = [], []
    for i, g in enumerate(good):
        if i == 2:
            tickets.append(srv.submit(asym["off"], asym["nbr"], None, 1, 1, O.NODEW_DEGREE))
            kinds.append(("bad", (L.LCC_ERR_NOT_SYMMETRIC, L.LCC_ERR_INVALID)))
        if i == 4:
            tickets.append(srv.submit(loop["off"], loop["nbr"], None, 1, 1, O.NODEW_DEGREE))
            kinds.append(("bad", (L.LCC_ERR_SELF_LOOP, L.LCC_ERR_NOT_SYMMETRIC)))
        fault = 3 if i == 5 else 0
        tickets.append(srv.submit(g["off"], g["nbr"], None, 1, 1, O.NODEW_DEGREE,
                                  inject_fault_tick=fault))
        kinds.append(("fault", (L.LCC_ERR_CUDA,)) if fault else ("good", g))
        if i % 3 == 2:
            time.sleep(0.005)
    srv.wait_idle(600000)
    for t, (kind, x) in zip(tickets, kinds):
        if kind == "good":
            labels, obj, lat = srv.poll(t)
            wl, num, den, _ = O.cluster(x["off"], x["nbr"], None, 1, 1, mode=O.NODEW_DEGREE)
            assert np.array_equal(labels, wl)
        else:
            with pytest.raises(L.LccError) as e:
                srv.poll(t)
            assert e.value.status in x, (kind, e.value)
            if kind == "fault":
                assert "injected fault" in str(e.value)
    assert srv.counters()["done"] == len(tickets)
    srv.close()


def test_server_rejects_oversize_and_cancels(L):
    g = GRAPHS["sbm"]
    srv = L.Server(hbm_budget_bytes=1 << 20, max_slots=2)
    with pytest.raises(L.LccError) as e:
        srv.submit(g["off"], g["nbr"], None, 1, 50, O.NODEW_UNIT)
    assert e.value.status == L.LCC_ERR_OOM
    srv.close()
    srv = L.Server(hbm_budget_bytes=4 << 30, max_slots=1)
    t1 = srv.submit(g["off"], g["nbr"], None, 1, 50, O.NODEW_UNIT)
    t2 = srv.submit(g["off"], g["nbr"], None, 1, 50, O.NODEW_UNIT)
    srv.cancel(t2)
    srv.wait_idle(600000)
    assert srv.poll(t1) is not None
    with pytest.raises(L.LccError) as e:
        srv.poll(t2)
    assert e.value.status == L.LCC_ERR_CANCELLED
    srv.close()


def test_hub_tables_in_many_windows(L, monkeypatch):
    """Hub hash tables processed in small windows (many passes per round),
    and the tables of long coarse rows in Compress likewise, give the same
    desired clusters, the same coarse graph and the same clustering."""
    monkeypatch.setenv("LCC_HUB_WINDOW_SLOTS", "4096")
    monkeypatch.setenv("LCC_ROW_WINDOW_SLOTS", "4096")
    g = GRAPHS["giant"]
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
    k = np.ones(g["n"], np.int64)
    Lb = I.random_labels(g["n"], g["n"] // 3, seed=78).numpy()
    mp, C = L.lcc_compress(G, O.NODEW_UNIT, Lb)
    got = L.lcc_graph_export(C)
    want = O.compress(g["off"], g["nbr"], g["w"], k, Lb)
    assert np.array_equal(mp, want[0])
    for a, b in zip(got, want[1:]):
        assert np.array_equal(a, b)
    C.free()
    G.free()
    g = GRAPHS["hubs_w"]
    n = g["n"]
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
    Lb = I.random_labels(n, n // 40, seed=77).numpy()
    K = np.zeros(n, np.int64)
    np.add.at(K, Lb, 1)
    got = L.lcc_desired(G, 1, 9, O.NODEW_UNIT, Lb)
    want = O.desired(g["off"], g["nbr"], g["w"], np.ones(n, np.int64), 1, 9, Lb, K)
    assert np.array_equal(got, want)
    labels, obj, st = L.lcc_cluster(G, 1, 9, O.NODEW_UNIT)
    wl, num, den, _ = O.cluster(g["off"], g["nbr"], g["w"], 1, 9)
    assert np.array_equal(labels, wl) and st["obj_num"] == num
    G.free()
