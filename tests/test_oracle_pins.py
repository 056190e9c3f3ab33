"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these tests re-derives the oracle's own formulas: the objective is
checked against the ordered-pair definition evaluated pair by pair, against
networkx's modularity, and against closed forms; the best-move rule is checked
by brute force (move the vertex, re-evaluate the definition); Compress by the
contraction identity and by a dictionary rebuild; whole runs by closed forms
on disjoint cliques and the oscillating edge.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2108_01731_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers --

def dense(g):
    n = g["n"]
    W = np.zeros((n, n), dtype=object)
    E = np.zeros((n, n), dtype=bool)
    off, nbr = g["off"], g["nbr"]
    w = g["w"] if g["w"] is not None else np.ones(len(nbr), np.int64)
    for u in range(n):
        for e in range(off[u], off[u + 1]):
            W[u, nbr[e]] += int(w[e])
            E[u, nbr[e]] = True
    return W, E


def cc_definition(W, E, k, lam, labels):
    """CC(x) = sum over ordered (i, j) in V x V of w'_ij (1 - x_ij), Sec. 2."""
    n = len(labels)
    tot = Fraction(0)
    for i in range(n):
        for j in range(n):
            if i == j or labels[i] != labels[j]:
                continue
            wp = -lam * int(k[i]) * int(k[j])
            if E[i, j]:
                wp += W[i, j]
            tot += wp
    return tot


def small_graph(seed, n=7, p=0.5, lo=-3, hi=5):
    return I.to_numpy(I.random_signed_graph(n, p, lo, hi, seed))


def brute_desired(g, W, E, k, p, q, L, v):
    """Desired cluster of v by brute force: try every candidate target
    (neighbouring clusters, and the empty cluster v when it is empty), score
    each by re-evaluating the objective definition, keep the best (ties to
    the smallest id) and move only if strictly better than staying."""
    lam = Fraction(p, q)
    off, nbr = g["off"], g["nbr"]
    cands = set(int(L[u]) for u in nbr[off[v]:off[v + 1]])
    cands.discard(int(L[v]))
    K = {}
    for x in range(g["n"]):
        K[int(L[x])] = K.get(int(L[x]), 0) + int(k[x])
    if int(L[v]) != v and K.get(v, 0) == 0:
        cands.add(v)
    base = cc_definition(W, E, k, lam, L)
    best, best_c = None, None
    for c in sorted(cands):
        L2 = L.copy()
        L2[v] = c
        val = cc_definition(W, E, k, lam, L2)
        if best is None or val > best:
            best, best_c = val, c
    if best is not None and best > base:
        return best_c
    return int(L[v])


def set_partitions(n):
    """All set partitions of range(n) as restricted growth strings."""
    def rec(i, a, m):
        if i == n:
            yield list(a)
            return
        for c in range(m + 1):
            a.append(c)
            yield from rec(i + 1, a, max(m, c + 1))
            a.pop()
    yield from rec(0, [], 0)


# ------------------------------------------------------------- objective --

@pytest.mark.parametrize("seed", range(6))
def test_objective_matches_ordered_pair_definition(seed):
    g = small_graph(seed)
    W, E = dense(g)
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 4, g["n"])
    for p, q in [(1, 3), (2, 5), (7, 2)]:
        for trial in range(4):
            L = rng.integers(0, g["n"], g["n"]).astype(np.int32)
            want = cc_definition(W, E, k, Fraction(p, q), L) * q
            assert want.denominator == 1
            got = O.objective_num(g["off"], g["nbr"], g["w"], k, p, q, L)
            got_lit = O.objective_num(g["off"], g["nbr"], g["w"], k, p, q, L,
                                      literal=True)
            assert got == want.numerator
            assert got_lit == want.numerator


def test_objective_singletons_is_zero_and_one_cluster_closed_form():
    g = I.to_numpy(I.random_signed_graph(30, 0.3, -4, 9, 11))
    n = g["n"]
    k = np.arange(n) % 5
    assert O.objective_num(g["off"], g["nbr"], g["w"], k, 3, 7,
                           np.arange(n, dtype=np.int32)) == 0
    # everything in one cluster: q * sum_{ordered edges} w - p ((sum k)^2 - sum k^2)
    S = int(np.sum(g["w"].astype(np.int64)))
    want = 7 * S - 3 * (int(k.sum()) ** 2 - int((k.astype(np.int64) ** 2).sum()))
    assert O.objective_num(g["off"], g["nbr"], g["w"], k, 3, 7,
                           np.zeros(n, np.int32)) == want


def test_modularity_mode_matches_networkx():
    """Sec. 2: with k_v = d_v and lambda = gamma / 2m, CC / 2m is the
    modularity of Reichardt-Bornholdt without the i = j terms; networkx
    includes them, so Q_paper = Q_nx + gamma * sum_i d_i^2 / (2m)^2."""
    nx = pytest.importorskip("networkx")
    G = nx.karate_club_graph()
    n = G.number_of_nodes()
    rows = [[] for _ in range(n)]
    for a, b in G.edges():
        rows[a].append(b)
        rows[b].append(a)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    nbr = np.array([x for r in rows for x in sorted(r)], np.int32)
    labels, num, den, _ = O.cluster(off, nbr, None, 1, 1, mode=O.NODEW_DEGREE)
    two_m = 2 * G.number_of_edges()
    assert den == two_m
    comms = {}
    for v, c in enumerate(labels):
        comms.setdefault(int(c), set()).add(v)
    q_nx = nx.community.modularity(G, list(comms.values()), weight=None, resolution=1.0)
    deg = np.diff(off)
    q_paper = num / den / two_m
    assert abs(q_paper - (q_nx + float((deg ** 2).sum()) / two_m ** 2)) < 1e-12
    # and for arbitrary labels, with a resolution gamma = 3/4
    rng = np.random.default_rng(0)
    for _ in range(5):
        L = rng.integers(0, 5, n).astype(np.int32)
        cs = {}
        for v, c in enumerate(L):
            cs.setdefault(int(c), set()).add(v)
        qn = nx.community.modularity(G, list(cs.values()), weight=None, resolution=0.75)
        num = O.objective_num(off, nbr, None, deg, 3, 4 * two_m, L)
        qp = Fraction(num, 4 * two_m) / two_m
        assert abs(float(qp) - (qn + 0.75 * float((deg ** 2).sum()) / two_m ** 2)) < 1e-12


# ------------------------------------------------------------- best move --

@pytest.mark.parametrize("seed", range(8))
def test_desired_cluster_by_brute_force(seed):
    """Appendix A gain, the stay term, ties and the empty-cluster move, all
    against re-evaluation of the objective definition."""
    g = small_graph(100 + seed, n=7, p=0.55)
    W, E = dense(g)
    rng = np.random.default_rng(seed)
    n = g["n"]
    for p, q in [(1, 2), (1, 5), (3, 1)]:
        for trial in range(5):
            k = rng.integers(0, 3, n)
            L = rng.integers(0, n, n).astype(np.int32)
            if trial == 0:
                L = np.arange(n, dtype=np.int32)
            K = np.zeros(n, np.int64)
            np.add.at(K, L, k)
            D = O.desired(g["off"], g["nbr"], g["w"], k, p, q, L, K)
            for v in range(n):
                assert D[v] == brute_desired(g, W, E, k, p, q, L, v), (v, L, k)


def test_sync_round_is_simultaneous_application_of_brute_force_moves():
    g = small_graph(7, n=8, p=0.5)
    W, E = dense(g)
    n = g["n"]
    k = np.ones(n, np.int64)
    L0 = np.arange(n, dtype=np.int32)
    for p, q in [(1, 4), (1, 2)]:
        want = np.array([brute_desired(g, W, E, k, p, q, L0, v) for v in range(n)],
                        np.int32)
        L1, moved, rounds = O.best_moves(g["off"], g["nbr"], g["w"], k, p, q, L0, 1)
        assert rounds == 1
        assert np.array_equal(L1, want)


@pytest.mark.parametrize("vset", [O.VSET_ALL, O.VSET_NBR_VERTICES, O.VSET_NBR_CLUSTERS])
def test_best_moves_rounds_and_vertex_subsets(vset):
    """Algorithm 1's loop: V' = V, then the Sec. 3.2.2 subset after each
    round; stop when a round makes no move."""
    for seed in range(3):
        g = small_graph(40 + seed, n=8, p=0.45, lo=-1, hi=4)
        W, E = dense(g)
        n = g["n"]
        k = np.ones(n, np.int64)
        p, q = 1, 3
        L = np.arange(n, dtype=np.int32)
        vp = np.ones(n, bool)
        off, nbr = g["off"], g["nbr"]
        sims = [L.copy()]
        for _ in range(4):
            D = L.copy()
            for v in range(n):
                if vp[v]:
                    D[v] = brute_desired(g, W, E, k, p, q, L, v)
            moved = D != L
            if not moved.any():
                break
            left = set(int(x) for x in L[moved])
            L = D
            nxt = np.zeros(n, bool)
            if vset == O.VSET_ALL:
                nxt[:] = True
            elif vset == O.VSET_NBR_VERTICES:
                for v in np.nonzero(moved)[0]:
                    nxt[nbr[off[v]:off[v + 1]]] = True
            else:
                for x in range(n):
                    if int(L[x]) in left:
                        nxt[nbr[off[x]:off[x + 1]]] = True
            vp = nxt
            sims.append(L.copy())
        for r in range(1, len(sims)):
            Lr, _, _ = O.best_moves(off, nbr, g["w"], k, p, q,
                                    np.arange(n, dtype=np.int32), r, vset=vset)
            assert np.array_equal(Lr, sims[r]), (seed, r)


def test_sequential_moves_strictly_raise_objective():
    """Algorithm 2's inner loop: a single best move never lowers CC."""
    for seed in range(4):
        g = I.to_numpy(I.random_signed_graph(25, 0.25, -2, 6, 200 + seed))
        n = g["n"]
        k = (np.arange(n) % 3).astype(np.int64)
        p, q = 1, 6
        L = np.arange(n, dtype=np.int32)
        prev = O.objective_num(g["off"], g["nbr"], g["w"], k, p, q, L)
        steps = 0
        while steps < 200:
            L2, mv = O.sequential_sweep(g["off"], g["nbr"], g["w"], k, p, q, L, 1)
            if mv == 0:
                break
            cur = O.objective_num(g["off"], g["nbr"], g["w"], k, p, q, L2)
            assert cur > prev
            prev, L = cur, L2
            steps += 1
        assert steps > 0


def test_figure1_concurrent_moves_lower_objective():
    """Sec. 3.1, Figure 1 (weights are this project's reading; the caption's
    numbers are the paper's)."""
    fx = json.load(open(os.path.join(GOLDEN, "fig1_reading.json")))
    n = 3
    rows = [[] for _ in range(n)]
    for a, b, w in fx["edges"]:
        rows[a].append((b, w))
        rows[b].append((a, w))
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    nbr = np.array([x for r in rows for x, _ in sorted(r)], np.int32)
    w = np.array([y for r in rows for _, y in sorted(r)], np.int64)
    k = np.ones(n, np.int64)
    p, q = fx["lambda_p"], fx["lambda_q"]
    L = np.arange(n, dtype=np.int32)
    assert O.objective_num(off, nbr, w, k, p, q, L) == 2 * fx["objective_before_unordered"]
    K = np.ones(n, np.int64)
    D = O.desired(off, nbr, w, k, p, q, L, K)
    # b and c each choose the cluster {a}; a is not scheduled in the caption
    assert D[1] == 0 and D[2] == 0
    L2 = L.copy()
    L2[1], L2[2] = D[1], D[2]
    got = O.objective_num(off, nbr, w, k, p, q, L2)
    assert got == 2 * fx["objective_after_unordered"] * q


# -------------------------------------------------------------- compress --

def test_compress_dictionary_rebuild_and_node_weights():
    for seed in range(5):
        g = I.to_numpy(I.random_signed_graph(40, 0.15, -3, 7, 300 + seed))
        n = g["n"]
        rng = np.random.default_rng(seed)
        L = rng.integers(0, n, n).astype(np.int32)
        k = rng.integers(0, 5, n).astype(np.int64)
        mp, off2, nbr2, w2, k2 = O.compress(g["off"], g["nbr"], g["w"], k, L)
        occ = sorted(set(int(x) for x in L))
        rank = {c: i for i, c in enumerate(occ)}
        assert np.array_equal(mp, np.array([rank[int(x)] for x in L], np.int32))
        want = {}
        for u in range(n):
            for e in range(g["off"][u], g["off"][u + 1]):
                a, b = rank[int(L[u])], rank[int(L[g["nbr"][e]])]
                if a != b:
                    want[(a, b)] = want.get((a, b), 0) + int(g["w"][e])
        got = {}
        for a in range(len(occ)):
            row = nbr2[off2[a]:off2[a + 1]]
            assert np.all(np.diff(row) > 0)
            for e in range(off2[a], off2[a + 1]):
                got[(a, int(nbr2[e]))] = int(w2[e])
        assert got == want
        kw = np.zeros(len(occ), np.int64)
        np.add.at(kw, mp, k)
        assert np.array_equal(k2, kw)


def test_contraction_preserves_objective():
    """CC_G(flatten(C')) = CC_G'(C') + CC_G(C): Compress keeps every
    inter-cluster pair's weight and k' = K, so the objective splits exactly."""
    for seed in range(6):
        g = I.to_numpy(I.random_signed_graph(30, 0.2, -3, 6, 400 + seed))
        n = g["n"]
        rng = np.random.default_rng(seed)
        L = rng.integers(0, 10, n).astype(np.int32)
        k = rng.integers(0, 4, n).astype(np.int64)
        p, q = 2, 9
        mp, off2, nbr2, w2, k2 = O.compress(g["off"], g["nbr"], g["w"], k, L)
        n2 = len(k2)
        L2 = rng.integers(0, n2, n2).astype(np.int32)
        flat = L2[mp]
        lhs = O.objective_num(g["off"], g["nbr"], g["w"], k, p, q, flat)
        rhs = (O.objective_num(off2, nbr2, w2, k2, p, q, L2)
               + O.objective_num(g["off"], g["nbr"], g["w"], k, p, q, L))
        assert lhs == rhs


# ------------------------------------------------------------ whole runs --

def cliques(r, s, seed):
    n = r * s
    perm = np.random.default_rng(seed).permutation(n)
    a, b = [], []
    for c in range(r):
        for i in range(s):
            for j in range(i + 1, s):
                a.append(perm[c * s + i])
                b.append(perm[c * s + j])
    import torch
    a = torch.tensor(a, dtype=torch.int64)
    b = torch.tensor(b, dtype=torch.int64)
    g = I.to_numpy(I.pairs_to_csr(torch.minimum(a, b), torch.maximum(a, b), n))
    members = [sorted(perm[c * s:(c + 1) * s]) for c in range(r)]
    return g, members


@pytest.mark.parametrize("r,s,p,q", [(5, 3, 1, 2), (4, 5, 1, 3), (3, 8, 2, 3), (6, 4, 1, 100)])
def test_disjoint_cliques_closed_form(r, s, p, q):
    g, members = cliques(r, s, r * 100 + s)
    labels, num, den, st = O.cluster(g["off"], g["nbr"], None, p, q)
    for mem in members:
        assert all(labels[v] == mem[0] for v in mem)
    assert den == q
    assert num == r * s * (s - 1) * (q - p)
    # rounds: 3 at level 0 (two moving rounds, one quiet), 1 at level 1
    # (no edges), 1 refinement round at level 0
    assert st[0] == 2
    assert st[1] == 5


def test_isolated_edge_oscillates_then_stops():
    import torch
    g = I.to_numpy(I.pairs_to_csr(torch.tensor([0]), torch.tensor([1]), 2))
    for it in (1, 2, 5, 10):
        L, moved, rounds = O.best_moves(g["off"], g["nbr"], None, np.ones(2), 1, 3,
                                        np.arange(2, dtype=np.int32), it)
        assert rounds == it
        assert list(L) == ([1, 0] if it % 2 else [0, 1])
    labels, num, den, st = O.cluster(g["off"], g["nbr"], None, 1, 3, num_iter=7)
    assert list(labels) == [0, 1] and num == 0 and st[1] == 7


def test_never_worse_than_best_partition_bound_and_exact_on_cliques():
    for seed in range(3):
        g = small_graph(500 + seed, n=7, p=0.5, lo=-2, hi=4)
        W, E = dense(g)
        n = g["n"]
        k = np.ones(n)
        p, q = 1, 4
        labels, num, den, _ = O.cluster(g["off"], g["nbr"], g["w"], p, q)
        best = max(cc_definition(W, E, k, Fraction(p, q), np.array(a))
                   for a in set_partitions(n))
        assert Fraction(num, den) <= best
    g, members = cliques(2, 4, 1)
    W, E = dense(g)
    labels, num, den, _ = O.cluster(g["off"], g["nbr"], None, 1, 2)
    best = max(cc_definition(W, E, np.ones(8), Fraction(1, 2), np.array(a))
               for a in set_partitions(8))
    assert Fraction(num, den) == best


def test_planted_partition_easy_regime():
    """In the easy regime p_in >> lambda >> p_out the run reaches at least the
    planted partition's objective; at lambda = 1/40 it recovers it exactly."""
    g = I.to_numpy(I.sbm([50] * 20, 0.3, 0.002, seed=9))
    n = g["n"]
    planted = g["planted"].astype(np.int32)
    for q, exact in [(20, False), (40, True)]:
        labels, num, den, _ = O.cluster(g["off"], g["nbr"], None, 1, q, num_iter=20)
        planted_num = O.objective_num(g["off"], g["nbr"], None, np.ones(n), 1, q, planted)
        assert num >= planted_num
        if exact:
            pairs = {}
            for a, b in zip(labels, planted):
                pairs.setdefault(int(b), set()).add(int(a))
            assert all(len(s) == 1 for s in pairs.values())
            assert len(set(int(x) for x in labels)) == 20


def test_resolution_orders_cluster_counts():
    """Sec. 4.1: lower lambda gives fewer (larger) clusters."""
    g = I.to_numpy(I.sbm([40] * 10, 0.25, 0.02, seed=3))
    counts = []
    for p, q in [(1, 1000), (1, 40), (1, 8), (1, 2)]:
        labels, *_ = O.cluster(g["off"], g["nbr"], None, p, q)
        counts.append(len(set(int(x) for x in labels)))
    assert counts == sorted(counts)
    assert counts[0] < counts[-1]


def test_deterministic_and_refinement_flag():
    g = I.to_numpy(I.chung_lu(2000, 2.1, 8, seed=5))
    a = O.cluster(g["off"], g["nbr"], None, 1, 1, mode=O.NODEW_DEGREE)
    b = O.cluster(g["off"], g["nbr"], None, 1, 1, mode=O.NODEW_DEGREE)
    assert np.array_equal(a[0], b[0]) and a[1:] == b[1:]
    c = O.cluster(g["off"], g["nbr"], None, 1, 1, mode=O.NODEW_DEGREE, refine=False)
    assert c[3][1] < a[3][1]


# ------------------------------------- whole method, every level by brute force --

def rows_graph(n, rows):
    """CSR dict of a level given as rows[u] = [(v, w), ...] (sorted by v)."""
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    nbr = np.array([v for r in rows for v, _ in r], np.int32)
    w = np.array([x for r in rows for _, x in r], np.int64)
    return {"n": n, "off": off, "nbr": nbr, "w": w}


def brute_best_moves(g, k, p, q, L, num_iter, vset, trace, rows=None, depth=0, phase=0,
                     coin_seed=None):
    """Algorithm 1's Best-Moves with every desired cluster found by brute
    force (re-evaluating the Sec. 2 definition per candidate), the moves of a
    round applied together (Sec. 3.2.1) and V' per Sec. 3.2.2.  L is updated
    in place; the moves of each round are appended to `trace`, and with
    `rows` a record (depth, phase, round, |V'|, entries, moved, held) too.
    With coin_seed, a vertex that wants to move does so only when the
    SplitMix64 coin of (seed, phase, depth, round, vertex) allows it; one held
    back keeps its label and is evaluated again next round, and the call ends
    when no vertex wants to move."""
    W, E = dense(g)
    n = g["n"]
    off, nbr = g["off"], g["nbr"]
    vp = np.ones(n, bool)
    any_moved = False
    for t in range(num_iter):
        D = L.copy()
        for v in range(n):
            if vp[v]:
                D[v] = brute_desired(g, W, E, k, p, q, L, v)
        want = D != L
        held = np.zeros(n, bool)
        if coin_seed is not None:
            held = np.array([bool(want[v]) and not coin(coin_seed, phase, depth, t, v)
                             for v in range(n)], bool)
            D[held] = L[held]
        moved = D != L
        trace.append(int(moved.sum()))
        if rows is not None:
            deg = np.diff(off)
            rows.append((depth, phase, len(trace) - 1, int(vp.sum()), int(deg[vp].sum()),
                         int(moved.sum()), int(held.sum())))
        if not want.any():
            break
        any_moved |= bool(moved.any())
        left = set(int(x) for x in L[moved])
        L[:] = D
        vp = np.zeros(n, bool)
        if vset == O.VSET_ALL:
            vp[:] = True
        elif vset == O.VSET_NBR_VERTICES:
            for v in np.nonzero(moved)[0]:
                vp[nbr[off[v]:off[v + 1]]] = True
        else:
            for x in range(n):
                if int(L[x]) in left:
                    vp[nbr[off[x]:off[x + 1]]] = True
        vp |= held
    return any_moved


def brute_parallel_cc(g, k, p, q, num_iter, vset, refine, depth, log, coin_seed=None,
                      max_levels=64):
    """Parallel-CC (Algorithm 1) on one level: singletons, Best-Moves, and
    unless nothing moved, the level did not shrink or the level cap is
    reached (at most max_levels levels), Compress (a dictionary keyed by the
    two endpoint clusters, intra-cluster pairs dropped, coarse node weight =
    cluster weight, coarse ids = occupied ids in order), recursion, Flatten
    and -- with refinement (Sec. 3.2.3) -- a full Best-Moves on this level
    from the flattened labels, at every depth (coin phase 0 on the way down,
    1 in refinement)."""
    n = g["n"]
    log["levels"] = max(log["levels"], depth + 1)
    L = np.arange(n, dtype=np.int32)
    trace = []
    moved = brute_best_moves(g, k, p, q, L, num_iter, vset, trace, log.get("rows"), depth, 0,
                             coin_seed)
    log["rounds"] += len(trace)
    if not moved or depth + 1 >= max_levels:
        return L
    occupied = sorted(set(int(c) for c in L))
    if len(occupied) == n:
        return L
    rank = {c: i for i, c in enumerate(occupied)}
    n2 = len(occupied)
    acc = {}
    off, nbr, w = g["off"], g["nbr"], g["w"]
    for u in range(n):
        for e in range(off[u], off[u + 1]):
            a, b = rank[int(L[u])], rank[int(L[nbr[e]])]
            if a != b:
                acc[(a, b)] = acc.get((a, b), 0) + int(w[e])
    rows = [[] for _ in range(n2)]
    for (a, b), x in sorted(acc.items()):
        rows[a].append((b, x))
    k2 = np.zeros(n2, np.int64)
    for v in range(n):
        k2[rank[int(L[v])]] += int(k[v])
    L2 = brute_parallel_cc(rows_graph(n2, rows), k2, p, q, num_iter, vset, refine, depth + 1, log,
                           coin_seed, max_levels)
    L = np.array([L2[rank[int(c)]] for c in L], np.int32)
    if refine:
        trace = []
        brute_best_moves(g, k, p, q, L, num_iter, vset, trace, log.get("rows"), depth, 1,
                         coin_seed)
        log["rounds"] += len(trace)
        log["refine"].append((depth, trace))
    return L


# (seed, n, lambda p, q, V' rule, node weights 1 or 1 + v mod 3): signed
# graphs on which the method goes three or four levels deep
DEEP_CASES = [(4, 9, 1, 3, O.VSET_ALL, 0), (0, 10, 1, 3, O.VSET_ALL, 0),
              (8, 8, 1, 2, O.VSET_NBR_CLUSTERS, 1), (2, 9, 1, 4, O.VSET_NBR_VERTICES, 0),
              (3, 10, 1, 4, O.VSET_NBR_VERTICES, 0)]


@pytest.mark.parametrize("case", DEEP_CASES)
@pytest.mark.parametrize("num_iter", [2, 4, 10])
def test_multilevel_run_with_refinement_by_brute_force(case, num_iter):
    """The oracle's whole run (labels, exact objective, levels, rounds)
    equals Algorithm 1 simulated level by level from brute-force moves.  The
    cases are chosen so that refinement moves vertices below the top level
    and keeps moving for more than one round, which a refinement limited to
    depth 0 or to a single round would not reproduce."""
    seed, n, p, q, vset, kmode = case
    g = small_graph(seed * 7 + n, n=n, p=0.45, lo=-2, hi=5)
    k = np.ones(n, np.int64) if kmode == 0 else (np.arange(n) % 3 + 1).astype(np.int64)
    log = {"levels": 0, "rounds": 0, "refine": []}
    L = brute_parallel_cc(g, k, p, q, num_iter, vset, True, 0, log)
    first = {}
    for v in range(n):
        first.setdefault(int(L[v]), v)
    want = np.array([first[int(c)] for c in L], np.int32)
    W, E = dense(g)
    cc = cc_definition(W, E, k, Fraction(p, q), want)
    labels, num, den, st = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=O.NODEW_CUSTOM,
                                     k=k, num_iter=num_iter, vset=vset)
    assert np.array_equal(labels, want)
    assert Fraction(num, den) == cc
    assert st[0] == log["levels"] and st[1] == log["rounds"]
    assert log["levels"] >= 3
    assert any(d >= 1 and sum(t) > 0 for d, t in log["refine"])
    assert any(sum(1 for m in t if m > 0) >= 2 for _, t in log["refine"])


@pytest.mark.parametrize("case", DEEP_CASES[1:4])
def test_round_trace_by_brute_force(case):
    """The oracle's per-round record (depth, phase, round, |V'|, entries,
    moved) of a whole multi-level run equals the brute-force Algorithm 1's,
    round by round, in the same order (coarsening calls on the way down,
    refinement calls on the way up)."""
    seed, n, p, q, vset, kmode = case
    g = small_graph(seed * 7 + n, n=n, p=0.45, lo=-2, hi=5)
    k = np.ones(n, np.int64) if kmode == 0 else (np.arange(n) % 3 + 1).astype(np.int64)
    log = {"levels": 0, "rounds": 0, "refine": [], "rows": []}
    brute_parallel_cc(g, k, p, q, 4, vset, True, 0, log)
    *_, tr = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=O.NODEW_CUSTOM, k=k, num_iter=4,
                       vset=vset, trace=True)
    assert [tuple(int(x) for x in r) for r in tr] == log["rows"]
    assert any(r[3] < n for r in log["rows"])  # V' shrank below V in some round


def test_round_trace_counts_isolated_vertices_in_the_first_v_prime():
    """V' starts as all of V (Algorithm 1), vertices without an edge included:
    the first round's |V'| counts them (they cannot move), on a graph with
    three vertices appended that have no edge, at every level of the run."""
    seed, n, p, q, vset, kmode = DEEP_CASES[1]
    g0 = small_graph(seed * 7 + n, n=n, p=0.45, lo=-2, hi=5)
    iso = 3
    g = {"n": n + iso, "off": np.concatenate([g0["off"], np.repeat(g0["off"][-1], iso)]),
         "nbr": g0["nbr"], "w": g0["w"]}
    k = np.ones(n + iso, np.int64)
    log = {"levels": 0, "rounds": 0, "refine": [], "rows": []}
    brute_parallel_cc(g, k, p, q, 4, vset, True, 0, log)
    *_, tr = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=O.NODEW_CUSTOM, k=k, num_iter=4,
                       vset=vset, trace=True)
    assert [tuple(int(x) for x in r) for r in tr] == log["rows"]
    assert log["rows"][0][3] == n + iso


@pytest.mark.parametrize("case", DEEP_CASES[:4])
def test_level_cap_by_brute_force(case):
    """With a cap of 1, 2 or 3 levels the oracle stops coarsening exactly
    where Algorithm 1 simulated with the same cap does: labels, exact
    objective, levels and rounds."""
    seed, n, p, q, vset, kmode = case
    g = small_graph(seed * 7 + n, n=n, p=0.45, lo=-2, hi=5)
    k = np.ones(n, np.int64) if kmode == 0 else (np.arange(n) % 3 + 1).astype(np.int64)
    W, E = dense(g)
    for cap in (1, 2, 3):
        log = {"levels": 0, "rounds": 0, "refine": []}
        L = brute_parallel_cc(g, k, p, q, 10, vset, True, 0, log, max_levels=cap)
        first = {}
        for v in range(n):
            first.setdefault(int(L[v]), v)
        want = np.array([first[int(c)] for c in L], np.int32)
        labels, num, den, st = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=O.NODEW_CUSTOM,
                                         k=k, num_iter=10, vset=vset, max_levels=cap)
        assert np.array_equal(labels, want), cap
        assert Fraction(num, den) == cc_definition(W, E, k, Fraction(p, q), want), cap
        assert st[0] == log["levels"] == min(cap, log["levels"]) and st[1] == log["rounds"], cap
        if cap == 1:
            assert st[0] == 1


@pytest.mark.parametrize("ci, cseed", [(1, 2), (1, 8), (2, 26)])
def test_coin_multilevel_run_by_brute_force(ci, cseed):
    """With the symmetry-breaking coin, the oracle's whole multi-level run
    (labels, exact objective, levels, rounds, and the per-round record with
    the held-back counts) equals Algorithm 1 simulated with brute-force moves
    and the SplitMix64 coin keyed by (seed, phase, depth, round, vertex),
    phase 1 in refinement.  The graphs and seeds are ones on which the coin
    holds vertices back during refinement, so a coin keyed without the phase
    would change the run."""
    seed, n, p, q, vset, kmode = DEEP_CASES[ci]
    g = small_graph(seed * 7 + n, n=n, p=0.45, lo=-2, hi=5)
    k = np.ones(n, np.int64) if kmode == 0 else (np.arange(n) % 3 + 1).astype(np.int64)
    W, E = dense(g)
    log = {"levels": 0, "rounds": 0, "refine": [], "rows": []}
    L = brute_parallel_cc(g, k, p, q, 10, vset, True, 0, log, coin_seed=cseed)
    first = {}
    for v in range(n):
        first.setdefault(int(L[v]), v)
    want = np.array([first[int(c)] for c in L], np.int32)
    labels, num, den, st, tr = O.cluster(g["off"], g["nbr"], g["w"], p, q, mode=O.NODEW_CUSTOM,
                                         k=k, num_iter=10, vset=vset, coin=True, seed=cseed,
                                         trace=True)
    assert np.array_equal(labels, want)
    assert Fraction(num, den) == cc_definition(W, E, k, Fraction(p, q), want)
    assert st[0] == log["levels"] and st[1] == log["rounds"]
    assert [tuple(int(x) for x in r) for r in tr] == log["rows"]
    assert sum(r[6] for r in log["rows"] if r[1] == 1) > 0  # held back in refinement


# ------------------------------------------- range of the exact arithmetic --

def heavy_graph(scale):
    """Five vertices, six undirected edges whose weights are `scale` minus
    small offsets (both directions stored)."""
    edges = [(0, 1, 1), (1, 2, 3), (2, 3, 0), (3, 4, 5), (0, 4, 2), (1, 3, 7)]
    rows = [[] for _ in range(5)]
    for a, b, d in edges:
        rows[a].append((b, scale - d))
        rows[b].append((a, scale - d))
    return rows_graph(5, [sorted(r) for r in rows])


def brute_whole_run(g, k, p, q, num_iter=10):
    log = {"levels": 0, "rounds": 0, "refine": []}
    L = brute_parallel_cc(g, k, p, q, num_iter, O.VSET_NBR_VERTICES, True, 0, log)
    first = {}
    for v in range(g["n"]):
        first.setdefault(int(L[v]), v)
    return np.array([first[int(c)] for c in L], np.int32)


def test_exact_range_degree_mode_refuses_at_the_bound():
    """Modularity mode at gamma = 8 on a graph whose total weight 2m is just
    above 2^61: p * (sum k)^2 = 8 (2m)^2 passes 2^125, so the run is refused
    rather than computed with wrapped 128-bit gains.  Just below 2^61 it is
    accepted, and then its labels and exact objective equal the brute-force
    Algorithm 1 evaluated in unbounded Python integers."""
    base = (1 << 61) // 12  # twelve entries
    over = heavy_graph(base + 64)
    assert int(np.abs(over["w"]).sum()) > 1 << 61
    with pytest.raises(OverflowError):
        O.cluster(over["off"], over["nbr"], over["w"], 8, 1, mode=O.NODEW_DEGREE)
    under = heavy_graph(base - 64)
    two_m = int(under["w"].sum())
    assert two_m < 1 << 61 and 8 * two_m * two_m < 1 << 125
    k = np.array([int(under["w"][under["off"][v]:under["off"][v + 1]].sum())
                  for v in range(5)], np.int64)
    labels, num, den, _ = O.cluster(under["off"], under["nbr"], under["w"], 8, 1,
                                    mode=O.NODEW_DEGREE)
    assert den == two_m
    want = brute_whole_run(under, k, 8, two_m)
    assert np.array_equal(labels, want)
    W, E = dense(under)
    assert Fraction(num, den) == cc_definition(W, E, k, Fraction(8, two_m), want)


def test_exact_range_custom_node_weights_boundary():
    """Custom node weights summing to 2^32: p = 2^61 puts p * (sum k)^2 at
    exactly 2^125 and is refused; p = 2^61 - 1 is accepted and matches the
    brute-force run.  The same holds for the single-round and objective
    entry points."""
    g = heavy_graph(1000)
    k = np.full(5, 1 << 30, np.int64)
    k[4] = (1 << 32) - 4 * (1 << 30)
    k[3] -= 5
    k[4] += 5
    assert int(k.sum()) == 1 << 32 and (k >= 0).all()
    L = np.arange(5, dtype=np.int32)
    for fn in (lambda p: O.cluster(g["off"], g["nbr"], g["w"], p, 1, mode=O.NODEW_CUSTOM, k=k),
               lambda p: O.objective_num(g["off"], g["nbr"], g["w"], k, p, 1, L),
               lambda p: O.desired(g["off"], g["nbr"], g["w"], k, p, 1, L, k),
               lambda p: O.best_moves(g["off"], g["nbr"], g["w"], k, p, 1, L, 3)):
        with pytest.raises(OverflowError):
            fn(1 << 61)
        fn((1 << 61) - 1)
    p = (1 << 61) - 1
    labels, num, den, _ = O.cluster(g["off"], g["nbr"], g["w"], p, 1, mode=O.NODEW_CUSTOM, k=k)
    assert np.array_equal(labels, brute_whole_run(g, k, p, 1))
    W, E = dense(g)
    assert Fraction(num, den) == cc_definition(W, E, k, Fraction(p, 1), labels)


def test_weighted_degrees_match_numpy():
    for seed in range(3):
        g = I.to_numpy(I.random_signed_graph(50, 0.2, 0, 9, 600 + seed))
        k, tot = O.weighted_degrees(g["off"], g["w"])
        want = np.zeros(g["n"], np.int64)
        np.add.at(want, np.repeat(np.arange(g["n"]), np.diff(g["off"])), g["w"].astype(np.int64))
        assert np.array_equal(k, want) and tot == int(want.sum())
        k1, t1 = O.weighted_degrees(g["off"], None)
        assert np.array_equal(k1, np.diff(g["off"])) and t1 == g["nnz"]


def test_desired_list_equals_range():
    g = I.to_numpy(I.random_signed_graph(60, 0.2, -2, 5, 701))
    n = g["n"]
    rng = np.random.default_rng(3)
    k = rng.integers(0, 4, n)
    L = rng.integers(0, n, n).astype(np.int32)
    K = np.zeros(n, np.int64)
    np.add.at(K, L, k)
    full = O.desired(g["off"], g["nbr"], g["w"], k, 1, 7, L, K)
    verts = rng.permutation(n)[:25]
    rows = [np.arange(g["off"][v], g["off"][v + 1]) for v in verts]
    off_l = np.zeros(len(verts) + 1, np.int64)
    off_l[1:] = np.cumsum([len(r) for r in rows])
    idx = np.concatenate(rows)
    D = O.desired_list(n, verts, off_l, g["nbr"][idx], g["w"][idx], k, 1, 7, L, K)
    assert np.array_equal(D, full[verts])


# --------------------------------------------------------- Sequential-CC --

def improving_neighbour_move(g, W, E, k, lam, labels):
    """A vertex and neighbouring cluster whose move strictly raises the
    objective definition, or None."""
    off, nbr = g["off"], g["nbr"]
    base = cc_definition(W, E, k, lam, labels)
    for v in range(g["n"]):
        for c in sorted(set(int(labels[u]) for u in nbr[off[v]:off[v + 1]]) - {int(labels[v])}):
            L2 = labels.copy()
            L2[v] = c
            if cc_definition(W, E, k, lam, L2) > base:
                return v, c
    return None


@pytest.mark.parametrize("seed", range(5))
def test_sequential_cc_level_ends_at_local_optimum(seed):
    """Sec. 3.1: local moving repeats until no vertex moves, so one level ends
    where no vertex gains by joining a neighbouring cluster (checked by
    re-evaluating the definition for every such move)."""
    g = small_graph(800 + seed, n=8, p=0.5, lo=-3, hi=5)
    W, E = dense(g)
    k = np.ones(g["n"])
    for p, q in [(1, 4), (1, 1)]:
        labels, num, den, st = O.sequential_cc(g["off"], g["nbr"], g["w"], p, q,
                                               seed=seed, max_levels=1)
        assert improving_neighbour_move(g, W, E, k, Fraction(p, q), labels) is None
        assert Fraction(num, den) == cc_definition(W, E, k, Fraction(p, q), labels)
        assert st[0] == 1 and (num > 0) == (st[2] > 0) and num >= 0


@pytest.mark.parametrize("r,s,p,q", [(5, 3, 1, 2), (4, 5, 1, 3), (3, 8, 2, 3)])
def test_sequential_cc_recovers_disjoint_cliques_for_any_order(r, s, p, q):
    """Inside a clique with lambda < 1 a vertex gains (1 - lambda)(s2 - s1 + 1)
    by leaving its part of size s1 for another of size s2, so the only local
    optimum is the whole clique: CC = r s (s - 1)(1 - lambda) whatever the
    random order; the coarse level has no edges and ends the recursion."""
    g, members = cliques(r, s, r * 10 + s)
    for seed in range(4):
        labels, num, den, st = O.sequential_cc(g["off"], g["nbr"], None, p, q, seed=seed)
        for mem in members:
            assert all(labels[v] == mem[0] for v in mem)
        assert den == q and num == r * s * (s - 1) * (q - p)
        assert st[0] == 2 and st[2] >= r * (s - 1)


def test_sequential_cc_merges_the_edge_sync_rounds_swap():
    """The isolated edge that the synchronous rounds swap forever (Sec. 3.1,
    Figure 1's pathology) is merged by the sequential method: CC = 2 (1 - lambda)."""
    import torch
    g = I.to_numpy(I.pairs_to_csr(torch.tensor([0]), torch.tensor([1]), 2))
    for seed in range(3):
        labels, num, den, st = O.sequential_cc(g["off"], g["nbr"], None, 1, 3, seed=seed)
        assert list(labels) == [0, 0] and (num, den) == (2 * (3 - 1), 3)
        assert st == (2, 3, 1)  # level 0: a moving pass and a quiet one; level 1: one pass


def test_sequential_cc_bounded_by_best_partition_and_deterministic():
    for seed in range(3):
        g = small_graph(900 + seed, n=7, p=0.5, lo=-2, hi=4)
        W, E = dense(g)
        k = np.ones(g["n"])
        labels, num, den, _ = O.sequential_cc(g["off"], g["nbr"], g["w"], 1, 4, seed=seed)
        best = max(cc_definition(W, E, k, Fraction(1, 4), np.array(a))
                   for a in set_partitions(g["n"]))
        assert Fraction(num, den) <= best
        again = O.sequential_cc(g["off"], g["nbr"], g["w"], 1, 4, seed=seed)
        assert np.array_equal(again[0], labels) and again[1:] == (num, den, again[3])


def test_sequential_cc_planted_partition():
    """Easy regime (as for the synchronous run): at least the planted
    partition's objective, and the partition itself at lambda = 1/40."""
    g = I.to_numpy(I.sbm([50] * 20, 0.3, 0.002, seed=9))
    n = g["n"]
    planted = g["planted"].astype(np.int32)
    for q, exact in [(20, False), (40, True)]:
        labels, num, den, _ = O.sequential_cc(g["off"], g["nbr"], None, 1, q, seed=1)
        assert num >= O.objective_num(g["off"], g["nbr"], None, np.ones(n), 1, q, planted)
        if exact:
            assert len(set(int(x) for x in labels)) == 20
            for b in range(20):
                assert len(set(int(x) for x in labels[planted == b])) == 1


# ------------------------------------------------- symmetry-breaking coin --

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def splitmix64_output(seed, i):
    """Output i (i >= 1) of the SplitMix64 stream seeded with `seed`, from its
    published definition (Vigna; Steele, Lea and Flood 2014)."""
    z = (seed + i * GAMMA) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def coin(seed, phase, depth, t, v):
    key = v + (t << 32) + (depth << 48) + (phase << 56)
    return splitmix64_output(seed, key + 1) >> 63 == 1


def test_coin_is_fair():
    hits = sum(coin(7, 0, 0, t, v) for t in range(20) for v in range(10000))
    assert abs(hits / 200000 - 0.5) < 0.005


@pytest.mark.parametrize("vset", [O.VSET_ALL, O.VSET_NBR_VERTICES, O.VSET_NBR_CLUSTERS])
def test_coin_rounds_by_brute_force(vset):
    """With the coin, a round moves the vertices whose brute-force best move
    differs from their label and whose coin allows it; the others keep their
    label and are evaluated again next round, and the call ends when no
    vertex wants to move."""
    for gseed in range(3):
        g = small_graph(60 + gseed, n=9, p=0.45, lo=-1, hi=4)
        W, E = dense(g)
        n = g["n"]
        k = np.ones(n, np.int64)
        p, q, seed = 1, 3, 1000 + gseed
        off, nbr = g["off"], g["nbr"]
        L = np.arange(n, dtype=np.int32)
        vp = np.ones(n, bool)
        sims, ended = [L.copy()], None
        for t in range(8):
            D = L.copy()
            for v in range(n):
                if vp[v]:
                    D[v] = brute_desired(g, W, E, k, p, q, L, v)
            want = D != L
            if not want.any():
                ended = t + 1
                break
            held = np.array([want[v] and not coin(seed, 0, 0, t, v) for v in range(n)])
            D[held] = L[held]
            moved = D != L
            left = set(int(x) for x in L[moved])
            L = D
            nxt = np.zeros(n, bool)
            if vset == O.VSET_ALL:
                nxt[:] = True
            elif vset == O.VSET_NBR_VERTICES:
                for v in np.nonzero(moved)[0]:
                    nxt[nbr[off[v]:off[v + 1]]] = True
            else:
                for x in range(n):
                    if int(L[x]) in left:
                        nxt[nbr[off[x]:off[x + 1]]] = True
            vp = nxt | held
            sims.append(L.copy())
        for r in range(1, len(sims)):
            Lr, _, rounds = O.best_moves(off, nbr, g["w"], k, p, q, np.arange(n, dtype=np.int32),
                                         r, vset=vset, coin=True, seed=seed)
            assert np.array_equal(Lr, sims[r]) and rounds == r, (gseed, r)
        if ended is not None:
            Lr, _, rounds = O.best_moves(off, nbr, g["w"], k, p, q, np.arange(n, dtype=np.int32),
                                         50, vset=vset, coin=True, seed=seed)
            assert rounds == ended and np.array_equal(Lr, sims[-1])


def test_coin_level_ends_at_local_optimum():
    """With V' = V every round, a coin run stops only when no vertex wants to
    move, i.e. at a local optimum (the plain rounds may stop at the round cap
    while swapping)."""
    for gseed in range(4):
        g = small_graph(70 + gseed, n=8, p=0.5, lo=-3, hi=5)
        W, E = dense(g)
        for p, q in [(1, 4), (1, 1)]:
            labels, num, den, _ = O.cluster(g["off"], g["nbr"], g["w"], p, q, vset=O.VSET_ALL,
                                            max_levels=1, num_iter=200, coin=True, seed=gseed)
            assert improving_neighbour_move(g, W, E, np.ones(g["n"]), Fraction(p, q),
                                            labels) is None


def test_coin_merges_the_swapping_edge_and_recovers_cliques():
    import torch
    e = I.to_numpy(I.pairs_to_csr(torch.tensor([0]), torch.tensor([1]), 2))
    for seed in range(5):
        labels, num, den, _ = O.cluster(e["off"], e["nbr"], None, 1, 3, num_iter=20,
                                        coin=True, seed=seed)
        assert list(labels) == [0, 0] and (num, den) == (2 * (3 - 1), 3)
    for r, s, p, q in [(5, 3, 1, 2), (3, 8, 2, 3)]:
        g, members = cliques(r, s, r * 7 + s)
        for seed in range(3):
            labels, num, den, _ = O.cluster(g["off"], g["nbr"], None, p, q, num_iter=100,
                                            coin=True, seed=seed)
            for mem in members:
                assert all(labels[v] == mem[0] for v in mem)
            assert num == r * s * (s - 1) * (q - p)


def test_coin_planted_partition():
    g = I.to_numpy(I.sbm([50] * 20, 0.3, 0.002, seed=9))
    n = g["n"]
    planted = g["planted"].astype(np.int32)
    for q in (20, 40):
        _, num, _, _ = O.cluster(g["off"], g["nbr"], None, 1, q, num_iter=20, coin=True, seed=3)
        assert num >= O.objective_num(g["off"], g["nbr"], None, np.ones(n), 1, q, planted)
