"""Seeded synthetic graph generators shared by the tests, the smoke check and
the benchmark.

This module draws random graphs and lays them out as CSR; it holds none of the
clustering arithmetic.  Every generator takes a seed and a torch device, so
the same code builds small graphs on the CPU and the billion-edge R-MAT graph
on the GPU.  A graph is returned as a dict with

  off  int64[n+1]   row offsets (both directions of every undirected edge)
  nbr  int32[nnz]   neighbour ids, ascending within each row
  w    int32[nnz]   edge weights, or None for an unweighted graph
  n, nnz            sizes

All graphs are symmetric, loop-free and without parallel edges, and their
vertex ids are randomly permuted so that ids carry no locality.
"""
import math

import numpy as np
import torch

BASE_SEED = 0x1CC02108


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & ((1 << 63) - 1))
    return g


def pairs_to_csr(a, b, n, w=None):
    """Symmetric CSR from unique undirected pairs a < b (int64 tensors).

    Row x lists its smaller neighbours (from pairs (u, x)) and then its larger
    ones (from pairs (x, v)), each ascending, so rows come out sorted."""
    dev = a.device
    m = a.numel()
    k1 = a * n + b
    o1 = torch.argsort(k1)
    del k1
    a1, b1 = a[o1], b[o1]
    w1 = w[o1] if w is not None else None
    del o1
    k2 = b * n + a
    o2 = torch.argsort(k2)
    del k2
    a2, b2 = a[o2], b[o2]
    w2 = w[o2] if w is not None else None
    del o2
    cnt_up = torch.bincount(a1, minlength=n)
    cnt_lo = torch.bincount(b2, minlength=n)
    deg = cnt_up + cnt_lo
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(deg, 0)
    nnz = 2 * m
    nbr = torch.empty(nnz, dtype=torch.int32, device=dev)
    wout = torch.empty(nnz, dtype=torch.int32, device=dev) if w is not None else None
    st_up = torch.cumsum(cnt_up, 0) - cnt_up
    idx = torch.arange(m, dtype=torch.int64, device=dev)
    pos = off[a1] + cnt_lo[a1] + (idx - st_up[a1])
    nbr[pos] = b1.to(torch.int32)
    if w is not None:
        wout[pos] = w1
    del pos, st_up
    st_lo = torch.cumsum(cnt_lo, 0) - cnt_lo
    pos = off[b2] + (idx - st_lo[b2])
    nbr[pos] = a2.to(torch.int32)
    if w is not None:
        wout[pos] = w2
    return {"off": off, "nbr": nbr, "w": wout, "n": int(n), "nnz": int(nnz)}


def canonical_unique(u, v, n):
    """Drop loops, orient each pair as (min, max) and merge duplicates."""
    keep = u != v
    u, v = u[keep], v[keep]
    a = torch.minimum(u, v)
    b = torch.maximum(u, v)
    key = torch.unique(a * n + b)
    return key // n, key % n


def permute_ids(a, b, n, gen):
    perm = torch.randperm(n, generator=gen, device=a.device)
    return perm[a], perm[b], perm


def sbm(sizes, p_in, p_out, seed, device="cpu"):
    """Planted-partition (stochastic block model) graph.

    Block i has sizes[i] vertices; each intra-block pair is an edge with
    probability p_in and each inter-block pair with probability p_out.  The
    edge counts are drawn exactly (binomial); the pairs themselves are drawn
    with replacement and merged, which for sparse blocks differs from the
    exact model only by the rare repeated pair.  Returns the graph plus
    ``planted`` (block of each vertex, after the id permutation)."""
    gen = _gen(seed, device)
    sizes_t = torch.as_tensor(sizes, dtype=torch.int64, device=device)
    n = int(sizes_t.sum())
    starts = torch.cumsum(sizes_t, 0) - sizes_t
    nb = sizes_t.numel()
    sz = sizes_t.to(torch.float64)
    intra_pairs = sz * (sz - 1) / 2
    x_in = torch.binomial(intra_pairs, torch.full_like(intra_pairs, float(p_in)),
                          generator=gen).to(torch.int64)
    tot_in = int(x_in.sum())
    blk = torch.repeat_interleave(torch.arange(nb, device=device), x_in)
    s_blk = sizes_t[blk]
    r1 = torch.rand(tot_in, generator=gen, device=device, dtype=torch.float64)
    r2 = torch.rand(tot_in, generator=gen, device=device, dtype=torch.float64)
    u_in = starts[blk] + (r1 * s_blk).to(torch.int64).clamp_max(s_blk - 1)
    v_in = starts[blk] + (r2 * s_blk).to(torch.int64).clamp_max(s_blk - 1)
    all_pairs = n * (n - 1) / 2
    inter_pairs = all_pairs - float(intra_pairs.sum())
    if inter_pairs > 0 and p_out > 0:
        x_out = int(torch.binomial(torch.tensor([inter_pairs], dtype=torch.float64,
                                                device=device),
                                   torch.tensor([float(p_out)], dtype=torch.float64,
                                                device=device),
                                   generator=gen).item())
    else:
        x_out = 0
    block_of = torch.repeat_interleave(torch.arange(nb, device=device), sizes_t)
    us, vs = [u_in], [v_in]
    if x_out > 0:
        frac = inter_pairs / all_pairs
        need = x_out
        while need > 0:
            draw = int(need / frac * 1.1) + 64
            u = torch.randint(0, n, (draw,), generator=gen, device=device)
            v = torch.randint(0, n, (draw,), generator=gen, device=device)
            ok = block_of[u] != block_of[v]
            u, v = u[ok][:need], v[ok][:need]
            us.append(u)
            vs.append(v)
            need -= u.numel()
    a, b = canonical_unique(torch.cat(us), torch.cat(vs), n)
    a, b, perm = permute_ids(a, b, n, gen)
    a, b = torch.minimum(a, b), torch.maximum(a, b)
    g = pairs_to_csr(a, b, n)
    planted = torch.empty(n, dtype=torch.int64, device=device)
    planted[perm] = block_of
    g["planted"] = planted
    return g


def chung_lu(n, beta, mean_deg, seed, device="cpu", i0=1.0):
    """Chung-Lu power-law graph: expected degree of vertex i proportional to
    (i + i0)^(-1/(beta-1)), scaled to the mean degree and capped at the square
    root of the total; n * mean_deg / 2 endpoint pairs are drawn in proportion
    to the expected degrees, then loops and repeats are dropped."""
    gen = _gen(seed, device)
    i = torch.arange(n, dtype=torch.float64, device=device)
    wt = (i + i0) ** (-1.0 / (beta - 1.0))
    wt = wt * (n * mean_deg / wt.sum())
    wt = torch.clamp(wt, max=math.sqrt(float(wt.sum())))
    cdf = torch.cumsum(wt, 0)
    cdf = cdf / cdf[-1]
    m = int(n * mean_deg // 2)
    u = torch.searchsorted(cdf, torch.rand(m, generator=gen, device=device,
                                           dtype=torch.float64))
    v = torch.searchsorted(cdf, torch.rand(m, generator=gen, device=device,
                                           dtype=torch.float64))
    u = u.clamp_max(n - 1)
    v = v.clamp_max(n - 1)
    a, b = canonical_unique(u, v, n)
    a, b, _ = permute_ids(a, b, n, gen)
    a, b = torch.minimum(a, b), torch.maximum(a, b)
    return pairs_to_csr(a, b, n)


def rmat(scale, m_edges, a=0.57, b=0.19, c=0.19, seed=0, device="cpu",
         chunk=1 << 27, weighted=True):
    """R-MAT graph with 2^scale vertices and exactly m_edges unique undirected
    edges (both directions stored).  Endpoints are drawn level by level from
    the quadrant probabilities (a, b, c, d = 1 - a - b - c); draws continue
    until enough unique loop-free pairs exist, and a seeded random subset of
    exactly m_edges is kept.  With weighted=True every edge carries a stored
    int32 weight of 1."""
    gen = _gen(seed, device)
    n = 1 << scale
    keys = torch.empty(0, dtype=torch.int64, device=device)
    target = int(m_edges)
    draw_total = int(target * 1.15) + 1024
    while keys.numel() < target:
        parts = [keys]
        left = draw_total
        while left > 0:
            cnt = min(chunk, left)
            src = torch.zeros(cnt, dtype=torch.int64, device=device)
            dst = torch.zeros(cnt, dtype=torch.int64, device=device)
            for _ in range(scale):
                r = torch.rand(cnt, generator=gen, device=device)
                bit_s = (r >= a + b).to(torch.int64)
                bit_d = ((r >= a) & (r < a + b)) | (r >= a + b + c)
                src = src * 2 + bit_s
                dst = dst * 2 + bit_d.to(torch.int64)
                del r, bit_s, bit_d
            keep = src != dst
            src, dst = src[keep], dst[keep]
            lo = torch.minimum(src, dst)
            hi = torch.maximum(src, dst)
            parts.append(lo * n + hi)
            del src, dst, lo, hi, keep
            left -= cnt
        keys = torch.unique(torch.cat(parts))
        del parts
        draw_total = int((target - keys.numel()) * 1.5) + 1024
    if keys.numel() > target:
        sel = torch.randperm(keys.numel(), generator=gen, device=device)[:target]
        keys = keys[sel]
        del sel
    a_, b_ = keys // n, keys % n
    del keys
    a_, b_, _ = permute_ids(a_, b_, n, gen)
    a2, b2 = torch.minimum(a_, b_), torch.maximum(a_, b_)
    del a_, b_
    g = pairs_to_csr(a2, b2, n)
    if weighted:
        g["w"] = torch.ones(g["nnz"], dtype=torch.int32, device=device)
    return g


def knn(n_points, dim, n_centers, sigma, k, seed, device="cpu", scale=1 << 16,
        chunk=4096):
    """Weighted k-nearest-neighbour similarity graph on a Gaussian mixture.

    Centres are normalised Gaussian vectors; each point is a random centre
    plus N(0, sigma^2 I) noise.  Each point links to its k most cosine-similar
    other points; the union of these links is symmetrised and each undirected
    edge gets weight round(cos * scale) (signed int32), computed once per pair
    in float64 so that both directions carry the same weight."""
    gen = _gen(seed, device)
    cent = torch.randn(n_centers, dim, generator=gen, device=device)
    cent = cent / cent.norm(dim=1, keepdim=True)
    which = torch.randint(0, n_centers, (n_points,), generator=gen, device=device)
    pts = cent[which] + sigma * torch.randn(n_points, dim, generator=gen,
                                            device=device)
    pts = pts / pts.norm(dim=1, keepdim=True)
    us, vs = [], []
    for s in range(0, n_points, chunk):
        e = min(n_points, s + chunk)
        sim = pts[s:e] @ pts.T
        sim[torch.arange(e - s, device=device),
            torch.arange(s, e, device=device)] = -float("inf")
        idx = torch.topk(sim, k, dim=1).indices
        us.append(torch.arange(s, e, device=device).repeat_interleave(k))
        vs.append(idx.reshape(-1))
        del sim, idx
    a, b = canonical_unique(torch.cat(us), torch.cat(vs), n_points)
    p64 = pts.to(torch.float64)
    wts = torch.empty(a.numel(), dtype=torch.int32, device=device)
    step = 1 << 22
    for s in range(0, a.numel(), step):
        cos = (p64[a[s:s + step]] * p64[b[s:s + step]]).sum(1)
        wts[s:s + step] = torch.round(cos * scale).to(torch.int32)
    a, b, perm = permute_ids(a, b, n_points, gen)
    a2, b2 = torch.minimum(a, b), torch.maximum(a, b)
    g = pairs_to_csr(a2, b2, n_points, w=wts)
    centre = torch.empty(n_points, dtype=torch.int64, device=device)
    centre[perm] = which
    g["planted"] = centre
    return g


def serving_params(index, base_seed=BASE_SEED + 5):
    """Parameters of graph `index` of the serving stream: n log-uniform in
    [100, 200000]; communities log-uniform in [5, 500] (at most n/10); target
    mean degree log-uniform in [8, 64]; inter-community fraction mu uniform in
    [0.1, 0.4]; p_in = d(1-mu)/(n/B - 1), p_out = d mu/(n - n/B)."""
    rs = np.random.default_rng([base_seed, index])
    n = int(round(math.exp(rs.uniform(math.log(100), math.log(200000)))))
    nb = int(round(math.exp(rs.uniform(math.log(5), math.log(500)))))
    nb = max(1, min(nb, n // 10))
    d = math.exp(rs.uniform(math.log(8), math.log(64)))
    mu = rs.uniform(0.1, 0.4)
    s = n / nb
    p_in = min(1.0, d * (1 - mu) / max(s - 1, 1))
    p_out = min(1.0, d * mu / max(n - s, 1))
    base = n // nb
    sizes = [base + (1 if i < n % nb else 0) for i in range(nb)]
    return {"n": n, "blocks": nb, "sizes": sizes, "p_in": p_in, "p_out": p_out,
            "mean_deg": d, "mu": mu, "seed": base_seed * 1000003 + index}


def serving_graph(index, device="cpu"):
    pr = serving_params(index)
    return sbm(pr["sizes"], pr["p_in"], pr["p_out"], pr["seed"], device)


def to_numpy(g):
    """Host copy of a graph (numpy arrays)."""
    out = {"n": g["n"], "nnz": g["nnz"]}
    for key in ("off", "nbr", "w", "planted"):
        if key in g and g[key] is not None:
            out[key] = g[key].cpu().numpy()
        else:
            out[key] = None
    return out


def random_labels(n, n_clusters, seed, device="cpu"):
    """Arbitrary labels in [0, n): n_clusters distinct ids drawn at random."""
    gen = _gen(seed, device)
    ids = torch.randperm(n, generator=gen, device=device)[:max(1, n_clusters)]
    pick = torch.randint(0, ids.numel(), (n,), generator=gen, device=device)
    return ids[pick].to(torch.int32)


def random_signed_graph(n, p_edge, w_lo, w_hi, seed, device="cpu"):
    """Small Erdos-Renyi graph with integer weights uniform in [w_lo, w_hi]."""
    gen = _gen(seed, device)
    iu = torch.triu_indices(n, n, 1, device=device)
    keep = torch.rand(iu.shape[1], generator=gen, device=device) < p_edge
    a, b = iu[0][keep], iu[1][keep]
    w = torch.randint(w_lo, w_hi + 1, (a.numel(),), generator=gen,
                      device=device).to(torch.int32)
    return pairs_to_csr(a.to(torch.int64), b.to(torch.int64), n, w=w)


def hub_graph(n, mean_deg, hubs, hub_deg, seed, device="cpu", w_lo=None, w_hi=None):
    """Sparse random graph plus `hubs` vertices joined to hub_deg random others
    each (hub_deg may be a list, one draw count per hub), so that every degree
    bucket (including rows of tens of thousands of entries) is populated.
    Optional integer weights uniform in [w_lo, w_hi]."""
    gen = _gen(seed, device)
    m = int(n * mean_deg // 2)
    u = torch.randint(0, n, (m,), generator=gen, device=device)
    v = torch.randint(0, n, (m,), generator=gen, device=device)
    degs = list(hub_deg) if isinstance(hub_deg, (list, tuple)) else [hub_deg] * hubs
    hu = torch.repeat_interleave(torch.arange(len(degs), device=device),
                                 torch.tensor(degs, device=device))
    hv = torch.randint(0, n, (int(sum(degs)),), generator=gen, device=device)
    a, b = canonical_unique(torch.cat([u, hu]), torch.cat([v, hv]), n)
    a, b, _ = permute_ids(a, b, n, gen)
    a2, b2 = torch.minimum(a, b), torch.maximum(a, b)
    w = None
    if w_lo is not None:
        w = torch.randint(w_lo, w_hi + 1, (a2.numel(),), generator=gen,
                          device=device).to(torch.int32)
    return pairs_to_csr(a2, b2, n, w=w)
