"""The allocation-free entry point lcc_desired_noalloc.

It serves callers that may not allocate GPU memory when they call (their own
runtime owns every device allocation), so its working memory is a fixed array
inside the library.  These tests call it through the C ABI on caller-owned
device buffers and compare its output with lcc_desired's, and with the CPU
oracle's, on two consecutive calls (the second call must not see leftovers of
the first).  Results are integers, so the comparison is exact.  It must also
refuse what the other entry points refuse: ids outside [0, n), negative
weights and inputs outside the exact integer range.  The file is named to be
collected last.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_01731_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _noalloc(L, g, k, p, q, labels, K=None):
    import torch
    n = g["n"]
    if K is None:
        K = np.zeros(n, np.int64)
        np.add.at(K, labels, k)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()  # noqa: E731
    d_w = None if g["w"] is None else dev(g["w"], np.int32)
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    L.lcc_desired_noalloc(dev(g["off"], np.int64), dev(g["nbr"], np.int32), d_w,
                          dev(k, np.int64), p, q, dev(labels, np.int32), dev(K, np.int64), out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), K


def _case(L, g, k, p, q, labels):
    got, K = _noalloc(L, g, k, p, q, labels)
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], node_w=k)
    want = L.lcc_desired(G, p, q, L.LCC_NODEW_CUSTOM, labels)
    G.free()
    orc = O.desired(g["off"], g["nbr"], g["w"], k, p, q, labels, K)
    assert np.array_equal(want, orc)
    return got, want


def test_noalloc_matches_lcc_desired_on_two_calls():
    import torch
    torch.cuda.set_device(0)
    from paper_2108_01731_gb300 import lcc as L
    L.load()
    g1 = I.to_numpy(I.hub_graph(30000, 8, 3, 2500, seed=41, w_lo=-2, w_hi=7))
    assert np.diff(g1["off"]).max() <= 4096
    k1 = np.random.default_rng(1).integers(0, 5, g1["n"]).astype(np.int64)
    lab1 = I.random_labels(g1["n"], 900, seed=42).numpy()
    got, want = _case(L, g1, k1, 2, 11, lab1)
    assert np.array_equal(got, want)
    # second call in a row, other graph and labels: the shared array is reused
    g2 = I.to_numpy(I.sbm([80] * 40, 0.2, 0.01, seed=43))
    k2 = np.ones(g2["n"], np.int64)
    lab2 = np.arange(g2["n"], dtype=np.int32)
    got2, want2 = _case(L, g2, k2, 1, 30, lab2)
    assert np.array_equal(got2, want2)


def test_noalloc_rejects_rows_beyond_its_limit():
    import torch
    torch.cuda.set_device(0)
    from paper_2108_01731_gb300 import lcc as L
    L.load()
    g = I.to_numpy(I.hub_graph(20000, 4, 1, 9000, seed=44))
    assert np.diff(g["off"]).max() > 4096
    k = np.ones(g["n"], np.int64)
    labels = np.arange(g["n"], dtype=np.int32)
    with pytest.raises(L.LccError) as e:
        _case(L, g, k, 1, 10, labels)
    assert e.value.status == L.LCC_ERR_INVALID
    assert "at most 4096" in str(e.value)


def test_noalloc_refuses_what_it_cannot_compute_exactly():
    """Ids outside [0, n) and negative weights give LCC_ERR_INVALID (the
    kernel skips those entries and reports them); node weights whose total
    puts p * (sum k)^2 at 2^125 give LCC_ERR_OVERFLOW, as in lcc_desired and
    the oracle.  A valid call afterwards still matches the oracle."""
    import torch
    torch.cuda.set_device(0)
    from paper_2108_01731_gb300 import lcc as L
    L.load()
    g = I.to_numpy(I.random_signed_graph(300, 0.1, -4, 6, seed=6))
    n = g["n"]
    k = np.ones(n, np.int64)
    lab = np.arange(n, dtype=np.int32)
    bad = lab.copy()
    bad[17] = n  # one label out of range
    with pytest.raises(L.LccError) as e:
        _noalloc(L, g, k, 1, 5, bad, K=np.ones(n, np.int64))
    assert e.value.status == L.LCC_ERR_INVALID
    kneg = k.copy()
    kneg[3] = -1
    with pytest.raises(L.LccError) as e:
        _noalloc(L, g, kneg, 1, 5, lab)
    assert e.value.status == L.LCC_ERR_INVALID
    kbig = k.copy()
    kbig[n // 2] = 1 << 40
    kt = int(kbig.sum())
    pmax = ((1 << 125) - 1) // (kt * kt)
    with pytest.raises(L.LccError) as e:
        _noalloc(L, g, kbig, pmax + 1, 1 << 62, lab)
    assert e.value.status == L.LCC_ERR_OVERFLOW
    with pytest.raises(OverflowError):
        O.desired(g["off"], g["nbr"], g["w"], kbig, pmax + 1, 1 << 62, lab, kbig)
    got, K = _noalloc(L, g, kbig, pmax, 1 << 62, lab)
    want = O.desired(g["off"], g["nbr"], g["w"], kbig, pmax, 1 << 62, lab, K)
    assert np.array_equal(got, want) and (got != lab).any()
