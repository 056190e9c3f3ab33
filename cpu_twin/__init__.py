"""Multi-core CPU twin of the LambdaCC best-move / contraction path (OpenMP).

A measured CPU baseline: the same deterministic synchronous schedule as the
GPU library (Algorithm 1, Sec. 3.2), run on all host cores, with the oracle's
labels, objective and counters bit for bit at every thread count.  The
benchmark's CPU leg and the tests load it; the GPU library never does.  The
arithmetic lives in ``lcc_twin.c``; this module only marshals numpy arrays.

Weights are passed as int32 (input graphs) or int64 (coarse graphs) arrays, or
None for an unweighted graph.
"""
import ctypes as C

import numpy as np

from .build import build, LIB

NODEW_UNIT, NODEW_DEGREE, NODEW_CUSTOM = 0, 1, 2
VSET_ALL, VSET_NBR_VERTICES, VSET_NBR_CLUSTERS = 0, 1, 2

_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB)
        P, I64, I = C.c_void_p, C.c_int64, C.c_int
        U64 = C.c_uint64
        _lib.tw_cluster.argtypes = [I64, P, P, P, P, P, I, I64, I64, I, I, I, I, I, U64, I,
                                    P, I64, P, P, P, P, P, P, P]
        _lib.tw_best_moves.argtypes = [I64, P, P, P, P, P, I64, I64, I, I, I, U64, I,
                                       P, P, P]
        _lib.tw_compress.argtypes = [I64, P, P, P, P, P, P, I, P, P, P, P, P, P, P]
        _lib.tw_first_round.argtypes = [I64, P, P, P, P, I64, I64, I, P, P, P, P]
        _lib.tw_free.argtypes = [P]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _graph(off, nbr, w):
    off = np.ascontiguousarray(off, dtype=np.int64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    w32 = w64 = None
    if w is not None:
        w = np.asarray(w)
        if w.dtype == np.int64:
            w64 = np.ascontiguousarray(w)
        else:
            w32 = np.ascontiguousarray(w, dtype=np.int32)
    return off, nbr, w32, w64


def _check(rc, what):
    if rc:
        raise ValueError("cpu twin %s failed: status %d" % (what, rc))


def cluster(off, nbr, w, p, q, mode=NODEW_UNIT, k=None, num_iter=10, max_levels=64,
            refine=True, vset=VSET_NBR_VERTICES, coin=False, seed=0, threads=0):
    """Parallel-CC (Algorithm 1, synchronous; coin=True adds the seeded
    symmetry-breaking coin) on `threads` cores (0 = all).

    Returns (labels, num, den, stats, threads_used) with CC = num / den
    exactly and stats = (levels, rounds, entries scanned)."""
    return _cluster(off, nbr, w, p, q, mode, k, num_iter, max_levels, refine, vset, coin, seed,
                    threads, None)


TRACE_COLUMNS = ("level", "phase", "round", "vprime", "entries", "moved", "held")


def cluster_trace(off, nbr, w, p, q, mode=NODEW_UNIT, k=None, num_iter=10, max_levels=64,
                  refine=True, vset=VSET_NBR_VERTICES, coin=False, seed=0, threads=0,
                  max_rounds=100000):
    """cluster() plus one row per best-move round (TRACE_COLUMNS): level
    depth, phase (1 = refinement), round within the call, |V'|, entries
    scanned, vertices moved and vertices the coin held back."""
    buf = np.zeros((max_rounds, len(TRACE_COLUMNS)), np.int64)
    res = _cluster(off, nbr, w, p, q, mode, k, num_iter, max_levels, refine, vset, coin, seed,
                   threads, buf)
    rows = res[-1]
    if rows > max_rounds:
        raise ValueError("more than %d rounds; raise max_rounds" % max_rounds)
    return res[:-1], buf[:rows]


def _cluster(off, nbr, w, p, q, mode, k, num_iter, max_levels, refine, vset, coin, seed,
             threads, trace):
    off, nbr, w32, w64 = _graph(off, nbr, w)
    n = len(off) - 1
    kk = None if k is None else np.ascontiguousarray(k, dtype=np.int64)
    labels = np.empty(max(n, 1), np.int32)
    hi, lo, den, nt, tl = C.c_int64(), C.c_uint64(), C.c_int64(), C.c_int(), C.c_int64()
    st = np.zeros(3, np.int64)
    rc = lib().tw_cluster(n, _p(off), _p(nbr), _p(w32), _p(w64), _p(kk), mode, p, q,
                          num_iter, max_levels, int(bool(refine)), vset, int(bool(coin)),
                          seed & ((1 << 64) - 1), threads, _p(trace),
                          0 if trace is None else trace.shape[0], C.byref(tl),
                          _p(labels), C.byref(hi), C.byref(lo), C.byref(den), _p(st),
                          C.byref(nt))
    _check(rc, "cluster")
    v = (int(hi.value) << 64) | int(lo.value)
    if v >= 1 << 127:
        v -= 1 << 128
    out = (labels[:n], v, den.value, tuple(int(x) for x in st), nt.value)
    return out + (tl.value,) if trace is not None else out


def best_moves(off, nbr, w, k, p, q, L, num_iter, vset=VSET_NBR_VERTICES, coin=False, seed=0,
               threads=0):
    """Best-Moves on one level from labels L; returns (labels, moved, rounds)."""
    off, nbr, w32, w64 = _graph(off, nbr, w)
    k = np.ascontiguousarray(k, dtype=np.int64)
    L = np.array(L, dtype=np.int32, copy=True)
    moved, rounds = C.c_int(), C.c_int64()
    rc = lib().tw_best_moves(len(off) - 1, _p(off), _p(nbr), _p(w32), _p(w64), _p(k), p, q,
                             num_iter, vset, int(bool(coin)), seed & ((1 << 64) - 1), threads,
                             _p(L), C.byref(moved), C.byref(rounds))
    _check(rc, "best_moves")
    return L, bool(moved.value), rounds.value


def compress(off, nbr, w, k, L, threads=0):
    """Coarse graph of the clustering L: (map, off', nbr', w', k')."""
    off, nbr, w32, w64 = _graph(off, nbr, w)
    n = len(off) - 1
    k = np.ascontiguousarray(k, dtype=np.int64)
    L = np.ascontiguousarray(L, dtype=np.int32)
    mp = np.empty(max(n, 1), np.int32)
    n2, nnz2 = C.c_int64(), C.c_int64()
    po, pn, pw, pk = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
    rc = lib().tw_compress(n, _p(off), _p(nbr), _p(w32), _p(w64), _p(k), _p(L), threads,
                           _p(mp), C.byref(n2), C.byref(nnz2), C.byref(po), C.byref(pn),
                           C.byref(pw), C.byref(pk))
    _check(rc, "compress")

    def take(ptr, count, ctype, dtype):
        out = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=(count,)).copy() \
            if count else np.zeros(0, dtype)
        lib().tw_free(ptr)
        return out.astype(dtype, copy=False)

    a, b = n2.value, nnz2.value
    return (mp[:n], take(po, a + 1, C.c_int64, np.int64), take(pn, b, C.c_int32, np.int32),
            take(pw, b, C.c_int64, np.int64), take(pk, a, C.c_int64, np.int64))


def first_round(off, nbr, w32, k, p, q, threads=0):
    """One full-frontier best-move round from singletons.  k=None selects
    modularity (k = weighted degree, lambda = p / (q 2m)).

    Returns (D, entries scanned, seconds of the round alone, threads used)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    w32 = None if w32 is None else np.ascontiguousarray(w32, dtype=np.int32)
    k = None if k is None else np.ascontiguousarray(k, dtype=np.int64)
    n = len(off) - 1
    D = np.empty(max(n, 1), np.int32)
    ent, secs, nt = C.c_int64(), C.c_double(), C.c_int()
    rc = lib().tw_first_round(n, _p(off), _p(nbr), _p(w32), _p(k), p, q, threads, _p(D),
                              C.byref(ent), C.byref(secs), C.byref(nt))
    _check(rc, "first_round")
    return D[:n], ent.value, secs.value, nt.value
