"""CPU oracle for the LambdaCC best-move / contraction path.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the library never does.  The
arithmetic lives in ``lcc_oracle.c`` (plain single-threaded C, exact int128
gains); this module only marshals numpy arrays through ctypes.

Graphs are CSR triples ``(off int64[n+1], nbr int32[nnz], w int64[nnz])``;
an unweighted graph passes ``w`` of ones.
"""
import ctypes as C
import os

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
        P = C.c_void_p
        I64 = C.c_int64
        _lib.orc_objective.argtypes = [I64, P, P, P, P, I64, I64, P, P, P]
        _lib.orc_objective_pairs.argtypes = [I64, P, P, P, P, I64, I64, P, P, P]
        _lib.orc_desired_range.argtypes = [I64, I64, I64, P, P, P, P, I64, I64,
                                           P, P, P]
        _lib.orc_compress.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, P, P]
        _lib.orc_free.argtypes = [P]
        _lib.orc_cluster.argtypes = [I64, P, P, P, P, C.c_int, I64, I64,
                                     C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_uint64, P, P, P, P, P, P, I64, P]
        _lib.orc_best_moves.argtypes = [I64, P, P, P, P, I64, I64, C.c_int,
                                        C.c_int, C.c_int, C.c_uint64, P, P]
        _lib.orc_sequential_cc.argtypes = [I64, P, P, P, P, C.c_int, I64, I64,
                                           C.c_uint64, C.c_int, C.c_int, P, P, P,
                                           P, P]
        _lib.orc_sequential_sweep.argtypes = [I64, P, P, P, P, I64, I64, P, I64]
        _lib.orc_sequential_sweep.restype = I64
        _lib.orc_weighted_degrees_i32.argtypes = [I64, P, P, P]
        _lib.orc_desired_list.argtypes = [I64, I64, P, P, P, P, P, I64, I64, P, P, P]
        _lib.orc_scratch_new.argtypes = [I64]
        _lib.orc_scratch_new.restype = P
        _lib.orc_scratch_free.argtypes = [P]
        _lib.orc_desired_scratch.argtypes = [P, I64, I64, I64, P, P, P, P, I64, I64,
                                             P, P, P]
        _lib.orc_weighted_degrees_i32.restype = I64
    return _lib


ERR_OVERFLOW = 5


def _check(rc, what):
    """Raise for an oracle status: OverflowError when the exact 128-bit range
    would be left (q * sum|w| or p * (sum k)^2 reaching 2^125), else
    ValueError."""
    if rc == ERR_OVERFLOW:
        raise OverflowError("oracle %s: outside the exact integer range" % what)
    if rc:
        raise ValueError("oracle %s failed: %d" % (what, rc))


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _i128(hi, lo):
    return (int(hi) << 64) | int(lo)


def _graph(off, nbr, w):
    off = _c(off, np.int64)
    nbr = _c(nbr, np.int32)
    w = np.ones(len(nbr), np.int64) if w is None else _c(w, np.int64)
    return off, nbr, w


def objective_num(off, nbr, w, k, p, q, labels, literal=False):
    """Exact q * CC(labels) as a Python int (Sec. 2 objective, ordered pairs).

    literal=True evaluates the O(n^2) double sum of the definition."""
    off, nbr, w = _graph(off, nbr, w)
    k = _c(k, np.int64)
    labels = _c(labels, np.int32)
    hi = C.c_int64()
    lo = C.c_uint64()
    fn = lib().orc_objective_pairs if literal else lib().orc_objective
    rc = fn(len(off) - 1, _p(off), _p(nbr), _p(w), _p(k), p, q, _p(labels),
            C.byref(hi), C.byref(lo))
    _check(rc, "objective")
    v = _i128(hi.value, lo.value)
    if v >= 1 << 127:
        v -= 1 << 128
    return v


def desired(off, nbr, w, k, p, q, L, K, v0=0, v1=None):
    """Desired cluster D[v] of every v in [v0, v1) under the snapshot (L, K)."""
    off, nbr, w = _graph(off, nbr, w)
    n = len(off) - 1
    v1 = n if v1 is None else v1
    offw = _c(off[v0:v1 + 1] - off[v0], np.int64)
    nbrw = nbr[off[v0]:off[v1]]
    ww = w[off[v0]:off[v1]]
    k = _c(k, np.int64)
    L = _c(L, np.int32)
    K = _c(K, np.int64)
    D = np.empty(v1 - v0, np.int32)
    rc = lib().orc_desired_range(n, v0, v1, _p(offw), _p(nbrw), _p(ww), _p(k),
                                 p, q, _p(L), _p(K), _p(D))
    _check(rc, "desired")
    return D


class Scratch:
    """The oracle's per-vertex aggregation scratch for an n-vertex graph, made
    (and its pages touched) once, for many desired_window calls."""

    def __init__(self, n):
        self.n = n
        self.h = lib().orc_scratch_new(n)
        if not self.h:
            raise MemoryError("oracle scratch")

    def close(self):
        if self.h:
            lib().orc_scratch_free(self.h)
            self.h = None

    def __del__(self):
        self.close()


def desired_window(n, v0, v1, offw, nbrw, ww, k, p, q, L, K, scratch=None):
    """As desired(), with rows [v0, v1) already cut out as a CSR window;
    `scratch` (a Scratch of n) avoids re-making the scratch per call."""
    offw = _c(offw, np.int64)
    nbrw = _c(nbrw, np.int32)
    ww = _c(ww, np.int64)
    k = _c(k, np.int64)
    L = _c(L, np.int32)
    K = _c(K, np.int64)
    D = np.empty(v1 - v0, np.int32)
    if scratch is not None:
        assert scratch.n == n
        rc = lib().orc_desired_scratch(scratch.h, n, v0, v1, _p(offw), _p(nbrw), _p(ww),
                                       _p(k), p, q, _p(L), _p(K), _p(D))
    else:
        rc = lib().orc_desired_range(n, v0, v1, _p(offw), _p(nbrw), _p(ww), _p(k),
                                     p, q, _p(L), _p(K), _p(D))
    _check(rc, "desired")
    return D


def desired_list(n, verts, off_l, nbr_l, w_l, k, p, q, L, K):
    """Desired cluster of each listed vertex; its rows given as a compact CSR."""
    verts = _c(verts, np.int64)
    off_l = _c(off_l, np.int64)
    nbr_l = _c(nbr_l, np.int32)
    w_l = np.ones(len(nbr_l), np.int64) if w_l is None else _c(w_l, np.int64)
    k = _c(k, np.int64)
    L = _c(L, np.int32)
    K = _c(K, np.int64)
    D = np.empty(len(verts), np.int32)
    rc = lib().orc_desired_list(n, len(verts), _p(verts), _p(off_l), _p(nbr_l), _p(w_l), _p(k),
                                p, q, _p(L), _p(K), _p(D))
    _check(rc, "desired_list")
    return D


def compress(off, nbr, w, k, L):
    """Compress (Sec. 3.1): returns (map, off2, nbr2, w2, k2)."""
    off, nbr, w = _graph(off, nbr, w)
    n = len(off) - 1
    k = _c(k, np.int64)
    L = _c(L, np.int32)
    mp = np.empty(n, np.int32)
    n2 = C.c_int64()
    nnz2 = C.c_int64()
    po = C.c_void_p()
    pn = C.c_void_p()
    pw = C.c_void_p()
    pk = C.c_void_p()
    rc = lib().orc_compress(n, _p(off), _p(nbr), _p(w), _p(k), _p(L), _p(mp),
                            C.byref(n2), C.byref(nnz2), C.byref(po),
                            C.byref(pn), C.byref(pw), C.byref(pk))
    _check(rc, "compress")

    def take(ptr, cnt, ct, dt):
        if cnt == 0:
            out = np.empty(0, dt)
        else:
            out = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ct)),
                                        shape=(cnt,)).astype(dt, copy=True)
        lib().orc_free(ptr)
        return out

    off2 = take(po, n2.value + 1, C.c_int64, np.int64)
    nbr2 = take(pn, nnz2.value, C.c_int32, np.int32)
    w2 = take(pw, nnz2.value, C.c_int64, np.int64)
    k2 = take(pk, n2.value, C.c_int64, np.int64)
    return mp, off2, nbr2, w2, k2


TRACE_COLUMNS = ("level", "phase", "round", "vprime", "entries", "moved", "held")


def cluster(off, nbr, w, p, q, mode=NODEW_UNIT, k=None, num_iter=10,
            max_levels=64, refine=True, vset=VSET_NBR_VERTICES, coin=False, seed=0,
            trace=False, max_rounds=100000):
    """Parallel-CC (Algorithm 1, synchronous; coin=True adds the seeded
    symmetry-breaking coin of the library's LCC_SCHED_COIN schedule).

    Returns (labels, num, den, stats): the objective is CC = num / den exactly
    (den = q, or q * 2m in DEGREE mode); stats = (levels, rounds, edges).
    With trace=True a fifth element holds one row per best-move round
    (TRACE_COLUMNS): depth, phase (1 = refinement after Flatten), round of
    the call, |V'|, entries scanned, vertices moved, vertices held back."""
    off, nbr, w = _graph(off, nbr, w)
    n = len(off) - 1
    kk = _c(k, np.int64) if k is not None else np.zeros(1, np.int64)
    labels = np.empty(n, np.int32)
    hi = C.c_int64()
    lo = C.c_uint64()
    den = C.c_int64()
    st = np.zeros(3, np.int64)
    buf = np.zeros((max_rounds if trace else 1, len(TRACE_COLUMNS)), np.int64)
    tl = C.c_int64()
    rc = lib().orc_cluster(n, _p(off), _p(nbr), _p(w), _p(kk), mode, p, q,
                           num_iter, max_levels, int(bool(refine)), vset,
                           int(bool(coin)), seed & ((1 << 64) - 1),
                           _p(labels), C.byref(hi), C.byref(lo), C.byref(den),
                           _p(st), _p(buf) if trace else None,
                           max_rounds if trace else 0, C.byref(tl))
    _check(rc, "cluster")
    v = _i128(hi.value, lo.value)
    if v >= 1 << 127:
        v -= 1 << 128
    out = (labels, v, den.value, tuple(int(x) for x in st))
    if trace:
        if tl.value > max_rounds:
            raise ValueError("more than %d rounds; raise max_rounds" % max_rounds)
        out = out + (buf[:tl.value].copy(),)
    return out


def sequential_cc(off, nbr, w, p, q, mode=NODEW_UNIT, k=None, seed=0,
                  max_passes=1000, max_levels=64):
    """Sequential-CC (Sec. 3.1, Algorithm 2): random-order local moving until a
    pass moves nothing, then Compress, recursion and Flatten.

    Returns (labels, num, den, stats) with CC = num / den exactly and
    stats = (levels, passes, moves)."""
    off, nbr, w = _graph(off, nbr, w)
    n = len(off) - 1
    kk = _c(k, np.int64) if k is not None else np.zeros(1, np.int64)
    labels = np.empty(max(n, 1), np.int32)
    hi, lo, den = C.c_int64(), C.c_uint64(), C.c_int64()
    st = np.zeros(3, np.int64)
    rc = lib().orc_sequential_cc(n, _p(off), _p(nbr), _p(w), _p(kk), mode, p, q,
                                 seed & ((1 << 64) - 1), max_passes, max_levels,
                                 _p(labels), C.byref(hi), C.byref(lo), C.byref(den),
                                 _p(st))
    _check(rc, "sequential_cc")
    v = _i128(hi.value, lo.value)
    if v >= 1 << 127:
        v -= 1 << 128
    return labels[:n], v, den.value, tuple(int(x) for x in st)


def best_moves(off, nbr, w, k, p, q, L, num_iter, vset=VSET_NBR_VERTICES, coin=False,
               seed=0):
    """Best-Moves on one level from labels L (modified copy returned)."""
    off, nbr, w = _graph(off, nbr, w)
    k = _c(k, np.int64)
    L = _c(L, np.int32).copy()
    rounds = C.c_int64()
    rc = lib().orc_best_moves(len(off) - 1, _p(off), _p(nbr), _p(w), _p(k), p,
                              q, num_iter, vset, int(bool(coin)), seed & ((1 << 64) - 1),
                              _p(L), C.byref(rounds))
    if rc < 0:
        _check(-rc, "best_moves")
    return L, bool(rc), rounds.value


def sequential_sweep(off, nbr, w, k, p, q, L, max_moves):
    off, nbr, w = _graph(off, nbr, w)
    k = _c(k, np.int64)
    L = _c(L, np.int32).copy()
    mv = lib().orc_sequential_sweep(len(off) - 1, _p(off), _p(nbr), _p(w),
                                    _p(k), p, q, _p(L), max_moves)
    if mv < 0:
        raise MemoryError("oracle sweep failed")
    return L, mv


def weighted_degrees(off, w32=None):
    """Modularity node weights k_v = sum_u w_uv (Sec. 2) from int32 weights
    (None = unweighted); returns (k, 2m)."""
    off = _c(off, np.int64)
    n = len(off) - 1
    k = np.empty(n, np.int64)
    wp = None if w32 is None else _c(w32, np.int32)
    tot = lib().orc_weighted_degrees_i32(n, _p(off), None if wp is None else _p(wp), _p(k))
    return k, int(tot)
