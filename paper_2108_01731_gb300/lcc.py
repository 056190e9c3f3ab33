"""ctypes binding of liblcc.so (include/lcc.h), with the same entry-point names.

Argument marshalling only: every step of the clustering runs inside the CUDA
library.  Arrays may be numpy arrays (host memory) or torch CUDA tensors
(device memory); the memory space is passed to the library accordingly.
Loading fails loudly when the library has not been built.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblcc.so")

LCC_OK = 0
LCC_ERR_INVALID = 1
LCC_ERR_NOT_SYMMETRIC = 2
LCC_ERR_SELF_LOOP = 3
LCC_ERR_OOM = 4
LCC_ERR_OVERFLOW = 5
LCC_ERR_TIMEOUT = 6
LCC_ERR_CUDA = 7
LCC_ERR_BUSY = 8
LCC_ERR_CANCELLED = 9

LCC_NODEW_UNIT, LCC_NODEW_DEGREE, LCC_NODEW_CUSTOM = 0, 1, 2
LCC_VSET_ALL, LCC_VSET_NBR_VERTICES, LCC_VSET_NBR_CLUSTERS = 0, 1, 2
LCC_MEM_HOST, LCC_MEM_DEVICE = 0, 1
LCC_SCHED_TIMING = 1
LCC_SCHED_MARK_ONLY = 2
LCC_SCHED_COIN = 4


class lcc_schedule(C.Structure):
    _fields_ = [("num_iter", C.c_int32), ("max_levels", C.c_int32),
                ("refine", C.c_int32), ("vset", C.c_int32), ("sync", C.c_int32),
                ("flags", C.c_int32), ("seed", C.c_uint64)]


class lcc_tuning(C.Structure):
    _fields_ = [("warp_max", C.c_int32), ("fuse_small", C.c_int32), ("prefetch", C.c_int32),
                ("pregather", C.c_int32), ("part_min", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class lcc_stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("rounds_total", C.c_int32),
                ("edges_scanned", C.c_int64), ("vertices_scanned", C.c_int64),
                ("candidates", C.c_int64), ("num_clusters", C.c_int64),
                ("obj_num_hi", C.c_int64), ("obj_num_lo", C.c_uint64),
                ("obj_den", C.c_int64), ("objective", C.c_double),
                ("ms_bestmove", C.c_double), ("ms_round_other", C.c_double),
                ("ms_contract", C.c_double), ("ms_other", C.c_double),
                ("ms_total", C.c_double), ("bytes_bestmove", C.c_int64),
                ("pairs_sorted", C.c_int64), ("kernel_launches", C.c_int64),
                ("ms_bucket", C.c_double * 16), ("bucket_entries", C.c_int64 * 16),
                ("bucket_vertices", C.c_int64 * 16), ("bytes_contract_min", C.c_int64),
                ("calls", C.c_int64), ("calls_capped", C.c_int64), ("ms_gather", C.c_double)]


class lcc_round(C.Structure):
    _fields_ = [("level", C.c_int32), ("phase", C.c_int32), ("round", C.c_int32),
                ("pad", C.c_int32), ("vprime", C.c_int64), ("entries", C.c_int64),
                ("moved", C.c_int64), ("held", C.c_int64)]


ROUND_COLUMNS = ("level", "phase", "round", "vprime", "entries", "moved", "held")


class lcc_server_cfg(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32),
                ("reserved", C.c_int32), ("sched", lcc_schedule)]


class lcc_job(C.Structure):
    _fields_ = [("offsets", C.c_void_p), ("nbrs", C.c_void_p),
                ("weights", C.c_void_p), ("n", C.c_int64), ("nnz", C.c_int64),
                ("lambda_p", C.c_int64), ("lambda_q", C.c_int64),
                ("mode", C.c_int32), ("inject_fault_tick", C.c_int32)]


class LccError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (status_str(status), status, msg))
        self.status = status


_lib = None
P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
_SIGS = {
    "lcc_load_csr": [P, P, P, I64, I64, P, I32, P, P],
    "lcc_graph_info": [P, P, P],
    "lcc_free_graph": [P],
    "lcc_cluster": [P, I64, I64, I32, P, P, I32, P, P],
    "lcc_cluster_trace": [P, I64, I64, I32, P, P, I32, P, P, P, I64, P],
    "lcc_desired": [P, I64, I64, I32, P, P, P],
    "lcc_best_moves": [P, I64, I64, I32, I32, I32, P, P, P],
    "lcc_compress": [P, I32, P, P, P],
    "lcc_graph_export": [P, P, P, P, P],
    "lcc_objective": [P, I64, I64, I32, P, P, P, P],
    "lcc_desired_noalloc": [P, P, P, P, I64, I64, I64, P, P, P, P],
    "lcc_cluster_batch": [P, I32, P, P, P, P, P, P],
    "lcc_server_create": [P, P],
    "lcc_submit": [P, P, P],
    "lcc_poll": [P, U64, P, P, P],
    "lcc_cancel": [P, U64],
    "lcc_server_wait_idle": [P, I64],
    "lcc_server_counters": [P, P],
    "lcc_server_destroy": [P],
    "lcc_get_tuning": [I32, P],
    "lcc_set_tuning": [I32, P],
    "lcc_autotune": [P, I64, I64, I32, C.c_char_p, P],
    "lcc_status_str": [I32],
    "lcc_last_error": [],
}


def load():
    """Load liblcc.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblcc.so is not built (%s); run __graft_entry__.build()"
                               % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            if name == "lcc_free_graph":
                fn.restype = None
            elif name in ("lcc_status_str", "lcc_last_error"):
                fn.restype = C.c_char_p
            else:
                fn.restype = C.c_int
        _lib = lib
    return _lib


def status_str(st):
    try:
        return load().lcc_status_str(st).decode()
    except Exception:
        return "status"


def _check(st):
    if st != LCC_OK:
        raise LccError(st, load().lcc_last_error().decode())


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a, dtype):
    """(pointer, keepalive) of a contiguous array of the given numpy dtype."""
    if a is None:
        return None, None
    if _is_torch_cuda(a):
        import torch
        tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}[dtype]
        a = a.contiguous().to(tdt)
        return C.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(a, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), a


def schedule(num_iter=10, max_levels=64, refine=True, vset=LCC_VSET_NBR_VERTICES,
             timing=False, mark_only=False, coin=False, seed=0):
    """An lcc_schedule: rounds per Best-Moves call, level cap, refinement, the
    V' rule, per-phase timing, V' by marking only, and the seeded
    symmetry-breaking coin (LCC_SCHED_COIN; results are deterministic for a
    seed)."""
    flags = ((LCC_SCHED_TIMING if timing else 0) | (LCC_SCHED_MARK_ONLY if mark_only else 0)
             | (LCC_SCHED_COIN if coin else 0))
    return lcc_schedule(int(num_iter), int(max_levels), int(bool(refine)), int(vset), 1, flags,
                        int(seed) & ((1 << 64) - 1))


class Graph:
    """Owns an lcc_graph handle."""

    def __init__(self, handle, n, nnz):
        self.handle = handle
        self.n = n
        self.nnz = nnz

    def free(self):
        if self.handle:
            load().lcc_free_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def lcc_load_csr(off, nbr, w=None, node_w=None, stream=None):
    """Copy a CSR graph into the library (numpy = host, torch CUDA = device)."""
    lib = load()
    dev = _is_torch_cuda(off)
    po, ko = _ptr(off, np.int64)
    pn, kn = _ptr(nbr, np.int32)
    pw, kw = _ptr(w, np.int32)
    pk, kk = _ptr(node_w, np.int64)
    n = (off.numel() if dev else len(off)) - 1
    nnz = nbr.numel() if dev else len(nbr)
    h = C.c_void_p()
    st = C.c_void_p(int(stream)) if stream else None
    _check(lib.lcc_load_csr(po, pn, pw, n, nnz, pk, LCC_MEM_DEVICE if dev else LCC_MEM_HOST,
                            st, C.byref(h)))
    return Graph(h, n, nnz)


def lcc_graph_info(g):
    n = C.c_int64()
    nnz = C.c_int64()
    _check(load().lcc_graph_info(g.handle, C.byref(n), C.byref(nnz)))
    return n.value, nnz.value


def lcc_free_graph(g):
    g.free()


def _stats_dict(s):
    d = {f: getattr(s, f) for f, _ in lcc_stats._fields_}
    d["ms_bucket"] = list(d["ms_bucket"])
    d["bucket_entries"] = list(d["bucket_entries"])
    d["bucket_vertices"] = list(d["bucket_vertices"])
    num = (d["obj_num_hi"] << 64) | d["obj_num_lo"]
    if num >= 1 << 127:
        num -= 1 << 128
    d["obj_num"] = num
    return d


def lcc_cluster(g, lambda_p, lambda_q, mode=LCC_NODEW_UNIT, sched=None, labels_out=None):
    """Parallel-CC.  Returns (labels, objective, stats dict).  labels_out may
    be a torch CUDA int32 tensor to keep the labels on the device."""
    lib = load()
    sched = sched or schedule()
    if labels_out is None:
        labels_out = np.empty(g.n, np.int32)
    dev = _is_torch_cuda(labels_out)
    pl = C.c_void_p(labels_out.data_ptr()) if dev else labels_out.ctypes.data_as(C.c_void_p)
    obj = C.c_double()
    st = lcc_stats()
    _check(lib.lcc_cluster(g.handle, int(lambda_p), int(lambda_q), int(mode), C.byref(sched),
                           pl, LCC_MEM_DEVICE if dev else LCC_MEM_HOST, C.byref(obj),
                           C.byref(st)))
    return labels_out, obj.value, _stats_dict(st)


def lcc_cluster_trace(g, lambda_p, lambda_q, mode=LCC_NODEW_UNIT, sched=None, max_rounds=100000):
    """lcc_cluster plus its per-round record.  Returns (labels, objective,
    stats dict, rows) with one row per Best-Moves round (ROUND_COLUMNS):
    depth, phase (1 = refinement), round of the call, |V'|, entries scanned,
    vertices moved, vertices held back by the coin."""
    lib = load()
    sched = sched or schedule()
    labels = np.empty(g.n, np.int32)
    obj = C.c_double()
    st = lcc_stats()
    buf = (lcc_round * max_rounds)()
    tl = C.c_int64()
    _check(lib.lcc_cluster_trace(g.handle, int(lambda_p), int(lambda_q), int(mode),
                                 C.byref(sched), labels.ctypes.data_as(C.c_void_p),
                                 LCC_MEM_HOST, C.byref(obj), C.byref(st), buf, max_rounds,
                                 C.byref(tl)))
    if tl.value > max_rounds:
        raise ValueError("more than %d rounds; raise max_rounds" % max_rounds)
    rows = np.array([[getattr(buf[i], f) for f in ROUND_COLUMNS] for i in range(tl.value)],
                    np.int64).reshape(-1, len(ROUND_COLUMNS))
    return labels, obj.value, _stats_dict(st), rows


def lcc_desired(g, lambda_p, lambda_q, mode, labels, frontier=None):
    lib = load()
    labels = np.ascontiguousarray(labels, np.int32)
    fr = None if frontier is None else np.ascontiguousarray(frontier, np.uint8)
    out = np.empty(g.n, np.int32)
    _check(lib.lcc_desired(g.handle, int(lambda_p), int(lambda_q), int(mode),
                           labels.ctypes.data_as(C.c_void_p),
                           None if fr is None else fr.ctypes.data_as(C.c_void_p),
                           out.ctypes.data_as(C.c_void_p)))
    return out


def lcc_best_moves(g, lambda_p, lambda_q, mode, num_iter, vset, labels):
    lib = load()
    L = np.ascontiguousarray(labels, np.int32).copy()
    rounds = C.c_int32()
    moved = C.c_int32()
    _check(lib.lcc_best_moves(g.handle, int(lambda_p), int(lambda_q), int(mode), int(num_iter),
                              int(vset), L.ctypes.data_as(C.c_void_p), C.byref(rounds),
                              C.byref(moved)))
    return L, bool(moved.value), rounds.value


def lcc_compress(g, mode, labels):
    lib = load()
    L = np.ascontiguousarray(labels, np.int32)
    mp = np.empty(g.n, np.int32)
    h = C.c_void_p()
    _check(lib.lcc_compress(g.handle, int(mode), L.ctypes.data_as(C.c_void_p),
                            mp.ctypes.data_as(C.c_void_p), C.byref(h)))
    n, nnz = C.c_int64(), C.c_int64()
    _check(lib.lcc_graph_info(h, C.byref(n), C.byref(nnz)))
    return mp, Graph(h, n.value, nnz.value)


def lcc_graph_export(g):
    lib = load()
    off = np.empty(g.n + 1, np.int64)
    nbr = np.empty(g.nnz, np.int32)
    w = np.empty(g.nnz, np.int64)
    k = np.empty(g.n, np.int64)
    _check(lib.lcc_graph_export(g.handle, off.ctypes.data_as(C.c_void_p),
                                nbr.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p),
                                k.ctypes.data_as(C.c_void_p)))
    return off, nbr, w, k


def lcc_objective(g, lambda_p, lambda_q, mode, labels):
    """Exact objective: returns (num, den) with CC = num / den."""
    lib = load()
    L = np.ascontiguousarray(labels, np.int32)
    hi, lo, den = C.c_int64(), C.c_uint64(), C.c_int64()
    _check(lib.lcc_objective(g.handle, int(lambda_p), int(lambda_q), int(mode),
                             L.ctypes.data_as(C.c_void_p), C.byref(hi), C.byref(lo),
                             C.byref(den)))
    num = (hi.value << 64) | lo.value
    if num >= 1 << 127:
        num -= 1 << 128
    return num, den.value


def _tuning_dict(t):
    return {"warp_max": t.warp_max, "fuse_small": t.fuse_small, "prefetch": t.prefetch,
            "pregather": t.pregather, "part_min": t.part_min}


def lcc_get_tuning(device=0):
    """The kernel tuning used on `device`: {"warp_max", "fuse_small", "prefetch",
    "pregather", "part_min"}."""
    t = lcc_tuning()
    _check(load().lcc_get_tuning(int(device), C.byref(t)))
    return _tuning_dict(t)


def lcc_set_tuning(device, warp_max, fuse_small=1, prefetch=0, pregather=1, part_min=8192):
    t = lcc_tuning()
    t.warp_max = int(warp_max)
    t.fuse_small = int(fuse_small)
    t.prefetch = int(prefetch)
    t.pregather = int(pregather)
    t.part_min = int(part_min)
    _check(load().lcc_set_tuning(int(device), C.byref(t)))


def lcc_autotune(g, lambda_p, lambda_q, mode, cache_path=None):
    """Times tunings on three best-move rounds of g, one field at a time
    (warp_max, then fuse_small, prefetch, pregather and part_min), or reads the cache file's line
    for this device, and applies the fastest; returns it as a dict."""
    t = lcc_tuning()
    path = cache_path.encode() if cache_path else None
    _check(load().lcc_autotune(g.handle, int(lambda_p), int(lambda_q), int(mode), path,
                               C.byref(t)))
    return _tuning_dict(t)


def lcc_desired_noalloc(off, nbr, w, k, lambda_p, lambda_q, labels, K, out, stream=None):
    """Allocation-free evaluation on device tensors (all torch CUDA tensors;
    `out` int32[n] receives the desired clusters).  The library allocates
    nothing for this call; see include/lcc.h."""
    n = off.numel() - 1
    st = C.c_void_p(int(stream)) if stream else None

    def p(t):
        return None if t is None else C.c_void_p(t.data_ptr())
    _check(load().lcc_desired_noalloc(p(off), p(nbr), p(w), p(k), n, int(lambda_p),
                                      int(lambda_q), p(labels), p(K), p(out), st))
    return out


def lcc_cluster_batch(graphs, lambda_p, lambda_q, mode, sched=None):
    lib = load()
    cnt = len(graphs)
    sched = sched or schedule()
    hs = (C.c_void_p * cnt)(*[g.handle for g in graphs])
    ps = np.ascontiguousarray(lambda_p, np.int64)
    qs = np.ascontiguousarray(lambda_q, np.int64)
    ms = np.ascontiguousarray(mode, np.int32)
    outs = [np.empty(g.n, np.int32) for g in graphs]
    po = (C.c_void_p * cnt)(*[o.ctypes.data_as(C.c_void_p) for o in outs])
    objs = np.empty(cnt, np.float64)
    _check(lib.lcc_cluster_batch(hs, cnt, ps.ctypes.data_as(C.c_void_p),
                                 qs.ctypes.data_as(C.c_void_p), ms.ctypes.data_as(C.c_void_p),
                                 C.byref(sched), po, objs.ctypes.data_as(C.c_void_p)))
    return outs, objs


class Server:
    """Serving engine handle (lcc_server_create / lcc_submit / lcc_poll)."""

    def __init__(self, hbm_budget_bytes, max_slots, sched=None):
        lib = load()
        cfg = lcc_server_cfg(int(hbm_budget_bytes), int(max_slots), 0, sched or schedule())
        self.h = C.c_void_p()
        _check(lib.lcc_server_create(C.byref(cfg), C.byref(self.h)))
        self.sizes = {}

    def submit(self, off, nbr, w, lambda_p, lambda_q, mode, inject_fault_tick=0):
        """Queue a job; inject_fault_tick > 0 is the fault-injection hook of
        lcc_job (the job fails at the start of that engine tick)."""
        off = np.ascontiguousarray(off, np.int64)
        nbr = np.ascontiguousarray(nbr, np.int32)
        w = None if w is None else np.ascontiguousarray(w, np.int32)
        job = lcc_job(off.ctypes.data, nbr.ctypes.data, None if w is None else w.ctypes.data,
                      len(off) - 1, len(nbr), int(lambda_p), int(lambda_q), int(mode),
                      int(inject_fault_tick))
        t = C.c_uint64()
        _check(load().lcc_submit(self.h, C.byref(job), C.byref(t)))
        self.sizes[t.value] = len(off) - 1
        return t.value

    def poll(self, ticket):
        """None while running; else (labels, objective, latency_ms)."""
        n = self.sizes[ticket]
        out = np.empty(n, np.int32)
        obj = C.c_double()
        lat = C.c_double()
        st = load().lcc_poll(self.h, C.c_uint64(ticket), out.ctypes.data_as(C.c_void_p),
                             C.byref(obj), C.byref(lat))
        if st == LCC_ERR_BUSY:
            return None
        del self.sizes[ticket]
        _check(st)
        return out, obj.value, lat.value

    def cancel(self, ticket):
        _check(load().lcc_cancel(self.h, C.c_uint64(ticket)))

    def wait_idle(self, timeout_ms=600000):
        _check(load().lcc_server_wait_idle(self.h, int(timeout_ms)))

    def counters(self):
        out = np.zeros(5, np.int64)
        _check(load().lcc_server_counters(self.h, out.ctypes.data_as(C.c_void_p)))
        return dict(zip(["done", "ticks", "peak_bytes", "peak_jobs", "rejected"],
                        [int(x) for x in out]))

    def close(self):
        if self.h:
            _check(load().lcc_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
