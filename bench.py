#!/usr/bin/env python3
"""Benchmark of the LambdaCC best-move / contraction path on GB300.

Workload (default): R-MAT graph, 2^26 vertices, exactly 2^30 undirected edges
stored in both directions (2^31 CSR entries, int32 ids and int32 weights,
int64 offsets), modularity mode (k = degree, lambda = 1/2m), full multi-level
Parallel-CC (Algorithm 1, synchronous, 10 rounds per Best-Moves, refinement
on).  One step = one whole lcc_cluster call on the resident graph: every
best-move round, every contraction, flatten/refine, canonical labels and the
exact objective.

Metric: best-move GEdges/s = directed CSR entries scanned by the best-move
rounds of a step (the sum of deg(v) over every evaluated vertex) / step time.
`roofline` reports the best-move kernels' algorithmic bytes / their device
time against the measured HBM copy bandwidth.  `e2e` times the same call with
the CSR in pinned host memory (load + validate + cluster + labels to host).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched by torchrun, one replica of the workload per GPU (the
path has no exchange step), value = sum of edges over ranks / max time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Degree buckets of the best-move kernels (row lengths), as in lcc_stats.
BUCKETS = ["<=4", "<=8", "<=16", "<=32", "<=64", "<=128", "<=256", "<=1024", "<=2048",
           "<=4096", "<=8192", "<=16384", "<=32768", "<=65536", "<=131072", ">131072"]

WORKLOADS = {
    # name: generator, node-weight mode, lambda p/q, rounds per Best-Moves
    "rmat26": dict(kind="rmat", scale=26, m=1 << 30, mode=1, p=1, q=1, num_iter=10,
                   desc="R-MAT a=0.57 b=c=0.19 d=0.05, 2^26 vertices, 2^30 undirected edges "
                        "(2^31 CSR entries), int32 weights, modularity (gamma=1)"),
    "chunglu20": dict(kind="chunglu", n=1 << 20, beta=2.1, deg=32, mode=1, p=1, q=1,
                      num_iter=10, desc="Chung-Lu beta=2.1, 2^20 vertices, ~16M edges, "
                                        "modularity (gamma=1)"),
    "rmat24": dict(kind="rmat", scale=24, m=1 << 28, mode=1, p=1, q=1, num_iter=10,
                   desc="R-MAT a=0.57 b=c=0.19 d=0.05, 2^24 vertices, 2^28 undirected edges "
                        "(2^29 CSR entries), modularity (gamma=1): the benchmark graph at a "
                        "quarter of its size, for kernel profiles"),
    "rmat22": dict(kind="rmat", scale=22, m=1 << 26, mode=1, p=1, q=1, num_iter=10,
                   desc="R-MAT a=0.57 b=c=0.19 d=0.05, 2^22 vertices, 2^26 undirected edges, "
                        "modularity (gamma=1)"),
    # the paper's R-MAT density sweep (Sec. 4, scalability; its generator's
    # a=0.5, b=c=0.1, d=0.3) at 2^20 vertices: m = 5n, 50n and n^1.5
    "rmat20_5n": dict(kind="rmat", scale=20, m=5 << 20, abc=(0.5, 0.1, 0.1), mode=1, p=1, q=1,
                      num_iter=10, desc="R-MAT a=0.5 b=c=0.1 d=0.3, 2^20 vertices, m = 5n, "
                                        "modularity (gamma=1)"),
    "rmat20_50n": dict(kind="rmat", scale=20, m=50 << 20, abc=(0.5, 0.1, 0.1), mode=1, p=1,
                       q=1, num_iter=10, desc="R-MAT a=0.5 b=c=0.1 d=0.3, 2^20 vertices, "
                                               "m = 50n, modularity (gamma=1)"),
    "rmat20_n15": dict(kind="rmat", scale=20, m=1 << 30, abc=(0.5, 0.1, 0.1), mode=1, p=1, q=1,
                       num_iter=10, desc="R-MAT a=0.5 b=c=0.1 d=0.3, 2^20 vertices, "
                                         "m = n^1.5 = 2^30, modularity (gamma=1)"),
    "sbm1e4": dict(kind="sbm", mode=0, p=1, q=100, num_iter=20,
                   desc="planted partition, 100 blocks of 100, p_in 0.05, p_out 0.0005, "
                        "lambda 1/100, 20 rounds"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat26")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--serving", type=int, default=160,
                    help="graphs of the serving stream to run (0 = skip)")
    ap.add_argument("--serving-large", type=int, default=3000,
                    help="graphs of the stream for one more saturation run in which the "
                         "HBM admission budget binds (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-twin", action="store_true",
                    help="skip the OpenMP CPU twin's timed first round")
    ap.add_argument("--no-coin", action="store_true",
                    help="skip the extra step with the symmetry-breaking coin")
    ap.add_argument("--sweep", action="store_true",
                    help="also run the R-MAT density sweep (2^20 vertices, m = 5n, 50n, n^1.5) "
                         "and report it as density_sweep")
    ap.add_argument("--tuning-cache", default=None,
                    help="tuning file for lcc_autotune: reuse this GPU's line if present, "
                         "else measure and append (keeps the routing fixed across runs)")
    return ap.parse_args()


# ---------------------------------------------------------- distributed --

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_scalar(x, world, op, device):
    """max/sum of a float over ranks (identity at world 1)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------- inputs --

def make_graph(wl, device):
    from paper_2108_01731_gb300 import inputs as I
    seed = I.BASE_SEED
    if wl["kind"] == "rmat":
        a, b, c = wl.get("abc", (0.57, 0.19, 0.19))
        return I.rmat(wl["scale"], wl["m"], a=a, b=b, c=c, seed=seed + 4, device=device)
    if wl["kind"] == "chunglu":
        return I.chung_lu(wl["n"], wl["beta"], wl["deg"], seed=seed + 2, device=device)
    if wl["kind"] == "sbm":
        return I.sbm([100] * 100, 0.05, 0.0005, seed=seed + 1, device=device)
    raise ValueError(wl["kind"])


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def random_gather_rate(dev):
    """Random-access ceiling of this GPU for the best-move gathers: 8-byte words
    gathered at uniform random positions of a 512 MB table (PyTorch's index
    kernel; every best-move entry gathers one such word), in gathers/s."""
    import torch
    tab = torch.arange(1 << 26, dtype=torch.int64, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(0x1CC02108)
    idx = torch.randint(0, 1 << 26, (1 << 28,), generator=gen, device=dev)
    out = torch.empty(1 << 28, dtype=torch.int64, device=dev)
    for _ in range(2):
        torch.index_select(tab, 0, idx, out=out)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        torch.index_select(tab, 0, idx, out=out)
    e1.record()
    torch.cuda.synchronize()
    rate = 5 * (1 << 28) / (e0.elapsed_time(e1) / 1e3)
    del tab, idx, out
    torch.cuda.empty_cache()
    return rate


# DRAM bytes per scanned entry of the best-move kernels (dram__bytes_read.sum
# + dram__bytes_write.sum over every best-move launch of one step, per
# scanned entry), from one ncu capture of the R-MAT 2^22 step (the capture and
# its scaling are recorded under profiles/bestmove_dram_rmat22.md), the
# sha256[:16] of the k_round.cu it was taken on and the pregather tuning it
# ran with.  The figure is reported only while that source is unchanged and
# the timed run uses the same pregather choice (the flat gather pass moves
# about 12 bytes per entry of its own).
BESTMOVE_TRAFFIC = {"k_round.cu": "83f4e7da07330cea", "pregather": 1,
                    "dram_bytes_per_entry": 39.16}


def profile_traffic(src=None, measured=None, pregather=None):
    """DRAM bytes per scanned entry of the best-move kernels, if measured on
    the current kernel source with the run's pregather choice (else None)."""
    measured = measured or BESTMOVE_TRAFFIC
    src = src or os.path.join(ROOT, "paper_2108_01731_gb300", "csrc", "k_round.cu")
    if not measured.get("k_round.cu") or not os.path.exists(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != measured["k_round.cu"]:
        return None
    if pregather is not None and measured.get("pregather") not in (None, pregather):
        return None
    return measured["dram_bytes_per_entry"]


# ----------------------------------------------------------------- clocks --

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200",
                                       "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle --

def oracle_sample(host, wl, seconds):
    """Times the CPU oracle on the first best-move round of the same graph for
    a window of vertices [0, X) sized to take about `seconds`.  Returns
    (GEdges/s, description, oracle seconds)."""
    import numpy as np
    import oracle as O
    off = host["off"]
    n = len(off) - 1
    if wl["mode"] == 1:
        k, two_m = O.weighted_degrees(off, host["w"])
        p, q = wl["p"], wl["q"] * two_m
    else:
        k = np.ones(n, np.int64)
        p, q = wl["p"], wl["q"]
    L = np.arange(n, dtype=np.int32)
    K = k
    scratch = O.Scratch(n)  # made once, outside the timed windows
    x = min(n, 4096)
    done_edges, done_t, v0 = 0, 0.0, 0
    while done_t < seconds and v0 < n:
        v1 = min(n, v0 + x)
        e0, e1 = int(off[v0]), int(off[v1])
        offw = off[v0:v1 + 1] - off[v0]
        nbrw = host["nbr"][e0:e1]
        ww = (host["w"][e0:e1].astype(np.int64) if host["w"] is not None
              else np.ones(e1 - e0, np.int64))
        t0 = time.perf_counter()
        O.desired_window(n, v0, v1, offw, nbrw, ww, k, p, q, L, K, scratch=scratch)
        dt = time.perf_counter() - t0
        done_edges += e1 - e0
        done_t += dt
        v0 = v1
        if dt < seconds / 8:
            x *= 2
    return (done_edges / done_t / 1e9, "first best-move round of the same graph, vertices "
            "[0, %d) (%d of %d vertices, %d entries scanned), single-threaded oracle"
            % (v0, v0, n, done_edges), done_t)


# --------------------------------------------------- symmetry-breaking coin --

def modularity(st, q):
    """Q = CC / 2m of a modularity-mode run (obj_den = q 2m)."""
    return st["obj_num"] / st["obj_den"] / (st["obj_den"] / q)


def coin_leg(run, wl):
    """One whole step with the symmetry-breaking coin (LCC_SCHED_COIN, seed 0)
    on the resident graph, beside the plain synchronous steps: its device
    time, scanned entries, objective and clusters.  run() -> (ms, stats).
    Any failure is reported, not raised: the headline numbers have been taken
    before this leg runs."""
    try:
        ms, st = run()
    except Exception as e:  # noqa: BLE001
        return {"unavailable": "%s: %s" % (type(e).__name__, e)}
    out = {"schedule": "LCC_SCHED_COIN, seed 0", "ms_per_step": round(ms, 3),
           "edges_scanned": int(st["edges_scanned"]),
           "gedges_per_s": round(st["edges_scanned"] / (ms / 1e3) / 1e9, 4),
           "levels": int(st["levels"]), "rounds": int(st["rounds_total"]),
           "num_clusters": int(st["num_clusters"]), "objective": st["objective"]}
    if wl["mode"] == 1:
        out["modularity"] = modularity(st, wl["q"])
    return out


# ------------------------------------------------------- CPU OpenMP twin --

def twin_round(host, wl, gpu_desired):
    """Times the OpenMP CPU twin on the first full-frontier best-move round of
    the same graph (every vertex, every host core) and compares its desired
    clusters with the GPU library's for that round (gpu_desired(labels), the
    library's lcc_desired on the resident graph)."""
    import numpy as np
    n = len(host["off"]) - 1
    try:
        import cpu_twin as T
        k = None if wl["mode"] == 1 else np.ones(n, np.int64)
        D, ent, secs, cores = T.first_round(host["off"], host["nbr"], host["w"], k,
                                            wl["p"], wl["q"])
    except Exception as e:  # no OpenMP toolchain or no host memory for it
        return {"unavailable": "%s: %s" % (type(e).__name__, e)}
    Dg = gpu_desired(np.arange(n, dtype=np.int32))
    return {"value": round(ent / secs / 1e9, 4), "unit": "GEdges/s", "cores": cores,
            "kind": "openmp twin (same synchronous schedule, all host cores)",
            "seconds": round(secs, 3),
            "sample": "first best-move round of the same graph over all %d vertices "
                      "(%d entries scanned)" % (n, ent),
            "desired_equal_gpu": bool(np.array_equal(D, Dg))}


def degree_shares(off):
    """Share of CSR entries in each degree bucket of the best-move kernels."""
    import numpy as np
    d = np.diff(off)
    tot = max(1, int(d.sum()))
    edges = [0, 4, 8, 16, 32, 256, 1024, 4096, None]
    names = ["<=4", "<=8", "<=16", "<=32", "<=256", "<=1024", "<=4096", ">4096"]
    out = {}
    for i, nm in enumerate(names):
        lo, hi = edges[i], edges[i + 1]
        m = (d > lo) if hi is None else ((d > lo) & (d <= hi))
        out[nm] = {"vertices": int(m.sum()), "entry_share": round(float(d[m].sum()) / tot, 4)}
    out["max_degree"] = int(d.max()) if len(d) else 0
    return out


def host_copy(g):
    import numpy as np
    out = {}
    for key in ("off", "nbr", "w"):
        t = g.get(key)
        out[key] = None if t is None else t.cpu().numpy()
    return out


# ---------------------------------------------------------------- serving --

def serving_bench(L, count, device, large=0):
    """Config-5 stream: the plain one-graph-per-call path against the
    continuous-batching server, on the first `count` graphs of the stream:
    graphs/s at saturation (every graph submitted at once) with its p50/p99,
    and p50/p99 under Poisson arrivals at 0.25 ... 8 times the plain path's
    rate.  With large > 0, the first `large` graphs of the stream also run
    through the server at saturation, which is long enough for the 120 GB
    admission budget to bind."""
    import numpy as np
    from paper_2108_01731_gb300 import inputs as I

    def make(k):
        out = []
        for i in range(k):
            g = I.serving_graph(i, device=device)
            out.append({x: (v.cpu().numpy() if hasattr(v, "cpu") else v) for x, v in g.items()
                        if x in ("off", "nbr", "n", "nnz")})
        return out

    mode = L.LCC_NODEW_DEGREE
    budget = 120 << 30

    def plain_run(graphs):
        t0 = time.perf_counter()
        labs = []
        for g in graphs:
            G = L.lcc_load_csr(g["off"], g["nbr"])
            lab, _, _ = L.lcc_cluster(G, 1, 1, mode)
            labs.append(lab)
            G.free()
        return labs, time.perf_counter() - t0

    def run_server(graphs, ref, rate):
        srv = L.Server(budget, 1 << 14)
        rs = np.random.default_rng(12345)
        gaps = rs.exponential(1.0 / rate, len(graphs)) if rate else np.zeros(len(graphs))
        t_start = time.perf_counter()
        tickets = []
        t_next = t_start
        for g, gap in zip(graphs, gaps):
            t_next += gap
            while time.perf_counter() < t_next:
                time.sleep(min(0.0005, max(0.0, t_next - time.perf_counter())))
            tickets.append(srv.submit(g["off"], g["nbr"], None, 1, 1, mode))
        srv.wait_idle(3600 * 1000)
        t_end = time.perf_counter()
        lats, same = [], True
        for t, r in zip(tickets, ref):
            lab, obj, lat = srv.poll(t)
            lats.append(lat)
            same &= bool(np.array_equal(lab, r))
        c = srv.counters()
        srv.close()
        return len(graphs) / (t_end - t_start), lats, same, c

    def pct(lats):
        return (round(float(np.percentile(lats, 50)), 3), round(float(np.percentile(lats, 99)), 3))

    graphs = make(count)
    plain, t_plain = plain_run(graphs)
    gps_plain = count / t_plain
    gps_batched, lats_sat, same_sat, c_sat = run_server(graphs, plain, 0)
    p50, p99 = pct(lats_sat)
    out = {"graphs": count, "config": "planted-partition stream, n log-uniform [100, 200000], "
                                      "5-500 communities, mean degree 8-64, modularity",
           "sample": "the first %d graphs of the 20,000-graph stream" % count,
           "plain_graphs_per_s": round(gps_plain, 3),
           "batched_graphs_per_s": round(gps_batched, 3),
           "batched_over_plain": round(gps_batched / gps_plain, 3),
           "labels_identical": same_sat,
           "saturation_p50_ms": p50, "saturation_p99_ms": p99,
           "peak_concurrent_jobs": c_sat["peak_jobs"], "budget_bytes": budget, "rates": []}
    for frac in (0.25, 0.5, 1.0, 2.0, 4.0, 8.0):
        rate = frac * gps_plain
        gps, lats, same, c = run_server(graphs, plain, rate)
        p50, p99 = pct(lats)
        out["rates"].append({"arrival_per_s": round(rate, 3), "x_plain": frac,
                             "graphs_per_s": round(gps, 3), "p50_ms": p50, "p99_ms": p99,
                             "labels_identical": same, "peak_concurrent_jobs": c["peak_jobs"]})
    if large > count:
        try:
            graphs = make(large)
            plain, t_plain = plain_run(graphs)
            gps, lats, same, c = run_server(graphs, plain, 0)
        except Exception as e:  # noqa: BLE001  (the longer stream is extra: reported)
            out["large_stream"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
            return out
        p50, p99 = pct(lats)
        out["large_stream"] = {"graphs": large,
                               "sample": "the first %d graphs of the 20,000-graph stream" % large,
                               "plain_graphs_per_s": round(large / t_plain, 3),
                               "batched_graphs_per_s": round(gps, 3),
                               "batched_over_plain": round(gps / (large / t_plain), 3),
                               "saturation_p50_ms": p50, "saturation_p99_ms": p99,
                               "labels_identical": same, "peak_concurrent_jobs": c["peak_jobs"],
                               "peak_resident_bytes": c["peak_bytes"],
                               "total_entries": int(sum(g["nnz"] for g in graphs))}
    return out


def density_sweep(L, dev, steps):
    """The paper's scalability sweep over edge density (Sec. 4): R-MAT with
    its generator parameters at 2^20 vertices and m = 5n, 50n and n^1.5, one
    whole modularity run per step; time is linear in m if the throughput per
    entry stays flat."""
    import torch
    out = []
    for name in ("rmat20_5n", "rmat20_50n", "rmat20_n15"):
        wl = WORKLOADS[name]
        g = make_graph(wl, dev)
        G = L.lcc_load_csr(g["off"], g["nbr"], g["w"])
        n, nnz = g["n"], g["nnz"]
        del g
        torch.cuda.empty_cache()
        sched = L.schedule(num_iter=wl["num_iter"], timing=True)
        L.lcc_cluster(G, wl["p"], wl["q"], wl["mode"], sched)  # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            _, _, st = L.lcc_cluster(G, wl["p"], wl["q"], wl["mode"], sched)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        G.free()
        out.append({"workload": name, "n": n, "m": nnz // 2, "csr_entries": nnz,
                    "ms_per_step": round(ms, 3),
                    "gedges_per_s": round(st["edges_scanned"] / (ms / 1e3) / 1e9, 3),
                    "edges_scanned": int(st["edges_scanned"]), "levels": int(st["levels"]),
                    "rounds": int(st["rounds_total"]),
                    "ms_bestmove": round(st["ms_bestmove"], 3),
                    "ms_contract": round(st["ms_contract"], 3),
                    "modularity": modularity(st, wl["q"])})
    return out


# ------------------------------------------------------------------- arms --

def run_reference(args, rank, world, local):
    """The oracle (the CPU restatement of the method) as the reference arm."""
    wl = WORKLOADS[args.workload]
    if rank != 0:
        return 0
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    g = make_graph(wl, dev)
    host = host_copy(g)
    del g
    n_entries = len(host["nbr"])
    vals, secs = [], []
    desc = ""
    per = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        v, desc, t = oracle_sample(host, wl, per)
        if i >= args.warmup:
            vals.append(v)
            secs.append(t)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": "best-move GEdges/s", "value": round(value, 6),
            "unit": "GEdges/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * statistics.mean(secs), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int128", "data": "synthetic",
            "config": {"workload": args.workload, "description": wl["desc"],
                       "csr_entries": n_entries, "l2": "inputs larger than L2",
                       "step": "a bounded sample of the workload: the oracle's first best-move "
                               "round over a prefix of the vertices (see cpu_baseline.sample)"},
            "cpu_baseline": {"value": round(value, 6), "unit": "GEdges/s", "cores": 1,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 6), "unit": "GEdges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import torch
    from paper_2108_01731_gb300 import lcc as L
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    L.load()
    gather_rate = random_gather_rate(dev)
    t_gen = time.perf_counter()
    g = make_graph(wl, dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    n, nnz = g["n"], g["nnz"]
    csr_bytes = (n + 1) * 8 + nnz * (8 if g["w"] is not None else 4)
    stream = torch.cuda.current_stream().cuda_stream
    G = L.lcc_load_csr(g["off"], g["nbr"], g["w"], stream=stream)
    host = None
    if not args.no_e2e or rank == 0:
        host = host_copy(g)
    del g
    torch.cuda.empty_cache()
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    sched = L.schedule(num_iter=wl["num_iter"], timing=True)
    # degree routing for this GPU and graph, chosen before the timed region
    t_tune = time.perf_counter()
    tuning = L.lcc_autotune(G, wl["p"], wl["q"], wl["mode"], args.tuning_cache)
    t_tune = time.perf_counter() - t_tune

    def step():
        return L.lcc_cluster(G, wl["p"], wl["q"], wl["mode"], sched, labels_out=labels)[2]

    for _ in range(args.warmup):
        step()
    ref_labels = labels.clone() if args.warmup > 0 else None
    barrier(world)
    torch.cuda.synchronize()
    clk = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    stats = [step() for _ in range(args.steps)]
    e1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = reduce_scalar(ms, world, "max", dev)
    edges = stats[-1]["edges_scanned"]
    assert all(s["edges_scanned"] == edges for s in stats)
    if ref_labels is None:
        ref_labels = labels.clone()
    assert torch.equal(labels, ref_labels), "labels changed between steps"
    tot_edges = reduce_scalar(edges, world, "sum", dev)
    value = tot_edges / (ms_max / 1e3) / 1e9
    launches = sum(s["kernel_launches"] for s in stats)

    bm_bytes = statistics.mean(s["bytes_bestmove"] for s in stats)
    bm_ms = statistics.mean(s["ms_bestmove"] for s in stats)
    rounds = stats[-1]["rounds_total"]
    peak, peak_kind = measured_peaks()
    achieved = bm_bytes / (bm_ms / 1e3) / 1e9
    tpe = profile_traffic(pregather=tuning["pregather"])
    roofline = {"kernel": "best-move (all degree buckets), per round", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "traffic": (round(tpe * edges / rounds) if tpe else None),
                "algorithmic_bytes_per_round": int(bm_bytes / rounds),
                "ms_per_round": round(bm_ms / rounds, 4), "rounds_per_step": rounds,
                "bestmove_only_gedges_s": round(edges / (bm_ms / 1e3) / 1e9, 3),
                # every entry gathers one packed label word: the entry rate
                # against this GPU's uniform random 8-byte gather rate
                "random_gather": {"ceiling_g_per_s": round(gather_rate / 1e9, 2),
                                  "entries_g_per_s": round(edges / (bm_ms / 1e3) / 1e9, 3),
                                  "frac": round(edges / (bm_ms / 1e3) / gather_rate, 4),
                                  "source": "torch.index_select, 2^28 uniform indices "
                                            "into a 2^26-word int64 table, timed here"},
                "ms_gather_pass": round(statistics.mean(s["ms_gather"] for s in stats), 2),
                "ms_per_bucket": dict(zip(BUCKETS,
                                          [round(statistics.mean(s["ms_bucket"][i]
                                                                 for s in stats), 2)
                                           for i in range(len(BUCKETS))])),
                "entries_per_bucket": [int(statistics.mean(s["bucket_entries"][i] for s in stats))
                                       for i in range(len(BUCKETS))],
                "vertices_per_bucket": [int(statistics.mean(s["bucket_vertices"][i]
                                                            for s in stats))
                                        for i in range(len(BUCKETS))]}

    # contraction against its minimum traffic: each contracted level's CSR and
    # labels read once, the coarse CSR written once
    c_ms = statistics.mean(s["ms_contract"] for s in stats)
    c_min = statistics.mean(s["bytes_contract_min"] for s in stats)
    contraction = {"ms_per_step": round(c_ms, 3), "min_bytes_per_step": int(c_min),
                   "pairs_sorted_per_step": int(stats[-1]["pairs_sorted"]),
                   "achieved": (round(c_min / (c_ms / 1e3) / 1e9, 1) if c_ms > 0 else None),
                   "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
                   "frac": (round(c_min / (c_ms / 1e3) / 1e9 / peak, 4) if c_ms > 0 else None),
                   "bytes": "least bytes over the contraction's device time"}

    # the legs that use the device-resident graph run first; it is freed
    # before the end-to-end leg loads the same graph again from host memory,
    # so that the two copies and their levels never share the device
    coin = None
    twin = None
    if rank == 0 and not args.no_coin:
        def run_coin():
            sc = L.schedule(num_iter=wl["num_iter"], coin=True, seed=0)
            torch.cuda.synchronize()
            e0.record()
            st = L.lcc_cluster(G, wl["p"], wl["q"], wl["mode"], sc, labels_out=labels)[2]
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), st
        coin = coin_leg(run_coin, wl)
    if rank == 0 and not args.no_twin:
        twin = twin_round(host, wl, lambda lab: L.lcc_desired(G, wl["p"], wl["q"],
                                                              wl["mode"], lab))
    torch.cuda.synchronize()
    G.free()
    G = None
    torch.cuda.empty_cache()

    def run_e2e():
        pinned = {k: (torch.from_numpy(v).pin_memory() if v is not None else None)
                  for k, v in host.items()}
        hl = torch.empty(n, dtype=torch.int32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in pinned.values() if t is not None)

        def e2e_step():
            Gh = L.lcc_load_csr(pinned["off"].numpy(), pinned["nbr"].numpy(),
                                None if pinned["w"] is None else pinned["w"].numpy(),
                                stream=stream)
            try:
                out = L.lcc_cluster(Gh, wl["p"], wl["q"], wl["mode"], sched,
                                    labels_out=hl.numpy())
            finally:
                Gh.free()
            return out[2]

        e2e_step()  # warm-up of the host path (pinned buffers, pool)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        ms_e2e = (time.perf_counter() - t0) * 1e3 / args.steps
        ms_e2e = reduce_scalar(ms_e2e, world, "max", dev)
        assert np.array_equal(hl.numpy(), ref_labels.cpu().numpy())
        return {"value": round(tot_edges / (ms_e2e / 1e3) / 1e9, 4), "unit": "GEdges/s",
                "ms_per_step": round(ms_e2e, 3), "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(n * 4)}

    e2e = None
    if not args.no_e2e:
        if world > 1:
            e2e = run_e2e()  # every rank takes the same path through the barriers
        else:
            # on one GPU a failure of this leg (say, no device memory left for
            # the second load) is reported in the line instead of losing it
            try:
                e2e = run_e2e()
            except Exception as e:  # noqa: BLE001
                e2e = {"unavailable": "%s: %s" % (type(e).__name__, e)}

    cpu = None
    serving = None
    if rank == 0:
        v, desc, _ = oracle_sample(host, wl, args.cpu_seconds)
        cpu = {"value": round(v, 6), "unit": "GEdges/s", "cores": 1, "kind": "oracle",
               "sample": desc}
        if args.serving > 0:
            try:
                serving = serving_bench(L, args.serving, dev, args.serving_large)
            except Exception as e:  # noqa: BLE001  (an extra leg: reported, never fatal)
                serving = {"unavailable": "%s: %s" % (type(e).__name__, e)}
    line = {"metric": "best-move GEdges/s", "value": round(value, 4), "unit": "GEdges/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_max, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.workload, "description": wl["desc"], "n": n,
                       "csr_entries": nnz, "edges_scanned_per_step": edges,
                       "levels": stats[-1]["levels"], "rounds_per_step": rounds,
                       "num_clusters": stats[-1]["num_clusters"],
                       "objective": stats[-1]["objective"],
                       "ms_bestmove": round(bm_ms, 3),
                       "ms_contract": round(statistics.mean(s["ms_contract"] for s in stats), 3),
                       "ms_round_other": round(statistics.mean(s["ms_round_other"]
                                                              for s in stats), 3),
                       "ms_other": round(statistics.mean(s["ms_other"] for s in stats), 3),
                       "pairs_sorted": stats[-1]["pairs_sorted"],
                       "generation_s": round(t_gen, 2),
                       "tuning": {"warp_max": tuning["warp_max"],
                                  "fuse_small": tuning["fuse_small"],
                                  "prefetch": tuning["prefetch"],
                                  "pregather": tuning["pregather"],
                                  "part_min": tuning["part_min"],
                                  "autotune_s": round(t_tune, 2),
                                  "chosen_by": ("lcc_autotune on this graph before timing "
                                                "(3 best-move rounds per routing)"
                                                if not args.tuning_cache else
                                                "lcc_autotune with the tuning file "
                                                + args.tuning_cache)},
                       "degree_buckets": degree_shares(host["off"]) if host else None,
                       "l2": ("inputs larger than L2 (CSR %.1f GB vs 129 MB L2)" % (csr_bytes / 1e9)
                              if csr_bytes > (129 << 20) else
                              "CSR of %.1f MB fits L2; no flush between steps" % (csr_bytes / 1e6)),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "contraction": contraction, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clocks}
    if twin is not None:
        line["cpu_parallel"] = twin
    if serving is not None:
        line["serving"] = serving
    if wl["mode"] == 1:
        line["config"]["modularity"] = modularity(stats[-1], wl["q"])
    if coin is not None:
        line["coin_schedule"] = coin
    if rank == 0 and args.sweep:
        try:
            line["density_sweep"] = density_sweep(L, dev, max(1, min(args.steps, 3)))
        except Exception as e:  # noqa: BLE001  (an extra leg: reported, never fatal)
            line["density_sweep"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


import numpy as np  # noqa: E402  (used by run_ours' e2e check)


def main():
    args = parse()
    rank, world, local = dist_env()
    if world != args.gpus and world > 1:
        print("warning: WORLD_SIZE=%d but --gpus %d" % (world, args.gpus), file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, rank, world, local)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
