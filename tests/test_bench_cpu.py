"""Host-side logic of bench.py (no GPU): the source check behind
roofline.traffic, and the reference arm's JSON line on a small workload."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_profile_traffic_only_for_the_measured_source_and_tuning(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    m = {"k_round.cu": sha, "dram_bytes_per_entry": 21.5}
    assert bench.profile_traffic(str(src), m) == 21.5
    m1 = dict(m, pregather=1)
    assert bench.profile_traffic(str(src), m1, pregather=1) == 21.5
    assert bench.profile_traffic(str(src), m1, pregather=0) is None
    src.write_text("changed kernel source\n")
    assert bench.profile_traffic(str(src), m) is None
    assert bench.profile_traffic(str(src), {"k_round.cu": None}) is None


@pytest.mark.slow
def test_reference_arm_line_on_cpu():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "sbm1e4", "--steps", "1", "--warmup", "0",
                          "--cpu-seconds", "1"], capture_output=True, text=True, cwd=ROOT,
                         timeout=600, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_twin_leg_reports_rate_and_agreement():
    """The bench's OpenMP-twin leg on a small graph, with the oracle standing
    in for the GPU's desired clusters: a positive rate, the cores used, and
    agreement with the stand-in (or its absence when it differs)."""
    import numpy as np
    import oracle as O
    from paper_2108_01731_gb300 import inputs as I
    g = I.to_numpy(I.rmat(12, 30000, seed=3))
    host = {"off": g["off"], "nbr": g["nbr"], "w": g["w"]}
    wl = dict(bench.WORKLOADS["rmat22"])
    k, two_m = O.weighted_degrees(g["off"], g["w"])

    def oracle_desired(lab):
        return O.desired(g["off"], g["nbr"], g["w"], k, 1, two_m, lab, k)

    out = bench.twin_round(host, wl, oracle_desired)
    assert out["value"] > 0 and out["cores"] >= 1 and out["desired_equal_gpu"] is True
    assert "%d entries" % g["nnz"] in out["sample"]
    out = bench.twin_round(host, wl, lambda lab: oracle_desired(lab)[::-1].copy())
    assert out["desired_equal_gpu"] is False


def test_coin_leg_reports_or_degrades():
    wl = dict(bench.WORKLOADS["rmat22"])
    st = {"edges_scanned": 2_000_000_000, "levels": 5, "rounds_total": 60, "num_clusters": 10,
          "objective": 1000.0, "obj_num": 1000 * 8, "obj_den": 8}
    out = bench.coin_leg(lambda: (500.0, st), wl)
    assert out["gedges_per_s"] == 4.0 and out["rounds"] == 60
    assert out["modularity"] == 1000.0 / 8  # CC / 2m with obj_den = q 2m, q = 1

    def boom():
        raise RuntimeError("CUDA error (status 7)")
    out = bench.coin_leg(boom, wl)
    assert "unavailable" in out and "status 7" in out["unavailable"]
