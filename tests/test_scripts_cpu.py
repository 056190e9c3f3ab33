"""The committed analysis scripts run and print their tables (CPU only)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    out = subprocess.run([sys.executable, *args], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [ln for ln in out.stdout.splitlines() if ln.startswith("| ")]


def test_quality_table():
    rows = run(os.path.join("oracle", "quality.py"))
    assert len(rows) == 1 + 3  # header and three graphs
    assert all(r.count("|") == 5 for r in rows)


def test_schedule_table_small_scale():
    rows = run(os.path.join("cpu_twin", "schedules.py"), "12")
    assert len(rows) == 1 + 2 * 8  # header, then two graphs x eight options
    coin = [r for r in rows if "| coin, V' = neighbours of moved vertices, refinement |" in r]
    plain = [r for r in rows if "| synchronous, V' = neighbours of moved vertices" in r]
    assert len(coin) == 2 and len(plain) == 2


def test_vprime_table_small_scale():
    rows = run(os.path.join("cpu_twin", "vprime.py"), "12")
    assert len(rows) == 1 + 2 * 2 * 2  # header, then two graphs x two schedules x two rules
    for r in rows[1:]:
        first = r.rstrip(" |").split("|")[-1].split()[0]
        assert first == "100.0"  # round 0 evaluates every vertex
