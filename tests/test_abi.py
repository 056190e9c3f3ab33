"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/lcc.h declares; the binding's
signature table matches the header."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lcc.h")).read()
    return sorted(set(re.findall(r"LCC_API[^;{(]*?\b(lcc_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lcc_load_csr", "lcc_cluster", "lcc_free_graph", "lcc_status_str",
                 "lcc_last_error", "lcc_server_create", "lcc_submit", "lcc_poll",
                 "lcc_server_destroy", "lcc_cluster_batch"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2108_01731_gb300.build import build
    path = build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2108_01731_gb300 import lcc
    assert sorted(lcc._SIGS) == declared_functions()
    lib = lcc.load()
    assert lib.lcc_status_str(lcc.LCC_ERR_NOT_SYMMETRIC).decode() == "graph not symmetric"


def test_struct_layouts_match_header_sizes():
    from paper_2108_01731_gb300 import lcc
    assert ctypes.sizeof(lcc.lcc_schedule) == 24
    assert ctypes.sizeof(lcc.lcc_stats) == 4 * 2 + 8 * 7 + 8 * 6 + 8 * 3 + 8 * 16 * 3
    assert ctypes.sizeof(lcc.lcc_job) == 8 * 7 + 8
