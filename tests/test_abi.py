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


def test_struct_layouts_match_header_sizes(tmp_path):
    """The ctypes structs against the C compiler's view of include/lcc.h:
    the size of every struct and the offset of every field."""
    import subprocess
    from paper_2108_01731_gb300 import lcc
    structs = [lcc.lcc_schedule, lcc.lcc_stats, lcc.lcc_tuning, lcc.lcc_server_cfg, lcc.lcc_job,
               lcc.lcc_round]
    lines = []
    for st in structs:
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (st.__name__, st.__name__))
        for f in st._fields_:
            lines.append('printf("%%s.%%s %%zu\\n", "%s", "%s", offsetof(%s, %s));'
                         % (st.__name__, f[0], st.__name__, f[0]))
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"lcc.h\"\n"
                   "int main(void) {\n%s\nreturn 0;\n}\n" % "\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    want = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for st in structs:
        assert int(want[st.__name__]) == ctypes.sizeof(st), st.__name__
        for f in st._fields_:
            assert int(want["%s.%s" % (st.__name__, f[0])]) == getattr(st, f[0]).offset, f[0]
    assert ctypes.sizeof(lcc.lcc_schedule) == 32 and lcc.lcc_schedule.seed.offset == 24
