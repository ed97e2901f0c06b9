"""The C ABI library builds for sm_103a, loads, and exports every function include/gc.h declares.
No compute calls are made (this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gc_\w+)\s*\(", text)))


def test_header_is_plain_c():
    text = open(os.path.join(ROOT, "include", "gc.h")).read()
    assert 'extern "C"' in text
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for bad in ("torch", "at::", "c10", "std::"):
        assert bad not in text


def test_library_exports_every_declared_symbol(gclib):
    lib = ctypes.CDLL(gclib.LIB_PATH)
    names = declared_functions()
    assert "gc_color" in names and "gc_color_batch" in names and "gc_server_submit" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string(gclib):
    lib = gclib.load()
    assert lib.gc_version() >= 100
    assert isinstance(lib.gc_last_error(), bytes)


def test_header_compiles_as_c_and_cpp(tmp_path):
    # the stats struct tag and the gc_server_stats function share a name, which C and C++ allow
    import subprocess
    src = tmp_path / "use.c"
    src.write_text('#include "gc.h"\nint f(gc_server *s) { struct gc_server_stats st; return gc_server_stats(s, &st) '
                   '+ gc_server_stats_get(s, &st); }\n')
    inc = os.path.join(ROOT, "include")
    for cmd in (["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                ["g++", "-x", "c++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_binding_structs_match_header(tmp_path):
    # the Python binding's ctypes mirrors have the header's sizes and field offsets
    import subprocess
    import paper_1509_08267_gb300 as gc
    pairs = {"gc_options": gc._Options, "gc_stats": gc._Stats, "gc_server_config": gc._ServerConfig,
             "struct gc_server_stats": gc._ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gc.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    want = {}
    for cname, py in pairs.items():
        want[f"{cname} size"] = ctypes.sizeof(py)
        for f, _ in py._fields_:
            want[f"{cname} {f}"] = getattr(py, f).offset
    got = {ln.rsplit(" ", 1)[0]: int(ln.rsplit(" ", 1)[1]) for ln in out if ln}
    assert got == want
