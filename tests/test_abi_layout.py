"""The binding's ctypes structures and NumPy record types against the C
structs of include/ht.h: every field at the same offset and every struct of
the same size, read from a C program compiled against the header."""
import os
import shutil
import subprocess

import pytest

from paper_1507_03074_gb300 import ht

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [
    ("ht_binning", ht.c_binning), ("ht_ranges", ht.c_ranges), ("ht_tuning", ht.c_tuning),
    ("ht_server_cfg", ht.c_server_cfg), ("ht_server_stats", ht.c_server_stats),
    ("ht_kernel_time", ht.c_kernel_time), ("ht_peak", ht.PEAK_DTYPE), ("ht_track", ht.TRACK_DTYPE),
]


def _python_layout(t):
    if hasattr(t, "_fields_"):
        return __import__("ctypes").sizeof(t), [(n, getattr(t, n).offset) for n, *_ in t._fields_]
    return t.itemsize, [(n, t.fields[n][1]) for n in t.names]


def test_struct_layouts_match_header(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not found")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ht.h"', "int main(void) {"]
    want = {}
    for cname, t in PAIRS:
        size, fields = _python_layout(t)
        want[cname] = (size, dict(fields))
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in fields:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    b = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert b.returncode == 0, b.stderr      # a field the header lacks fails here
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in filter(None, out):
        cname, f, v = line.split()
        got.setdefault(cname, {})[f] = int(v)
    for cname, (size, fields) in want.items():
        assert got[cname]["sizeof"] == size, (cname, got[cname]["sizeof"], size)
        for f, off in fields.items():
            assert got[cname][f] == off, (cname, f, got[cname][f], off)
