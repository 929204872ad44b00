"""The ctypes structures of the Python binding have the layout of the C structs in
include/iga.h: a small C program compiled against the header (gcc, host only)
prints sizeof and every field offset, which must equal the ctypes values."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["iga_space_desc", "iga_space_info", "iga_ops_info", "iga_wave_desc", "iga_wave_stats",
           "iga_interface"]


def _binding():
    from paper_2004_05197_gb300 import build
    build.build()
    from paper_2004_05197_gb300 import iga
    return iga


def test_ctypes_structs_match_the_header():
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    iga = _binding()
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "iga.h"', "int main(void) {"]
    for sname in STRUCTS:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (sname, sname))
        for fname, _ in getattr(iga, sname)._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (sname, fname, sname, fname))
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines))
        subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for sname in STRUCTS:
        st = getattr(iga, sname)
        assert int(got["%s size" % sname]) == __import__("ctypes").sizeof(st), sname
        for fname, _ in st._fields_:
            assert int(got["%s.%s" % (sname, fname)]) == getattr(st, fname).offset, (sname, fname)
