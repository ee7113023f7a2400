"""CPU test that the binding's ctypes mirror of fmmfft_stats matches the C
struct of include/fmmfft.h field by field.

fmmfft_plan_stats writes sizeof(fmmfft_stats) bytes into the caller's struct,
so a mirror that is shorter, or whose fields sit at other offsets, would have
the library write past the Python buffer or the binding read the wrong
values.  The C side is measured by compiling a few offsetof lines against the
header with the host compiler."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stats_struct_matches_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    import paper_2010_00520_gb300 as F
    fields = [name for name, _ in F._Stats._fields_]
    src = tmp_path / "layout.c"
    src.write_text(
        "#include <stdio.h>\n#include <stddef.h>\n#include \"fmmfft.h\"\nint main(void) {\n"
        '  printf("size %zu\\n", sizeof(fmmfft_stats));\n'
        + "".join(f'  printf("{n} %zu %zu\\n", offsetof(fmmfft_stats, {n}), sizeof(((fmmfft_stats*)0)->{n}));\n'
                  for n in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, stdout=subprocess.PIPE, text=True).stdout.split("\n")
    import ctypes
    got = {}
    for line in out:
        if line:
            k, *v = line.split()
            got[k] = tuple(int(x) for x in v)
    assert got.pop("size") == (ctypes.sizeof(F._Stats),)
    for name in fields:
        f = getattr(F._Stats, name)
        assert got[name] == (f.offset, f.size), name
