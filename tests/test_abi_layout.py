"""The ctypes structures of the Python binding have the layout of the C
structures include/mhd.h declares: gcc compiles a probe that prints
sizeof and offsetof of every field the binding names (a misspelt or missing
field fails to compile), and each must equal ctypes' own figure."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(tmp_path, ctype, names):
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "mhd.h"', "int main(void) {",
           f'  printf("%zu\\n", sizeof({ctype}));']
    src += [f'  printf("%zu\\n", offsetof({ctype}, {n}));' for n in names]
    src += ["  return 0;", "}"]
    c = tmp_path / "probe.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "probe"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("pyname,ctype", [("Params", "mhd_params"), ("Stats", "mhd_stats"),
                                          ("GranParams", "mhd_gran_params")])
def test_struct_layout_matches_the_header(tmp_path, pyname, ctype):
    from paper_1908_08557_gb300 import binding
    cls = getattr(binding, pyname)
    names = [n for n, _ in cls._fields_]
    size, offs = _c_layout(tmp_path, ctype, names)
    assert ctypes.sizeof(cls) == size
    for n, o in zip(names, offs):
        assert getattr(cls, n).offset == o, n
