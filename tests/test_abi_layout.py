"""The binding's ctypes structures match the C header's layout (CPU only): a small C program,
compiled with the host compiler against include/sfft.h, prints the size of each struct of the
boundary and the offset of each member, and the ctypes mirrors must agree field by field."""
import os
import shutil
import subprocess

import pytest

from paper_1606_07407_gb300 import sfft as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"sfft_pschedule": S._PSchedule, "sfft_tilts": S._Tilts, "sfft_opts": S._Opts, "sfft_stats": S._Stats}


def test_ctypes_mirrors_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sfft.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for name, cls in STRUCTS.items():
        assert got[(name, "size")] == __import__("ctypes").sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
