"""The Python mirrors of the C ABI's structs (ctypes structures and numpy
record dtypes in paper_2203_02527_gb300/_lib.py) match include/ph0.h: a C
program, generated from the mirrors' field names and compiled by the host C
compiler against the header, prints every struct's size and every field's
offset (a field the header does not have fails to compile), and the test
compares them with the mirrors'.  Host only."""
import os
import shutil
import subprocess

import pytest

from paper_2203_02527_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "ph0_stats": _lib.Stats,
    "ph0_tuning": _lib.Tuning,
    "ph0_profile": _lib.Profile,
    "ph0_options": _lib.Options,
    "ph0_h1_stats": _lib.H1Stats,
    "ph0_inf_bar": _lib.InfBar,
    "ph0_result": _lib.Result,
}
DTYPES = {"ph0_bar": _lib.BAR_DTYPE, "ph0_h1bar": _lib.H1_DTYPE}


def mirror_layout():
    want = {}
    for cname, cls in STRUCTS.items():
        want[cname] = ctypes_sizeof(cls)
        for name, _ in cls._fields_:
            want[f"{cname}.{name}"] = getattr(cls, name).offset
    for cname, dt in DTYPES.items():
        want[cname] = dt.itemsize
        for name in dt.names:
            want[f"{cname}.{name}"] = dt.fields[name][1]
    return want


def ctypes_sizeof(cls):
    import ctypes
    return ctypes.sizeof(cls)


def test_python_mirrors_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    want = mirror_layout()
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ph0.h"', "int main(void) {"]
    for key in want:
        if "." in key:
            cname, field = key.split(".")
            lines.append(f'    printf("{key} %zu\\n", offsetof({cname}, {field}));')
        else:
            lines.append(f'    printf("{key} %zu\\n", sizeof({key}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "abi_layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "abi_layout")
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", exe, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines():
        key, val = line.split()
        got[key] = int(val)
    assert got == want
