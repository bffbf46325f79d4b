"""The ctypes structures of the binding against the C header: a C program compiled
from include/sphvisc.h prints sizeof and offsetof of every field, which must match
ctypes' layout (CPU only; needs a C compiler)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "paper_2206_14780_gb300", "_build", "abi_probe")


def _structs():
    from paper_2206_14780_gb300 import binding as b

    return [b.sph_scene, b.sph_visc_params, b.sph_solve_opts, b.sph_solve_report, b.sph_profile_counters,
            b.sph_state, b.sph_step_params, b.sph_step_report]


def _c_layout(structs):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sphvisc.h"', "int main(void) {"]
    for s in structs:
        name = s.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in s._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    os.makedirs(OUT, exist_ok=True)
    src, exe = os.path.join(OUT, "probe.c"), os.path.join(OUT, "probe")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


def test_ctypes_structs_match_the_header():
    structs = _structs()
    layout = _c_layout(structs)
    for s in structs:
        name = s.__name__
        assert ctypes.sizeof(s) == layout[(name, "sizeof")], name
        for f, _ in s._fields_:
            assert getattr(s, f).offset == layout[(name, f)], (name, f)
