"""The C-ABI library loads and exports every symbol include/sphvisc.h declares (no GPU calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sphvisc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sph_build_neighbors", "sph_visc_apply", "sph_visc_solve"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2206_14780_gb300 import binding, build

    if not os.path.exists(binding.LIB_PATH):
        build.build()
    lib = binding.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(binding.EXPORTS) == _declared()
    assert b"sm_103a" in lib.sph_version()


def test_missing_library_fails_loudly():
    """No fallback: without the compiled library the binding raises instead of computing."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("from paper_2206_14780_gb300 import binding; "
            "binding.load(binding.LIB_PATH + '.absent')")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True)
    assert out.returncode != 0 and "is missing" in out.stderr, (out.returncode, out.stderr[-300:])
