"""The oracle and the CUDA path share no code: the product package and the input
generators never import the oracle, the oracle never touches the product package,
and importing the binding or the benchmark does not load the oracle (CPU only)."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
IMPORT_ORACLE = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)", re.M)


def _files(top, exts):
    for dirpath, dirs, files in os.walk(os.path.join(ROOT, top)):
        dirs[:] = [d for d in dirs if not d.startswith(("_", "."))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_product_and_generators_never_import_the_oracle():
    checked = 0
    for top in ("paper_2206_14780_gb300", "scenes"):
        for path in _files(top, (".py",)):
            with open(path) as fh:
                assert not IMPORT_ORACLE.search(fh.read()), path
            checked += 1
    for path in _files("paper_2206_14780_gb300", (".cu", ".cuh", ".h")):
        with open(path) as fh:
            assert "oracle" not in fh.read(), path
        checked += 1
    assert checked > 20


def test_oracle_never_touches_the_product():
    for path in _files("oracle", (".py",)):
        with open(path) as fh:
            text = fh.read()
        assert "paper_2206_14780_gb300" not in text and "csrc" not in text and "sphvisc" not in text, path


def test_importing_binding_and_bench_leaves_the_oracle_unloaded():
    code = ("import sys; import bench; from paper_2206_14780_gb300 import binding; "
            "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, check=True)
    assert out.stdout.strip() == "[]", out.stdout
