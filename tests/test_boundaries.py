"""Static checks of the separation between the product and the oracle: the
package (Python and CUDA sources) never refers to the oracle, and the oracle
never imports the package; the only shared module is synth (inputs)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2509_21694_gb300")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_use_the_oracle():
    for p in _files(PKG, (".py", ".cu", ".cuh", ".h")):
        src = open(p).read()
        assert not re.search(r"\boracle\b", src), p


def test_oracle_does_not_import_the_package():
    for p in _files(os.path.join(ROOT, "oracle"), (".py",)):
        src = open(p).read()
        assert "paper_2509_21694_gb300" not in src, p
        assert "libmpip" not in src, p


def test_synth_imports_neither_side():
    for p in _files(os.path.join(ROOT, "synth"), (".py",)):
        src = open(p).read()
        assert not re.search(r"^\s*(from|import)\s+(oracle|paper_2509_21694_gb300)", src, re.M), p
