"""The oracle and the library share no code: the package never imports or loads anything from
oracle/, the oracle never imports the package, and the CUDA sources include nothing from oracle/.
Only synth/ (seeded input generators, none of the method's arithmetic) serves both."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(sub, exts):
    for dp, _, fns in os.walk(os.path.join(ROOT, sub)):
        if "_build" in dp or "__pycache__" in dp:
            continue
        for fn in fns:
            if fn.endswith(exts):
                yield os.path.join(dp, fn)


def test_package_does_not_use_oracle():
    for f in _files("paper_1010_5636_gb300", (".py", ".cu", ".cuh", ".h", ".cpp")):
        src = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", src, re.M), f
        assert "oracle/" not in src and '"oracle' not in src, f


def test_oracle_does_not_use_package():
    for f in _files("oracle", (".py", ".c", ".h")):
        src = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+paper_1010_5636_gb300\b", src, re.M), f
        assert "libnd" not in src and "csrc/" not in src, f


def test_synth_holds_no_method_code():
    for f in _files("synth", (".py",)):
        src = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+(oracle|paper_1010_5636_gb300)\b", src, re.M), f
