"""The oracle and the CUDA path share no code: the oracle never imports the package or
its library, the package never imports the oracle, and the only module both use is the
seeded input generator (which holds none of the method's arithmetic)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sources(folder, exts):
    for dirpath, _, files in os.walk(os.path.join(ROOT, folder)):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_oracle_does_not_use_the_product():
    for p in sources("oracle", (".py", ".c", ".h")):
        text = open(p).read()
        assert "paper_2212_05159_gb300" not in text, p
        assert "libspx" not in text and "spx.h" not in text, p


def test_product_does_not_use_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)", re.M)
    for p in sources("paper_2212_05159_gb300", (".py", ".cu", ".cuh")):
        text = open(p).read()
        assert not pat.search(text), p
        assert "spx_oracle" not in text and "liboracle" not in text, p


def test_generators_hold_no_method_arithmetic():
    """synth/ builds inputs only: no products, solves or gradients of the method."""
    text = open(os.path.join(ROOT, "synth", "__init__.py")).read()
    for word in ("spmm", "sddmm", "spgemm", "transpose", "pcg", "gradient", "import oracle",
                 "paper_2212_05159_gb300"):
        assert word not in text.lower(), word
