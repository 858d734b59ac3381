"""The C-ABI library builds, loads and exports every entry point include/lbm.h
declares (no compute calls: this runs without a GPU)."""

import os
import re

from paper_1712_08288_gb300 import _build, binding

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = binding.load_library(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_product_path_does_not_touch_the_oracle_and_fails_loudly_without_the_library():
    """The package and its binding never import the oracle, and a missing library
    is an ImportError, not a fallback."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_1712_08288_gb300, paper_1712_08288_gb300.binding as B, "
        "paper_1712_08288_gb300.workloads\n"
        "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules), 'oracle imported'\n"
        "try:\n"
        "    B.load_library('/nonexistent/liblbm.so')\n"
        "    raise SystemExit('no error')\n"
        "except ImportError:\n"
        "    pass\n" % root)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
