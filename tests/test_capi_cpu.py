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
