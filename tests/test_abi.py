"""The C ABI library loads and exports every entry point include/clot.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(clot_\w+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2304_09180_gb300.build import build
    so = build()
    lib = ctypes.CDLL(so)
    names = declared()
    assert {"clot_mesh_create", "clot_species_step", "clot_reaction_step"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_2304_09180_gb300 import binding
    assert declared() <= set(binding.EXPORTED)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2304_09180_gb300")
    for dp, _, fns in os.walk(pkg):
        for fn in fns:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dp, fn)).read()
                assert "import oracle" not in src and "from oracle" not in src, fn
                assert "clot_oracle" not in src, fn
