"""The C ABI library loads and exports every entry point include/clot.h
declares, and the binding's ctypes structures lay out exactly like the
header's structs (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil
import subprocess
import tempfile

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


STRUCTS = ("clot_mesh_desc", "clot_mesh_info_t", "clot_fields", "clot_fluxes", "clot_params", "clot_profile_t",
           "clot_channel", "clot_tune_t", "clot_mlp")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_binding_structs_match_the_header_layout():
    """A C program compiled against include/clot.h prints sizeof and offsetof
    of every field the ctypes structure names; both must agree (a field the
    header lacks fails the compile)."""
    from paper_2304_09180_gb300 import binding
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "clot.h"', "int main(void) {"]
    for st in STRUCTS:
        cls = getattr(binding, st)
        lines.append(f'  printf("{st} sizeof %zu\\n", sizeof({st}));')
        for name, _ in cls._fields_:
            lines.append(f'  printf("{st} {name} %zu\\n", offsetof({st}, {name}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as td:
        src, exe = os.path.join(td, "layout.c"), os.path.join(td, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        st, name, v = line.split()
        got[(st, name)] = int(v)
    for st in STRUCTS:
        cls = getattr(binding, st)
        assert got[(st, "sizeof")] == ctypes.sizeof(cls), st
        for name, _ in cls._fields_:
            assert got[(st, name)] == getattr(cls, name).offset, (st, name)


def test_every_declaration_cites_the_paper_or_says_it_has_no_counterpart():
    """Each entry point of include/clot.h is documented by the comment right
    above it with the passage of the paper it implements (Sec. / App. / Eq.),
    or with a plain statement that the paper has none."""
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(clot_\w+)\s*\(", src, re.M):
            before = src[:m.start()]
            end = before.rfind("*/")
            assert end >= 0 and before[end + 2:].strip() == "", (fn, m.group(1), "no comment right above")
            comment = " ".join(re.sub(r"^\s*\*", " ", ln) for ln in before[before.rfind("/*", 0, end):end].splitlines())
            comment = re.sub(r"\s+", " ", comment)
            assert re.search(r"Sec\.|App\.|Eq\.|not (part of|in) the paper|no counterpart", comment, re.I), \
                (fn, m.group(1))


def test_noalloc_binding_rejects_undersized_or_misplaced_tensors_before_any_launch():
    """The C side of clot_eta_solve_noalloc cannot see tensor sizes or devices;
    the binding checks them and raises ValueError before calling the library
    (CPU tensors here: no CUDA call is made)."""
    import torch

    import paper_2304_09180_gb300 as clot
    import synthetic as S
    p = S.params_default()
    d = S.config("channel_40x12", p)["desc"]
    nc = 40 * 12
    prm = type("P", (), {"c": None})()          # never reached
    good_c, good_eta = torch.zeros((15, 512)), torch.zeros(nc)
    with pytest.raises(ValueError, match="pitch"):
        clot.clot_eta_solve_noalloc(d, good_c, nc - 1, good_eta, prm)
    with pytest.raises(ValueError, match="c holds"):
        clot.clot_eta_solve_noalloc(d, torch.zeros((15, 100)), 512, good_eta, prm)
    with pytest.raises(ValueError, match="eta holds"):
        clot.clot_eta_solve_noalloc(d, good_c, 512, torch.zeros(nc - 1), prm)
    with pytest.raises(ValueError, match="current CUDA device"):
        clot.clot_eta_solve_noalloc(d, good_c, 512, good_eta, prm)
