"""The C-ABI library loads, exports every entry point of include/ifmm.h, and its
host-side tree / lists / Algorithm 3 coloring equal the oracle's bit for bit."""

import os
import re
import subprocess

import numpy as np
import pytest

from oracle.tree import Tree, greedy_coloring
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_directions, fibonacci_sphere, torus

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ifmm.h")


def test_exports_every_declared_symbol():
    decl = set(re.findall(r"^\s*(?:ifmm_status|void|const char\*)\s+(\w+)\s*\(", open(HEADER).read(), re.M))
    out = subprocess.run(["nm", "-D", "--defined-only", ifmm._LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert decl, "no declarations parsed"
    assert decl <= exported, decl - exported
    assert set(ifmm.EXPORTED) <= decl


def _csr(tree, level, name):
    ptr = ifmm.ifmm_tree_query(tree, level, name + "_ptr")
    val = ifmm.ifmm_tree_query(tree, level, name)
    return [list(val[ptr[i]:ptr[i + 1]]) for i in range(len(ptr) - 1)]


@pytest.mark.parametrize("case", [("sphere", 2048, 3), ("bumpy", 5000, 4), ("torus", 4000, 4), ("sphere", 300, 2)])
@pytest.mark.parametrize("sigma", [3, 6])
def test_tree_and_coloring_match_oracle(case, sigma):
    shape, n, depth = case
    pts = {"sphere": fibonacci_sphere, "bumpy": bumpy_sphere, "torus": torus}[shape](n, 5)
    ref = Tree(pts, depth)
    t = ifmm.ifmm_build_tree(pts, depth)
    ncol = ifmm.ifmm_color(t, sigma)
    assert np.array_equal(ifmm.ifmm_tree_query(t, 0, "perm"), ref.perm)
    assert np.array_equal(ifmm.ifmm_tree_query(t, 0, "leaf_ptr"), ref.leaf_start)
    for kappa in range(0, depth + 1):
        L = ref.levels[kappa]
        assert np.array_equal(ifmm.ifmm_tree_query(t, kappa, "cells").reshape(-1, 3), L.cells)
        if kappa >= 1:
            assert np.array_equal(ifmm.ifmm_tree_query(t, kappa, "parent"), L.parent)
        assert _csr(t, kappa, "nbr") == [list(v) for v in L.nbrs]
        assert _csr(t, kappa, "il") == [list(v) for v in L.il]
        if kappa >= 2:
            color, groups = greedy_coloring(L, sigma)
            assert ncol[kappa] == len(groups)
            assert np.array_equal(ifmm.ifmm_tree_query(t, kappa, "color"), color)
            assert _csr(t, kappa, "group") == groups


def test_table1_through_the_library():
    """Table 1 (Sec. 5.2) reproduced by the library's own tree and coloring."""
    t = ifmm.ifmm_build_tree(fibonacci_directions(1003520), 5)
    ncol = ifmm.ifmm_color(t, 3)
    want = {2: (56, 19, 2, 8), 3: (272, 26, 7, 16), 4: (1160, 27, 8, 70), 5: (4742, 27, 84, 245)}
    for kappa, (nodes, ng, gmin, gmax) in want.items():
        gp = ifmm.ifmm_tree_query(t, kappa, "group_ptr")
        sizes = np.diff(gp)
        assert len(ifmm.ifmm_tree_query(t, kappa, "cells")) // 3 == nodes
        assert ncol[kappa] == ng and sizes.min() == gmin and sizes.max() == gmax


def test_invalid_arguments_fail_cleanly():
    with pytest.raises(ifmm.IFMMError) as e:
        ifmm.ifmm_build_tree(np.zeros((5, 3)), 1)
    assert e.value.code == 1
    t = ifmm.ifmm_build_tree(fibonacci_sphere(100, 1), 2)
    with pytest.raises(ifmm.IFMMError):
        ifmm.ifmm_color(t, 2)
    with pytest.raises(ifmm.IFMMError):
        ifmm.ifmm_tree_query(t, 9, "cells")
    with pytest.raises(ifmm.IFMMError):
        ifmm.ifmm_factor(t, 3, 1e-6)  # not colored yet


@pytest.mark.parametrize("tau", [2, 3, 4])
def test_color_levels_sequential_below_tau(tau):
    """Sec. 4.2, Table 2: levels below tau get one node per color in node order
    (matrix-parallel), levels tau..depth the Algorithm 3 coloring."""
    pts = bumpy_sphere(5000, 2)
    a = ifmm.ifmm_build_tree(pts, 4)
    b = ifmm.ifmm_build_tree(pts, 4)
    na = ifmm.ifmm_color(a, 3)
    nb = ifmm.ifmm_color_levels(b, 3, tau)
    for lvl in range(2, 5):
        n = len(ifmm.ifmm_tree_query(b, lvl, "parent"))
        if lvl < tau:
            assert nb[lvl] == n
            assert list(ifmm.ifmm_tree_query(b, lvl, "group")) == list(range(n))
            assert list(ifmm.ifmm_tree_query(b, lvl, "group_ptr")) == list(range(n + 1))
        else:
            assert nb[lvl] == na[lvl]
            for what in ("color", "group", "group_ptr"):
                assert np.array_equal(ifmm.ifmm_tree_query(a, lvl, what), ifmm.ifmm_tree_query(b, lvl, what))
    with pytest.raises(ifmm.IFMMError):
        ifmm.ifmm_color_levels(b, 3, 5)
