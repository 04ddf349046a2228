"""Pins for the oracle's tree, lists and coloring (Sec. 2.1, Sec. 3, Algorithm 3)."""

import itertools
import os

import numpy as np
import pytest

from oracle.tree import Level, Tree, dist, greedy_coloring
from paper_1905_10602_gb300.workloads import fibonacci_directions, fibonacci_sphere, torus

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_sphere_sigma3.txt")


def test_table1_sphere_statistics():
    """Table 1 (Sec. 5.2): node counts and sigma=3 group statistics, levels 2-5."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    T = Tree(fibonacci_directions(1003520), 5)
    for row in rows:
        kappa, nodes, ngroups, gmin = int(row[0]), int(row[1]), int(row[2]), int(row[3])
        gave, gmax = float(row[4]), int(row[5])
        L = T.levels[kappa]
        _, groups = greedy_coloring(L, 3)
        sizes = [len(g) for g in groups]
        assert L.n == nodes
        assert len(groups) == ngroups
        assert min(sizes) == gmin and max(sizes) == gmax
        assert abs(np.mean(sizes) - gave) < 1e-6


def _complete_level(kappa):
    m = 1 << kappa
    cells = np.array([(i, j, k) for k in range(m) for j in range(m) for i in range(m)])
    return Level(kappa, cells)


@pytest.mark.parametrize("sigma", [2, 3, 4])
def test_complete_grid_sigma_cubed_colors(sigma):
    """Sec. 3.4: on a complete grid the coloring uses sigma^3 colors, each a stride-sigma sub-grid."""
    L = _complete_level(3)
    color, groups = greedy_coloring(L, sigma)
    assert len(groups) == sigma ** 3
    for g in groups:
        c = L.cells[g]
        assert len(set(map(tuple, c % sigma))) == 1


def _check_coloring_properties(T, kappa, sigma):
    L = T.levels[kappa]
    color, groups = greedy_coloring(L, sigma)
    assert sorted(itertools.chain(*groups)) == list(range(L.n))
    assert len(groups) <= sigma ** 3
    nb = [set(map(int, v)) for v in L.nbrs]
    il = [set(map(int, v)) for v in L.il]
    for g in groups:
        c = L.cells[g]
        D = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2)
        np.fill_diagonal(D, 10 ** 6)
        assert D.min() >= sigma  # Eq. (sep)
        if sigma >= 3:  # Sec. 3.1 (b): neighbour sets disjoint
            for a, b in itertools.combinations(g, 2):
                assert not (nb[a] & nb[b])
        if sigma >= 6:  # Sec. 3.1 (c): q in N_i, q' in N_i' => q not in IL_q'
            for a, b in itertools.combinations(g, 2):
                for q in nb[a]:
                    assert not (il[q] & nb[b])


@pytest.mark.parametrize("sigma", [3, 6])
def test_coloring_separation_sphere(sigma):
    T = Tree(fibonacci_sphere(8192, 7), 5)
    for kappa in (3, 4, 5):
        _check_coloring_properties(T, kappa, sigma)


def test_coloring_separation_torus():
    T = Tree(torus(6000, 3), 4)
    for kappa in (3, 4):
        _check_coloring_properties(T, kappa, 3)
        _check_coloring_properties(T, kappa, 6)


def test_lists_against_definitions():
    """Eq. (dist): neighbours at distance 1, interaction list at 2 or 3; brute force
    over all same-level pairs against the Sec. 2.1 definitions."""
    T = Tree(fibonacci_sphere(3000, 11), 4)
    for kappa in range(2, 5):
        L, P = T.levels[kappa], T.levels[kappa - 1]
        for u in range(L.n):
            want_nb, want_il = [], []
            for v in range(L.n):
                if u == v:
                    continue
                d = dist(L, u, v)
                dp = dist(P, L.parent[u], L.parent[v])
                if d == 1:
                    want_nb.append(v)
                elif d >= 2 and dp == 1:
                    want_il.append(v)
                    assert d in (2, 3)
            assert list(L.nbrs[u]) == want_nb
            assert list(L.il[u]) == want_il


def test_points_partitioned_into_leaves():
    pts = fibonacci_sphere(5000, 2)
    T = Tree(pts, 4)
    leaf = T.levels[4]
    seen = np.concatenate([T.leaf_points(i) for i in range(leaf.n)])
    assert sorted(seen) == list(range(len(pts)))
    h = T.side / 16
    for i in range(leaf.n):
        lo = T.origin + leaf.cells[i] * h
        P = pts[T.leaf_points(i)]
        assert np.all(P >= lo - 1e-12) and np.all(P <= lo + h + 1e-12)
