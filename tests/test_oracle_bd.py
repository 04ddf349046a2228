"""Pins of the block-diagonal preconditioner oracle (Sec. 4.3, Algorithm 5)
against what its definition fixes: level 0 is one block (M = A^-1); M is block
diagonal over the cells of the level; each diagonal block of M A is the identity;
the blocks at a level are the unions of their children's points."""

import numpy as np
import pytest

from oracle.bd import bd_apply, cell_points
from oracle.operators import dense_matrix
from oracle.tree import Tree
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_sphere


def test_level0_is_the_exact_inverse():
    pts = fibonacci_sphere(700, 2)
    tree = Tree(pts, 3)
    r = np.random.default_rng(1).standard_normal(len(pts))
    assert np.linalg.norm(bd_apply(tree, 0, r) - np.linalg.solve(dense_matrix(pts), r)) < 1e-12 * np.linalg.norm(r)


@pytest.mark.parametrize("level", [1, 2, 3])
def test_block_diagonal_structure_and_identity_blocks(level):
    pts = bumpy_sphere(900, 4)
    tree = Tree(pts, 3)
    A = dense_matrix(pts)
    cells = cell_points(tree, level)
    assert sorted(np.concatenate(cells).tolist()) == list(range(len(pts)))
    rng = np.random.default_rng(level)
    for idx in cells[:: max(1, len(cells) // 5)]:
        # a right-hand side on one cell stays on that cell
        r = np.zeros(len(pts))
        r[idx] = rng.standard_normal(len(idx))
        v = bd_apply(tree, level, r)
        outside = np.setdiff1d(np.arange(len(pts)), idx)
        assert np.all(v[outside] == 0.0)
        # and (M A)_cc = I on the cell's own block
        assert np.allclose(A[np.ix_(idx, idx)] @ v[idx], r[idx], rtol=0, atol=1e-12 * np.abs(r).max())


def test_cells_are_unions_of_their_children():
    pts = fibonacci_sphere(1200, 5)
    tree = Tree(pts, 4)
    for level in (2, 3):
        parent = tree.levels[level + 1].parent
        fine = cell_points(tree, level + 1)
        coarse = cell_points(tree, level)
        for a, idx in enumerate(coarse):
            kids = np.concatenate([fine[c] for c in range(len(fine)) if parent[c] == a])
            assert sorted(idx.tolist()) == sorted(kids.tolist())
