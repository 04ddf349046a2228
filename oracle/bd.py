"""Oracle: the block-diagonal preconditioner BD / BDbot l_BD.

TEST INFRASTRUCTURE ONLY (see oracle/tree.py).

Sec. 4.3 and Algorithm 5: the preconditioner M is block diagonal, one block per
non-empty cell i of level l_BD, M_ii = (A_ii)^{-1} with A_ii the self block of A
over the points of cell i (at the leaf level, the self P2P operator); applying
M solves A_ii v_i = r_i for every cell independently.  Plain NumPy, FP64, one
cell at a time (the paper factorizes each block by LU; a dense solve is the
same operator).
"""

from __future__ import annotations

import numpy as np

from .operators import kernel_block
from .tree import Tree


def cell_points(tree: Tree, level: int) -> list[np.ndarray]:
    """User indices of the points of every non-empty cell of `level`, each cell's
    points in tree order (its leaves in leaf order)."""
    leaf = tree.levels[tree.depth]
    out = [[] for _ in range(tree.levels[level].n)]
    for i in range(leaf.n):
        a = i
        for kappa in range(tree.depth, level, -1):
            a = int(tree.levels[kappa].parent[a])
        out[a].append(tree.leaf_points(i))
    return [np.concatenate(x) if x else np.zeros(0, dtype=np.int64) for x in out]


def bd_apply(tree: Tree, level: int, r: np.ndarray) -> np.ndarray:
    """v = M r: the self block of every cell of `level` solved against r's entries there."""
    pts = tree.pts
    N = len(pts)
    v = np.zeros_like(np.asarray(r, dtype=np.float64))
    for idx in cell_points(tree, level):
        if len(idx) == 0:
            continue
        Aii = kernel_block(N, pts[idx], pts[idx], same=True)
        v[idx] = np.linalg.solve(Aii, r[idx])
    return v
