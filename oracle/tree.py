"""Oracle: uniform octree, neighbour / interaction lists and the greedy coloring.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import or run anything under oracle/.  The product path
never does.

Follows the paper:
  * Sec. 2.1  hierarchical decomposition: uniform tree, neighbours N_i (adjacent
    cells, excluding i), interaction list IL_i (non-adjacent children of the
    neighbours of i's parent).
  * Sec. 3, Eq. (dist)  normalised infinity-norm distance between same-level cells.
  * Sec. 3.4, Algorithm 3  greedy coloring at separation sigma.
Only non-empty cells are kept and colored (Sec. 3.4).

Readings where the paper is silent:
  * root cube: the tight bounding cube of the points, side = max extent * (1+1e-12),
    centred on the bounding-box midpoint;
  * a cell's grid index along one axis is floor((x - origin) / cell size), clamped;
  * nodes of a level are numbered in the scan order of Algorithm 3
    (z slowest, then y, then x), i.e. ascending lin = (iz*m + iy)*m + ix;
  * points are ordered by (leaf lin, original index).
"""

from __future__ import annotations

import numpy as np

NEAR_OFFSETS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


class Level:
    """All non-empty cells of one level."""

    def __init__(self, kappa: int, cells: np.ndarray):
        self.kappa = kappa
        self.m = 1 << kappa
        m = self.m
        lin = (cells[:, 2].astype(np.int64) * m + cells[:, 1]) * m + cells[:, 0]
        order = np.argsort(lin, kind="stable")
        self.cells = np.ascontiguousarray(cells[order]).astype(np.int64)
        self.lin = lin[order]
        self.index = {int(v): k for k, v in enumerate(self.lin)}
        self.n = len(self.lin)
        self.parent = None
        self.children = None
        self.nbrs: list[np.ndarray] = []
        self.il: list[np.ndarray] = []

    def find(self, ix: int, iy: int, iz: int) -> int:
        m = self.m
        if min(ix, iy, iz) < 0 or max(ix, iy, iz) >= m:
            return -1
        return self.index.get((iz * m + iy) * m + ix, -1)


def dist(level: Level, u: int, v: int) -> int:
    """Normalised distance: infinity norm of the centre difference over the cell size."""
    return int(np.max(np.abs(level.cells[u] - level.cells[v])))


class Tree:
    def __init__(self, pts: np.ndarray, depth: int):
        if depth < 2:
            raise ValueError("depth must be >= 2")
        pts = np.asarray(pts, dtype=np.float64)
        self.pts = pts
        self.N = len(pts)
        self.depth = depth
        lo, hi = pts.min(axis=0), pts.max(axis=0)
        self.center = 0.5 * (lo + hi)
        self.side = float(np.max(hi - lo)) * (1.0 + 1e-12)
        self.origin = self.center - 0.5 * self.side
        m = 1 << depth
        h = self.side / m
        g = np.floor((pts - self.origin) / h).astype(np.int64)
        g = np.clip(g, 0, m - 1)
        leaf_lin = (g[:, 2] * m + g[:, 1]) * m + g[:, 0]
        self.perm = np.argsort(leaf_lin, kind="stable")  # tree order -> user index
        self.leaf_of_point_sorted = None
        self.levels: dict[int, Level] = {}
        cells = np.unique(g, axis=0)
        for kappa in range(depth, -1, -1):
            self.levels[kappa] = Level(kappa, cells)
            cells = np.unique(cells // 2, axis=0)
        # parent / children links
        for kappa in range(depth, 0, -1):
            L, P = self.levels[kappa], self.levels[kappa - 1]
            L.parent = np.array([P.find(*(c // 2)) for c in L.cells], dtype=np.int64)
            ch = [[] for _ in range(P.n)]
            for k, p in enumerate(L.parent):
                ch[p].append(k)
            P.children = [np.array(c, dtype=np.int64) for c in ch]
        # points of each leaf, in tree order
        leaf = self.levels[depth]
        lin_sorted = leaf_lin[self.perm]
        node_of_sorted = np.array([leaf.index[int(v)] for v in lin_sorted], dtype=np.int64)
        starts = np.searchsorted(node_of_sorted, np.arange(leaf.n + 1))
        self.leaf_start = starts  # points of leaf i are perm[starts[i]:starts[i+1]]
        # neighbour lists and interaction lists (Sec. 2.1)
        for kappa in range(0, depth + 1):
            L = self.levels[kappa]
            L.nbrs = []
            for c in L.cells:
                nb = []
                for (dx, dy, dz) in NEAR_OFFSETS:
                    if dx == dy == dz == 0:
                        continue
                    k = L.find(c[0] + dx, c[1] + dy, c[2] + dz)
                    if k >= 0:
                        nb.append(k)
                L.nbrs.append(np.array(sorted(nb), dtype=np.int64))
        for kappa in range(0, depth + 1):
            L = self.levels[kappa]
            L.il = []
            cl = [tuple(int(v) for v in c) for c in L.cells]
            for k in range(L.n):
                if kappa < 2:
                    L.il.append(np.zeros(0, dtype=np.int64))
                    continue
                P = self.levels[kappa - 1]
                p = L.parent[k]
                a = cl[k]
                cand = []
                for pn in P.nbrs[p]:
                    for c in P.children[pn]:
                        b = cl[c]
                        if max(abs(a[0] - b[0]), abs(a[1] - b[1]), abs(a[2] - b[2])) >= 2:
                            cand.append(int(c))
                L.il.append(np.array(sorted(cand), dtype=np.int64))

    def leaf_points(self, i: int) -> np.ndarray:
        """User indices of the points in leaf node i (tree order)."""
        return self.perm[self.leaf_start[i]:self.leaf_start[i + 1]]

    def cell_center(self, kappa: int, node: int) -> np.ndarray:
        h = self.side / (1 << kappa)
        return self.origin + (self.levels[kappa].cells[node] + 0.5) * h

    def cell_halfwidth(self, kappa: int) -> float:
        return 0.5 * self.side / (1 << kappa)


def greedy_coloring(level: Level, sigma: int):
    """Algorithm 3: scan (k0, j0, i0); each non-empty uncolored cell opens a new
    color, then the grid is searched for further cells of that color with a
    stride of sigma after every hit (in i), and after rows (j) and planes (k)
    that received a hit.  Returns (color per node, groups in discovery order).

    The innermost scan over i visits only the occupied cells of the row: a miss
    moves i by one cell, so jumping straight to the next occupied cell at or
    after i is the same walk."""
    m = level.m
    rows: dict[tuple[int, int], list[tuple[int, int]]] = {}
    for node, c in enumerate(level.cells):
        rows.setdefault((int(c[2]), int(c[1])), []).append((int(c[0]), node))
    for v in rows.values():
        v.sort()
    occ = {(int(c[2]), int(c[1]), int(c[0])): node for node, c in enumerate(level.cells)}
    color = [-1] * level.n
    groups: list[list[int]] = []

    def scan_row(j, k, i, g, grp):
        """Walk row (j, k) from i; return True if any cell got color g."""
        hit = False
        for (ix, node) in rows.get((k, j), ()):
            if ix < i or color[node] >= 0:
                continue
            color[node] = g
            grp.append(node)
            hit = True
            i = ix + sigma
        return hit

    g = 0
    for k0 in range(m):
        for j0 in range(m):
            if (k0, j0) not in rows:
                continue
            for i0 in range(m):
                node0 = occ.get((k0, j0, i0), -1)
                if node0 < 0 or color[node0] >= 0:
                    continue
                grp = [node0]
                color[node0] = g
                j_stride = True
                k_stride = True
                k = k0
                while k < m:
                    j = j0 if k == k0 else 0
                    while j < m:
                        i = i0 + sigma if (j == j0 and k == k0) else 0
                        if scan_row(j, k, i, g, grp):
                            j_stride = True
                            k_stride = True
                        j = j + sigma if j_stride else j + 1
                        j_stride = False
                    k = k + sigma if k_stride else k + 1
                    k_stride = False
                groups.append(grp)
                g += 1
    return np.array(color, dtype=np.int64), groups
