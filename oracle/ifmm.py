"""Oracle: IFMM factorization and solve on the extended sparse system.

TEST INFRASTRUCTURE ONLY (see oracle/tree.py).  Plain NumPy, FP64, one node at
a time, no blocking or fusion beyond what the steps below state.

Passages followed: Eq. (1) (extended sparse system), Algorithm 1 (factorization,
Sec. 2.3), Algorithm 2 (solve, Sec. 2.4), Sec. 3.2/3.3 (colors processed in
order, nodes of a color independent; sigma=3 serializes the interaction-list
updates), Sec. 5.1 (low-rank compression at relative error eps).

Variables and rows of node i at level kappa (Eq. (1)):
    x_i (n_i)   particles / the children's multipoles,
    y_i (r_i)   multipole coefficients,   row E_y,i:  P2M_i x_i - y_i = 0
    z_i (r_i)   local coefficients,       row R_i:    -z_i + sum_{l in IL_i} M2L_il y_l + L2L_i z_parent = 0
                                          row E_x,i:  P2P_ii x_i + sum_q P2P_iq x_q + L2P_i z_i = b_i
Eliminating node i removes (x_i, z_i) with the pivot rows (E_x,i, E_y,i); y_i
stays with row R_i and becomes part of the parent's x (Sec. 2.3 "aggregate").

Readings of the paper (where it is silent or ambiguous):
  R1 pivot: Pi_i = [[P2P_ii, L2P_i], [P2M_i, 0]] is inverted as a whole
     ("factorize P2P_ii and eliminate node i", Alg. 1).
  R2 block state: between nodes p, q with dist <= 1 there is one current block,
     row E_x,p (p live) or R_p (p eliminated) times column x_q (q live) or y_q
     (q eliminated): P2P, P2L, M2P or M2L in the paper's names.
  R3 fill-ins of pairs (p, q) in N_i x N_i at distance 2 (p in IL_q, because the
     parents are adjacent) are far fields: both eliminated -> add to M2L (Case 1);
     otherwise fold into the live node's basis and add the coefficients to M2L
     (Cases 2-4).
  R4 weighted recompression: the row basis of live q is recomputed from the SVD
     of G = [R P2M_q ; F_1 ; F_2 ...] where R is the R factor of
     Z_q = [M2L_lq (l in IL_q) ; M2M_q] and the F are the far fill-ins in
     column x_q; the column basis likewise from [L2P_q R'^T, F'_1, ...] with R'
     the R factor of [M2L_ql ..., L2L_q]^T.  Keep singular values s_j > eps*s_1
     (eps = 0: s_j > max(m, n) * 2^-52 * s_1).  Both bases of a node share one
     rank, the larger of the two counts (Pi_i must be square).
  R5 each level starts by recompressing every node with no fill-ins (the
     initial leaf rank can exceed the number of points).
  R6 Case 2's "l in IL_p" (Alg. 1) is read as l in IL_q: the node whose basis
     changes is q.
  R7 order: colors ascending, nodes of a color in discovery order; per color,
     phase A eliminates every node and computes every new basis from the state
     at the start of the color, phase B re-expresses the touched M2L, M2M, L2L
     blocks (M <- T'_a M T_b), phase C adds the fill-in coefficients.
  R8 top level: levels ell..2 are eliminated; the remaining y of level 2 with
     their R rows form the dense system that is solved by LU (Sec. 2.3, Alg. 1
     remark; Sec. 2.4 remark "level 1").
"""

from __future__ import annotations

import math
from collections import defaultdict

import numpy as np
import scipy.linalg

from .operators import Operators
from .tree import Tree, greedy_coloring

DBL_EPS = 2.0 ** -52


class Flops:
    """Algorithmic work: GEMM 2mnk; inverse 2n^3 (Gauss-Jordan); Householder QR
    (R only) 2mn^2 - 2n^3/3 with n = min; SVD 6mn^2 + 20n^3 (R-SVD: S, U1, V);
    LU 2n^3/3."""

    def __init__(self):
        self.by_kind = defaultdict(float)

    def gemm(self, m, n, k):
        self.by_kind["gemm"] += 2.0 * m * n * k

    def inv(self, n):
        self.by_kind["inv"] += 2.0 * n ** 3

    def qr(self, m, n):
        a, b = max(m, n), min(m, n)
        self.by_kind["qr"] += 2.0 * a * b * b - 2.0 * b ** 3 / 3.0

    def svd(self, m, n):
        a, b = max(m, n), min(m, n)
        self.by_kind["svd"] += 6.0 * a * b * b + 20.0 * b ** 3

    def lu(self, n):
        self.by_kind["lu"] += 2.0 * n ** 3 / 3.0

    @property
    def total(self):
        return sum(self.by_kind.values())


def _mm(fl: Flops, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    fl.gemm(A.shape[0], B.shape[1], A.shape[1])
    return A @ B


def _h(A: np.ndarray) -> np.ndarray:
    """Conjugate transpose (the transpose for real data): the adjoint an
    orthonormal basis is inverted by."""
    return A.conj().T


def kept_count(s: np.ndarray, shape, eps: float) -> int:
    """Number of singular values kept at relative error eps (reading R4)."""
    if len(s) == 0 or s[0] <= 0.0:
        return 0
    thr = eps * s[0] if eps > 0.0 else max(shape) * DBL_EPS * s[0]
    return int(np.count_nonzero(s > thr))


class RankPolicy:
    """Rank of each recompression event.  Event key: (level, node, k) with k the
    count of earlier events of that node at that level (k = 0: level start).

    The rule is pinned against the mathematics (strict threshold, the eps = 0
    numerical-rank threshold, the larger of the two counts, and the weighted
    re-basing reproducing every far block within eps).  The paper prints no
    ranks for this kernel, so the absolute ranks of a whole factorization are
    not pinned beyond that rule; the CUDA path is compared with them replayed."""

    def __init__(self, eps: float, replay: dict | None = None):
        self.eps = eps
        self.replay = replay
        self.log: dict = {}

    def choose(self, key, s_row, shape_row, s_col, shape_col) -> int:
        k_row = kept_count(s_row, shape_row, self.eps)
        k_col = kept_count(s_col, shape_col, self.eps)
        cap = min(len(s_row), len(s_col))
        k = min(max(k_row, k_col), cap)
        if self.replay is not None:
            k = int(self.replay[key])
            if k > cap:
                raise ValueError(f"replayed rank {k} exceeds available {cap} at {key}")
        self.log[key] = k
        return k


def rebase(fl: Flops, Zrow: list, Zcol: list, P2M_old, L2P_old, Frows: list, Fcols: list, policy, key):
    """Reading R4: new orthonormal row/column bases of one live node.

    Returns (P2M_new, L2P_new, T, T') with T = P2M_old V (old y = T new y) and
    T' = U^T L2P_old (new z = T' old z)."""
    n = P2M_old.shape[1]
    r_old = P2M_old.shape[0]
    if Zrow:
        Z = np.vstack(Zrow)
        fl.qr(*Z.shape)
        Rr = np.linalg.qr(Z, mode="r")
    else:
        Rr = np.zeros((0, r_old))
    if Zcol:
        Zc = np.hstack(Zcol)
        fl.qr(*Zc.shape)
        Rc = np.linalg.qr(_h(Zc), mode="r")
    else:
        Rc = np.zeros((0, r_old))
    Grow = np.vstack([_mm(fl, Rr, P2M_old)] + list(Frows))
    Gcol = np.hstack([_mm(fl, L2P_old, _h(Rc))] + list(Fcols))
    if Grow.size:
        fl.svd(*Grow.shape)
        _, s_r, Vt = np.linalg.svd(Grow, full_matrices=False)
    else:
        s_r, Vt = np.zeros(0), np.zeros((0, n))
    if Gcol.size:
        fl.svd(*Gcol.shape)
        U, s_c, _ = np.linalg.svd(Gcol, full_matrices=False)
    else:
        s_c, U = np.zeros(0), np.zeros((n, 0))
    k = policy.choose(key, s_r, Grow.shape, s_c, Gcol.shape)
    P2M_new = np.ascontiguousarray(Vt[:k])
    L2P_new = np.ascontiguousarray(U[:, :k])
    T = _mm(fl, P2M_old, _h(P2M_new))
    Tp = _mm(fl, _h(L2P_new), L2P_old)
    return P2M_new, L2P_new, T, Tp


class LevelFactor:
    """What the solve needs from one level."""

    def __init__(self, kappa):
        self.kappa = kappa
        self.order = []  # colors: lists of node ids
        self.piv = {}  # i -> (PiInv, clique, was_elim, Lc, Ur, n_i, r_i)
        self.n = None  # x dims
        self.r_final = None  # y dims at the end of the level
        self.children = None  # parent-level children lists (for x_parent = stack y_c)


class IFMMOracle:
    """IFMM factorization (Algorithm 1 with colors, Sec. 3) and solve (Algorithm 2)."""

    def __init__(self, pts, depth, cheb_order, eps, sigma=6, rank_replay=None, color_groups=None, wavenumber=0.0):
        self.tree = Tree(pts, depth)
        self.ops = Operators(self.tree, cheb_order, wavenumber)
        self.eps = eps
        self.sigma = sigma
        self.flops = Flops()
        self.policy = RankPolicy(eps, rank_replay)
        self.colors = {}
        for kappa in range(2, depth + 1):
            if color_groups is not None and kappa in color_groups:
                self.colors[kappa] = [list(g) for g in color_groups[kappa]]
            else:
                _, groups = greedy_coloring(self.tree.levels[kappa], sigma)
                self.colors[kappa] = groups
        self.levels: dict[int, LevelFactor] = {}
        self.top = None
        self.rank_events = defaultdict(int)

    # ---------------------------------------------------------------- factor
    def factor(self):
        T, ops, fl = self.tree, self.ops, self.flops
        ell = T.depth
        carry = None
        for kappa in range(ell, 1, -1):
            L = T.levels[kappa]
            S = self._init_level(kappa, carry)
            lf = LevelFactor(kappa)
            lf.n = dict(S["n"])
            for grp in self.colors[kappa]:
                self._eliminate_color(S, kappa, grp, lf)
                lf.order.append(list(grp))
            lf.r_final = dict(S["r"])
            self.levels[kappa] = lf
            if kappa > 2:
                carry = self._aggregate(S, kappa)
            else:
                self._top(S)
        return self

    def _init_level(self, kappa, carry):
        """Level start: operators at this level, then reading R5."""
        T, ops, fl = self.tree, self.ops, self.flops
        L = T.levels[kappa]
        S = {"near": {}, "far": {}, "P2M": {}, "L2P": {}, "M2M": {}, "L2L": {}, "n": {}, "r": {},
             "elim": set(), "nbrset": [set(int(v) for v in nb) for nb in L.nbrs]}
        if carry is None:  # leaf level
            for i in range(L.n):
                for j in [i] + [int(v) for v in L.nbrs[i]]:
                    S["near"][(i, j)] = ops.p2p(i, j)
                S["n"][i] = len(T.leaf_points(i))
            P2M0 = {i: ops.p2m_leaf(i) for i in range(L.n)}
            L2P0 = {i: P2M0[i].T.copy() for i in range(L.n)}
        else:
            S["near"], S["n"], P2M0, L2P0 = carry
        far0 = {}
        for a in range(L.n):
            for b in L.il[a]:
                far0[(a, int(b))] = ops.m2l(kappa, a, int(b))
        M2M0, L2L0 = {}, {}
        if kappa > 2:
            for q in range(L.n):
                M2M0[q] = ops.m2m(kappa, q)
                L2L0[q] = M2M0[q].T.copy()
        new = {}
        for q in range(L.n):
            Zrow = [far0[(int(l), q)] for l in L.il[q]] + ([M2M0[q]] if kappa > 2 else [])
            Zcol = [far0[(q, int(l))] for l in L.il[q]] + ([L2L0[q]] if kappa > 2 else [])
            key = (kappa, q, self.rank_events[(kappa, q)])
            self.rank_events[(kappa, q)] += 1
            new[q] = rebase(fl, Zrow, Zcol, P2M0[q], L2P0[q], [], [], self.policy, key)
        for q in range(L.n):
            P2M, L2P, Tq, Tpq = new[q]
            S["P2M"][q], S["L2P"][q], S["r"][q] = P2M, L2P, P2M.shape[0]
            if kappa > 2:
                S["M2M"][q] = _mm(fl, M2M0[q], Tq)
                S["L2L"][q] = _mm(fl, Tpq, L2L0[q])
        for (a, b), K in far0.items():
            S["far"][(a, b)] = _mm(fl, _mm(fl, new[a][3], K), new[b][2])
        return S

    def _eliminate_color(self, S, kappa, grp, lf):
        """One color (reading R7)."""
        fl = self.flops
        L = self.tree.levels[kappa]
        near, far = S["near"], S["far"]
        fills_far = []
        Frows, Fcols = defaultdict(list), defaultdict(list)
        rebase_set = []
        # ---- phase A: eliminate every node of the color
        for i in grp:
            ni, ri = S["n"][i], S["r"][i]
            Pi = np.block([[near[(i, i)], S["L2P"][i]], [S["P2M"][i], np.zeros((ri, ri))]])
            fl.inv(ni + ri)
            PiInv = np.linalg.inv(Pi)
            clique = [int(v) for v in L.nbrs[i]]
            was_elim = {q: (q in S["elim"]) for q in clique}
            Lc = {q: near[(q, i)] for q in clique}
            Ur = {q: near[(i, q)] for q in clique}
            lf.piv[i] = (PiInv, clique, was_elim, Lc, Ur, ni, ri)
            A11, A12 = PiInv[:ni, :ni], PiInv[:ni, ni:]
            A21, A22 = PiInv[ni:, :ni], PiInv[ni:, ni:]
            near[(i, i)] = -A22
            for q in clique:
                near[(i, q)] = _mm(fl, A21, Ur[q])
                near[(q, i)] = _mm(fl, Lc[q], A12)
            S["elim"].add(i)
            for q in clique:
                X = _mm(fl, Lc[q], A11)
                for q2 in clique:
                    F = -_mm(fl, X, Ur[q2])
                    if q2 == q or q2 in S["nbrset"][q]:
                        near[(q, q2)] = near[(q, q2)] + F
                    else:  # q2 in IL_q (reading R3)
                        fills_far.append((q, q2, F))
                        if not was_elim[q]:
                            Fcols[q].append(F)
                        if not was_elim[q2]:
                            Frows[q2].append(F)
            for q in clique:
                if not was_elim[q] and (Fcols[q] or Frows[q]) and q not in rebase_set:
                    rebase_set.append(q)
        # ---- phase A (cont.): new bases from the start-of-color state
        new = {}
        for q in rebase_set:
            Zrow = [far[(int(l), q)] for l in L.il[q]] + ([S["M2M"][q]] if kappa > 2 else [])
            Zcol = [far[(q, int(l))] for l in L.il[q]] + ([S["L2L"][q]] if kappa > 2 else [])
            key = (kappa, q, self.rank_events[(kappa, q)])
            self.rank_events[(kappa, q)] += 1
            new[q] = rebase(fl, Zrow, Zcol, S["P2M"][q], S["L2P"][q], Frows[q], Fcols[q], self.policy, key)
        # ---- phase B: re-express blocks touching a re-based node
        touched = set()
        for q in rebase_set:
            P2M, L2P, Tq, Tpq = new[q]
            S["P2M"][q], S["L2P"][q], S["r"][q] = P2M, L2P, P2M.shape[0]
            if kappa > 2:
                S["M2M"][q] = _mm(fl, S["M2M"][q], Tq)
                S["L2L"][q] = _mm(fl, Tpq, S["L2L"][q])
            for l in L.il[q]:
                touched.add((q, int(l)))
                touched.add((int(l), q))
        for (a, b) in sorted(touched):
            M = far[(a, b)]
            if a in new:
                M = _mm(fl, new[a][3], M)
            if b in new:
                M = _mm(fl, M, new[b][2])
            far[(a, b)] = M
        # ---- phase C: fill-in coefficients in the new bases
        for (a, b, F) in fills_far:
            C = F
            if a not in S["elim"]:
                C = _mm(fl, _h(S["L2P"][a]), C)
            if b not in S["elim"]:
                C = _mm(fl, C, _h(S["P2M"][b]))
            far[(a, b)] = far[(a, b)] + C

    def _block_R_y(self, S, L, a, b):
        """Block R_a x y_b once both are eliminated."""
        if a == b or b in S["nbrset"][a]:
            return S["near"][(a, b)]
        return S["far"][(a, b)]

    def _aggregate(self, S, kappa):
        """Algorithm 1, end of a level: children's R rows / y columns become the
        parent's P2P; [M2M_c] the parent's P2M; stacked L2L_c its L2P."""
        T = self.tree
        L, P = T.levels[kappa], T.levels[kappa - 1]
        near_p, n_p, P2M0, L2P0 = {}, {}, {}, {}
        for a in range(P.n):
            ch = [int(c) for c in P.children[a]]
            n_p[a] = sum(S["r"][c] for c in ch)
            P2M0[a] = np.hstack([S["M2M"][c] for c in ch])
            L2P0[a] = np.vstack([S["L2L"][c] for c in ch])
        for a in range(P.n):
            cha = [int(c) for c in P.children[a]]
            for b in [a] + [int(v) for v in P.nbrs[a]]:
                chb = [int(c) for c in P.children[b]]
                near_p[(a, b)] = np.block([[self._block_R_y(S, L, c, d) for d in chb] for c in cha])
        return near_p, n_p, P2M0, L2P0

    def _top(self, S):
        """Reading R8: dense LU of the level-2 R rows on the level-2 y."""
        L = self.tree.levels[2]
        D = np.block([[self._block_R_y(S, L, a, b) for b in range(L.n)] for a in range(L.n)])
        self.flops.lu(D.shape[0])
        self.top = scipy.linalg.lu_factor(D)
        self.top_dims = [S["r"][a] for a in range(L.n)]

    # ---------------------------------------------------------------- solve
    def solve(self, b: np.ndarray) -> np.ndarray:
        """Algorithm 2 on the extended system: forward (upward, colors ascending),
        dense top solve, backward (downward, colors descending)."""
        T = self.tree
        ell = T.depth
        bt = np.asarray(b)
        if not np.iscomplexobj(bt):
            bt = bt.astype(np.float64)
        rhs_x = {}
        leaf = T.levels[ell]
        for i in range(leaf.n):
            rhs_x[i] = bt[T.leaf_points(i)].copy()
        saved_rhs = {}
        for kappa in range(ell, 1, -1):
            lf = self.levels[kappa]
            rhs_R = {}
            for grp in lf.order:
                for i in grp:
                    PiInv, clique, was_elim, Lc, Ur, ni, ri = lf.piv[i]
                    t = PiInv @ np.concatenate([rhs_x[i], np.zeros(ri)])
                    for q in clique:
                        if was_elim[q]:
                            rhs_R[q] = rhs_R[q] - Lc[q] @ t[:ni]
                        else:
                            rhs_x[q] = rhs_x[q] - Lc[q] @ t[:ni]
                    rhs_R[i] = t[ni:].copy()
            saved_rhs[kappa] = (rhs_x, rhs_R)
            if kappa > 2:
                P = T.levels[kappa - 1]
                rhs_x = {a: np.concatenate([rhs_R[int(c)] for c in P.children[a]]) for a in range(P.n)}
        L2 = T.levels[2]
        _, rhs_R2 = saved_rhs[2]
        ytop = scipy.linalg.lu_solve(self.top, np.concatenate([rhs_R2[a] for a in range(L2.n)]))
        y = {}
        off = 0
        for a in range(L2.n):
            y[a] = ytop[off:off + self.top_dims[a]]
            off += self.top_dims[a]
        x_leaf = None
        for kappa in range(2, ell + 1):
            lf = self.levels[kappa]
            rhs_x, _ = saved_rhs[kappa]
            x = {}
            for grp in reversed(lf.order):
                for i in grp:
                    PiInv, clique, was_elim, Lc, Ur, ni, ri = lf.piv[i]
                    s = rhs_x[i].copy()
                    for q in clique:
                        s -= Ur[q] @ (y[q] if was_elim[q] else x[q])
                    xz = PiInv @ np.concatenate([s, y[i]])
                    x[i] = xz[:ni]
            if kappa < ell:
                Lc_ = T.levels[kappa]
                y = {}
                for a in range(Lc_.n):
                    off = 0
                    for c in Lc_.children[a]:
                        rc = self.levels[kappa + 1].r_final[int(c)]
                        y[int(c)] = x[a][off:off + rc]
                        off += rc
            else:
                x_leaf = x
        out = np.empty(T.N, dtype=np.result_type(bt, *[v.dtype for v in x_leaf.values()]))
        for i in range(leaf.n):
            out[T.leaf_points(i)] = x_leaf[i]
        return out

    def ranks(self):
        return dict(self.policy.log)
