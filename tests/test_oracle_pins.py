"""Pins of the oracle's rank rule, weighted re-basing and coloring against what
the paper and the mathematics fix, each chosen so that a plausible slip fails:

* the truncation rule of Sec. 5.1 ("relative error eps"): singular values kept
  strictly above eps * s_1 (a tie is dropped), the eps = 0 numerical-rank
  threshold max(m, n) * 2^-52 * s_1, and eps applied to s_j, not s_j^2;
* the shared rank of a node's two bases: the larger of the row and column
  counts, capped by the available width (both truncations must meet eps);
* the R_Z weighting of the re-basing: after a re-base every far-field block the
  old basis fed (M2L_lq for l in IL_q, M2M_q), every fill-in, and the column-side
  blocks are reproduced through the new basis to within eps * s_1(G); an
  unweighted variant fails that bound on a constructed case;
* Algorithm 3, restated here on the dense m^3 grid with its own walk, gives the
  oracle's colors on random occupancies.
"""

import numpy as np
import pytest

from oracle.ifmm import Flops, RankPolicy, kept_count, rebase
from oracle.operators import Operators
from oracle.tree import Level, Tree, greedy_coloring
from paper_1905_10602_gb300.workloads import fibonacci_sphere

U52 = 2.0 ** -52


# ------------------------------------------------------------------ rank rule
def test_kept_count_strict_tie_is_dropped():
    # s_2 equals eps * s_1 exactly (1e-6 * 1.0 is exact): a strict ">" drops it
    assert kept_count(np.array([1.0, 1e-6, 5e-7]), (10, 10), 1e-6) == 1
    # just above the threshold it is kept
    assert kept_count(np.array([1.0, 1.0000001e-6, 5e-7]), (10, 10), 1e-6) == 2


def test_kept_count_applies_eps_to_sigma_not_sigma_squared():
    # thr = 1e-6 * 2 = 2e-6: s = 1e-5 is kept (on squares it would not be: 1e-10 < 4e-6)
    assert kept_count(np.array([2.0, 1e-5, 1e-7]), (8, 5), 1e-6) == 2


def test_kept_count_eps0_uses_max_dimension():
    # eps = 0: thr = max(m, n) * 2^-52 * s_1 = 100 * 2^-52 = 2.22e-14; with
    # min(m, n) = 50 it would be 1.11e-14 and keep 1.5e-14
    assert kept_count(np.array([1.0, 1.5e-14, 1e-17]), (100, 50), 0.0) == 1
    assert kept_count(np.array([1.0, 1.5e-14, 1e-17]), (50, 100), 0.0) == 1
    assert kept_count(np.array([1.0, 3e-14, 1e-17]), (100, 50), 0.0) == 2


def test_kept_count_degenerate():
    assert kept_count(np.zeros(0), (0, 4), 1e-6) == 0
    assert kept_count(np.zeros(3), (3, 3), 1e-6) == 0


def test_kept_count_on_matrices_with_prescribed_spectra():
    """G = U diag(s) V^T: the count from G's computed singular values equals the
    number of prescribed values above eps * s_1 (none within rounding of it)."""
    rng = np.random.default_rng(5)
    for m, n, s in [(30, 12, [3.0, 1.0, 2e-3, 7e-6, 2e-6, 4e-7, 1e-9]),
                    (9, 20, [1.0, 0.5, 0.25, 1e-4, 3.1e-6, 2.9e-6, 1e-8, 1e-12, 0.0])]:
        k = len(s)
        U = np.linalg.qr(rng.standard_normal((m, k)))[0]
        V = np.linalg.qr(rng.standard_normal((n, k)))[0]
        G = U @ np.diag(s) @ V.T
        sv = np.linalg.svd(G, compute_uv=False)
        expect = sum(1 for x in s if x > 3e-6 * max(s))
        assert kept_count(sv, G.shape, 3e-6) == expect


def test_rank_policy_takes_the_larger_count_capped_by_width():
    pol = RankPolicy(1e-6)
    s_row = np.array([1.0, 0.1, 1e-3, 1e-9, 1e-10])           # 3 kept
    s_col = np.array([1.0, 0.5, 0.2, 0.1, 1e-2, 1e-12])       # 5 kept
    assert pol.choose(("a",), s_row, (5, 9), s_col, (9, 6)) == 5
    # the row side offers only 4 directions: the rank cannot exceed 4
    assert pol.choose(("b",), s_row[:4], (4, 9), s_col, (9, 6)) == 4
    # the column side keeps fewer: still the larger (row) count
    assert pol.choose(("c",), s_col, (6, 9), s_row, (9, 5)) == 5
    # replay overrides the choice; beyond the width it is an error
    rep = RankPolicy(1e-6, replay={("d",): 2, ("e",): 9})
    assert rep.choose(("d",), s_row, (5, 9), s_col, (9, 6)) == 2
    with pytest.raises(ValueError):
        rep.choose(("e",), s_row, (5, 9), s_col, (9, 6))


# ------------------------------------------------------------------ weighted re-basing
def _orth(rng, m, k):
    return np.linalg.qr(rng.standard_normal((m, k)))[0]


def _represented_errors(Zrow, Zcol, P2M_old, L2P_old, Frows, Fcols, new):
    """Largest 2-norm error, relative to s_1 of the weighted stacks, with which the
    new bases reproduce what the old ones fed: row side M2L_lq P2M_old (each block
    of Zrow) and the row fill-ins; column side L2P_old M2L_ql (each block of Zcol)
    and the column fill-ins."""
    P2M_new, L2P_new, T, Tp = new
    Grow = np.vstack([np.linalg.qr(np.vstack(Zrow), mode="r") @ P2M_old] + list(Frows))
    Gcol = np.hstack([L2P_old @ np.linalg.qr(np.hstack(Zcol).T, mode="r").T] + list(Fcols))
    s1r = np.linalg.norm(Grow, 2)
    s1c = np.linalg.norm(Gcol, 2)
    e = []
    for B in Zrow:  # M2L_lq <- M2L_lq T, acting through P2M_new
        e.append(np.linalg.norm(B @ T @ P2M_new - B @ P2M_old, 2) / s1r)
    for F in Frows:  # fill-in coefficient F P2M_new^T, acting through P2M_new
        e.append(np.linalg.norm(F @ P2M_new.T @ P2M_new - F, 2) / s1r)
    for C in Zcol:  # M2L_ql <- T' M2L_ql, reached through L2P_new
        e.append(np.linalg.norm(L2P_new @ Tp @ C - L2P_old @ C, 2) / s1c)
    for F in Fcols:
        e.append(np.linalg.norm(L2P_new @ L2P_new.T @ F - F, 2) / s1c)
    return max(e)


def _anisotropic_case(seed=3):
    """Old bases whose weakest directions the far field weighs most: P2M_old has
    singular values sp along V_p, and the weight stack Z maps P2M_old's output
    directions U_p with gains w, so Z P2M_old has singular values w * sp."""
    rng = np.random.default_rng(seed)
    n, r = 14, 8
    sp = np.array([1.0, 0.3, 1e-2, 1e-4, 1e-7, 1e-9, 1e-10, 1e-12])
    w = np.array([1.0, 1.0, 1.0, 1.0, 1e6, 1e6, 1e2, 1.0])  # w * sp: 1 .3 1e-2 1e-4 .1 1e-3 1e-8 1e-12
    Up, Vp = _orth(rng, r, r), _orth(rng, n, r)
    P2M_old = Up @ np.diag(sp) @ Vp.T
    Z = _orth(rng, 30, r) @ np.diag(w) @ Up.T  # 30 x r: three IL blocks and an M2M
    Zrow = [Z[:8], Z[8:16], Z[16:24], Z[24:]]
    # column side: L2P_old (n x r) and blocks M2L_ql (r x c) with gains wc
    sc = np.array([1.0, 0.5, 1e-3, 1e-5, 1e-8, 1e-8, 1e-11, 1e-13])
    wc = np.array([1.0, 1.0, 1.0, 1.0, 1e5, 1e4, 1e5, 1.0])  # wc * sc: 1 .5 1e-3 1e-5 1e-3 1e-4 1e-6 1e-13
    Uc, Vc = _orth(rng, n, r), _orth(rng, r, r)
    L2P_old = Uc @ np.diag(sc) @ Vc.T
    Zc = Vc @ np.diag(wc) @ _orth(rng, 24, r).T  # r x 24
    Zcol = [Zc[:, :8], Zc[:, 8:16], Zc[:, 16:]]
    return Zrow, Zcol, P2M_old, L2P_old


def test_rebase_weighted_reproduces_every_far_block_within_eps():
    eps = 1e-6
    Zrow, Zcol, P2M_old, L2P_old = _anisotropic_case()
    pol = RankPolicy(eps)
    new = rebase(Flops(), Zrow, Zcol, P2M_old, L2P_old, [], [], pol, ("k",))
    # row side keeps w*sp > 1e-6: 1 .3 1e-2 1e-4 .1 1e-3 -> 6; column side wc*sc >
    # 1e-6 (the tie at 1e-6 * 1 = 1e-6 is dropped): 1 .5 1e-3 1e-5 1e-3 1e-4 -> 6
    assert pol.log[("k",)] == 6
    assert _represented_errors(Zrow, Zcol, P2M_old, L2P_old, [], [], new) <= 1.01 * eps


def test_rebase_unweighted_variant_fails_the_bound():
    """Deliberately dropping R_Z (weights = identity) truncates the directions the
    far field amplifies: the represented blocks miss by far more than eps."""
    eps = 1e-6
    Zrow, Zcol, P2M_old, L2P_old = _anisotropic_case()
    r = P2M_old.shape[0]
    unweighted = rebase(Flops(), [np.eye(r)], [np.eye(r)], P2M_old, L2P_old, [], [], RankPolicy(eps), ("u",))
    assert unweighted[0].shape[0] == 4  # sp > 1e-6: 1 .3 1e-2 1e-4; sc: 1 .5 1e-3 1e-5
    assert _represented_errors(Zrow, Zcol, P2M_old, L2P_old, [], [], unweighted) > 1e3 * eps


def test_rebase_keeps_fill_ins_and_uses_the_larger_side():
    """Fill-ins stacked under the weighted basis are reproduced within eps; the
    column side needs more directions than the row side, and the shared rank
    (the larger count) meets both bounds, where the smaller would not."""
    eps = 1e-6
    rng = np.random.default_rng(8)
    Zrow, Zcol, P2M_old, L2P_old = _anisotropic_case(4)
    n = P2M_old.shape[1]
    Frows = [rng.standard_normal((5, n)) @ np.diag(np.logspace(0, -9, n)) for _ in range(2)]
    Fcols = [np.diag(np.logspace(0, -12, n)) @ rng.standard_normal((n, 6)) for _ in range(3)]
    pol = RankPolicy(eps)
    new = rebase(Flops(), Zrow, Zcol, P2M_old, L2P_old, Frows, Fcols, pol, ("f",))
    assert _represented_errors(Zrow, Zcol, P2M_old, L2P_old, Frows, Fcols, new) <= 1.01 * eps
    Grow = np.vstack([np.linalg.qr(np.vstack(Zrow), mode="r") @ P2M_old] + Frows)
    Gcol = np.hstack([L2P_old @ np.linalg.qr(np.hstack(Zcol).T, mode="r").T] + Fcols)
    s_r = np.linalg.svd(Grow, compute_uv=False)
    s_c = np.linalg.svd(Gcol, compute_uv=False)
    kr, kc = int(np.sum(s_r > eps * s_r[0])), int(np.sum(s_c > eps * s_c[0]))
    assert kr != kc and pol.log[("f",)] == max(kr, kc)
    # with the smaller count one side misses its bound
    small = RankPolicy(eps, replay={("g",): min(kr, kc)})
    low = rebase(Flops(), Zrow, Zcol, P2M_old, L2P_old, Frows, Fcols, small, ("g",))
    assert _represented_errors(Zrow, Zcol, P2M_old, L2P_old, Frows, Fcols, low) > 2 * eps


def test_rebase_on_real_operators_meets_the_bound():
    """A level-start re-base on the Chebyshev operators of a real tree: every
    M2L_lq, M2M_q and column-side block is reproduced within eps."""
    eps = 1e-6
    pts = fibonacci_sphere(1500, 2)
    tree = Tree(pts, 3)
    ops = Operators(tree, 3)
    L = tree.levels[3]
    checked = 0
    for q in range(0, L.n, 37):
        il = [int(l) for l in L.il[q]]
        if not il:
            continue
        Zrow = [ops.m2l(3, l, q) for l in il] + [ops.m2m(3, q)]
        Zcol = [ops.m2l(3, q, l) for l in il] + [ops.m2m(3, q).T]
        P2M0 = ops.p2m_leaf(q)
        new = rebase(Flops(), Zrow, Zcol, P2M0, P2M0.T.copy(), [], [], RankPolicy(eps), ("r", q))
        assert _represented_errors(Zrow, Zcol, P2M0, P2M0.T.copy(), [], [], new) <= 1.01 * eps
        checked += 1
    assert checked >= 3


# ------------------------------------------------------------------ Algorithm 3
def _alg3_dense(occ: np.ndarray, sigma: int) -> np.ndarray:
    """Algorithm 3 (Sec. 3.4) on the full m^3 grid (occ[k, j, i]: cell non-empty).
    Cells are scanned with x fastest; each non-empty uncolored cell u opens a
    color, and one sweep over the rest of the grid (from u's row on) gives that
    color to every non-empty uncolored cell it lands on.  The sweep moves sigma
    cells after a hit along x and one cell after a miss; it moves to the next
    row sigma rows ahead if the row (or u's own row) had a hit, else one row;
    and likewise between planes."""
    m = occ.shape[0]
    color = -np.ones(occ.shape, dtype=np.int64)
    g = 0
    for u in range(m ** 3):
        k0, j0, i0 = u // (m * m), (u // m) % m, u % m
        if not occ[k0, j0, i0] or color[k0, j0, i0] >= 0:
            continue
        color[k0, j0, i0] = g
        k = k0
        while k < m:
            plane_hit = k == k0
            j = j0 if k == k0 else 0
            while j < m:
                row_hit = (k == k0 and j == j0)
                i = i0 + sigma if row_hit else 0
                while i < m:
                    if occ[k, j, i] and color[k, j, i] < 0:
                        color[k, j, i] = g
                        row_hit = True
                        i += sigma
                    else:
                        i += 1
                plane_hit = plane_hit or row_hit
                j += sigma if row_hit else 1
            k += sigma if plane_hit else 1
        g += 1
    return color


@pytest.mark.parametrize("m,sigma,density,seed", [(8, 3, 0.3, 1), (8, 6, 0.5, 2), (16, 3, 0.08, 3),
                                                  (16, 6, 0.15, 4), (16, 3, 1.0, 5), (12, 6, 0.02, 6)])
def test_oracle_coloring_is_algorithm3(m, sigma, density, seed):
    rng = np.random.default_rng(seed)
    occ = rng.random((m, m, m)) < density
    occ[0, 0, 0] |= density >= 1.0
    kz, jy, ix = np.nonzero(occ)
    cells = np.stack([ix, jy, kz], axis=1)
    kappa = int(np.log2(m)) if (m & (m - 1)) == 0 else None
    if kappa is None:  # a grid that is not a power of two: embed it in the next level
        kappa = int(np.ceil(np.log2(m)))
        big = np.zeros((1 << kappa,) * 3, dtype=bool)
        big[:m, :m, :m] = occ
        occ = big
    level = Level(kappa, cells)
    col_oracle, groups = greedy_coloring(level, sigma)
    dense = _alg3_dense(occ, sigma)
    expect = np.array([dense[c[2], c[1], c[0]] for c in level.cells])
    assert np.array_equal(col_oracle, expect)
    # groups list the nodes of each color in discovery (scan) order
    for g, grp in enumerate(groups):
        assert all(col_oracle[v] == g for v in grp)
