"""CUDA path against the oracle, element by element, through the C ABI.

Tolerances: the FP64 path must reproduce the oracle's applied inverse to a
relative 2-norm difference <= 1e-9 (rank replay at finite eps, so both sides
truncate to the same ranks); at eps = 0 both equal A~^{-1} (1e-11); the
direct-summation matvec matches the dense product to 1e-13.
"""

import numpy as np
import pytest

from oracle.dense import direct_matvec, fmm_matrix
from oracle.gmres import gmres as oracle_gmres
from oracle.ifmm import IFMMOracle
from oracle.operators import dense_matrix
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_sphere, point_source_rhs, torus

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _gpu(pts, depth, p, eps, sigma, replay=None, **kw):
    t = ifmm.ifmm_build_tree(pts, depth)
    ifmm.ifmm_color(t, sigma)
    rep = None if replay is None else [list(k) + [v] for k, v in replay.items()]
    f = ifmm.ifmm_factor(t, p, eps, rank_mode="replay" if rep else "svd", replay=rep, **kw)
    return t, f


@pytest.mark.parametrize("N,depth,p,sigma", [(200, 2, 2, 3), (600, 2, 3, 6), (1024, 3, 3, 6), (1024, 3, 3, 3),
                                             (1500, 3, 4, 3)])
def test_exact_at_eps0(N, depth, p, sigma):
    """eps = 0: the GPU factorization is exact Gaussian elimination on the extended
    system; its solve equals the oracle's and A~^{-1} b."""
    pts = fibonacci_sphere(N, 1)
    b = point_source_rhs(pts)
    o = IFMMOracle(pts, depth, p, 0.0, sigma).factor()
    t, f = _gpu(pts, depth, p, 0.0, sigma)
    xg = ifmm.ifmm_solve(f, b)
    assert _rel(xg, o.solve(b)) < 1e-11
    At = fmm_matrix(o.tree, o.ops)
    assert _rel(xg, np.linalg.solve(At, b)) < 1e-11


@pytest.mark.parametrize("shape,N,depth,p,eps,sigma", [
    ("sphere", 2048, 3, 3, 1e-6, 6),   # the 2,048-point sphere workload
    ("sphere", 2048, 3, 3, 1e-6, 3),
    ("bumpy", 3000, 4, 3, 1e-6, 3),    # ragged tail: 4 levels, bumpy surface
    ("torus", 2500, 3, 4, 1e-4, 6),
])
def test_replay_parity(shape, N, depth, p, eps, sigma):
    """Finite eps with the oracle's ranks replayed: applied inverse within 1e-9."""
    pts = {"sphere": fibonacci_sphere, "bumpy": bumpy_sphere, "torus": torus}[shape](N, 3)
    o = IFMMOracle(pts, depth, p, eps, sigma).factor()
    t, f = _gpu(pts, depth, p, eps, sigma, replay=o.ranks())
    rng = np.random.default_rng(7)
    R = rng.standard_normal((3, N))
    V = ifmm.ifmm_solve(f, R)
    for k in range(3):
        assert _rel(V[k], o.solve(R[k])) < 1e-9
    assert ifmm.ifmm_fact_ranks(f) == o.ranks()


def test_free_ranks_agree_with_oracle():
    """Without replay the GPU chooses its own ranks; they match the oracle's except
    for singular values within rounding of the threshold, and the solve is within eps."""
    pts = fibonacci_sphere(2048, 1)
    o = IFMMOracle(pts, 3, 3, 1e-6, 6).factor()
    t, f = _gpu(pts, 3, 3, 1e-6, 6)
    rg, ro = ifmm.ifmm_fact_ranks(f), o.ranks()
    assert rg.keys() == ro.keys()
    assert sum(rg[k] != ro[k] for k in ro) <= 0.01 * len(ro)
    b = point_source_rhs(pts)
    assert _rel(ifmm.ifmm_solve(f, b), o.solve(b)) < 1e-6


def test_sigma6_permutation_independent_of_node_order_within_color():
    """Sec. 3.2: the nodes of a sigma=6 color are independent; the GPU processes
    them in parallel, and the result equals the oracle's sequential order."""
    pts = bumpy_sphere(2500, 9)
    o = IFMMOracle(pts, 3, 3, 1e-8, 6).factor()
    t, f = _gpu(pts, 3, 3, 1e-8, 6, replay=o.ranks())
    b = point_source_rhs(pts)
    assert _rel(ifmm.ifmm_solve(f, b), o.solve(b)) < 1e-9


def test_matvec_matches_dense():
    for pts in (fibonacci_sphere(3000, 2), torus(1777, 1)):
        t = ifmm.ifmm_build_tree(pts, 3)
        x = np.random.default_rng(1).standard_normal(len(pts))
        assert _rel(ifmm.bem_matvec(t, x), dense_matrix(pts) @ x) < 1e-13


def test_matvec_sampled_rows_large():
    """N = 131,072 bumpy sphere: sampled rows against the oracle's direct sum."""
    pts = bumpy_sphere(131072, 3)
    t = ifmm.ifmm_build_tree(pts, 6)
    x = np.random.default_rng(2).standard_normal(len(pts))
    y = ifmm.bem_matvec(t, x)
    rows = np.random.default_rng(3).choice(len(pts), 64, replace=False)
    assert _rel(y[rows], direct_matvec(pts, x, rows)) < 1e-12


def test_gmres_matches_oracle_and_dense():
    pts = fibonacci_sphere(2048, 1)
    A = dense_matrix(pts)
    b = point_source_rhs(pts)
    t, f = _gpu(pts, 3, 3, 1e-6, 6)
    x, its, rel = ifmm.bem_gmres(t, b, precond=f, tol=1e-8)
    assert rel <= 1e-8 and np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 1.01e-8
    o = IFMMOracle(pts, 3, 3, 1e-6, 6).factor()
    _, its_o, _ = oracle_gmres(lambda v: A @ v, b, precond=o.solve, tol=1e-8)
    assert abs(its - its_o) <= 1
    x0, its0, rel0 = ifmm.bem_gmres(t, b, precond=None, tol=1e-8)
    assert its < its0


def test_solve_host_and_device_buffers_agree():
    import torch

    pts = fibonacci_sphere(1024, 4)
    t, f = _gpu(pts, 3, 3, 1e-6, 3)
    b = point_source_rhs(pts)
    xh = ifmm.ifmm_solve(f, b)
    xd = ifmm.ifmm_solve(f, torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.array_equal(xh, xd)


def test_empty_interaction_lists_small_tree():
    """Degenerate cases: a depth-2 tree over a few points (most cells adjacent,
    tiny or empty interaction lists) still factors exactly."""
    pts = fibonacci_sphere(40, 2)
    o = IFMMOracle(pts, 2, 2, 0.0, 3).factor()
    t, f = _gpu(pts, 2, 2, 0.0, 3)
    b = point_source_rhs(pts)
    assert _rel(ifmm.ifmm_solve(f, b), o.solve(b)) < 1e-11


def test_matvec_double_float_accuracy():
    """The float-pair matvec keeps FP64-level accuracy against the dense FP64 product."""
    for pts in (fibonacci_sphere(3000, 2), bumpy_sphere(2500, 5)):
        t = ifmm.ifmm_build_tree(pts, 3)
        x = np.random.default_rng(1).standard_normal(len(pts))
        y = ifmm.bem_matvec(t, x, kernel=ifmm.default_kernel(len(pts), "df"))
        assert _rel(y, dense_matrix(pts) @ x) < 1e-12


def test_matvec_double_float_sampled_large():
    pts = bumpy_sphere(131072, 3)
    t = ifmm.ifmm_build_tree(pts, 6)
    x = np.random.default_rng(2).standard_normal(len(pts))
    y = ifmm.bem_matvec(t, x, kernel=ifmm.default_kernel(len(pts), "df"))
    rows = np.random.default_rng(3).choice(len(pts), 64, replace=False)
    assert _rel(y[rows], direct_matvec(pts, x, rows)) < 1e-12


# applied-inverse error bound against the FP64 oracle (eps = 1e-6) and extra
# GMRES iterations allowed over FP64: FP32 (unit roundoff 6e-8, amplified by the
# conditioning of the pivots and the recompression) stays far below 1e-4;
# bfloat16 operands (unit roundoff 2^-8 = 3.9e-3) in the Schur GEMMs bound the
# error by a small multiple of that unit
MIXED_BOUNDS = {"fp32": (1e-4, 2), "bf16": (5e-2, 12)}


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_precision_error_and_gmres(prec):
    """Reduced-precision Schur updates and recompression: the applied inverse stays
    within the bound of its arithmetic of the FP64 oracle's, and GMRES with
    FP64-accurate residuals still reaches 1e-8."""
    bound, extra = MIXED_BOUNDS[prec]
    pts = bumpy_sphere(4096, 3)
    b = point_source_rhs(pts)
    o = IFMMOracle(pts, 4, 3, 1e-6, 3).factor()
    t = ifmm.ifmm_build_tree(pts, 4)
    ifmm.ifmm_color(t, 3)
    f = ifmm.ifmm_factor(t, 3, 1e-6, precision=prec)
    err = _rel(ifmm.ifmm_solve(f, b), o.solve(b))
    assert err < bound, err
    k = ifmm.default_kernel(len(pts), "df")
    x, its, rel = ifmm.bem_gmres(t, b, precond=f, tol=1e-8, kernel=k)
    f64 = ifmm.ifmm_factor(t, 3, 1e-6, precision="fp64")
    _, its64, _ = ifmm.bem_gmres(t, b, precond=f64, tol=1e-8)
    print(f"{prec}: applied-inverse error {err:.2e}, GMRES {its} iterations (FP64 {its64})")
    assert rel <= 1e-8 and its <= its64 + extra
    assert _rel(x, np.linalg.solve(dense_matrix(pts), b)) < 1e-7


def test_bf16_differs_from_fp32():
    """The BF16 mode really rounds the Schur operands: its factor differs from the
    FP32 one by about the bfloat16 unit, far more than FP32 rounding."""
    pts = bumpy_sphere(4096, 3)
    b = point_source_rhs(pts)
    t = ifmm.ifmm_build_tree(pts, 4)
    ifmm.ifmm_color(t, 3)
    v32 = ifmm.ifmm_solve(ifmm.ifmm_factor(t, 3, 1e-6, precision="fp32"), b)
    v16 = ifmm.ifmm_solve(ifmm.ifmm_factor(t, 3, 1e-6, precision="bf16"), b)
    d = _rel(v16, v32)
    assert 1e-5 < d < 5e-2, d


@pytest.mark.parametrize("tau,sigma", [(3, 3), (4, 6)])
def test_tau_switch_replay_parity(tau, sigma):
    """Levels below tau eliminated one node at a time (Table 2's top level tau):
    the GPU factor equals the oracle's with the same per-level order (singleton
    groups below tau), ranks replayed, within 1e-9."""
    pts = bumpy_sphere(3000, 5)
    depth = 4
    groups = None
    from oracle.tree import Tree

    tr = Tree(pts, depth)
    groups = {k: [[i] for i in range(tr.levels[k].n)] for k in range(2, tau)}
    o = IFMMOracle(pts, depth, 3, 1e-6, sigma, color_groups=groups).factor()
    t = ifmm.ifmm_build_tree(pts, depth)
    ifmm.ifmm_color_levels(t, sigma, tau)
    rep = [list(k) + [v] for k, v in o.ranks().items()]
    f = ifmm.ifmm_factor(t, 3, 1e-6, rank_mode="replay", replay=rep)
    R = np.random.default_rng(3).standard_normal((2, len(pts)))
    V = ifmm.ifmm_solve(f, R)
    for k in range(2):
        assert _rel(V[k], o.solve(R[k])) < 1e-9


@pytest.mark.parametrize("tile", ["sym", "128x1", "256x2"])
@pytest.mark.parametrize("n", [2, 129, 300, 3001])
def test_matvec_kernels_forced(tile, n, monkeypatch):
    """Each float-pair matvec kernel (the symmetric one included), forced on a
    fresh tree, against the dense FP64 product: two points, one tile plus one
    point, ragged tile tails."""
    monkeypatch.setenv("IFMM_MATVEC_TILE", tile)
    pts = bumpy_sphere(n, 6) if n > 2 else np.array([[0.1, 0.2, 0.3], [0.5, -0.4, 0.2]])
    t = ifmm.ifmm_build_tree(pts, 2)
    x = np.random.default_rng(n).standard_normal(n)
    y = ifmm.bem_matvec(t, x, kernel=ifmm.default_kernel(n, "df"))
    code = list(ifmm.ifmm_tree_query(t, 0, "matvec_block"))
    assert code[1] == (3 if tile == "sym" else int(tile.split("x")[1]))
    ref = dense_matrix(pts) @ x
    assert _rel(y, ref) < 1e-12
    assert np.array_equal(y, ifmm.bem_matvec(t, x, kernel=ifmm.default_kernel(n, "df")))
