"""Python binding of the C ABI in include/ifmm.h (ctypes, argument marshalling only).

Every function here has the name of the C entry point it calls.  Arrays may be
NumPy arrays (host memory) or torch CUDA tensors (device memory); results come
back on the same side as the inputs.  There is no fallback: if the shared
library is missing, importing this module raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libifmm.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with `python -m paper_1905_10602_gb300.build`")
lib = ctypes.CDLL(_LIB_PATH)

STATUS = {0: "IFMM_OK", 1: "IFMM_EINVAL", 2: "IFMM_ENOMEM", 3: "IFMM_ECUDA", 4: "IFMM_ESINGULAR",
          5: "IFMM_ENOCONV", 6: "IFMM_ETIMEOUT", 7: "IFMM_ERANK"}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
RANK_MODE = {"svd": 0, "replay": 1, "learned": 2}


class IFMMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Kernel(ctypes.Structure):
    _fields_ = [("scale", ctypes.c_double), ("diag", ctypes.c_double), ("arith", ctypes.c_int),
                ("order", ctypes.c_int), ("wavenumber", ctypes.c_double), ("diag_im", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("cheb_order", ctypes.c_int), ("eps", ctypes.c_double), ("precision", ctypes.c_int),
                ("rank_mode", ctypes.c_int), ("replay", ctypes.POINTER(ctypes.c_int32)),
                ("replay_len", ctypes.c_int64), ("max_rank", ctypes.c_int),
                ("mlp", ctypes.POINTER(ctypes.c_float)), ("seed", ctypes.c_uint64)]


_vp, _i64, _i32, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_sig = {
    "ifmm_build_tree": [_vp, _i64, ctypes.c_int, ctypes.POINTER(_vp)],
    "ifmm_color": [_vp, ctypes.c_int, _vp],
    "ifmm_color_levels": [_vp, ctypes.c_int, ctypes.c_int, _vp],
    "ifmm_tree_query": [_vp, ctypes.c_int, ctypes.c_char_p, _vp, _i64, ctypes.POINTER(_i64)],
    "ifmm_factor": [_vp, ctypes.POINTER(Kernel), ctypes.POINTER(Opts), _vp, ctypes.POINTER(_vp)],
    "ifmm_solve": [_vp, _vp, _vp, ctypes.c_int, _vp],
    "bem_gmres": [_vp, ctypes.POINTER(Kernel), _vp, _vp, _vp, ctypes.c_int, _dbl, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_dbl), _vp],
    "bem_matvec": [_vp, ctypes.POINTER(Kernel), _vp, _vp, _vp],
    "bem_matvec_noalloc": [_vp, ctypes.POINTER(Kernel), _vp, _vp, _vp],
    "ifmm_fact_ranks": [_vp, _vp, _i64, ctypes.POINTER(_i64)],
    "ifmm_factor_batched": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp],
    "bem_gmres_batched": [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _dbl, ctypes.c_int, _vp, _vp,
                          ctypes.c_int],
    "ifmm_fact_events": [_vp, _vp, _vp, _i64, ctypes.POINTER(_i64)],
    "ifmm_mlp_forward": [_vp, _vp, _i64, _vp, _vp],
    "ifmm_mlp_grad": [_vp, _vp, _vp, _i64, _vp, _vp, _vp],
    "ifmm_mlp_train": [_vp, _vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64, _vp, _vp, _vp],
    "ifmm_fact_stats": [_vp, _vp, _i64, ctypes.POINTER(_i64)],
    "ifmm_convert_check": [_vp, _i64, ctypes.c_int, _vp, _vp],
    "ifmm_probe_peak": [ctypes.c_int, ctypes.POINTER(_dbl)],
    "ifmm_bd_factor": [_vp, ctypes.POINTER(Kernel), ctypes.c_int, _vp, ctypes.POINTER(_vp)],
    "ifmm_gemm_check": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dbl, _vp,
                        ctypes.c_int, _vp, ctypes.c_int, _dbl, _vp, ctypes.c_int],
    "ifmm_inv_check": [ctypes.c_int, _vp, _vp, _vp],
    "ifmm_qr_check": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp],
}
for _name, _args in _sig.items():
    getattr(lib, _name).argtypes = _args
    getattr(lib, _name).restype = ctypes.c_int
lib.ifmm_profile.argtypes = [ctypes.c_int]
lib.ifmm_profile.restype = ctypes.c_int
lib.ifmm_profile_query.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_i64),
                                   ctypes.POINTER(_dbl)]
lib.ifmm_profile_query.restype = ctypes.c_int
lib.ifmm_fact_stat_name.argtypes = [_vp, _i64]
lib.ifmm_fact_stat_name.restype = ctypes.c_char_p
lib.ifmm_last_error.argtypes = []
lib.ifmm_last_error.restype = ctypes.c_char_p
lib.ifmm_tree_free.argtypes = [_vp]
lib.ifmm_tree_free.restype = None
lib.ifmm_fact_free.argtypes = [_vp]
lib.ifmm_fact_free.restype = None

EXPORTED = sorted(list(_sig) + ["ifmm_fact_stat_name", "ifmm_last_error", "ifmm_tree_free", "ifmm_fact_free",
                                 "ifmm_profile", "ifmm_profile_query"])


def _check(code):
    if code != 0:
        raise IFMMError(code, lib.ifmm_last_error().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _as_real(x):
    """A complex array as its interleaved (real, imaginary) float64 view, sharing
    memory (the layout the C ABI takes for the Helmholtz kernel); real arrays as
    they are."""
    if _is_torch(x):
        import torch

        return torch.view_as_real(x) if x.is_complex() else x
    return x.view(np.float64) if np.iscomplexobj(x) else x


def _ptr(x):
    """Pointer of a C-contiguous float64 NumPy array or torch tensor (complex:
    its interleaved float64 view)."""
    x = _as_real(x)
    if _is_torch(x):
        assert x.is_contiguous() and str(x.dtype) == "torch.float64"
        return ctypes.c_void_p(x.data_ptr())
    assert x.flags["C_CONTIGUOUS"] and x.dtype == np.float64
    return x.ctypes.data_as(ctypes.c_void_p)


def _stream(x=None):
    if x is not None and _is_torch(x) and x.is_cuda:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return ctypes.c_void_p(0)


ARITH = {"fp64": 0, "df": 1, "fmm": 2}


def default_kernel(n, arith: str = "fp64", order: int = 0):
    """A_ij = 1/(N |x_i - x_j|), A_ii = 0.5 + 1/sqrt(N); arith: the matvec as a
    direct sum in plain FP64 or in FP64-accurate float pairs ("df"), or the FMM
    representation A~ at Chebyshev order `order` ("fmm", 0 = 4)."""
    return Kernel(1.0 / n, 0.5 + 1.0 / np.sqrt(n), ARITH[arith], order, 0.0, 0.0)


def helmholtz_kernel(n, wavenumber: float):
    """A_ij = e^{ik|x_i - x_j|}/(N |x_i - x_j|), A_ii = 0.5 plus the kernel
    integrated over a disk panel of area 4 pi / N (radius rho = 2/sqrt(N)):
    (e^{ik rho} - 1)/(2ik).  Complex; FP64 direct-sum matvec."""
    k = float(wavenumber)
    rho = 2.0 / np.sqrt(n)
    return Kernel(1.0 / n, 0.5 + np.sin(k * rho) / (2.0 * k), 0, 0, k, (1.0 - np.cos(k * rho)) / (2.0 * k))


class Tree:
    def __init__(self, handle, n, depth, pts):
        self.h, self.n, self.depth, self._pts = handle, n, depth, pts

    def __del__(self):
        if getattr(self, "h", None):
            lib.ifmm_tree_free(self.h)
            self.h = None


class Fact:
    def __init__(self, handle, tree):
        self.h, self.tree = handle, tree

    def __del__(self):
        if getattr(self, "h", None):
            lib.ifmm_fact_free(self.h)
            self.h = None


def ifmm_build_tree(xyz, depth: int) -> Tree:
    """xyz: (N, 3) points, a NumPy array or a float64 CUDA tensor."""
    if not _is_torch(xyz):
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64))
    h = ctypes.c_void_p()
    _check(lib.ifmm_build_tree(_ptr(xyz), xyz.shape[0], depth, ctypes.byref(h)))
    return Tree(h, xyz.shape[0], depth, xyz)


def ifmm_color(tree: Tree, sigma: int) -> np.ndarray:
    out = np.zeros(tree.depth + 1, dtype=np.int32)
    _check(lib.ifmm_color(tree.h, sigma, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ifmm_color_levels(tree: Tree, sigma: int, tau: int) -> np.ndarray:
    """Coloring at sigma for levels tau..depth, one node per color below tau."""
    out = np.zeros(tree.depth + 1, dtype=np.int32)
    _check(lib.ifmm_color_levels(tree.h, sigma, tau, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ifmm_tree_query(tree: Tree, level: int, what: str) -> np.ndarray:
    cnt = _i64()
    _check(lib.ifmm_tree_query(tree.h, level, what.encode(), None, 0, ctypes.byref(cnt)))
    buf = np.zeros(cnt.value, dtype=np.int32)
    _check(lib.ifmm_tree_query(tree.h, level, what.encode(), buf.ctypes.data_as(ctypes.c_void_p), cnt.value,
                               ctypes.byref(cnt)))
    return buf


def ifmm_factor(tree: Tree, cheb_order: int, eps: float, kernel: Kernel | None = None, precision: str = "fp64",
                rank_mode: str = "svd", replay=None, max_rank: int = 0, mlp=None, seed: int = 0, stream=None) -> Fact:
    k = kernel if kernel is not None else default_kernel(tree.n)
    o = Opts()
    o.cheb_order, o.eps, o.precision, o.rank_mode = cheb_order, eps, PREC[precision], RANK_MODE[rank_mode]
    keep = []
    if replay is not None:
        arr = np.ascontiguousarray(np.asarray(replay, dtype=np.int32).reshape(-1, 4))
        keep.append(arr)
        o.replay = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        o.replay_len = arr.shape[0]
    if mlp is not None:
        w = np.ascontiguousarray(np.asarray(mlp, dtype=np.float32))
        keep.append(w)
        o.mlp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    o.max_rank, o.seed = max_rank, seed
    h = ctypes.c_void_p()
    _check(lib.ifmm_factor(tree.h, ctypes.byref(k), ctypes.byref(o), stream or ctypes.c_void_p(0), ctypes.byref(h)))
    return Fact(h, tree)


def ifmm_bd_factor(tree: Tree, level: int, kernel: Kernel | None = None, stream=None) -> Fact:
    """Block-diagonal preconditioner (BD / BDbot at `level`) as a factor handle."""
    k = kernel if kernel is not None else default_kernel(tree.n)
    h = ctypes.c_void_p()
    _check(lib.ifmm_bd_factor(tree.h, ctypes.byref(k), level, stream or ctypes.c_void_p(0), ctypes.byref(h)))
    return Fact(h, tree)


def ifmm_solve(fact: Fact, r, stream=None):
    """v ~ A~^{-1} r; r is (N,) or (nrhs, N) stacked rows (each row one right-hand side)."""
    if _is_torch(r):
        import torch

        v = torch.empty_like(r)
    else:
        r = np.asarray(r)
        r = np.ascontiguousarray(r if np.iscomplexobj(r) else r.astype(np.float64))
        v = np.empty_like(r)
    nrhs = 1 if r.ndim == 1 else r.shape[0]
    _check(lib.ifmm_solve(fact.h, _ptr(r), _ptr(v), nrhs, stream or _stream(r)))
    return v


def bem_matvec(tree: Tree, x, kernel: Kernel | None = None, stream=None):
    k = kernel if kernel is not None else default_kernel(tree.n)
    if _is_torch(x):
        import torch

        y = torch.empty_like(x)
    else:
        x = np.asarray(x)
        x = np.ascontiguousarray(x if np.iscomplexobj(x) else x.astype(np.float64))
        y = np.empty_like(x)
    _check(lib.bem_matvec(tree.h, ctypes.byref(k), _ptr(x), _ptr(y), stream or _stream(x)))
    return y


def bem_gmres(tree: Tree, b, precond: Fact | None = None, restart: int = 30, tol: float = 1e-8, maxit: int = 500,
              kernel: Kernel | None = None, stream=None, raise_on_noconv: bool = True):
    """Returns (x, iterations, true relative residual)."""
    k = kernel if kernel is not None else default_kernel(tree.n)
    if _is_torch(b):
        import torch

        x = torch.empty_like(b)
    else:
        b = np.asarray(b)
        b = np.ascontiguousarray(b if np.iscomplexobj(b) else b.astype(np.float64))
        x = np.empty_like(b)
    its, rel = ctypes.c_int(), ctypes.c_double()
    code = lib.bem_gmres(tree.h, ctypes.byref(k), precond.h if precond else None, _ptr(b), _ptr(x), restart, tol,
                         maxit, ctypes.byref(its), ctypes.byref(rel), stream or _stream(b))
    if code != 5 or raise_on_noconv:
        _check(code)
    return x, its.value, rel.value


def ifmm_fact_ranks(fact: Fact) -> dict:
    cnt = _i64()
    _check(lib.ifmm_fact_ranks(fact.h, None, 0, ctypes.byref(cnt)))
    buf = np.zeros(cnt.value, dtype=np.int32)
    _check(lib.ifmm_fact_ranks(fact.h, buf.ctypes.data_as(ctypes.c_void_p), cnt.value, ctypes.byref(cnt)))
    q = buf.reshape(-1, 4)
    return {(int(a), int(b), int(c)): int(d) for a, b, c, d in q}


def ifmm_fact_stats(fact: Fact) -> dict:
    cnt = _i64()
    _check(lib.ifmm_fact_stats(fact.h, None, 0, ctypes.byref(cnt)))
    buf = np.zeros(cnt.value, dtype=np.float64)
    _check(lib.ifmm_fact_stats(fact.h, buf.ctypes.data_as(ctypes.c_void_p), cnt.value, ctypes.byref(cnt)))
    return {lib.ifmm_fact_stat_name(fact.h, i).decode(): float(buf[i]) for i in range(cnt.value)}


def ifmm_profile(timing: bool = True) -> None:
    _check(lib.ifmm_profile(1 if timing else 0))


def ifmm_profile_query() -> dict:
    """{kernel name: (launches, milliseconds)} since the last ifmm_profile()."""
    out = {}
    i = 0
    while True:
        name, n, ms = ctypes.c_char_p(), _i64(), _dbl()
        if lib.ifmm_profile_query(i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms)) != 0:
            break
        out[name.value.decode()] = (int(n.value), float(ms.value))
        i += 1
    return out


def ifmm_convert_check(x: np.ndarray, shift: int = 0):
    """(f, back): the FP32 kernels' binary64 -> binary32 conversion of x * 2^shift
    on the device, and f * 2^-shift widened back (diagnostic)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.empty(x.shape, dtype=np.float32)
    back = np.empty(x.shape, dtype=np.float64)
    _check(lib.ifmm_convert_check(x.ctypes.data_as(ctypes.c_void_p), x.size, int(shift),
                                  f.ctypes.data_as(ctypes.c_void_p), back.ctypes.data_as(ctypes.c_void_p)))
    return f, back


def ifmm_gemm_check(precision: str, A, B, C=None, alpha: float = 1.0, beta: float = 0.0, ta=False, tb=False):
    """alpha op(A) op(B) + beta C through the library's batched GEMM kernels in
    `precision` ("fp64", "fp32", "bf16"); NumPy arrays (diagnostic)."""
    A = np.asfortranarray(A, dtype=np.float64)
    B = np.asfortranarray(B, dtype=np.float64)
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    C = np.asfortranarray(np.zeros((m, n)) if C is None else C, dtype=np.float64).copy(order="F")
    _check(lib.ifmm_gemm_check(PREC[precision], m, n, k, int(ta), int(tb), alpha, A.ctypes.data_as(_vp),
                               max(1, A.shape[0]), B.ctypes.data_as(_vp), max(1, B.shape[0]), beta,
                               C.ctypes.data_as(_vp), max(1, m)))
    return C


def ifmm_qr_check(A, precision: str = "fp64", pivoted: bool = False):
    """Householder QR of a NumPy matrix through the library's recompression QR
    kernels (diagnostic): returns R (min(m, n) x n), and with pivoted also the
    column order and the number of steps."""
    A = np.asfortranarray(A, dtype=np.float64).copy(order="F")
    m, n = A.shape
    jp = np.zeros(n, dtype=np.int32)
    k = ctypes.c_int(0)
    _check(lib.ifmm_qr_check(PREC[precision], int(pivoted), m, n, A.ctypes.data_as(_vp), m, jp.ctypes.data_as(_vp),
                             ctypes.byref(k)))
    R = np.triu(A[:min(m, n), :])
    return (R, jp, k.value) if pivoted else R


def ifmm_inv_check(mats):
    """Inverses of a list of square NumPy matrices through the library's FP64
    Gauss-Jordan pivot-block kernels (diagnostic); returns (inverses, info), info[i]
    = 0 or the 1-based step with no nonzero pivot."""
    ns = np.array([np.shape(a)[0] for a in mats], dtype=np.int32)
    for a, n in zip(mats, ns):
        assert np.shape(a) == (n, n)
    flat = np.concatenate([np.asarray(a, dtype=np.float64).ravel(order="F") for a in mats]) if len(mats) else \
        np.zeros(0)
    info = np.zeros(len(mats), dtype=np.int32)
    _check(lib.ifmm_inv_check(len(mats), ns.ctypes.data_as(_vp), flat.ctypes.data_as(_vp), info.ctypes.data_as(_vp)))
    out, off = [], 0
    for n in ns:
        out.append(flat[off:off + n * n].reshape((n, n), order="F").copy())
        off += n * n
    return out, info


PEAK_KINDS = {"fp32": 0, "fp64": 1, "tf32_mma": 2, "bf16_mma": 3, "fp64_mma": 4}


def ifmm_probe_peak(kind: str) -> float:
    """Measured TFLOP/s of one arithmetic unit of the current GPU (PEAK_KINDS)."""
    v = _dbl()
    _check(lib.ifmm_probe_peak(PEAK_KINDS[kind], ctypes.byref(v)))
    return float(v.value)


def bem_matvec_noalloc(tree: Tree, x, y, kernel: Kernel | None = None, stream=None) -> None:
    """y = A x into the caller's device tensor y, with no device allocation (for
    callers that cannot allocate device memory; see include/ifmm.h).  x and y
    are float64 CUDA tensors of N elements; the call returns once the work is
    enqueued on the stream."""
    k = kernel if kernel is not None else default_kernel(tree.n)
    _check(lib.bem_matvec_noalloc(tree.h, ctypes.byref(k), _ptr(x), _ptr(y), stream or _stream(x)))


MLP_INPUTS = 9
MLP_NWEIGHTS = 9025


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _fp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def ifmm_fact_events(fact: Fact):
    """(features (n, 9) float32, ranks (n,) int32) of every recompression event."""
    cnt = _i64()
    _check(lib.ifmm_fact_events(fact.h, None, None, 0, ctypes.byref(cnt)))
    X = np.zeros((cnt.value, MLP_INPUTS), dtype=np.float32)
    r = np.zeros(cnt.value, dtype=np.int32)
    _check(lib.ifmm_fact_events(fact.h, _fp(X), _fp(r), cnt.value, ctypes.byref(cnt)))
    return X, r


def ifmm_mlp_forward(weights, X):
    w, X = _f32(weights), _f32(X)
    y = np.zeros(X.shape[0], dtype=np.float32)
    _check(lib.ifmm_mlp_forward(_fp(w), _fp(X), X.shape[0], _fp(y), None))
    return y


def ifmm_mlp_grad(weights, X, t):
    w, X, t = _f32(weights), _f32(X), _f32(t)
    g = np.zeros(MLP_NWEIGHTS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(lib.ifmm_mlp_grad(_fp(w), _fp(X), _fp(t), X.shape[0], _fp(g), ctypes.byref(loss), None))
    return float(loss.value), g


def ifmm_mlp_train(X, t, epochs=200, batch=4096, lr=1e-3, seed=1):
    X, t = _f32(X), _f32(t)
    w = np.zeros(MLP_NWEIGHTS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(lib.ifmm_mlp_train(_fp(X), _fp(t), X.shape[0], epochs, batch, lr, seed, _fp(w), ctypes.byref(loss), None))
    return w, float(loss.value)


def ifmm_factor_batched(trees, cheb_order: int, eps: float, precision: str = "fp64", rank_mode: str = "svd",
                        mlp=None, nworkers: int = 8, kernels=None):
    """Factors independent problems concurrently (one stream per worker)."""
    n = len(trees)
    TA = ctypes.c_void_p * n
    KA = Kernel * n
    OA = Opts * n
    ks = KA(*[kernels[i] if kernels else default_kernel(t.n) for i, t in enumerate(trees)])
    os_ = OA()
    keep = []
    for i in range(n):
        os_[i].cheb_order, os_[i].eps, os_[i].precision = cheb_order, eps, PREC[precision]
        os_[i].rank_mode = RANK_MODE[rank_mode]
        if mlp is not None:
            w = np.ascontiguousarray(np.asarray(mlp, dtype=np.float32))
            keep.append(w)
            os_[i].mlp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    outs = TA()
    _check(lib.ifmm_factor_batched(TA(*[t.h for t in trees]), ks, os_, n, nworkers, outs))
    return [Fact(ctypes.c_void_p(outs[i]), trees[i]) for i in range(n)]


def bem_gmres_batched(trees, bs, facts=None, restart: int = 30, tol: float = 1e-8, maxit: int = 500,
                      kernels=None, nworkers: int = 8, raise_on_noconv: bool = True):
    """GMRES for independent problems concurrently; returns (xs, iters, relres)."""
    n = len(trees)
    TA = ctypes.c_void_p * n
    ks = (Kernel * n)(*[kernels[i] if kernels else default_kernel(t.n) for i, t in enumerate(trees)])
    bs = [np.ascontiguousarray(np.asarray(b, dtype=np.float64)) for b in bs]
    xs = [np.empty_like(b) for b in bs]
    its = (ctypes.c_int * n)()
    rel = (ctypes.c_double * n)()
    pre = TA(*[f.h if f is not None else None for f in facts]) if facts else None
    code = lib.bem_gmres_batched(TA(*[t.h for t in trees]), ks, pre, TA(*[_ptr(b).value for b in bs]),
                                 TA(*[_ptr(x).value for x in xs]), n, restart, tol, maxit, its, rel, nworkers)
    if code != 5 or raise_on_noconv:
        _check(code)
    return xs, list(its), list(rel)
