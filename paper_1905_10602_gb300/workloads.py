"""Seeded synthetic inputs: surfaces, right-hand sides and named workloads.

This module only generates inputs. It holds none of the method's arithmetic
(no kernel evaluation, no tree, no elimination), so both the CUDA path and the
CPU oracle can draw the same inputs from it.

The paper's meshes (a 1,003,520-element sphere, Sec. 5.2, and a 1,218,200-element
office building, Sec. 5.3) are not available; points on synthetic surfaces stand
in for them.  Like the paper's boundary meshes they are surface-like: the number
of occupied octree cells grows as ~4^kappa with the level (Table 1).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SOURCE_POINT = (0.1, 0.2, 0.3)


def fibonacci_directions(n: int) -> np.ndarray:
    """Unit vectors of the Fibonacci lattice: z_k = 1-(2k+1)/n, phi_k = k*pi*(3-sqrt5)."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def fibonacci_sphere(n: int, seed: int, jitter: float = 1e-3) -> np.ndarray:
    """Unit sphere: Fibonacci lattice, seeded Gaussian jitter, re-projected onto the sphere."""
    p = fibonacci_directions(n)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        p = p + jitter * rng.standard_normal(p.shape)
        p /= np.linalg.norm(p, axis=1, keepdims=True)
    return np.ascontiguousarray(p)


def _real_sph_harm_cos(l: int, m: int, ct: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonic (cos(m*phi) part) of degree l, order m>0.

    Y = sqrt(2) * sqrt((2l+1)/(4pi) * (l-m)!/(l+m)!) * P_l^m(cos theta) * cos(m phi),
    with P_l^m from the standard upward recurrence (no Condon-Shortley phase).
    """
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    # P_m^m = (2m-1)!! sin^m
    pmm = np.ones_like(ct)
    for i in range(1, m + 1):
        pmm = pmm * (2 * i - 1) * st
    if l == m:
        plm = pmm
    else:
        pm1 = ct * (2 * m + 1) * pmm
        if l == m + 1:
            plm = pm1
        else:
            p_prev, p_cur = pmm, pm1
            for ll in range(m + 2, l + 1):
                p_next = ((2 * ll - 1) * ct * p_cur - (ll + m - 1) * p_prev) / (ll - m)
                p_prev, p_cur = p_cur, p_next
            plm = p_cur
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
    return math.sqrt(2.0) * norm * plm * np.cos(m * phi)


def bumpy_sphere(n: int, seed: int, jitter: float = 1e-3) -> np.ndarray:
    """r(theta,phi) = 1 + 0.2 Y_3^2 + 0.1 Y_5^1 along jittered Fibonacci directions."""
    d = fibonacci_sphere(n, seed, jitter)
    ct = np.clip(d[:, 2], -1.0, 1.0)
    phi = np.arctan2(d[:, 1], d[:, 0])
    r = 1.0 + 0.2 * _real_sph_harm_cos(3, 2, ct, phi) + 0.1 * _real_sph_harm_cos(5, 1, ct, phi)
    return np.ascontiguousarray(d * r[:, None])


def torus(n: int, seed: int, R: float = 1.0, r: float = 0.3) -> np.ndarray:
    """Area-uniform points on a torus: rejection sampling of (u, v) with
    acceptance probability (R + r cos v)/(R + r)."""
    rng = np.random.default_rng(seed)
    out = []
    have = 0
    while have < n:
        m = 2 * (n - have) + 64
        u = rng.uniform(0.0, 2.0 * math.pi, m)
        v = rng.uniform(0.0, 2.0 * math.pi, m)
        w = rng.uniform(0.0, 1.0, m)
        keep = w < (R + r * np.cos(v)) / (R + r)
        u, v = u[keep], v[keep]
        pts = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], axis=1)
        out.append(pts)
        have += len(pts)
    return np.ascontiguousarray(np.concatenate(out)[:n])


def point_source_rhs(pts: np.ndarray, src=SOURCE_POINT) -> np.ndarray:
    """Right-hand side b_i = 1/(4 pi |x_i - s|): the field of a unit source at s."""
    d = np.linalg.norm(pts - np.asarray(src, dtype=np.float64)[None, :], axis=1)
    return 1.0 / (4.0 * math.pi * d)


def helmholtz_source_rhs(pts: np.ndarray, k: float, src=SOURCE_POINT) -> np.ndarray:
    """Right-hand side b_i = e^{ik|x_i - s|}/(4 pi |x_i - s|): a unit acoustic source at s."""
    d = np.linalg.norm(pts - np.asarray(src, dtype=np.float64)[None, :], axis=1)
    return np.exp(1j * k * d) / (4.0 * math.pi * d)


def surface(shape: str, n: int, seed: int) -> np.ndarray:
    if shape == "sphere":
        return fibonacci_sphere(n, seed)
    if shape == "bumpy":
        return bumpy_sphere(n, seed)
    if shape == "torus":
        return torus(n, seed)
    raise ValueError(f"unknown surface {shape!r}")


@dataclass
class Workload:
    """One BEM problem: points, octree depth, Chebyshev order, eps, coloring separation."""

    name: str
    shape: str
    n: int
    seed: int
    depth: int
    cheb_order: int
    eps: float
    sigma: int = 6
    extra: dict = field(default_factory=dict)

    def points(self) -> np.ndarray:
        return surface(self.shape, self.n, self.seed)

    def rhs(self, pts: np.ndarray | None = None) -> np.ndarray:
        return point_source_rhs(self.points() if pts is None else pts)


# Named workloads (sizes, shapes and parameters of the method's problem family).
WORKLOADS = {
    "sphere2k": Workload("sphere2k", "sphere", 2048, 1, 3, 3, 1e-6, 6),
    "sphere32k": Workload("sphere32k", "sphere", 32768, 2, 5, 4, 1e-8, 6),
    "bumpy131k": Workload("bumpy131k", "bumpy", 131072, 3, 6, 4, 1e-6, 3),
    "torus65k": Workload("torus65k", "torus", 65536, 4, 6, 4, 1e-6, 3),
    "torus262k": Workload("torus262k", "torus", 262144, 4, 6, 4, 1e-6, 3),
}


def batch_workloads(count: int = 64, seed: int = 5, cheb_order: int = 4, eps: float = 1e-6):
    """Independent problems with N log-uniform in [4096, 65536]; shapes cycle
    sphere / torus / bumpy; depth = clamp(round(log4(N/32)), 2, 6)."""
    rng = np.random.default_rng(seed)
    shapes = ("sphere", "torus", "bumpy")
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(4096), math.log(65536)))))
        depth = int(min(6, max(2, round(math.log(n / 32.0, 4)))))
        out.append(Workload(f"batch{k}", shapes[k % 3], n, seed * 1000 + k, depth, cheb_order, eps, 3))
    return out
