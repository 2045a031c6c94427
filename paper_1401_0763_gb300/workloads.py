"""Seeded synthetic inputs for the red-black SOR workloads.

This module holds no arithmetic of the method: it only draws boundary data,
source terms, grid sizes and request streams from numpy's PCG64 generator.
Both the oracle (tests, CPU baseline) and the CUDA path (tests, bench) take
their inputs from here, so the two sides see identical arrays.

Array convention: interior side ``n``, full array ``(n+2, n+2)`` row-major,
row 0 = north edge, ``x_j = j*h``, ``y_i = i*h`` with ``h = 1/(n+1)``
(paper Section 3.4: 2D steady heat conduction on a square plate, Dirichlet
edges).  Source arrays are the ``(n, n)`` interior of f for -Laplace(u) = f.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "rng", "heat_plate", "harmonic_xx_minus_yy", "quadratic_xx_plus_yy", "random_edges", "gaussian_source",
    "batch_sizes", "Request", "request_stream", "poisson_problem",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def heat_plate(n: int, top: float = 100.0, edge: str = "north") -> np.ndarray:
    """Heat plate of Section 3.4: one edge held at ``top``, the other three
    at 0, interior 0.  The two corners of the hot edge take the hot value
    (corners are never read by the 5-point stencil)."""
    u = np.zeros((n + 2, n + 2), dtype=np.float64)
    if edge == "north":
        u[0, :] = top
    elif edge == "south":
        u[-1, :] = top
    elif edge == "west":
        u[:, 0] = top
    elif edge == "east":
        u[:, -1] = top
    else:
        raise ValueError(edge)
    return u


def _coords(n: int):
    h = 1.0 / (n + 1)
    c = np.arange(n + 2, dtype=np.float64) * h
    return c[None, :], c[:, None]  # x (columns), y (rows)


def harmonic_xx_minus_yy(n: int) -> np.ndarray:
    """Boundary ring from u = x^2 - y^2 (harmonic), interior 0."""
    x, y = _coords(n)
    full = x * x - y * y
    u = np.zeros((n + 2, n + 2))
    u[0, :], u[-1, :], u[:, 0], u[:, -1] = full[0, :], full[-1, :], full[:, 0], full[:, -1]
    return u


def quadratic_xx_plus_yy(n: int):
    """Boundary ring from u = x^2 + y^2, interior 0, and the matching source
    f = -4 everywhere (-Laplace(x^2 + y^2) = -4)."""
    x, y = _coords(n)
    full = x * x + y * y
    u = np.zeros((n + 2, n + 2))
    u[0, :], u[-1, :], u[:, 0], u[:, -1] = full[0, :], full[-1, :], full[:, 0], full[:, -1]
    return u, np.full((n, n), -4.0)


def random_edges(n: int, seed: int, lo: float = 0.0, hi: float = 100.0) -> np.ndarray:
    """Edge cells i.i.d. uniform[lo, hi], drawn in the order top row (n+2),
    bottom row (n+2), left column without corners (n), right column without
    corners (n); interior 0."""
    g = rng(seed)
    v = g.uniform(lo, hi, size=4 * (n + 2) - 4)
    u = np.zeros((n + 2, n + 2))
    m = n + 2
    u[0, :] = v[0:m]
    u[-1, :] = v[m:2 * m]
    u[1:-1, 0] = v[2 * m:2 * m + n]
    u[1:-1, -1] = v[2 * m + n:2 * m + 2 * n]
    return u


def gaussian_source(n: int, seed: int, count: int = 8) -> np.ndarray:
    """f(x, y) = sum_k a_k exp(-((x-x_k)^2 + (y-y_k)^2) / (2 s_k^2)) on the
    interior nodes, with a_k ~ U[-1, 1], s_k ~ U[0.02, 0.2] and centres
    (x_k, y_k) ~ U[0, 1]^2, drawn in that order from one PCG64 stream."""
    g = rng(seed)
    a = g.uniform(-1.0, 1.0, size=count)
    s = g.uniform(0.02, 0.2, size=count)
    c = g.uniform(0.0, 1.0, size=(count, 2))
    h = 1.0 / (n + 1)
    xs = np.arange(1, n + 1, dtype=np.float64) * h
    ex = [np.exp(-((xs - c[k, 0]) ** 2) / (2.0 * s[k] ** 2)) for k in range(count)]
    ey = [np.exp(-((xs - c[k, 1]) ** 2) / (2.0 * s[k] ** 2)) for k in range(count)]
    # f = sum over k of a_k * (ey_k outer ex_k), terms added in order k = 0, 1, ...,
    # evaluated in blocks of rows that stay in cache (each element is rounded
    # exactly as in the unblocked expression: outer product, scaling, sum)
    f = np.zeros((n, n))
    rows = max(1, (1 << 15) // max(1, n))
    buf = np.empty((rows, n))
    for i0 in range(0, n, rows):
        i1 = min(n, i0 + rows)
        fb, tb = f[i0:i1], buf[:i1 - i0]
        for k in range(count):
            np.multiply.outer(ey[k][i0:i1], ex[k], out=tb)
            np.multiply(a[k], tb, out=tb)
            np.add(fb, tb, out=fb)
    return f


def poisson_problem(n: int, seed: int):
    """Zero Dirichlet boundary with the 8-Gaussian source: (u0, f)."""
    return np.zeros((n + 2, n + 2)), gaussian_source(n, seed)


def batch_sizes(count: int, seed: int, lo: int = 64, hi: int = 1024) -> np.ndarray:
    """Interior sides log-uniform in [lo, hi], rounded to integers."""
    g = rng(seed)
    return np.rint(np.exp(g.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)


@dataclass
class Request:
    arrival_s: float
    n: int
    tol: float
    seed: int


def request_stream(count: int, rate: float, seed: int, n_lo: int = 128, n_hi: int = 4096,
                   tol_lo: float = 1e-10, tol_hi: float = 1e-6):
    """Poisson arrivals (exponential gaps of mean 1/rate), interior side
    log-uniform in [n_lo, n_hi], tolerance log-uniform in [tol_lo, tol_hi];
    each request carries its own seed for its boundary and source."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    ns = np.rint(np.exp(g.uniform(np.log(n_lo), np.log(n_hi), size=count))).astype(np.int64)
    tols = np.exp(g.uniform(np.log(tol_lo), np.log(tol_hi), size=count))
    seeds = g.integers(0, 2 ** 31 - 1, size=count)
    return [Request(float(t[k]), int(ns[k]), float(tols[k]), int(seeds[k])) for k in range(count)]


def request_inputs(req: Request):
    """Boundary uniform[0, 100] and a Gaussian-sum source for one request."""
    return random_edges(req.n, req.seed), gaussian_source(req.n, req.seed + 1)


# ---------------------------------------------------------------------------
# Cubes (3D grids), arrays indexed [k, i, j] = plane (z), row (y), column (x).
# ---------------------------------------------------------------------------

def random_shell(n: int, seed: int, lo: float = 0.0, hi: float = 100.0) -> np.ndarray:
    """(n+2)^3 cube whose outer shell holds i.i.d. uniform[lo, hi] values
    (drawn for the whole cube in C order, interior then zeroed); interior 0."""
    g = rng(seed)
    u = g.uniform(lo, hi, size=(n + 2,) * 3)
    u[1:-1, 1:-1, 1:-1] = 0.0
    return u


def heat_cube(n: int, top: float = 100.0) -> np.ndarray:
    """Cube with the plane k = 0 held at `top`, the rest of the shell and the
    interior at 0 (the 3D counterpart of the heated plate)."""
    u = np.zeros((n + 2,) * 3)
    u[0] = top
    return u


def gaussian_source3(n: int, seed: int, count: int = 8) -> np.ndarray:
    """f(x, y, z) = sum_k a_k exp(-|p - p_k|^2 / (2 s_k^2)) on the interior
    nodes, a_k ~ U[-1, 1], s_k ~ U[0.02, 0.2], centres p_k ~ U[0, 1]^3, drawn
    in that order from one PCG64 stream."""
    g = rng(seed)
    a = g.uniform(-1.0, 1.0, size=count)
    s = g.uniform(0.02, 0.2, size=count)
    c = g.uniform(0.0, 1.0, size=(count, 3))
    h = 1.0 / (n + 1)
    t = np.arange(1, n + 1, dtype=np.float64) * h
    f = np.zeros((n, n, n))
    for k in range(count):
        ex = np.exp(-((t - c[k, 0]) ** 2) / (2.0 * s[k] ** 2))
        ey = np.exp(-((t - c[k, 1]) ** 2) / (2.0 * s[k] ** 2))
        ez = np.exp(-((t - c[k, 2]) ** 2) / (2.0 * s[k] ** 2))
        f += a[k] * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return f
