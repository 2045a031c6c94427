"""Independent mathematics the oracle is pinned to (test-side only).

Nothing here calls the oracle or the CUDA path.  The discrete problem is the
5-point Dirichlet problem on an n x n interior with h = 1/(n+1), scaled by h^2:

    4 u_ij - (u_N + u_S + u_W + u_E) = h^2 f_ij      (boundary values on the ring)

written as  A x = b  with the boundary moved to the right side.
"""
from __future__ import annotations

import numpy as np
import scipy.fft


def interior_index(n):
    return np.arange(n * n).reshape(n, n)


def dense_system(u0, f=None):
    """Dense A (n^2 x n^2, natural row-major ordering) and b for the grid u0."""
    n = u0.shape[0] - 2
    h2 = (1.0 / (n + 1)) ** 2
    A = np.zeros((n * n, n * n))
    b = np.zeros(n * n)
    idx = interior_index(n)
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            r = idx[i - 1, j - 1]
            A[r, r] = 4.0
            b[r] = h2 * f[i - 1, j - 1] if f is not None else 0.0
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if 1 <= ii <= n and 1 <= jj <= n:
                    A[r, idx[ii - 1, jj - 1]] = -1.0
                else:
                    b[r] += u0[ii, jj]
    return A, b


def dense_solve(u0, f=None):
    """Exact discrete solution on the full (n+2)^2 array (LAPACK)."""
    n = u0.shape[0] - 2
    A, b = dense_system(u0, f)
    x = np.linalg.solve(A, b)
    u = u0.copy()
    u[1:-1, 1:-1] = x.reshape(n, n)
    return u


def dst_solve(u0, f=None):
    """Exact discrete solution by the type-I discrete sine transform, which
    diagonalises the 5-point Dirichlet operator: eigenvalues
    (2 - 2cos(p pi/(n+1))) + (2 - 2cos(q pi/(n+1)))."""
    n = u0.shape[0] - 2
    h2 = (1.0 / (n + 1)) ** 2
    b = np.zeros((n, n)) if f is None else h2 * np.asarray(f, dtype=np.float64).copy()
    b[0, :] += u0[0, 1:-1]
    b[-1, :] += u0[-1, 1:-1]
    b[:, 0] += u0[1:-1, 0]
    b[:, -1] += u0[1:-1, -1]
    k = np.arange(1, n + 1)
    lam = 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))
    bh = scipy.fft.dstn(b, type=1)
    uh = bh / (lam[:, None] + lam[None, :])
    x = scipy.fft.idstn(uh, type=1)
    u = u0.copy()
    u[1:-1, 1:-1] = x
    return u


def red_black_iteration(u0, omega, iters, f=None):
    """Red-black SOR written as a matrix splitting (not as a sweep): with the
    unknowns ordered red first, A = D - L - U (D = 4I, L strictly lower, U
    strictly upper in that ordering), x_{k+1} = (D - wL)^{-1}[((1-w)D + wU) x_k + w b].
    Returns the list of full arrays u_1..u_iters."""
    n = u0.shape[0] - 2
    A, b = dense_system(u0, f)
    ii, jj = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    red = ((ii + jj) % 2 == 0).ravel()
    order = np.concatenate([np.nonzero(red)[0], np.nonzero(~red)[0]])
    P = A[np.ix_(order, order)]
    bp = b[order]
    D = np.diag(np.diag(P))
    L = -np.tril(P, -1)
    U = -np.triu(P, 1)
    lhs = D - omega * L
    M = np.linalg.solve(lhs, (1.0 - omega) * D + omega * U)
    c = np.linalg.solve(lhs, omega * bp)
    x = u0[1:-1, 1:-1].ravel()[order].copy()
    out = []
    for _ in range(iters):
        x = M @ x + c
        full = np.empty(n * n)
        full[order] = x
        u = u0.copy()
        u[1:-1, 1:-1] = full.reshape(n, n)
        out.append(u)
    return out


def ordered_sor_iteration(u0, omega, iters, order, f=None):
    """SOR with the unknowns updated in the given order (a permutation of the
    natural row-major interior indices), written as the matrix splitting
    x_{k+1} = (D - wL)^{-1}[((1-w)D + wU) x_k + w b] with L / U the strictly
    lower / upper parts of A in that order.  Returns u_1..u_iters."""
    n = u0.shape[0] - 2
    A, b = dense_system(u0, f)
    order = np.asarray(order)
    P = A[np.ix_(order, order)]
    bp = b[order]
    D = np.diag(np.diag(P))
    L = -np.tril(P, -1)
    U = -np.triu(P, 1)
    lhs = D - omega * L
    M = np.linalg.solve(lhs, (1.0 - omega) * D + omega * U)
    c = np.linalg.solve(lhs, omega * bp)
    x = u0[1:-1, 1:-1].ravel()[order].copy()
    out = []
    for _ in range(iters):
        x = M @ x + c
        full = np.empty(n * n)
        full[order] = x
        u = u0.copy()
        u[1:-1, 1:-1] = full.reshape(n, n)
        out.append(u)
    return out


def young_rate(omega, n):
    """Asymptotic SOR convergence factor for a consistently ordered matrix
    with Jacobi spectral radius mu = cos(pi h), for omega <= omega_opt."""
    mu = np.cos(np.pi / (n + 1))
    disc = omega * omega * mu * mu - 4.0 * (omega - 1.0)
    return ((omega * mu + np.sqrt(disc)) / 2.0) ** 2


def rel_err(a, b):
    """Normwise relative difference over the interior: max|a-b| / max|b|."""
    a, b = np.asarray(a)[1:-1, 1:-1], np.asarray(b)[1:-1, 1:-1]
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


# ---------------------------------------------------------------------------
# 3D: the 7-point Dirichlet problem on an n^3 interior, scaled by h^2:
#     6 u - (sum of the six neighbours) = h^2 f,  arrays indexed [k, i, j].
# ---------------------------------------------------------------------------

_NB3 = ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))


def dense_system3(u0, f=None):
    """Dense A (n^3 x n^3, natural ordering k, i, j) and b for the cube u0."""
    n = u0.shape[0] - 2
    h2 = (1.0 / (n + 1)) ** 2
    N = n ** 3
    A = np.zeros((N, N))
    b = np.zeros(N)
    idx = np.arange(N).reshape(n, n, n)
    for k in range(1, n + 1):
        for i in range(1, n + 1):
            for j in range(1, n + 1):
                r = idx[k - 1, i - 1, j - 1]
                A[r, r] = 6.0
                b[r] = h2 * f[k - 1, i - 1, j - 1] if f is not None else 0.0
                for dk, di, dj in _NB3:
                    kk, ii, jj = k + dk, i + di, j + dj
                    if 1 <= kk <= n and 1 <= ii <= n and 1 <= jj <= n:
                        A[r, idx[kk - 1, ii - 1, jj - 1]] = -1.0
                    else:
                        b[r] += u0[kk, ii, jj]
    return A, b


def dense_solve3(u0, f=None):
    """Exact discrete solution on the full (n+2)^3 cube (LAPACK)."""
    n = u0.shape[0] - 2
    A, b = dense_system3(u0, f)
    u = u0.copy()
    u[1:-1, 1:-1, 1:-1] = np.linalg.solve(A, b).reshape(n, n, n)
    return u


def dst_solve3(u0, f=None):
    """Exact discrete solution by the 3D type-I discrete sine transform
    (eigenvalues: the sum of three 1D terms 2 - 2cos(p pi/(n+1)))."""
    n = u0.shape[0] - 2
    h2 = (1.0 / (n + 1)) ** 2
    b = np.zeros((n, n, n)) if f is None else h2 * np.asarray(f, dtype=np.float64).copy()
    b[0] += u0[0, 1:-1, 1:-1]
    b[-1] += u0[-1, 1:-1, 1:-1]
    b[:, 0] += u0[1:-1, 0, 1:-1]
    b[:, -1] += u0[1:-1, -1, 1:-1]
    b[:, :, 0] += u0[1:-1, 1:-1, 0]
    b[:, :, -1] += u0[1:-1, 1:-1, -1]
    p = np.arange(1, n + 1)
    lam = 2.0 - 2.0 * np.cos(p * np.pi / (n + 1))
    uh = scipy.fft.dstn(b, type=1) / (lam[:, None, None] + lam[None, :, None] + lam[None, None, :])
    u = u0.copy()
    u[1:-1, 1:-1, 1:-1] = scipy.fft.idstn(uh, type=1)
    return u


def red_black_iteration3(u0, omega, iters, f=None):
    """3D red-black SOR as a matrix splitting, unknowns ordered red first
    ((i+j+k) even): x_{k+1} = (D - wL)^{-1}[((1-w)D + wU) x_k + w b]."""
    n = u0.shape[0] - 2
    A, b = dense_system3(u0, f)
    kk, ii, jj = np.meshgrid(*(np.arange(1, n + 1),) * 3, indexing="ij")
    red = ((kk + ii + jj) % 2 == 0).ravel()
    order = np.concatenate([np.nonzero(red)[0], np.nonzero(~red)[0]])
    P = A[np.ix_(order, order)]
    bp = b[order]
    D = np.diag(np.diag(P))
    L = -np.tril(P, -1)
    U = -np.triu(P, 1)
    lhs = D - omega * L
    M = np.linalg.solve(lhs, (1.0 - omega) * D + omega * U)
    c = np.linalg.solve(lhs, omega * bp)
    x = u0[1:-1, 1:-1, 1:-1].ravel()[order].copy()
    out = []
    for _ in range(iters):
        x = M @ x + c
        full = np.empty(n ** 3)
        full[order] = x
        u = u0.copy()
        u[1:-1, 1:-1, 1:-1] = full.reshape(n, n, n)
        out.append(u)
    return out


def rel_err3(a, b):
    """Normwise relative difference over the interior of two cubes."""
    a, b = np.asarray(a)[1:-1, 1:-1, 1:-1], np.asarray(b)[1:-1, 1:-1, 1:-1]
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


def cube_from(fn, n):
    """(n+2)^3 cube with the values fn(x, y, z) on the shell and 0 inside
    (x = j h, y = i h, z = k h)."""
    h = 1.0 / (n + 1)
    t = np.arange(n + 2) * h
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    u = fn(x, y, z)
    u[1:-1, 1:-1, 1:-1] = 0.0
    return u, fn(x, y, z)


# ---------------------------------------------------------------------------
# 9-point (compact) Laplacian, scaled by 6 h^2:
#     20 u - 4 (N + S + W + E) - (NW + NE + SW + SE) = 6 h^2 f.
# ---------------------------------------------------------------------------

_NB9 = (((-1, 0), 4.0), ((1, 0), 4.0), ((0, -1), 4.0), ((0, 1), 4.0),
        ((-1, -1), 1.0), ((-1, 1), 1.0), ((1, -1), 1.0), ((1, 1), 1.0))


def dense_system9(u0, f=None):
    """Dense A (n^2 x n^2) and b of the 9-point system for the grid u0."""
    n = u0.shape[0] - 2
    h2 = (1.0 / (n + 1)) ** 2
    A = np.zeros((n * n, n * n))
    b = np.zeros(n * n)
    idx = interior_index(n)
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            r = idx[i - 1, j - 1]
            A[r, r] = 20.0
            b[r] = 6.0 * h2 * f[i - 1, j - 1] if f is not None else 0.0
            for (di, dj), wgt in _NB9:
                ii, jj = i + di, j + dj
                if 1 <= ii <= n and 1 <= jj <= n:
                    A[r, idx[ii - 1, jj - 1]] = -wgt
                else:
                    b[r] += wgt * u0[ii, jj]
    return A, b


def dense_solve9(u0, f=None):
    n = u0.shape[0] - 2
    A, b = dense_system9(u0, f)
    u = u0.copy()
    u[1:-1, 1:-1] = np.linalg.solve(A, b).reshape(n, n)
    return u


def dst_solve9(u0, f=None):
    """Exact 9-point solution by the 2D DST-I: with cp = cos(p pi/(n+1)) the
    operator's eigenvalues are 20 - 8 cp - 8 cq - 4 cp cq."""
    n = u0.shape[0] - 2
    h2 = (1.0 / (n + 1)) ** 2
    b = np.zeros((n, n)) if f is None else 6.0 * h2 * np.asarray(f, dtype=np.float64).copy()
    # ring contributions: 4 x edge neighbours, 1 x diagonal neighbours
    b[0, :] += 4.0 * u0[0, 1:-1] + u0[0, :-2] + u0[0, 2:]
    b[-1, :] += 4.0 * u0[-1, 1:-1] + u0[-1, :-2] + u0[-1, 2:]
    b[:, 0] += 4.0 * u0[1:-1, 0] + u0[:-2, 0] + u0[2:, 0]
    b[:, -1] += 4.0 * u0[1:-1, -1] + u0[:-2, -1] + u0[2:, -1]
    # the four corner cells received their shared diagonal ring neighbour twice
    b[0, 0] -= u0[0, 0]
    b[0, -1] -= u0[0, -1]
    b[-1, 0] -= u0[-1, 0]
    b[-1, -1] -= u0[-1, -1]
    p = np.arange(1, n + 1)
    c = np.cos(p * np.pi / (n + 1))
    lam = 20.0 - 8.0 * c[:, None] - 8.0 * c[None, :] - 4.0 * c[:, None] * c[None, :]
    u = u0.copy()
    u[1:-1, 1:-1] = scipy.fft.idstn(scipy.fft.dstn(b, type=1) / lam, type=1)
    return u


def multicolour_iteration9(u0, omega, iters, f=None):
    """Four-colour SOR as a matrix splitting: unknowns ordered by colour
    2(i&1) + (j&1) = 0, 1, 2, 3, x_{k+1} = (D - wL)^{-1}[((1-w)D + wU) x_k + w b]."""
    n = u0.shape[0] - 2
    A, b = dense_system9(u0, f)
    ii, jj = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    colour = (2 * (ii & 1) + (jj & 1)).ravel()
    order = np.concatenate([np.nonzero(colour == c)[0] for c in range(4)])
    P = A[np.ix_(order, order)]
    bp = b[order]
    D = np.diag(np.diag(P))
    L = -np.tril(P, -1)
    U = -np.triu(P, 1)
    lhs = D - omega * L
    M = np.linalg.solve(lhs, (1.0 - omega) * D + omega * U)
    cvec = np.linalg.solve(lhs, omega * bp)
    x = u0[1:-1, 1:-1].ravel()[order].copy()
    out = []
    for _ in range(iters):
        x = M @ x + cvec
        full = np.empty(n * n)
        full[order] = x
        u = u0.copy()
        u[1:-1, 1:-1] = full.reshape(n, n)
        out.append(u)
    return out


def grid_from(fn, n):
    """(n+2)^2 grid with fn(x, y) on the ring (corners included) and 0 inside,
    plus fn on the whole grid (x = j h, y = i h)."""
    h = 1.0 / (n + 1)
    t = np.arange(n + 2) * h
    y, x = np.meshgrid(t, t, indexing="ij")
    full = fn(x, y)
    u = full.copy()
    u[1:-1, 1:-1] = 0.0
    return u, full
