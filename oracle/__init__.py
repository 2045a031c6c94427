"""Red-black SOR oracle: a plain FP64 (and FP32-sweep) CPU implementation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_1401_0763_gb300``) and neither
imports the other; the seeded input generators in
``paper_1401_0763_gb300.workloads`` hold no arithmetic of the method and are
the only thing both sides use.

What each function computes is stated in ``sor_oracle.c`` (2D),
``sor3d_oracle.c`` (3D) and ``sor9_oracle.c`` (four-colour, 9-point); in
short:

* :func:`sor_f64` -- Algorithm 1 of the paper (red phase, then black phase,
  convergence test every K iterations, Section 2.1 / Section 3.3) with the
  cell update of Eq. 1 taken with the 5-point Gauss-Seidel value.
* :func:`sor_f32` -- the same iteration in FP32 arithmetic and storage.
* :func:`sor_block_f64` -- block two-colour SOR, the reading of the
  block-parallel SOR that Section 3.1 names beside red-black SOR: blocks of
  by x bx cells coloured like a checkerboard, colour 0 first, row-major order
  inside a block; :func:`sor_block_f32` -- the same in FP32.
* :func:`residual` -- the scaled residual h^2 (f - A u) and its infinity
  norm relative to the right-hand side (boundary moved to the right).
* :func:`refine` -- FP64 defect correction around FP32 (or FP64) inner
  red-black SOR sweeps.
* :func:`sor3d_f64`, :func:`sor3d_f32`, :func:`residual3d` -- the same
  iteration and residual on a cube with the 7-point stencil (the 3D grids the
  paper names as its next step, Section 5); :func:`refine3d` -- the defect
  correction on a cube.
* :func:`sor9_f64`, :func:`sor9_f32`, :func:`residual9` -- multi-colour SOR
  (Section 3.1 names it beside red-black SOR): four colours for the compact
  9-point stencil; :func:`refine9` -- the defect correction with it.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``,
``tests/test_oracle_block_pins.py``, ``tests/test_oracle3d_pins.py`` and
``tests/test_oracle9_pins.py`` (dense
direct solves, the explicit SOR
iteration matrix, closed-form harmonic and quadratic solutions, a DST-I fast
Poisson solve, SOR convergence theory and superposition/symmetry invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "sor_oracle.c"), os.path.join(_HERE, "sor3d_oracle.c"),
         os.path.join(_HERE, "sor9_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle's C sources with gcc (contraction off) into ``_build/``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src) for src in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC", "-shared",
           "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_sor_f64.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _ip, _ip, _dp, _dp, _dp]
            lib.oracle_sor_block_f64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp,
                                                 _ip, _ip, _dp, _dp, _dp]
            lib.oracle_sor_block_f32.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _ip, _ip, _dp,
                                                 _dp]
            lib.oracle_sor_f32.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, _dp, _ip, _ip, _dp, _dp]
            lib.oracle_residual.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            lib.oracle_refine.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _ip, _ip, _ip, _dp, _dp]
            lib.oracle_sor3d_f64.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _ip, _ip, _dp, _dp,
                                             _dp]
            lib.oracle_sor3d_f32.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, _dp, _ip, _ip, _dp, _dp]
            lib.oracle_residual3d.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            lib.oracle_refine3d.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _ip, _ip, _ip, _dp,
                                            _dp]
            lib.oracle_sor9_f64.argtypes = lib.oracle_sor3d_f64.argtypes
            lib.oracle_sor9_f32.argtypes = lib.oracle_sor3d_f32.argtypes
            lib.oracle_residual9.argtypes = lib.oracle_residual3d.argtypes
            lib.oracle_refine9.argtypes = lib.oracle_refine3d.argtypes
            for fn in (lib.oracle_sor_f64, lib.oracle_sor_f32, lib.oracle_residual, lib.oracle_refine,
                       lib.oracle_sor3d_f64, lib.oracle_sor3d_f32, lib.oracle_residual3d, lib.oracle_refine3d,
                       lib.oracle_sor9_f64, lib.oracle_sor9_f32, lib.oracle_residual9, lib.oracle_refine9):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _grid(u0, n):
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    if u0.shape != (n + 2, n + 2):
        raise ValueError(f"u0 must be ({n + 2},{n + 2}), got {u0.shape}")
    return u0


def _src(f, n):
    if f is None:
        return None
    f = np.ascontiguousarray(f, dtype=np.float64)
    if f.shape != (n, n):
        raise ValueError(f"f must be ({n},{n}), got {f.shape}")
    return f


def omega_opt(n: int) -> float:
    """Optimal SOR factor for the 5-point Laplacian on an n x n interior,
    2 / (1 + sin(pi h)), h = 1/(n+1) (Young's theory; the paper's Eq. 1
    leaves the choice of the factor open)."""
    return 2.0 / (1.0 + np.sin(np.pi / (n + 1)))


def sor_f64(u0, omega, *, f=None, max_iters=5000, check_every=1, tol=1e-8, stop_mode=0, stall_window=0,
            trace=False):
    """Plain FP64 red-black SOR (Algorithm 1).  Returns a dict with ``u``,
    ``iterations``, ``converged``, ``final_maxdelta``, ``final_resid_rel`` and,
    when ``trace`` is set, ``trace`` = m_k for k = 1..iterations.  With
    stop_mode 1 and stall_window > 0 the loop also stops (not converged) once
    that many residual tests in a row gave no new smallest residual."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _grid(u0, n)
    f = _src(f, n)
    u = np.empty_like(u0)
    it, cv = ctypes.c_int(0), ctypes.c_int(0)
    md, rr = ctypes.c_double(0), ctypes.c_double(0)
    tr = np.zeros(max(max_iters, 1)) if trace else None
    rc = _load().oracle_sor_f64(n, float(omega), _ptr(u0), _ptr(f), int(max_iters), int(check_every), float(tol),
                                int(stop_mode), int(stall_window), _ptr(u), ctypes.byref(it), ctypes.byref(cv),
                                ctypes.byref(md), ctypes.byref(rr), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_sor_f64: bad arguments")
    out = dict(u=u, iterations=it.value, converged=bool(cv.value), final_maxdelta=md.value,
               final_resid_rel=rr.value)
    if trace:
        out["trace"] = tr[: it.value].copy()
    return out


def sor_block_f64(u0, omega, *, by, bx, f=None, max_iters=5000, check_every=1, tol=1e-8, stop_mode=0,
                  trace=False):
    """Block two-colour SOR in FP64 (the reading of block-parallel SOR stated
    in ``sor_oracle.c``): blocks of ``by`` x ``bx`` cells coloured (I + J) mod
    2, colour 0 first, row-major order inside a block.  Same loop, stopping
    test and result dict as :func:`sor_f64` (no stall rule)."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _grid(u0, n)
    f = _src(f, n)
    u = np.empty_like(u0)
    it, cv = ctypes.c_int(0), ctypes.c_int(0)
    md, rr = ctypes.c_double(0), ctypes.c_double(0)
    tr = np.zeros(max(max_iters, 1)) if trace else None
    rc = _load().oracle_sor_block_f64(n, int(by), int(bx), float(omega), _ptr(u0), _ptr(f), int(max_iters),
                                      int(check_every), float(tol), int(stop_mode), _ptr(u), ctypes.byref(it),
                                      ctypes.byref(cv), ctypes.byref(md), ctypes.byref(rr), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_sor_block_f64: bad arguments")
    out = dict(u=u, iterations=it.value, converged=bool(cv.value), final_maxdelta=md.value,
               final_resid_rel=rr.value)
    if trace:
        out["trace"] = tr[: it.value].copy()
    return out


def sor_block_f32(u0, omega, *, by, bx, f=None, max_iters=5000, check_every=1, tol=1e-8, trace=False):
    """Block two-colour SOR in FP32 arithmetic and storage, with the
    conventions of :func:`sor_f32` (stop on max|change|)."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _grid(u0, n)
    f = _src(f, n)
    u = np.empty_like(u0)
    it, cv = ctypes.c_int(0), ctypes.c_int(0)
    md = ctypes.c_double(0)
    tr = np.zeros(max(max_iters, 1)) if trace else None
    rc = _load().oracle_sor_block_f32(n, int(by), int(bx), float(omega), _ptr(u0), _ptr(f), int(max_iters),
                                      int(check_every), float(tol), _ptr(u), ctypes.byref(it), ctypes.byref(cv),
                                      ctypes.byref(md), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_sor_block_f32: bad arguments")
    out = dict(u=u, iterations=it.value, converged=bool(cv.value), final_maxdelta=md.value)
    if trace:
        out["trace"] = tr[: it.value].copy()
    return out


def sor_f32(u0, omega, *, f=None, max_iters=5000, check_every=1, tol=1e-8, trace=False):
    """Red-black SOR in FP32 arithmetic and storage (stop on max|change|)."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _grid(u0, n)
    f = _src(f, n)
    u = np.empty_like(u0)
    it, cv = ctypes.c_int(0), ctypes.c_int(0)
    md = ctypes.c_double(0)
    tr = np.zeros(max(max_iters, 1)) if trace else None
    rc = _load().oracle_sor_f32(n, float(omega), _ptr(u0), _ptr(f), int(max_iters), int(check_every), float(tol),
                                _ptr(u), ctypes.byref(it), ctypes.byref(cv), ctypes.byref(md), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_sor_f32: bad arguments")
    out = dict(u=u, iterations=it.value, converged=bool(cv.value), final_maxdelta=md.value)
    if trace:
        out["trace"] = tr[: it.value].copy()
    return out


def residual(u, *, f=None):
    """Scaled residual r~ = h^2 f + sum_nb(u) - 4u on the (n+2)^2 array (ring 0)
    and (max|r~|, max|b~|)."""
    n = int(np.asarray(u).shape[0]) - 2
    u = _grid(u, n)
    f = _src(f, n)
    r = np.zeros_like(u)
    rm, bm = ctypes.c_double(0), ctypes.c_double(0)
    rc = _load().oracle_residual(n, _ptr(u), _ptr(f), _ptr(r), ctypes.byref(rm), ctypes.byref(bm))
    if rc != 0:
        raise ValueError("oracle_residual: bad arguments")
    return r, rm.value, bm.value


def resid_rel(u, *, f=None):
    """max|r~| / max|b~| (or max|r~| when the right side is zero)."""
    _, rm, bm = residual(u, f=f)
    return rm / bm if bm > 0 else rm


def refine(u0, omega, *, f=None, inner_sweeps=20, inner_f32=True, tol=1e-10, max_outer=10000, stall_window=0,
           trace=False):
    """FP64 defect correction around reduced-precision red-black SOR sweeps
    (stall_window > 0: stop, not converged, after that many residual tests in
    a row without a new smallest residual)."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _grid(u0, n)
    f = _src(f, n)
    u = np.empty_like(u0)
    ou, sw, cv = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    rr = ctypes.c_double(0)
    tr = np.zeros(max_outer + 1) if trace else None
    rc = _load().oracle_refine(n, float(omega), _ptr(u0), _ptr(f), int(inner_sweeps), int(bool(inner_f32)),
                               float(tol), int(max_outer), int(stall_window), _ptr(u), ctypes.byref(ou),
                               ctypes.byref(sw),
                               ctypes.byref(cv), ctypes.byref(rr), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_refine: bad arguments")
    out = dict(u=u, outer_steps=ou.value, sweeps=sw.value, converged=bool(cv.value), final_resid_rel=rr.value)
    if trace:
        out["trace"] = tr[: ou.value + 1].copy()
    return out


def _cube(u0, n):
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    if u0.shape != (n + 2, n + 2, n + 2):
        raise ValueError(f"u0 must be ({n + 2},{n + 2},{n + 2}), got {u0.shape}")
    return u0


def _src3(f, n):
    if f is None:
        return None
    f = np.ascontiguousarray(f, dtype=np.float64)
    if f.shape != (n, n, n):
        raise ValueError(f"f must be ({n},{n},{n}), got {f.shape}")
    return f


def sor3d_f64(u0, omega, *, f=None, max_iters=5000, check_every=1, tol=1e-8, stop_mode=0, stall_window=0,
              trace=False):
    """Plain FP64 red-black SOR on an (n+2)^3 cube, 7-point stencil (index
    order [k, i, j] = plane, row, column; stall_window as for
    :func:`sor_f64`).  Returns a dict like :func:`sor_f64`."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _cube(u0, n)
    f = _src3(f, n)
    u = np.empty_like(u0)
    it, cv = ctypes.c_int(0), ctypes.c_int(0)
    md, rr = ctypes.c_double(0), ctypes.c_double(0)
    tr = np.zeros(max(max_iters, 1)) if trace else None
    rc = _load().oracle_sor3d_f64(n, float(omega), _ptr(u0), _ptr(f), int(max_iters), int(check_every), float(tol),
                                  int(stop_mode), int(stall_window), _ptr(u), ctypes.byref(it), ctypes.byref(cv),
                                  ctypes.byref(md), ctypes.byref(rr), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_sor3d_f64: bad arguments")
    out = dict(u=u, iterations=it.value, converged=bool(cv.value), final_maxdelta=md.value,
               final_resid_rel=rr.value)
    if trace:
        out["trace"] = tr[: it.value].copy()
    return out


def sor3d_f32(u0, omega, *, f=None, max_iters=5000, check_every=1, tol=1e-8, trace=False):
    """Red-black SOR on a cube in FP32 arithmetic and storage (stop on
    max|change|)."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _cube(u0, n)
    f = _src3(f, n)
    u = np.empty_like(u0)
    it, cv = ctypes.c_int(0), ctypes.c_int(0)
    md = ctypes.c_double(0)
    tr = np.zeros(max(max_iters, 1)) if trace else None
    rc = _load().oracle_sor3d_f32(n, float(omega), _ptr(u0), _ptr(f), int(max_iters), int(check_every), float(tol),
                                  _ptr(u), ctypes.byref(it), ctypes.byref(cv), ctypes.byref(md), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_sor3d_f32: bad arguments")
    out = dict(u=u, iterations=it.value, converged=bool(cv.value), final_maxdelta=md.value)
    if trace:
        out["trace"] = tr[: it.value].copy()
    return out


def residual3d(u, *, f=None):
    """Scaled residual r~ = h^2 f + sum_nb(u) - 6u on the (n+2)^3 cube (shell
    0) and (max|r~|, max|b~|)."""
    n = int(np.asarray(u).shape[0]) - 2
    u = _cube(u, n)
    f = _src3(f, n)
    r = np.zeros_like(u)
    rm, bm = ctypes.c_double(0), ctypes.c_double(0)
    rc = _load().oracle_residual3d(n, _ptr(u), _ptr(f), _ptr(r), ctypes.byref(rm), ctypes.byref(bm))
    if rc != 0:
        raise ValueError("oracle_residual3d: bad arguments")
    return r, rm.value, bm.value


def resid_rel3d(u, *, f=None):
    """max|r~| / max|b~| on a cube (or max|r~| when the right side is zero)."""
    _, rm, bm = residual3d(u, f=f)
    return rm / bm if bm > 0 else rm


def refine3d(u0, omega, *, f=None, inner_sweeps=20, inner_f32=True, tol=1e-10, max_outer=10000, stall_window=0,
             trace=False):
    """FP64 defect correction on a cube around FP32 (or FP64) inner red-black
    SOR sweeps (7-point stencil).  Returns a dict like :func:`refine`."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _cube(u0, n)
    f = _src3(f, n)
    u = np.empty_like(u0)
    ou, sw, cv = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    rr = ctypes.c_double(0)
    tr = np.zeros(max_outer + 1) if trace else None
    rc = _load().oracle_refine3d(n, float(omega), _ptr(u0), _ptr(f), int(inner_sweeps), int(bool(inner_f32)),
                                 float(tol), int(max_outer), int(stall_window), _ptr(u), ctypes.byref(ou),
                                 ctypes.byref(sw), ctypes.byref(cv), ctypes.byref(rr), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_refine3d: bad arguments")
    out = dict(u=u, outer_steps=ou.value, sweeps=sw.value, converged=bool(cv.value), final_resid_rel=rr.value)
    if trace:
        out["trace"] = tr[: ou.value + 1].copy()
    return out


def sor9_f64(u0, omega, *, f=None, max_iters=5000, check_every=1, tol=1e-8, stop_mode=0, stall_window=0,
             trace=False):
    """Four-colour SOR on the 9-point stencil, FP64 (colour 2(i&1) + (j&1),
    colours updated 0, 1, 2, 3; stall_window as for :func:`sor_f64`).
    Returns a dict like :func:`sor_f64`."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _grid(u0, n)
    f = _src(f, n)
    u = np.empty_like(u0)
    it, cv = ctypes.c_int(0), ctypes.c_int(0)
    md, rr = ctypes.c_double(0), ctypes.c_double(0)
    tr = np.zeros(max(max_iters, 1)) if trace else None
    rc = _load().oracle_sor9_f64(n, float(omega), _ptr(u0), _ptr(f), int(max_iters), int(check_every), float(tol),
                                 int(stop_mode), int(stall_window), _ptr(u), ctypes.byref(it), ctypes.byref(cv),
                                 ctypes.byref(md), ctypes.byref(rr), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_sor9_f64: bad arguments")
    out = dict(u=u, iterations=it.value, converged=bool(cv.value), final_maxdelta=md.value,
               final_resid_rel=rr.value)
    if trace:
        out["trace"] = tr[: it.value].copy()
    return out


def sor9_f32(u0, omega, *, f=None, max_iters=5000, check_every=1, tol=1e-8, trace=False):
    """Four-colour 9-point SOR in FP32 arithmetic and storage."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _grid(u0, n)
    f = _src(f, n)
    u = np.empty_like(u0)
    it, cv = ctypes.c_int(0), ctypes.c_int(0)
    md = ctypes.c_double(0)
    tr = np.zeros(max(max_iters, 1)) if trace else None
    rc = _load().oracle_sor9_f32(n, float(omega), _ptr(u0), _ptr(f), int(max_iters), int(check_every), float(tol),
                                 _ptr(u), ctypes.byref(it), ctypes.byref(cv), ctypes.byref(md), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_sor9_f32: bad arguments")
    out = dict(u=u, iterations=it.value, converged=bool(cv.value), final_maxdelta=md.value)
    if trace:
        out["trace"] = tr[: it.value].copy()
    return out


def residual9(u, *, f=None):
    """Scaled 9-point residual r~ = 6h^2 f + 4 s4 + sd - 20u (ring 0) and
    (max|r~|, max|b~|)."""
    n = int(np.asarray(u).shape[0]) - 2
    u = _grid(u, n)
    f = _src(f, n)
    r = np.zeros_like(u)
    rm, bm = ctypes.c_double(0), ctypes.c_double(0)
    rc = _load().oracle_residual9(n, _ptr(u), _ptr(f), _ptr(r), ctypes.byref(rm), ctypes.byref(bm))
    if rc != 0:
        raise ValueError("oracle_residual9: bad arguments")
    return r, rm.value, bm.value


def resid_rel9(u, *, f=None):
    _, rm, bm = residual9(u, f=f)
    return rm / bm if bm > 0 else rm


def refine9(u0, omega, *, f=None, inner_sweeps=20, inner_f32=True, tol=1e-10, max_outer=10000, stall_window=0,
             trace=False):
    """FP64 defect correction around FP32 (or FP64) inner four-colour 9-point
    SOR sweeps.  Returns a dict like :func:`refine`."""
    n = int(np.asarray(u0).shape[0]) - 2
    u0 = _grid(u0, n)
    f = _src(f, n)
    u = np.empty_like(u0)
    ou, sw, cv = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    rr = ctypes.c_double(0)
    tr = np.zeros(max_outer + 1) if trace else None
    rc = _load().oracle_refine9(n, float(omega), _ptr(u0), _ptr(f), int(inner_sweeps), int(bool(inner_f32)),
                                float(tol), int(max_outer), int(stall_window), _ptr(u), ctypes.byref(ou),
                                ctypes.byref(sw), ctypes.byref(cv), ctypes.byref(rr), _ptr(tr))
    if rc != 0:
        raise ValueError("oracle_refine9: bad arguments")
    out = dict(u=u, outer_steps=ou.value, sweeps=sw.value, converged=bool(cv.value), final_resid_rel=rr.value)
    if trace:
        out["trace"] = tr[: ou.value + 1].copy()
    return out
