"""All-core CPU baseline: red-black SOR on POSIX threads (``sor_cpu_mt.c``).

A measurement tool for the benchmark's CPU-baseline leg, not part of the
solver library: it splits the rows of each colour phase among the host's
cores with a barrier between the phases, as the paper's P-worker programs do
(Section 3.1, Section 3.2, Table 1).  It computes the plain FP64 iteration in
the same operation order as the single-threaded oracle and equals it bit for
bit at any thread count (``tests/test_cpu_baseline.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sor_cpu_mt.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsorcpu.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile with gcc: -O2, contraction off (every product and sum rounded
    on its own, as in the oracle), pthreads."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed:\n{r.stderr}")
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.cpu_sor_f64_mt.restype = ctypes.c_int
            lib.cpu_sor_f64_mt.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_int, _dp, _ip, _ip, _dp]
            _lib = lib
    return _lib


def host_cores() -> int:
    """Cores this process may run on (the affinity mask), else os.cpu_count()."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def sor_f64_mt(u0, omega, f=None, max_iters=1000, check_every=1, tol=-1.0, threads=None):
    """Plain FP64 red-black SOR with the max|change| stop on `threads` host
    threads (default: every core).  u0: (n+2)^2 array incl. the Dirichlet
    ring; f: n^2 interior source or None.  Returns a dict with u, iterations,
    converged, final_maxdelta and threads."""
    lib = _load()
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    n = u0.shape[0] - 2
    if u0.ndim != 2 or u0.shape[1] != n + 2 or n < 1:
        raise ValueError("u0 must be an (n+2) x (n+2) array with n >= 1")
    fp = None
    if f is not None:
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (n, n):
            raise ValueError("f must be n x n")
        fp = f.ctypes.data_as(_dp)
    threads = host_cores() if threads is None else int(threads)
    u = np.empty_like(u0)
    it, conv, mk = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    rc = lib.cpu_sor_f64_mt(n, float(omega), u0.ctypes.data_as(_dp), fp, int(max_iters), int(check_every),
                            float(tol), threads, u.ctypes.data_as(_dp), ctypes.byref(it), ctypes.byref(conv),
                            ctypes.byref(mk))
    if rc != 0:
        raise RuntimeError("cpu_sor_f64_mt failed")
    return {"u": u, "iterations": it.value, "converged": bool(conv.value), "final_maxdelta": mk.value,
            "threads": min(threads, n)}
