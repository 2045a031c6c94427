"""ctypes binding of the C ABI in ``include/sor.h`` (``libsorgb.so``).

The functions keep the C names (``sor_create``, ``sor_solve``,
``sor_batch_submit``, ``sor_poll``, ``sor_wait``, ``sor_destroy`` ...) and do
argument marshalling only: every step of the solve runs in the CUDA kernels of
the library.  There is no CPU fallback -- loading fails loudly when the
library has not been built or no CUDA device is present.

:class:`Context` wraps a ``sor_ctx*`` for Python callers and accepts numpy
arrays (host memory) or torch tensors (host or CUDA memory, float64,
contiguous); torch is used only to hold device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

SOR_OK = 0
SOR_NOT_READY = 1
SOR_ERR_INVALID_ARG = -1
SOR_ERR_BUDGET = -2
SOR_ERR_OOM = -3
SOR_ERR_CUDA = -4
SOR_ERR_TIMEOUT = -5
SOR_ERR_INTERNAL = -6
SOR_ERR_UNKNOWN_TICKET = -7
SOR_ERR_CANCELLED = -8

SOR_STOP_MAXDELTA = 0
SOR_STOP_RESID_REL = 1
SOR_FP64 = 0
SOR_FP32 = 1
SOR_FP32_REFINE = 2
SOR_FLAG_EXACT_ORDER = 1

SOR_OPT_TIMING = 1
SOR_OPT_GRAPHS = 2
SOR_OPT_CHUNK = 3
SOR_OPT_TEMPORAL_DEPTH = 4
SOR_OPT_AUTOTUNE = 5
SOR_OPT_BATCH_MAX_SLOTS = 6
SOR_OPT_CLUSTER = 7
SOR_OPT_FAST_CHAIN = 8
SOR_OPT_FUSED_KERNEL = 9
SOR_OPT_BATCH_PLAIN_STEP = 10
SOR_OPT_CUBE_DEPTH = 11
SOR_OPT_BLOCK_CHAIN = 12

EXPORTED = ("sor_create", "sor_solve", "sor_batch_submit", "sor_poll", "sor_wait", "sor_destroy",
            "sor_set_option", "sor_get_option", "sor_get_stats", "sor_reset_stats", "sor_last_error",
            "sor_status_string", "sor_omega_opt", "sor_solve_static", "sor_solve3d",
            "sor_solve9", "sor_diag_flow_wait", "sor_diag_fp64_rate", "sor_diag_bounds", "sor_batch_submit3d",
            "sor_solve_block")


class sor_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("precision", ctypes.c_int32), ("omega", ctypes.c_double),
                ("tol", ctypes.c_double), ("stop", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("inner_sweeps", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("stall_window", ctypes.c_int32)]


class sor_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("outer_steps", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("final_maxdelta", ctypes.c_double),
                ("final_resid_rel", ctypes.c_double), ("latency_s", ctypes.c_double),
                ("device_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class sor_stats(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_uint64), ("batch_completed", ctypes.c_uint64),
                ("sweep_launches", ctypes.c_uint64), ("lattice_updates", ctypes.c_uint64),
                ("sweep_ms", ctypes.c_double), ("timed_launches", ctypes.c_uint64),
                ("timed_updates", ctypes.c_uint64), ("bytes_reserved", ctypes.c_uint64),
                ("bytes_peak", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("batch_plain_step", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    """The library this process loads: the debug variant (device-side index
    checks) when SOR_DEBUG_BOUNDS=1 is set in the environment."""
    return _build.LIB_DEBUG if os.environ.get("SOR_DEBUG_BOUNDS") == "1" else _build.LIB


def load(build_if_missing: bool = False):
    """Load libsorgb.so (optionally building it first).  Raises when absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        debug = os.environ.get("SOR_DEBUG_BOUNDS") == "1"
        path = _build.build(debug=debug) if build_if_missing else library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1401_0763_gb300._build.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        lib.sor_create.argtypes = [P(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p, _alloc_fn,
                                   _free_fn, ctypes.c_void_p]
        lib.sor_solve.argtypes = [ctypes.c_void_p, P(sor_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  P(sor_result)]
        lib.sor_solve3d.argtypes = [ctypes.c_void_p, P(sor_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    P(sor_result)]
        lib.sor_solve9.argtypes = lib.sor_solve.argtypes
        lib.sor_solve_block.argtypes = [ctypes.c_void_p, P(sor_params), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, P(sor_result)]
        lib.sor_batch_submit.argtypes = [ctypes.c_void_p, P(sor_params), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, P(ctypes.c_uint64)]
        lib.sor_batch_submit3d.argtypes = lib.sor_batch_submit.argtypes
        lib.sor_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(sor_result)]
        lib.sor_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, P(sor_result)]
        lib.sor_destroy.argtypes = [ctypes.c_void_p]
        lib.sor_set_option.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]
        lib.sor_get_option.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int64)]
        lib.sor_get_stats.argtypes = [ctypes.c_void_p, P(sor_stats)]
        lib.sor_reset_stats.argtypes = [ctypes.c_void_p]
        lib.sor_last_error.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
        lib.sor_status_string.argtypes = [ctypes.c_int32]
        lib.sor_status_string.restype = ctypes.c_char_p
        lib.sor_solve_static.argtypes = [P(sor_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         P(sor_result), ctypes.c_void_p]
        lib.sor_diag_fp64_rate.argtypes = [ctypes.c_void_p, ctypes.c_int32, dp]
        lib.sor_diag_bounds.argtypes = [ctypes.c_void_p, P(ctypes.c_int32)]
        lib.sor_omega_opt.argtypes = [ctypes.c_int32]
        lib.sor_omega_opt.restype = ctypes.c_double
        for name in EXPORTED:
            if name not in ("sor_status_string", "sor_omega_opt"):
                getattr(lib, name).restype = ctypes.c_int32
        del dp
        _lib = lib
        return lib


class SorError(RuntimeError):
    def __init__(self, status, message=""):
        self.status = status
        super().__init__(f"{status_string(status)} ({status}){': ' + message if message else ''}")


def status_string(status: int) -> str:
    return load().sor_status_string(int(status)).decode()


def sor_omega_opt(n: int) -> float:
    return load().sor_omega_opt(int(n))


def make_params(n, *, precision=SOR_FP64, omega=0.0, tol=1e-8, stop=SOR_STOP_MAXDELTA, max_iters=5000,
                check_every=1, inner_sweeps=0, flags=0, stall_window=0) -> sor_params:
    return sor_params(int(n), int(precision), float(omega), float(tol), int(stop), int(max_iters),
                      int(check_every), int(inner_sweeps), int(flags), int(stall_window))


def _ptr(a):
    """Address of a float64 C-contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("arrays must be C-contiguous float64")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _numel(a):
    return a.size if isinstance(a, np.ndarray) else a.numel()


class Context:
    """A ``sor_ctx*`` on one device.  ``stream`` may be a torch.cuda.Stream,
    a raw ``cudaStream_t`` integer, or None (library-owned stream)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, stream=None):
        self._lib = load()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = ctypes.c_void_p()
        st = self._lib.sor_create(ctypes.byref(h), int(device), int(budget_bytes),
                                  ctypes.c_void_p(int(stream)) if stream else None, _alloc_fn(), _free_fn(), None)
        if st != SOR_OK:
            raise SorError(st, "sor_create")
        self._h = h
        self._keep = {}

    # -- lifecycle ----------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.sor_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls ---------------------------------------------------------------------------------------
    def last_error(self) -> str:
        buf = ctypes.create_string_buffer(1024)
        self._lib.sor_last_error(self._h, buf, 1024)
        return buf.value.decode(errors="replace")

    def _check(self, st, what):
        if st != SOR_OK:
            raise SorError(st, f"{what}: {self.last_error()}")

    def set_option(self, option: int, value: int):
        self._check(self._lib.sor_set_option(self._h, int(option), int(value)), "sor_set_option")

    def get_option(self, option: int) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.sor_get_option(self._h, int(option), ctypes.byref(v)), "sor_get_option")
        return v.value

    def stats(self) -> dict:
        s = sor_stats()
        self._check(self._lib.sor_get_stats(self._h, ctypes.byref(s)), "sor_get_stats")
        return s.as_dict()

    def reset_stats(self):
        self._check(self._lib.sor_reset_stats(self._h), "sor_reset_stats")

    def solve_raw(self, params: sor_params, u0_ptr, f_ptr, out_ptr):
        """sor_solve on raw addresses; returns (status, result)."""
        res = sor_result()
        st = self._lib.sor_solve(self._h, ctypes.byref(params), ctypes.c_void_p(u0_ptr),
                                 ctypes.c_void_p(f_ptr) if f_ptr else None, ctypes.c_void_p(out_ptr),
                                 ctypes.byref(res))
        return st, res

    def solve(self, u0, f=None, out=None, **kw) -> tuple:
        """Blocking solve.  ``u0`` is (n+2, n+2), ``f`` is (n, n) or None.
        Returns (u_out, result dict).  ``out`` defaults to a new array of
        u0's kind (numpy for numpy, a tensor on u0's device for torch)."""
        n = int(u0.shape[0]) - 2
        if tuple(u0.shape) != (n + 2, n + 2):
            raise ValueError("u0 must be square (n+2, n+2)")
        if f is not None and tuple(f.shape) != (n, n):
            raise ValueError("f must be (n, n)")
        if out is None:
            out = np.empty_like(u0) if isinstance(u0, np.ndarray) else u0.new_empty(u0.shape)
        p = make_params(n, **kw)
        st, res = self.solve_raw(p, _ptr(u0), _ptr(f), _ptr(out))
        self._check(st, "sor_solve")
        return out, res.as_dict()

    def solve3d_raw(self, params: sor_params, u0_ptr, f_ptr, out_ptr):
        """sor_solve3d on raw addresses; returns (status, result)."""
        res = sor_result()
        st = self._lib.sor_solve3d(self._h, ctypes.byref(params), ctypes.c_void_p(u0_ptr),
                                   ctypes.c_void_p(f_ptr) if f_ptr else None, ctypes.c_void_p(out_ptr),
                                   ctypes.byref(res))
        return st, res

    def solve3d(self, u0, f=None, out=None, **kw) -> tuple:
        """Blocking solve on a cube.  ``u0`` is (n+2, n+2, n+2) indexed
        [plane, row, column], ``f`` is (n, n, n) or None.  Returns (u_out,
        result dict)."""
        n = int(u0.shape[0]) - 2
        if tuple(u0.shape) != (n + 2,) * 3:
            raise ValueError("u0 must be a cube (n+2, n+2, n+2)")
        if f is not None and tuple(f.shape) != (n,) * 3:
            raise ValueError("f must be (n, n, n)")
        if out is None:
            out = np.empty_like(u0) if isinstance(u0, np.ndarray) else u0.new_empty(u0.shape)
        p = make_params(n, **kw)
        st, res = self.solve3d_raw(p, _ptr(u0), _ptr(f), _ptr(out))
        self._check(st, "sor_solve3d")
        return out, res.as_dict()

    def diag_flow_wait(self, polls: int, preset: int) -> int:
        """sor_diag_flow_wait: 1 when the bounded device wait gave up."""
        out = ctypes.c_int32(-1)
        st = self._lib.sor_diag_flow_wait(self._h, ctypes.c_int32(polls), ctypes.c_int32(preset),
                                          ctypes.byref(out))
        self._check(st, "sor_diag_flow_wait")
        return out.value

    def diag_fp64_rate(self, kind: int = 0) -> float:
        """sor_diag_fp64_rate: measured FP64 lane operations per second
        (kind 0: FMA chains, 1: addition chains)."""
        out = ctypes.c_double(0.0)
        st = self._lib.sor_diag_fp64_rate(self._h, ctypes.c_int32(kind), ctypes.byref(out))
        self._check(st, "sor_diag_fp64_rate")
        return out.value

    def diag_bounds(self) -> int:
        """sor_diag_bounds: 1 when the device-side index checks are compiled
        in (debug build) and refuse an out-of-range index, else 0."""
        out = ctypes.c_int32(-1)
        st = self._lib.sor_diag_bounds(self._h, ctypes.byref(out))
        self._check(st, "sor_diag_bounds")
        return out.value

    def solve9_raw(self, params: sor_params, u0_ptr, f_ptr, out_ptr):
        """sor_solve9 on raw addresses; returns (status, result)."""
        res = sor_result()
        st = self._lib.sor_solve9(self._h, ctypes.byref(params), ctypes.c_void_p(u0_ptr),
                                  ctypes.c_void_p(f_ptr) if f_ptr else None, ctypes.c_void_p(out_ptr),
                                  ctypes.byref(res))
        return st, res

    def solve9(self, u0, f=None, out=None, **kw) -> tuple:
        """Blocking four-colour SOR solve with the 9-point stencil.  ``u0`` is
        (n+2, n+2), ``f`` is (n, n) or None.  Returns (u_out, result dict)."""
        n = int(u0.shape[0]) - 2
        if tuple(u0.shape) != (n + 2, n + 2):
            raise ValueError("u0 must be square (n+2, n+2)")
        if f is not None and tuple(f.shape) != (n, n):
            raise ValueError("f must be (n, n)")
        if out is None:
            out = np.empty_like(u0) if isinstance(u0, np.ndarray) else u0.new_empty(u0.shape)
        p = make_params(n, **kw)
        st, res = self.solve9_raw(p, _ptr(u0), _ptr(f), _ptr(out))
        self._check(st, "sor_solve9")
        return out, res.as_dict()

    def solve_block_raw(self, params: sor_params, block_rows: int, block_cols: int, u0_ptr, f_ptr, out_ptr):
        """sor_solve_block on raw addresses; returns (status, result)."""
        res = sor_result()
        st = self._lib.sor_solve_block(self._h, ctypes.byref(params), int(block_rows), int(block_cols),
                                       ctypes.c_void_p(u0_ptr), ctypes.c_void_p(f_ptr) if f_ptr else None,
                                       ctypes.c_void_p(out_ptr), ctypes.byref(res))
        return st, res

    def solve_block(self, u0, f=None, out=None, *, block_rows: int, block_cols: int, **kw) -> tuple:
        """Blocking block two-colour SOR solve (blocks of block_rows x
        block_cols cells, colour (I + J) mod 2, row-major order inside a
        block).  ``u0`` is (n+2, n+2), ``f`` is (n, n) or None.  Returns
        (u_out, result dict)."""
        n = int(u0.shape[0]) - 2
        if tuple(u0.shape) != (n + 2, n + 2):
            raise ValueError("u0 must be square (n+2, n+2)")
        if f is not None and tuple(f.shape) != (n, n):
            raise ValueError("f must be (n, n)")
        if out is None:
            out = np.empty_like(u0) if isinstance(u0, np.ndarray) else u0.new_empty(u0.shape)
        p = make_params(n, **kw)
        st, res = self.solve_block_raw(p, block_rows, block_cols, _ptr(u0), _ptr(f), _ptr(out))
        self._check(st, "sor_solve_block")
        return out, res.as_dict()

    def submit(self, u0, f=None, out=None, **kw):
        """sor_batch_submit; returns (ticket, out).  Keep ``out`` alive until
        the ticket completes (this object also holds a reference)."""
        n = int(u0.shape[0]) - 2
        if out is None:
            out = np.empty_like(u0) if isinstance(u0, np.ndarray) else u0.new_empty(u0.shape)
        p = make_params(n, **kw)
        t = ctypes.c_uint64()
        st = self._lib.sor_batch_submit(self._h, ctypes.byref(p), ctypes.c_void_p(_ptr(u0)),
                                        ctypes.c_void_p(_ptr(f)) if f is not None else None,
                                        ctypes.c_void_p(_ptr(out)), ctypes.byref(t))
        self._check(st, "sor_batch_submit")
        self._keep[t.value] = out
        return t.value, out

    def submit3d(self, u0, f=None, out=None, **kw):
        """sor_batch_submit3d (a cube request); returns (ticket, out).  Keep
        ``out`` alive until the ticket completes (this object also holds a
        reference)."""
        n = int(u0.shape[0]) - 2
        if tuple(u0.shape) != (n + 2,) * 3:
            raise ValueError("u0 must be (n+2, n+2, n+2)")
        if f is not None and tuple(f.shape) != (n,) * 3:
            raise ValueError("f must be (n, n, n)")
        if out is None:
            out = np.empty_like(u0) if isinstance(u0, np.ndarray) else u0.new_empty(u0.shape)
        p = make_params(n, **kw)
        t = ctypes.c_uint64()
        st = self._lib.sor_batch_submit3d(self._h, ctypes.byref(p), ctypes.c_void_p(_ptr(u0)),
                                          ctypes.c_void_p(_ptr(f)) if f is not None else None,
                                          ctypes.c_void_p(_ptr(out)), ctypes.byref(t))
        self._check(st, "sor_batch_submit3d")
        self._keep[t.value] = out
        return t.value, out

    def poll(self, ticket: int):
        """(status, result dict or None); SOR_NOT_READY while pending."""
        res = sor_result()
        st = self._lib.sor_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(res))
        if st == SOR_NOT_READY:
            return st, None
        self._keep.pop(ticket, None)
        return st, res.as_dict()

    def wait(self, ticket: int, timeout_s: float = -1.0):
        res = sor_result()
        st = self._lib.sor_wait(self._h, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(res))
        if st != SOR_ERR_TIMEOUT:
            self._keep.pop(ticket, None)
        return st, (res.as_dict() if st == SOR_OK else None)
