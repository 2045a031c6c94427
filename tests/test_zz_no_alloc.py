"""sor_solve_static: the entry point for callers that cannot allocate device
memory (fixed memory plans, plug-ins whose framework owns the allocator, code
that may not call cudaMalloc).  Its working memory is one fixed array inside
the library, so it is checked against sor_solve -- the entry point that
allocates -- on two calls in a row: the second call must not see anything
the first left in the shared array.  Both run the exact-order FP64 path, so
the bar is bit-for-bit equality.

This file is collected last so a run that stops at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1401_0763_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    return capi, capi.load()


def _static_solve(capi, lib, u0, f, **kw):
    n = u0.shape[0] - 2
    u0d = torch.from_numpy(u0).cuda()
    fd = torch.from_numpy(f).cuda() if f is not None else None
    outd = torch.full_like(u0d, float("nan"))
    p = capi.make_params(n, **kw)
    res = capi.sor_result()
    torch.cuda.synchronize()
    st = lib.sor_solve_static(ctypes.byref(p), ctypes.c_void_p(u0d.data_ptr()),
                              ctypes.c_void_p(fd.data_ptr()) if fd is not None else None,
                              ctypes.c_void_p(outd.data_ptr()), ctypes.byref(res), None)
    torch.cuda.synchronize()
    return st, outd.cpu().numpy(), res.as_dict()


def test_static_solve_matches_sor_solve_twice_in_a_row():
    capi, lib = _lib()
    # a larger grid with a source first, then a smaller one without: the
    # second call reads a scratch array the first one filled
    n1 = 300
    u1 = wl.random_edges(n1, 5)
    f1 = wl.gaussian_source(n1, 6) * 40
    kw1 = dict(omega=oracle.omega_opt(n1), tol=1e-9, max_iters=4000, check_every=10,
               stop=capi.SOR_STOP_RESID_REL)
    n2 = 64
    u2 = wl.heat_plate(n2, 100.0)
    kw2 = dict(omega=oracle.omega_opt(n2), tol=1e-8, max_iters=3000, check_every=1)
    with capi.Context(0) as ctx:
        for u0, f, kw in ((u1, f1, kw1), (u2, None, kw2)):
            ref, rres = ctx.solve(u0, f, flags=capi.SOR_FLAG_EXACT_ORDER, **kw)
            st, got, res = _static_solve(capi, lib, u0, f, **kw)
            assert st == capi.SOR_OK, capi.status_string(st)
            assert res["converged"] and res["iterations"] == rres["iterations"]
            assert res["final_resid_rel"] == rres["final_resid_rel"]
            assert np.array_equal(got, ref)


def test_static_solve_rejects_what_it_cannot_hold():
    capi, lib = _lib()
    u0 = wl.heat_plate(513, 1.0)
    st, _, _ = _static_solve(capi, lib, u0, None, tol=1e-6, max_iters=10)  # one row past the limit
    assert st == capi.SOR_ERR_INVALID_ARG
    small = wl.heat_plate(16, 1.0)
    st, _, _ = _static_solve(capi, lib, small, None, precision=capi.SOR_FP32, max_iters=10)
    assert st == capi.SOR_ERR_INVALID_ARG
    # host pointers are refused: there is no staging memory to copy them through
    out = np.empty_like(small)
    p = capi.make_params(16, max_iters=10)
    st = lib.sor_solve_static(ctypes.byref(p), ctypes.c_void_p(small.ctypes.data), None,
                              ctypes.c_void_p(out.ctypes.data), None, None)
    assert st == capi.SOR_ERR_INVALID_ARG
