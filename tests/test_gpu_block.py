"""Parity of the block two-colour SOR CUDA path (sor_solve_block) with the
CPU oracle ``oracle.sor_block_f64``, through the C ABI.  Bar: bit identical
(the kernels evaluate every update in the oracle's operation order, one
rounding per operation, and the wavefront inside a block reads the same
values as the oracle's row-major order), with the same iteration count,
stop decision, max|change| and final residual.  Sizes cover 1 x 1 blocks
(red-black SOR), single blocks (natural order), ragged last blocks in both
directions, blocks of 1 to 32 rows (one block per warp, or two to 32 blocks
sharing a warp in segments of 16, 8, 4, 2 or 1 lanes), the degenerate
grids n = 1, 2, 3, and the full 4098^2 plate of the benchmark, in FP64 and
in FP32 (against the FP32 oracle)."""
import numpy as np
import pytest

import oracle
from paper_1401_0763_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    c = capi.Context(0)
    yield c
    c.close()


def capi_mod():
    from paper_1401_0763_gb300 import capi
    return capi


def run_block(ctx, u0, f=None, device=True, **kw):
    if device:
        u0t = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        ft = torch.from_numpy(np.ascontiguousarray(f)).cuda() if f is not None else None
        out, res = ctx.solve_block(u0t, ft, **kw)
        return out.cpu().numpy(), res
    return ctx.solve_block(np.ascontiguousarray(u0), f, **kw)


def check_equal(got, res, ref):
    assert res["iterations"] == ref["iterations"]
    assert res["converged"] == ref["converged"]
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    assert res["final_resid_rel"] == ref["final_resid_rel"]


CASES = [(1, 1, 1), (2, 1, 1), (3, 2, 2), (3, 32, 3), (31, 32, 31), (33, 32, 64), (33, 7, 5), (64, 1, 40),
         (100, 32, 1), (100, 16, 128), (100, 32, 100), (257, 32, 64), (257, 5, 300), (300, 32, 256), (130, 1, 1),
         (131, 2, 9), (129, 4, 33), (140, 8, 20), (150, 9, 17), (161, 16, 40), (170, 17, 3)]


@pytest.mark.parametrize("n,by,bx", CASES)
@pytest.mark.parametrize("with_f", [False, True])
def test_block_bitwise(ctx, n, by, bx, with_f):
    u0 = wl.random_edges(n, 700 + n)
    f = wl.gaussian_source(n, 710 + n) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor_block_f64(u0, w, by=by, bx=bx, f=f, max_iters=60, check_every=4, tol=1e-9)
    got, res = run_block(ctx, u0, f, block_rows=by, block_cols=bx, omega=w, max_iters=60, check_every=4, tol=1e-9)
    check_equal(got, res, ref)


@pytest.mark.parametrize("chain", [1, 2, 3, 7, 1000])
@pytest.mark.parametrize("n,by,bx", [(61, 4, 5), (100, 16, 9), (130, 32, 20), (97, 1, 3)])
def test_block_runs_of_blocks_bitwise(ctx, chain, n, by, bx):
    """SOR_OPT_BLOCK_CHAIN: a warp segment runs 1 .. many blocks of a block row back to back; the
    results are those of the oracle whatever the run length."""
    capi = capi_mod()
    u0 = wl.random_edges(n, 800 + n)
    f = wl.gaussian_source(n, 810 + n)
    ref = oracle.sor_block_f64(u0, 1.7, by=by, bx=bx, f=f, max_iters=25, check_every=5, tol=1e-12)
    ctx.set_option(capi.SOR_OPT_BLOCK_CHAIN, chain)
    try:
        got, res = run_block(ctx, u0, f, block_rows=by, block_cols=bx, omega=1.7, max_iters=25, check_every=5,
                             tol=1e-12)
    finally:
        ctx.set_option(capi.SOR_OPT_BLOCK_CHAIN, 0)
    check_equal(got, res, ref)


FP32_CASES = [(1, 1, 1), (3, 2, 2), (33, 7, 5), (100, 16, 128), (130, 32, 20), (257, 8, 64), (97, 1, 3),
              (300, 32, 300), (170, 17, 3)]


@pytest.mark.parametrize("n,by,bx", FP32_CASES)
@pytest.mark.parametrize("with_f", [False, True])
def test_block_fp32_bitwise(ctx, n, by, bx, with_f):
    """FP32 storage and arithmetic (blocks staged in shared memory): equal to the FP32 oracle bit for bit
    (the same roundings of u0, h^2 f and the coefficients); the final residual is the FP64 one of the
    returned values."""
    capi = capi_mod()
    u0 = wl.random_edges(n, 900 + n)
    f = wl.gaussian_source(n, 910 + n) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor_block_f32(u0, w, by=by, bx=bx, f=f, max_iters=60, check_every=4, tol=1e-5)
    got, res = run_block(ctx, u0, f, block_rows=by, block_cols=bx, omega=w, max_iters=60, check_every=4, tol=1e-5,
                         precision=capi.SOR_FP32)
    assert res["iterations"] == ref["iterations"] and res["converged"] == ref["converged"]
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    assert res["final_resid_rel"] == oracle.resid_rel(ref["u"], f=f)


def test_block_fp32_host_buffers_and_convergence(ctx):
    capi = capi_mod()
    n = 45
    u0 = wl.heat_plate(n, 100.0)
    ref = oracle.sor_block_f32(u0, 1.6, by=16, bx=16, max_iters=5000, check_every=3, tol=1e-4)
    assert ref["converged"]
    got, res = run_block(ctx, u0, device=False, block_rows=16, block_cols=16, omega=1.6, max_iters=5000,
                         check_every=3, tol=1e-4, precision=capi.SOR_FP32)
    assert res["iterations"] == ref["iterations"] and res["converged"]
    assert np.array_equal(got, ref["u"])


def test_block_fp32_full_plate_bitwise(ctx):
    capi = capi_mod()
    n = 4096
    u0 = wl.random_edges(n, 1)
    w = oracle.omega_opt(n)
    ref = oracle.sor_block_f32(u0, w, by=16, bx=128, max_iters=6, check_every=3, tol=-1.0)
    got, res = run_block(ctx, u0, block_rows=16, block_cols=128, omega=w, max_iters=6, check_every=3, tol=-1.0,
                         precision=capi.SOR_FP32)
    assert res["iterations"] == ref["iterations"]
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]


@pytest.mark.parametrize("n,by,bx", [(9, 1, 1), (20, 4, 6), (45, 32, 16)])
def test_block_runs_to_convergence(ctx, n, by, bx):
    u0 = wl.heat_plate(n, 100.0)
    ref = oracle.sor_block_f64(u0, 1.6, by=by, bx=bx, max_iters=5000, check_every=3, tol=1e-8)
    assert ref["converged"]
    got, res = run_block(ctx, u0, block_rows=by, block_cols=bx, omega=1.6, max_iters=5000, check_every=3, tol=1e-8)
    check_equal(got, res, ref)


@pytest.mark.parametrize("K", [1, 5])
def test_block_residual_stop(ctx, K):
    capi = capi_mod()
    n = 70
    u0 = wl.random_edges(n, 31)
    f = wl.gaussian_source(n, 32)
    ref = oracle.sor_block_f64(u0, 1.8, by=8, bx=24, f=f, max_iters=3000, check_every=K, tol=1e-7, stop_mode=1)
    assert ref["converged"]
    got, res = run_block(ctx, u0, f, block_rows=8, block_cols=24, omega=1.8, max_iters=3000, check_every=K,
                         tol=1e-7, stop=capi.SOR_STOP_RESID_REL)
    check_equal(got, res, ref)


def test_block_host_buffers_and_in_place(ctx):
    n = 77
    u0 = wl.random_edges(n, 41)
    f = wl.gaussian_source(n, 42)
    ref = oracle.sor_block_f64(u0, 1.4, by=12, bx=20, f=f, max_iters=40, check_every=7, tol=-1.0)
    got, res = run_block(ctx, u0, f, device=False, block_rows=12, block_cols=20, omega=1.4, max_iters=40,
                         check_every=7, tol=-1.0)
    check_equal(got, res, ref)
    # in place on a device tensor: u_out == u0
    u0t = torch.from_numpy(u0.copy()).cuda()
    ft = torch.from_numpy(f).cuda()
    out, res = ctx.solve_block(u0t, ft, out=u0t, block_rows=12, block_cols=20, omega=1.4, max_iters=40,
                               check_every=7, tol=-1.0)
    assert out.data_ptr() == u0t.data_ptr()
    check_equal(u0t.cpu().numpy(), res, ref)


def test_block_zero_iterations(ctx):
    n = 10
    u0 = wl.random_edges(n, 51)
    ref = oracle.sor_block_f64(u0, 1.3, by=3, bx=3, max_iters=0)
    got, res = run_block(ctx, u0, block_rows=3, block_cols=3, omega=1.3, max_iters=0)
    check_equal(got, res, ref)
    assert res["iterations"] == 0 and np.array_equal(got, u0)


def test_block_rejects_bad_arguments(ctx):
    capi = capi_mod()
    n = 8
    u0 = torch.from_numpy(wl.heat_plate(n, 1.0)).cuda()
    for kw in (dict(block_rows=0, block_cols=4), dict(block_rows=33, block_cols=4), dict(block_rows=4, block_cols=0),
               dict(block_rows=4, block_cols=4, precision=capi.SOR_FP32_REFINE),
               dict(block_rows=4, block_cols=4, precision=capi.SOR_FP32, stop=capi.SOR_STOP_RESID_REL),
               dict(block_rows=1, block_cols=4000, precision=capi.SOR_FP32),
               dict(block_rows=4, block_cols=4, stall_window=3), dict(block_rows=4, block_cols=4, omega=2.5)):
        with pytest.raises(RuntimeError):
            ctx.solve_block(u0, **kw)


@pytest.mark.parametrize("by,bx", [(32, 128), (16, 128), (8, 256)])
def test_block_full_plate_bitwise(ctx, by, bx):
    """The benchmark's plate and block shapes: 4098^2, 6 iterations."""
    n = 4096
    u0 = wl.random_edges(n, 0)
    w = oracle.omega_opt(n)
    ref = oracle.sor_block_f64(u0, w, by=by, bx=bx, max_iters=6, check_every=3, tol=-1.0)
    got, res = run_block(ctx, u0, block_rows=by, block_cols=bx, omega=w, max_iters=6, check_every=3, tol=-1.0)
    check_equal(got, res, ref)
