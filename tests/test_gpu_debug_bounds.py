"""The debug build's device-side index checks (SOR_DEBUG_BOUNDS).

Before a kernel touches a tile of a plate it checks that the rows and
columns it will read and write lie inside the slot's arrays; a tile that does
not is skipped and the solve fails with "device-side index check failed"
instead of touching other memory.  Here, in a fresh process that loads the
debug build:
* the probe entry point shows the check is compiled in and refuses an index
  outside its range (no memory is accessed at that index);
* small grids on every plate path -- exact-order and default FP64, FP32
  sweeps of both fused families, defect correction, the batch scheduler --
  and on the cube, 9-point and block-SOR paths (every precision, the cube's
  blocked sweeps at both depths, block runs of one and of several blocks) run
  with no check firing and give the oracle's results.
The release library reports the checks compiled away.
"""
import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, %r)
    import oracle
    from paper_1401_0763_gb300 import capi, workloads as wl
    capi.load(build_if_missing=True)
    assert capi.library_path().endswith("_build_debug/libsorgb.so")
    with capi.Context(0) as ctx:
        assert ctx.diag_bounds() == 1
        ctx.set_option(capi.SOR_OPT_CLUSTER, 0)
        for n in (1, 3, 130, 301):
            u0 = wl.random_edges(n, n)
            f = wl.gaussian_source(n, n + 1) * 10
            w = oracle.omega_opt(n)
            ref = oracle.sor_f64(u0, w, f=f, max_iters=23, check_every=7, tol=-1.0)
            got, res = ctx.solve(u0, f, omega=w, tol=-1.0, max_iters=23, check_every=7,
                                 flags=capi.SOR_FLAG_EXACT_ORDER)
            assert np.array_equal(got, ref["u"]), n
            got, res = ctx.solve(u0, f, omega=w, tol=-1.0, max_iters=23, check_every=7)
            assert np.max(np.abs(got - ref["u"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["u"]))), n
            ref32 = oracle.sor_f32(u0, w, f=f, max_iters=25, check_every=5, tol=-1.0)
            for family, depth in ((1, 6), (2, 3)):
                ctx.set_option(capi.SOR_OPT_FUSED_KERNEL, family)
                ctx.set_option(capi.SOR_OPT_TEMPORAL_DEPTH, depth)
                got, res = ctx.solve(u0, f, precision=capi.SOR_FP32, omega=w, tol=-1.0, max_iters=25, check_every=5)
                assert np.array_equal(got, ref32["u"]), (n, family, depth)
                refr = oracle.refine(u0, w, f=f, inner_sweeps=7, tol=1e-9, max_outer=500)
                got, res = ctx.solve(u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-9, max_iters=3500,
                                     inner_sweeps=7)
                assert np.array_equal(got, refr["u"]), (n, family, depth)
        jobs = []
        for k, n in enumerate((40, 90, 257)):
            u0, f = wl.poisson_problem(n, k)
            t, out = ctx.submit(u0, f, precision=capi.SOR_FP32_REFINE, omega=oracle.omega_opt(n), tol=1e-9,
                                max_iters=50000)
            jobs.append((t, out, u0, f, n))
        for t, out, u0, f, n in jobs:
            st, res = ctx.wait(t, 120.0)
            assert st == capi.SOR_OK, ctx.last_error()
            ref = oracle.refine(u0, oracle.omega_opt(n), f=f, inner_sweeps=20, tol=1e-9, max_outer=2500)
            assert np.array_equal(out, ref["u"]), n
        # cubes: FP64 default and exact order, FP32 per phase and blocked, defect correction
        for n in (1, 6, 33):
            u0 = wl.random_shell(n, n)
            f = wl.gaussian_source3(n, n + 2) * 5
            w = oracle.omega_opt(n)
            ref = oracle.sor3d_f64(u0, w, f=f, max_iters=21, check_every=7, tol=-1.0)
            got, res = ctx.solve3d(u0, f, omega=w, tol=-1.0, max_iters=21, check_every=7,
                                   flags=capi.SOR_FLAG_EXACT_ORDER)
            assert np.array_equal(got, ref["u"]), n
            got, res = ctx.solve3d(u0, f, omega=w, tol=-1.0, max_iters=21, check_every=7)
            assert np.max(np.abs(got - ref["u"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["u"]))), n
            ref32 = oracle.sor3d_f32(u0, w, f=f, max_iters=21, check_every=7, tol=-1.0)
            for depth in (0, 1, 2):
                ctx.set_option(capi.SOR_OPT_CUBE_DEPTH, depth)
                got, res = ctx.solve3d(u0, f, precision=capi.SOR_FP32, omega=w, tol=-1.0, max_iters=21,
                                       check_every=7)
                assert np.array_equal(got, ref32["u"]), (n, depth)
            ctx.set_option(capi.SOR_OPT_CUBE_DEPTH, 0)
            refr = oracle.refine3d(u0, w, f=f, inner_sweeps=20, tol=1e-9, max_outer=300)
            got, res = ctx.solve3d(u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-9, max_iters=6000)
            assert np.array_equal(got, refr["u"]), n
        # 9-point plates: FP64 default and exact order, FP32, defect correction
        for n in (1, 4, 77):
            u0 = wl.random_edges(n, n + 5)
            f = wl.gaussian_source(n, n + 6) * 5
            w = oracle.omega_opt(n)
            ref = oracle.sor9_f64(u0, w, f=f, max_iters=22, check_every=11, tol=-1.0)
            got, res = ctx.solve9(u0, f, omega=w, tol=-1.0, max_iters=22, check_every=11,
                                  flags=capi.SOR_FLAG_EXACT_ORDER)
            assert np.array_equal(got, ref["u"]), n
            got, res = ctx.solve9(u0, f, omega=w, tol=-1.0, max_iters=22, check_every=11)
            assert np.max(np.abs(got - ref["u"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["u"]))), n
            ref32 = oracle.sor9_f32(u0, w, f=f, max_iters=22, check_every=11, tol=-1.0)
            got, res = ctx.solve9(u0, f, precision=capi.SOR_FP32, omega=w, tol=-1.0, max_iters=22, check_every=11)
            assert np.array_equal(got, ref32["u"]), n
            refr = oracle.refine9(u0, w, f=f, inner_sweeps=20, tol=1e-9, max_outer=400)
            got, res = ctx.solve9(u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-9, max_iters=8000)
            assert np.array_equal(got, refr["u"]), n
        # block two-colour SOR: one-block runs and runs of several blocks
        for n, by, bx, chain in ((1, 1, 1, 0), (5, 2, 3, 0), (70, 7, 5, 0), (70, 32, 20, 3), (45, 16, 128, 0)):
            u0 = wl.random_edges(n, n + 9)
            f = wl.gaussian_source(n, n + 10) * 5
            ref = oracle.sor_block_f64(u0, 1.6, by=by, bx=bx, f=f, max_iters=12, check_every=4, tol=-1.0)
            ctx.set_option(capi.SOR_OPT_BLOCK_CHAIN, chain)
            got, res = ctx.solve_block(u0, f, block_rows=by, block_cols=bx, omega=1.6, tol=-1.0, max_iters=12,
                                       check_every=4)
            ctx.set_option(capi.SOR_OPT_BLOCK_CHAIN, 0)
            assert np.array_equal(got, ref["u"]), (n, by, bx, chain)
    print("debug build checks passed")
""") % ROOT


def test_debug_build_checks_fire_and_stay_quiet_on_valid_work():
    env = dict(os.environ, SOR_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug build checks passed" in r.stdout


def test_release_build_has_no_checks():
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    if os.environ.get("SOR_DEBUG_BOUNDS") == "1":
        pytest.skip("this process loads the debug build")
    with capi.Context(0) as ctx:
        assert ctx.diag_bounds() == 0
