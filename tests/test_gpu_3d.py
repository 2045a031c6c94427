"""Parity of the 3D (cube, 7-point) CUDA path with the CPU oracle, through
the C ABI (sor_solve3d).  Bars: with SOR_FLAG_EXACT_ORDER in FP64, and in
FP32, bit identical to the oracle (same operation order, every operation
rounded on its own), same iteration counts; the FP64 default path (rescaled
unknowns, shared pair sums) within a normwise relative difference of 1e-12
after equal iteration counts.  Sizes span several 32 x 128 tiles per plane,
ragged tails, two column tiles (n > 256), ragged warp strips, chunks cut by
the scale cap, and the degenerate cubes n = 1, 2."""
import numpy as np
import pytest

import oracle
from paper_1401_0763_gb300 import workloads as wl
from tests import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


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


def shell_of(a):
    """The 6 faces of a cube (the Dirichlet values), interior zeroed."""
    b = np.array(a, copy=True)
    b[1:-1, 1:-1, 1:-1] = 0.0
    return b


def run3(ctx, u0, f=None, device=True, **kw):
    if device:
        u0t = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        ft = torch.from_numpy(np.ascontiguousarray(f)).cuda() if f is not None else None
        out, res = ctx.solve3d(u0t, ft, **kw)
        return out.cpu().numpy(), res
    return ctx.solve3d(np.ascontiguousarray(u0), f, **kw)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 40, 65])
@pytest.mark.parametrize("with_f", [False, True])
def test_fp64_bitwise(ctx, n, with_f):
    capi = capi_mod()
    u0 = wl.random_shell(n, 100 + n)
    f = wl.gaussian_source3(n, 200 + n) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f64(u0, w, f=f, max_iters=60, check_every=5, tol=1e-9)
    got, res = run3(ctx, u0, f, omega=w, max_iters=60, check_every=5, tol=1e-9, precision=capi.SOR_FP64,
                    flags=capi.SOR_FLAG_EXACT_ORDER)
    assert res["iterations"] == ref["iterations"]
    assert res["converged"] == ref["converged"]
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    assert res["final_resid_rel"] == ref["final_resid_rel"]


@pytest.mark.parametrize("n", [3, 33, 64])
@pytest.mark.parametrize("with_f", [False, True])
def test_fp32_bitwise(ctx, n, with_f):
    capi = capi_mod()
    u0 = wl.random_shell(n, 300 + n)
    f = wl.gaussian_source3(n, 400 + n) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f32(u0, w, f=f, max_iters=50, check_every=10, tol=1e-4)
    got, res = run3(ctx, u0, f, omega=w, max_iters=50, check_every=10, tol=1e-4, precision=capi.SOR_FP32)
    assert res["iterations"] == ref["iterations"]
    assert res["converged"] == ref["converged"]
    assert np.array_equal(got, ref["u"])


def test_two_column_tiles_ragged(ctx):
    """n = 259: 130 packed columns (two column tiles, the second ragged) and
    a ragged last row tile in every plane."""
    capi = capi_mod()
    n = 259
    u0 = wl.random_shell(n, 7)
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f64(u0, w, max_iters=3, check_every=1, tol=0.0)
    got, res = run3(ctx, u0, omega=w, max_iters=3, check_every=1, tol=0.0, precision=capi.SOR_FP64,
                    flags=capi.SOR_FLAG_EXACT_ORDER)
    assert res["iterations"] == 3
    assert np.array_equal(got, ref["u"])
    got, res = run3(ctx, u0, omega=w, max_iters=3, check_every=1, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 3
    assert pins.rel_err3(got, ref["u"]) <= TOL64


def test_three_column_tiles_large_cube(ctx):
    """n = 513: 257 packed columns per row (three column tiles, the last one
    ragged), 16 row bands per plane; exact order bitwise and the
    default path within 1e-12 after 4 iterations (change measured at 2, 4)."""
    capi = capi_mod()
    n = 513
    u0 = wl.random_shell(n, 17)
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f64(u0, w, max_iters=4, check_every=2, tol=0.0)
    got, res = run3(ctx, u0, omega=w, max_iters=4, check_every=2, tol=0.0, precision=capi.SOR_FP64,
                    flags=capi.SOR_FLAG_EXACT_ORDER)
    assert res["iterations"] == 4 and np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    got, res = run3(ctx, u0, omega=w, max_iters=4, check_every=2, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 4 and pins.rel_err3(got, ref["u"]) <= TOL64


def test_residual_stop_matches(ctx):
    capi = capi_mod()
    n = 24
    u0 = wl.random_shell(n, 11)
    f = wl.gaussian_source3(n, 12)
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f64(u0, w, f=f, max_iters=2000, check_every=4, tol=1e-10, stop_mode=1)
    got, res = run3(ctx, u0, f, omega=w, max_iters=2000, check_every=4, tol=1e-10, precision=capi.SOR_FP64,
                    stop=capi.SOR_STOP_RESID_REL, flags=capi.SOR_FLAG_EXACT_ORDER)
    assert ref["converged"] and res["converged"]
    assert res["iterations"] == ref["iterations"]
    assert np.array_equal(got, ref["u"])
    assert res["final_resid_rel"] == ref["final_resid_rel"] < 1e-10
    got, res = run3(ctx, u0, f, omega=w, max_iters=2000, check_every=4, tol=1e-10, precision=capi.SOR_FP64,
                    stop=capi.SOR_STOP_RESID_REL)
    assert res["converged"] and res["iterations"] == ref["iterations"]
    assert pins.rel_err3(got, ref["u"]) <= TOL64
    assert res["final_resid_rel"] < 1e-10


def test_harmonic_quadratic_and_dst(ctx):
    """Converged cube against closed forms the oracle is pinned to."""
    capi = capi_mod()
    n = 48
    u0, exact = pins.cube_from(lambda x, y, z: x * x + y * y - 2.0 * z * z, n)
    got, res = run3(ctx, u0, max_iters=5000, check_every=10, tol=1e-14, precision=capi.SOR_FP64)
    assert res["converged"]
    assert np.max(np.abs(got - exact)) < 1e-11
    u0 = wl.random_shell(n, 5)
    f = wl.gaussian_source3(n, 6)
    got, res = run3(ctx, u0, f, max_iters=5000, check_every=10, tol=1e-11, precision=capi.SOR_FP64)
    assert res["converged"]
    assert pins.rel_err3(got, pins.dst_solve3(u0, f)) < 1e-11


def test_host_and_device_pointers_agree(ctx):
    capi = capi_mod()
    n = 20
    u0 = wl.random_shell(n, 3)
    a, ra = run3(ctx, u0, device=True, max_iters=30, tol=0.0, precision=capi.SOR_FP64)
    b, rb = run3(ctx, u0, device=False, max_iters=30, tol=0.0, precision=capi.SOR_FP64)
    assert np.array_equal(a, b) and ra["iterations"] == rb["iterations"] == 30


def test_full_size_cube_bitwise(ctx):
    """256^3 interior (258^3 array, the benchmark cube), 20 iterations with
    the change measured every 10: the whole cube against the oracle."""
    capi = capi_mod()
    n = 256
    u0 = wl.random_shell(n, 0)
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f64(u0, w, max_iters=20, check_every=10, tol=0.0)
    got, res = run3(ctx, u0, omega=w, max_iters=20, check_every=10, tol=0.0, precision=capi.SOR_FP64,
                    flags=capi.SOR_FLAG_EXACT_ORDER)
    assert res["iterations"] == 20
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    got, res = run3(ctx, u0, omega=w, max_iters=20, check_every=10, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 20
    assert pins.rel_err3(got, ref["u"]) <= TOL64
    assert abs(res["final_maxdelta"] - ref["final_maxdelta"]) <= 1e-10 * ref["final_maxdelta"]


@pytest.mark.parametrize("n", [1, 2, 5, 17, 40, 65, 130])
@pytest.mark.parametrize("with_f", [False, True])
def test_fp64_default_within_tolerance(ctx, n, with_f):
    """The default FP64 path: chunks of 5 rescaled iterations ending at the
    tested iterations, every strip of a plane ragged for n = 65, 130."""
    capi = capi_mod()
    u0 = wl.random_shell(n, 500 + n)
    f = wl.gaussian_source3(n, 600 + n) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f64(u0, w, f=f, max_iters=60, check_every=5, tol=0.0)
    got, res = run3(ctx, u0, f, omega=w, max_iters=60, check_every=5, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 60 and not res["converged"]
    assert pins.rel_err3(got, ref["u"]) <= TOL64
    assert np.array_equal(shell_of(got), shell_of(u0))  # shell back at scale 1 after every chunk
    scale = max(1.0, float(np.max(np.abs(ref["u"]))))
    assert abs(res["final_maxdelta"] - ref["final_maxdelta"]) <= 1e-12 * scale


@pytest.mark.parametrize("omega", [1.0, 0.6, 1.95])
def test_fp64_default_chunks_cut_by_scale_cap(ctx, omega):
    """Tests every 500 iterations, so the chunk length is set by the cap on
    the carried scale (w/6)^-2L (120 iterations at w = 1.95) and by the
    iteration cap; w = 1 drops the (1 - w) term, w < 1 under-relaxes."""
    capi = capi_mod()
    n = 19
    u0 = wl.random_shell(n, 31)
    f = wl.gaussian_source3(n, 32)
    ref = oracle.sor3d_f64(u0, omega, f=f, max_iters=300, check_every=500, tol=0.0)
    got, res = run3(ctx, u0, f, omega=omega, max_iters=300, check_every=500, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 300
    assert pins.rel_err3(got, ref["u"]) <= TOL64
    assert np.array_equal(shell_of(got), shell_of(u0))


def test_fp64_default_stops_like_oracle(ctx):
    """Max-change stop: the default path takes the oracle's iteration count
    (the tested changes sit far from the tolerance) and converges to the
    closed-form harmonic cube."""
    capi = capi_mod()
    n = 33
    u0 = wl.random_shell(n, 77)
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f64(u0, w, max_iters=3000, check_every=7, tol=1e-9)
    got, res = run3(ctx, u0, omega=w, max_iters=3000, check_every=7, tol=1e-9, precision=capi.SOR_FP64)
    assert ref["converged"] and res["converged"]
    assert res["iterations"] == ref["iterations"]
    assert pins.rel_err3(got, ref["u"]) <= TOL64
    u0, exact = pins.cube_from(lambda x, y, z: x * y + 2.0 * y * z - z * x + 3.0 * x, 40)
    got, res = run3(ctx, u0, max_iters=5000, check_every=10, tol=1e-14, precision=capi.SOR_FP64)
    assert res["converged"]
    assert np.max(np.abs(got - exact)) < 1e-11


@pytest.mark.parametrize("n", [1, 3, 12, 33, 65])
@pytest.mark.parametrize("with_f", [False, True])
def test_refine3d_bitwise(ctx, n, with_f):
    """Defect correction on a cube (FP32 inner sweeps, FP64 residual and
    correction): bit identical to the oracle, same correction count."""
    capi = capi_mod()
    u0 = wl.random_shell(n, 700 + n)
    f = wl.gaussian_source3(n, 800 + n) if with_f else None
    w = oracle.omega_opt(n)
    inner, cap = 7, 7 * 60
    ref = oracle.refine3d(u0, w, f=f, inner_sweeps=inner, tol=1e-11, max_outer=cap // inner)
    got, res = run3(ctx, u0, f, omega=w, tol=1e-11, max_iters=cap, inner_sweeps=inner,
                    precision=capi.SOR_FP32_REFINE)
    assert res["outer_steps"] == ref["outer_steps"] and bool(res["converged"]) == ref["converged"]
    assert res["iterations"] == ref["sweeps"]
    assert np.array_equal(got, ref["u"])
    assert res["final_resid_rel"] == ref["final_resid_rel"]


def test_refine3d_cap_and_solution(ctx):
    """The correction cap (max_iters / inner_sweeps) and a converged solve
    against the DST-I solution the oracle is pinned to."""
    capi = capi_mod()
    n = 40
    u0 = wl.random_shell(n, 21)
    f = wl.gaussian_source3(n, 22)
    w = oracle.omega_opt(n)
    ref = oracle.refine3d(u0, w, f=f, inner_sweeps=20, tol=1e-30, max_outer=3)
    got, res = run3(ctx, u0, f, omega=w, tol=1e-30, max_iters=69, inner_sweeps=20, precision=capi.SOR_FP32_REFINE)
    assert res["outer_steps"] == 3 and not res["converged"] and res["iterations"] == 60
    assert np.array_equal(got, ref["u"]) and res["final_resid_rel"] == ref["final_resid_rel"]
    got, res = run3(ctx, u0, f, tol=1e-11, max_iters=20000, precision=capi.SOR_FP32_REFINE, device=False)
    assert res["converged"] and res["final_resid_rel"] < 1e-11
    assert pins.rel_err3(got, pins.dst_solve3(u0, f)) < 1e-9


def test_stall_window_bitwise_and_default(ctx):
    """A tolerance below the FP64 floor with the stall rule: the exact-order
    path stops where the oracle does (same test, same bits); the default path
    also stops on the plateau, unconverged, long before the cap."""
    capi = capi_mod()
    n = 10
    u0 = wl.random_shell(n, 91)
    f = wl.gaussian_source3(n, 92) * 50
    w = oracle.omega_opt(n)
    kw = dict(omega=w, tol=1e-30, max_iters=3000, check_every=5, stall_window=6)
    ref = oracle.sor3d_f64(u0, w, f=f, stop_mode=1, **{k: v for k, v in kw.items() if k != "omega"})
    assert not ref["converged"] and ref["iterations"] < 3000
    got, res = run3(ctx, u0, f, precision=capi.SOR_FP64, stop=capi.SOR_STOP_RESID_REL,
                    flags=capi.SOR_FLAG_EXACT_ORDER, **kw)
    assert res["iterations"] == ref["iterations"] and not res["converged"]
    assert np.array_equal(got, ref["u"]) and res["final_resid_rel"] == ref["final_resid_rel"]
    got, res = run3(ctx, u0, f, precision=capi.SOR_FP64, stop=capi.SOR_STOP_RESID_REL, **kw)
    assert not res["converged"] and res["iterations"] < 3000
    assert res["final_resid_rel"] < 100 * ref["final_resid_rel"]


def test_bounded_wait_gives_up_and_context_survives(ctx):
    """The failure path of the data-flow kernels without a fault: their
    bounded device-side wait, run on a progress counter nothing advances,
    gives up and reports it; on a completed counter it does not; and the
    context solves normally afterwards."""
    capi = capi_mod()
    import time
    t0 = time.perf_counter()
    assert ctx.diag_flow_wait(4000, 0) == 1
    assert time.perf_counter() - t0 < 5.0
    assert ctx.diag_flow_wait(4000, 1) == 0
    for polls, preset in ((0, 0), (1 << 22, 0), (10, 2)):
        with pytest.raises(capi.SorError):
            ctx.diag_flow_wait(polls, preset)
    n = 12
    u0 = wl.random_shell(n, 4)
    ref = oracle.sor3d_f64(u0, oracle.omega_opt(n), max_iters=30, check_every=10, tol=0.0)
    got, res = run3(ctx, u0, omega=oracle.omega_opt(n), max_iters=30, check_every=10, tol=0.0,
                    precision=capi.SOR_FP64)
    assert res["iterations"] == 30 and pins.rel_err3(got, ref["u"]) <= TOL64


def test_invalid_arguments(ctx):
    capi = capi_mod()
    u0 = wl.random_shell(4, 1)
    for kw in (dict(precision=7), dict(stall_window=-1), dict(omega=2.5), dict(check_every=0), dict(flags=8),
               dict(precision=capi.SOR_FP32_REFINE, inner_sweeps=-1)):
        p = capi.make_params(4, **kw)
        out = np.empty_like(u0)
        st, _ = ctx.solve3d_raw(p, u0.ctypes.data, None, out.ctypes.data)
        assert st == capi.SOR_ERR_INVALID_ARG, kw
    p = capi.make_params(0)
    st, _ = ctx.solve3d_raw(p, u0.ctypes.data, None, u0.ctypes.data)
    assert st == capi.SOR_ERR_INVALID_ARG


def test_refine3d_stall_window_bitwise(ctx):
    """The defect correction with the stall rule below the FP64 floor: the
    same correction count and bits as the oracle, unconverged."""
    capi = capi_mod()
    n = 8
    u0 = wl.random_shell(n, 71)
    f = wl.gaussian_source3(n, 72) * 50
    w = oracle.omega_opt(n)
    ref = oracle.refine3d(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=400, stall_window=5)
    assert not ref["converged"] and ref["outer_steps"] < 400
    got, res = run3(ctx, u0, f, omega=w, tol=1e-30, max_iters=1200, inner_sweeps=3, stall_window=5,
                    precision=capi.SOR_FP32_REFINE)
    assert res["outer_steps"] == ref["outer_steps"] and not res["converged"]
    assert np.array_equal(got, ref["u"]) and res["final_resid_rel"] == ref["final_resid_rel"]


@pytest.mark.parametrize("budget_mb", [0, 200])
def test_cube_requests_in_the_batch_scheduler(budget_mb):
    """Cube requests through sor_batch_submit3d, mixed with plates: cubes run
    whole on worker streams beside the scheduler's plate steps; each result
    equals the lone sor_solve3d (sor_solve for the plates) bit for bit.  A
    200 MB budget makes cube requests wait for each other's memory."""
    capi = capi_mod()
    cubes = [
        (30, None, dict(precision=capi.SOR_FP64, tol=1e-9, max_iters=400, check_every=5)),
        (41, None, dict(precision=capi.SOR_FP64, tol=1e-9, max_iters=300, check_every=7,
                        flags=capi.SOR_FLAG_EXACT_ORDER)),
        (25, None, dict(precision=capi.SOR_FP32, tol=1e-4, max_iters=200, check_every=10)),
        (33, True, dict(precision=capi.SOR_FP32_REFINE, tol=1e-10, max_iters=20000)),
        (19, True, dict(precision=capi.SOR_FP64, tol=1e-8, max_iters=2000, check_every=4,
                        stop=capi.SOR_STOP_RESID_REL)),
    ]
    jobs = []
    for k, (n, with_f, kw) in enumerate(cubes):
        u0 = wl.random_shell(n, 500 + k)
        f = wl.gaussian_source3(n, 600 + k) if with_f else None
        jobs.append((u0, f, dict(kw, omega=oracle.omega_opt(n))))
    plates = []
    for k, n in enumerate((70, 130)):
        u0, f = wl.poisson_problem(n, 700 + k)
        plates.append((u0, f, dict(precision=capi.SOR_FP32_REFINE, omega=oracle.omega_opt(n), tol=1e-9,
                                   max_iters=50000)))
    with capi.Context(0) as solo:
        alone = [solo.solve3d(u0, f, **kw) for u0, f, kw in jobs]
        alone_p = [solo.solve(u0, f, **kw) for u0, f, kw in plates]
    with capi.Context(0, budget_bytes=budget_mb << 20) as ctx:
        t3 = [ctx.submit3d(u0, f, **kw) for u0, f, kw in jobs]
        t2 = [ctx.submit(u0, f, **kw) for u0, f, kw in plates]
        for (t, out), (ref, rres) in zip(t3, alone):
            st, res = ctx.wait(t, 300.0)
            assert st == capi.SOR_OK, ctx.last_error()
            assert res["iterations"] == rres["iterations"] and res["converged"] == rres["converged"]
            assert np.array_equal(out, ref)
        for (t, out), (ref, rres) in zip(t2, alone_p):
            st, res = ctx.wait(t, 300.0)
            assert st == capi.SOR_OK, ctx.last_error()
            assert np.array_equal(out, ref)
        assert ctx.stats()["batch_completed"] == len(jobs) + len(plates)
        if budget_mb:
            assert ctx.stats()["bytes_peak"] <= budget_mb << 20


def test_cube_requests_cancelled_by_destroy():
    """Closing the context with cube requests queued and running returns
    promptly (running solves stop at their next chunk) and the device stays
    usable."""
    capi = capi_mod()
    ctx = capi.Context(0)
    n = 200
    u0 = wl.random_shell(n, 1)
    for _ in range(6):
        ctx.submit3d(u0, precision=capi.SOR_FP64, tol=0.0, max_iters=100000, check_every=50)
    ctx.close()
    with capi.Context(0) as again:
        out, res = again.solve3d(wl.random_shell(10, 2), tol=1e-8, max_iters=500)
        assert res["converged"]


@pytest.mark.parametrize("depth", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 5, 17, 40, 65, 100])
@pytest.mark.parametrize("with_f", [False, True])
def test_fp32_blocked_sweeps_bitwise(depth, n, with_f):
    """FP32 cube sweeps with SOR_OPT_CUBE_DEPTH iterations fused per launch
    (each tile streamed through its planes, the phases a wavefront in shared
    memory, output to the other buffer pair) or one data-flow launch per run
    of iterations (depth 0): equal to the oracle bit for bit at every depth,
    on ragged sizes, for runs to the cap that end in a launch shorter than the
    depth (K = 7, 23 iterations) and for early stops (K = 3)."""
    capi = capi_mod()
    u0 = wl.random_shell(n, 900 + n)
    f = wl.gaussian_source3(n, 950 + n) * 5 if with_f else None
    w = oracle.omega_opt(n)
    with capi.Context(0) as c:
        c.set_option(capi.SOR_OPT_CUBE_DEPTH, depth)
        ref = oracle.sor3d_f32(u0, w, f=f, max_iters=23, check_every=7, tol=-1.0)
        got, res = run3(c, u0, f, omega=w, max_iters=23, check_every=7, tol=-1.0, precision=capi.SOR_FP32)
        assert res["iterations"] == 23 and not res["converged"]
        assert np.array_equal(got, ref["u"])
        assert res["final_maxdelta"] == ref["final_maxdelta"]
        ref = oracle.sor3d_f32(u0, w, f=f, max_iters=3000, check_every=3, tol=2e-2)
        got, res = run3(c, u0, f, omega=w, max_iters=3000, check_every=3, tol=2e-2, precision=capi.SOR_FP32)
        assert res["iterations"] == ref["iterations"] and res["converged"] == ref["converged"]
        assert np.array_equal(got, ref["u"])
        assert res["final_maxdelta"] == ref["final_maxdelta"]


def test_fp32_blocked_sweeps_large_cube():
    """A cube of several tiles in every direction, host and device buffers."""
    capi = capi_mod()
    n = 210
    u0 = wl.random_shell(n, 77)
    f = wl.gaussian_source3(n, 78) * 3
    w = oracle.omega_opt(n)
    ref = oracle.sor3d_f32(u0, w, f=f, max_iters=9, check_every=4, tol=-1.0)
    with capi.Context(0) as c:
        for depth in (1, 2):
            c.set_option(capi.SOR_OPT_CUBE_DEPTH, depth)
            for device in (True, False):
                got, res = run3(c, u0, f, device=device, omega=w, max_iters=9, check_every=4, tol=-1.0,
                                precision=capi.SOR_FP32)
                assert res["iterations"] == 9
                assert np.array_equal(got, ref["u"]), (depth, device)
                assert res["final_maxdelta"] == ref["final_maxdelta"]
