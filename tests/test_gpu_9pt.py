"""Parity of the four-colour 9-point CUDA path with the CPU oracle, through
the C ABI (sor_solve9).  Bars: with SOR_FLAG_EXACT_ORDER in FP64, and in
FP32, bit identical to the oracle (same operation order, every operation
rounded on its own), same iteration counts; the FP64 default path (shared
north / south triples, fused multiply-adds) within a normwise relative
difference of 1e-12 after equal iteration counts.  Sizes cover odd and even
n (the four quarters differ in extent), several strips of quarter rows, two
column tiles with a ragged tail (n > 256) and the degenerate grids
n = 1, 2, 3."""
import numpy as np
import pytest

import oracle
from paper_1401_0763_gb300 import workloads as wl
from tests import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
EXACT = 1  # SOR_FLAG_EXACT_ORDER


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


def run9(ctx, u0, f=None, device=True, **kw):
    if device:
        u0t = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        ft = torch.from_numpy(np.ascontiguousarray(f)).cuda() if f is not None else None
        out, res = ctx.solve9(u0t, ft, **kw)
        return out.cpu().numpy(), res
    return ctx.solve9(np.ascontiguousarray(u0), f, **kw)


@pytest.mark.parametrize("n", [1, 2, 3, 16, 37, 100, 129])
@pytest.mark.parametrize("with_f", [False, True])
def test_fp64_bitwise(ctx, n, with_f):
    capi = capi_mod()
    u0 = wl.random_edges(n, 500 + n)
    f = wl.gaussian_source(n, 600 + n) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor9_f64(u0, w, f=f, max_iters=80, check_every=4, tol=1e-9)
    got, res = run9(ctx, u0, f, omega=w, max_iters=80, check_every=4, tol=1e-9, precision=capi.SOR_FP64,
                    flags=EXACT)
    assert res["iterations"] == ref["iterations"]
    assert res["converged"] == ref["converged"]
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    assert res["final_resid_rel"] == ref["final_resid_rel"]


@pytest.mark.parametrize("n", [1, 2, 3, 16, 37, 100, 129, 300])
@pytest.mark.parametrize("with_f", [False, True])
def test_fp64_default_within_tolerance(ctx, n, with_f):
    capi = capi_mod()
    u0 = wl.random_edges(n, 900 + n)
    f = wl.gaussian_source(n, 950 + n) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor9_f64(u0, w, f=f, max_iters=70, check_every=7, tol=0.0)
    got, res = run9(ctx, u0, f, omega=w, max_iters=70, check_every=7, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 70 and not res["converged"]
    assert pins.rel_err(got, ref["u"]) <= TOL64
    ring = np.ones_like(u0, dtype=bool)
    ring[1:-1, 1:-1] = False
    assert np.array_equal(got[ring], u0[ring])
    scale = max(1.0, float(np.max(np.abs(ref["u"]))))
    assert abs(res["final_maxdelta"] - ref["final_maxdelta"]) <= 1e-12 * scale


@pytest.mark.parametrize("omega", [1.0, 0.7, 1.97])
def test_fp64_default_relaxation_factors(ctx, omega):
    capi = capi_mod()
    n = 41
    u0 = wl.random_edges(n, 61)
    f = wl.gaussian_source(n, 62) * 30
    ref = oracle.sor9_f64(u0, omega, f=f, max_iters=150, check_every=1000, tol=0.0)
    got, res = run9(ctx, u0, f, omega=omega, max_iters=150, check_every=1000, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 150
    assert pins.rel_err(got, ref["u"]) <= TOL64


@pytest.mark.parametrize("n", [5, 64, 131])
@pytest.mark.parametrize("with_f", [False, True])
def test_fp32_bitwise(ctx, n, with_f):
    capi = capi_mod()
    u0 = wl.random_edges(n, 700 + n)
    f = wl.gaussian_source(n, 800 + n) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor9_f32(u0, w, f=f, max_iters=60, check_every=5, tol=1e-4)
    got, res = run9(ctx, u0, f, omega=w, max_iters=60, check_every=5, tol=1e-4, precision=capi.SOR_FP32)
    assert res["iterations"] == ref["iterations"]
    assert res["converged"] == ref["converged"]
    assert np.array_equal(got, ref["u"])


@pytest.mark.parametrize("n", [517, 1030])
def test_two_column_tiles_and_more(ctx, n):
    """(n+1)/2 > 256 packed columns: several column tiles, ragged last one."""
    capi = capi_mod()
    u0 = wl.random_edges(n, n)
    w = oracle.omega_opt(n)
    ref = oracle.sor9_f64(u0, w, max_iters=6, check_every=3, tol=0.0)
    got, res = run9(ctx, u0, omega=w, max_iters=6, check_every=3, tol=0.0, precision=capi.SOR_FP64, flags=EXACT)
    assert res["iterations"] == 6
    assert np.array_equal(got, ref["u"])
    got, res = run9(ctx, u0, omega=w, max_iters=6, check_every=3, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 6
    assert pins.rel_err(got, ref["u"]) <= TOL64


def test_residual_stop_matches(ctx):
    capi = capi_mod()
    n = 50
    u0 = wl.random_edges(n, 21)
    f = wl.gaussian_source(n, 22)
    w = oracle.omega_opt(n)
    ref = oracle.sor9_f64(u0, w, f=f, max_iters=5000, check_every=5, tol=1e-10, stop_mode=1)
    got, res = run9(ctx, u0, f, omega=w, max_iters=5000, check_every=5, tol=1e-10, precision=capi.SOR_FP64,
                    stop=capi.SOR_STOP_RESID_REL, flags=EXACT)
    assert ref["converged"] and res["converged"]
    assert res["iterations"] == ref["iterations"]
    assert np.array_equal(got, ref["u"])
    assert res["final_resid_rel"] == ref["final_resid_rel"] < 1e-10
    got, res = run9(ctx, u0, f, omega=w, max_iters=5000, check_every=5, tol=1e-10, precision=capi.SOR_FP64,
                    stop=capi.SOR_STOP_RESID_REL)
    assert res["converged"] and res["iterations"] == ref["iterations"]
    assert pins.rel_err(got, ref["u"]) <= TOL64 and res["final_resid_rel"] < 1e-10


def test_quartic_harmonic_and_dst(ctx):
    """Converged solutions against the closed forms the oracle is pinned to:
    the quartic harmonic the 9-point operator reproduces exactly, and the
    DST-I solution of a Poisson problem."""
    capi = capi_mod()
    n = 96
    u0, exact = pins.grid_from(lambda x, y: x ** 4 - 6.0 * x * x * y * y + y ** 4, n)
    got, res = run9(ctx, u0, max_iters=20000, check_every=10, tol=1e-13, precision=capi.SOR_FP64)
    assert res["converged"]
    assert np.max(np.abs(got - exact)) < 1e-12
    u0 = wl.random_edges(n, 8)
    f = wl.gaussian_source(n, 9)
    got, res = run9(ctx, u0, f, max_iters=20000, check_every=10, tol=1e-11, precision=capi.SOR_FP64)
    assert res["converged"]
    assert pins.rel_err(got, pins.dst_solve9(u0, f)) < 1e-10


@pytest.mark.parametrize("n", [1, 2, 7, 37, 129, 300])
@pytest.mark.parametrize("with_f", [False, True])
def test_refine9_bitwise(ctx, n, with_f):
    """Defect correction with FP32 four-colour inner sweeps, FP64 residual
    and correction: bit identical to the oracle, same correction count."""
    capi = capi_mod()
    u0 = wl.random_edges(n, 1100 + n)
    f = wl.gaussian_source(n, 1200 + n) if with_f else None
    w = oracle.omega_opt(n)
    inner, cap = 6, 6 * 80
    ref = oracle.refine9(u0, w, f=f, inner_sweeps=inner, tol=1e-11, max_outer=cap // inner)
    got, res = run9(ctx, u0, f, omega=w, tol=1e-11, max_iters=cap, inner_sweeps=inner,
                    precision=capi.SOR_FP32_REFINE)
    assert res["outer_steps"] == ref["outer_steps"] and bool(res["converged"]) == ref["converged"]
    assert res["iterations"] == ref["sweeps"]
    assert np.array_equal(got, ref["u"])
    assert res["final_resid_rel"] == ref["final_resid_rel"]


def test_refine9_cap_and_solution(ctx):
    capi = capi_mod()
    n = 90
    u0 = wl.random_edges(n, 31)
    f = wl.gaussian_source(n, 32)
    w = oracle.omega_opt(n)
    ref = oracle.refine9(u0, w, f=f, inner_sweeps=20, tol=1e-30, max_outer=4)
    got, res = run9(ctx, u0, f, omega=w, tol=1e-30, max_iters=99, inner_sweeps=20, precision=capi.SOR_FP32_REFINE)
    assert res["outer_steps"] == 4 and not res["converged"] and res["iterations"] == 80
    assert np.array_equal(got, ref["u"]) and res["final_resid_rel"] == ref["final_resid_rel"]
    got, res = run9(ctx, u0, f, tol=1e-11, max_iters=40000, precision=capi.SOR_FP32_REFINE, device=False)
    assert res["converged"] and res["final_resid_rel"] < 1e-11
    assert pins.rel_err(got, pins.dst_solve9(u0, f)) < 1e-8


def test_stall_window_bitwise_and_default(ctx):
    """A tolerance below the FP64 floor with the stall rule: the exact-order
    path stops where the oracle does; the default path stops on the plateau,
    unconverged, long before the cap."""
    capi = capi_mod()
    n = 24
    u0 = wl.random_edges(n, 93)
    f = wl.gaussian_source(n, 94) * 50
    w = oracle.omega_opt(n)
    kw = dict(omega=w, tol=1e-30, max_iters=4000, check_every=4, stall_window=6)
    ref = oracle.sor9_f64(u0, w, f=f, stop_mode=1, **{k: v for k, v in kw.items() if k != "omega"})
    assert not ref["converged"] and ref["iterations"] < 4000
    got, res = run9(ctx, u0, f, precision=capi.SOR_FP64, stop=capi.SOR_STOP_RESID_REL, flags=EXACT, **kw)
    assert res["iterations"] == ref["iterations"] and not res["converged"]
    assert np.array_equal(got, ref["u"]) and res["final_resid_rel"] == ref["final_resid_rel"]
    got, res = run9(ctx, u0, f, precision=capi.SOR_FP64, stop=capi.SOR_STOP_RESID_REL, **kw)
    assert not res["converged"] and res["iterations"] < 4000
    assert res["final_resid_rel"] < 100 * ref["final_resid_rel"]


def test_host_and_device_pointers_agree(ctx):
    capi = capi_mod()
    n = 45
    u0 = wl.random_edges(n, 3)
    a, ra = run9(ctx, u0, device=True, max_iters=25, tol=0.0, precision=capi.SOR_FP64)
    b, rb = run9(ctx, u0, device=False, max_iters=25, tol=0.0, precision=capi.SOR_FP64)
    assert np.array_equal(a, b) and ra["iterations"] == rb["iterations"] == 25


def test_full_size_plate_bitwise(ctx):
    """4096^2 interior, 10 iterations: the whole plate against the oracle."""
    capi = capi_mod()
    n = 4096
    u0 = wl.random_edges(n, 0)
    w = oracle.omega_opt(n)
    ref = oracle.sor9_f64(u0, w, max_iters=10, check_every=5, tol=0.0)
    got, res = run9(ctx, u0, omega=w, max_iters=10, check_every=5, tol=0.0, precision=capi.SOR_FP64, flags=EXACT)
    assert res["iterations"] == 10
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    got, res = run9(ctx, u0, omega=w, max_iters=10, check_every=5, tol=0.0, precision=capi.SOR_FP64)
    assert res["iterations"] == 10
    assert pins.rel_err(got, ref["u"]) <= TOL64


def test_invalid_arguments(ctx):
    capi = capi_mod()
    u0 = wl.random_edges(6, 1)
    for kw in (dict(precision=7), dict(stall_window=-2), dict(omega=2.0), dict(check_every=0), dict(flags=4),
               dict(precision=capi.SOR_FP32_REFINE, inner_sweeps=-1)):
        p = capi.make_params(6, **kw)
        out = np.empty_like(u0)
        st, _ = ctx.solve9_raw(p, u0.ctypes.data, None, out.ctypes.data)
        assert st == capi.SOR_ERR_INVALID_ARG, kw


def test_refine9_stall_window_bitwise(ctx):
    """The defect correction with the stall rule below the FP64 floor: the
    same correction count and bits as the oracle, unconverged."""
    capi = capi_mod()
    n = 20
    u0 = wl.random_edges(n, 73)
    f = wl.gaussian_source(n, 74) * 50
    w = oracle.omega_opt(n)
    ref = oracle.refine9(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=400, stall_window=5)
    assert not ref["converged"] and ref["outer_steps"] < 400
    got, res = run9(ctx, u0, f, omega=w, tol=1e-30, max_iters=1200, inner_sweeps=3, stall_window=5,
                    precision=capi.SOR_FP32_REFINE)
    assert res["outer_steps"] == ref["outer_steps"] and not res["converged"]
    assert np.array_equal(got, ref["u"]) and res["final_resid_rel"] == ref["final_resid_rel"]
