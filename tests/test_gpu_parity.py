"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars:
* FP64 with SOR_FLAG_EXACT_ORDER, FP32 sweeps and FP32-refinement: bit
  identical to the oracle (same operation order, every operation rounded on
  its own on both sides), same iteration / correction counts.
* FP64 default path: normwise relative difference <= 1e-12 after equal
  iteration counts.
Sizes span several 32 x 128 tiles plus ragged tails and the degenerate
grids n = 1, 2, 3.
"""
import numpy as np
import pytest

import oracle
from paper_1401_0763_gb300 import workloads as wl
from tests import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def ctxs():
    """Four contexts: the default one (small plain plates solved in one
    launch on a cooperative grid of many SMs, with point-to-point exchanges
    between bands and the stop test decided behind the sweeps; in one
    thread-block cluster when the stop test is the residual), one whose grid
    takes a grid-wide barrier per colour phase instead, one that always takes
    the cluster, and one with the one-launch paths switched off, so the
    chunked multi-CTA kernels are exercised at every size."""
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    made = {"grid": capi.Context(0), "gridbar": capi.Context(0), "cluster": capi.Context(0),
            "multi": capi.Context(0)}
    made["gridbar"].set_option(capi.SOR_OPT_CLUSTER, 3)
    made["cluster"].set_option(capi.SOR_OPT_CLUSTER, 2)
    made["multi"].set_option(capi.SOR_OPT_CLUSTER, 0)
    yield made
    for c in made.values():
        c.close()


@pytest.fixture(scope="module")
def ctx(ctxs):
    return ctxs["grid"]


@pytest.fixture(scope="module")
def ctx_mc(ctxs):
    return ctxs["multi"]


PATHS = ["grid", "gridbar", "cluster", "multi"]


def capi_mod():
    from paper_1401_0763_gb300 import capi
    return capi


def run(ctx, u0, f=None, device=True, **kw):
    if device:
        u0t = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        ft = torch.from_numpy(np.ascontiguousarray(f)).cuda() if f is not None else None
        out, res = ctx.solve(u0t, ft, **kw)
        torch.cuda.synchronize()
        return out.cpu().numpy(), res
    return ctx.solve(np.ascontiguousarray(u0), None if f is None else np.ascontiguousarray(f), **kw)


SIZES = [1, 2, 3, 5, 31, 64, 127, 128, 129, 255, 256, 257, 300]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("path", PATHS)
def test_fp64_exact_bitwise(ctxs, path, n):
    ctx = ctxs[path]
    capi = capi_mod()
    u0 = wl.random_edges(n, n)
    f = wl.gaussian_source(n, n + 1) * 50 if n % 2 else None
    w = oracle.omega_opt(n)
    iters = 37
    ref = oracle.sor_f64(u0, w, f=f, max_iters=iters, check_every=5, tol=-1.0)
    got, res = run(ctx, u0, f, omega=w, tol=-1.0, max_iters=iters, check_every=5,
                   flags=capi.SOR_FLAG_EXACT_ORDER)
    assert res["iterations"] == iters and not res["converged"]
    assert np.array_equal(got, ref["u"]), pins.rel_err(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    assert res["final_resid_rel"] == ref["final_resid_rel"]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("path", PATHS)
def test_fp64_default_within_tolerance(ctxs, path, n):
    ctx = ctxs[path]
    u0 = wl.random_edges(n, 2 * n)
    f = wl.gaussian_source(n, n) * 20 if n % 3 == 0 else None
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, f=f, max_iters=60, check_every=1, tol=-1.0)
    got, res = run(ctx, u0, f, omega=w, tol=-1.0, max_iters=60, check_every=1)
    assert res["iterations"] == 60
    assert pins.rel_err(got, ref["u"]) <= TOL64


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("path", PATHS)
def test_fp32_bitwise(ctxs, path, n):
    ctx = ctxs[path]
    capi = capi_mod()
    u0 = wl.random_edges(n, 3 * n)
    f = wl.gaussian_source(n, n) * 30 if n % 2 == 0 else None
    w = oracle.omega_opt(n)
    ref = oracle.sor_f32(u0, w, f=f, max_iters=41, check_every=4, tol=-1.0)
    got, res = run(ctx, u0, f, precision=capi.SOR_FP32, omega=w, tol=-1.0, max_iters=41, check_every=4)
    assert res["iterations"] == 41
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]


def test_config1_heat_plate_converges_like_oracle(ctx):
    """258 x 258 plate, top edge 100, w_opt, stop on max|change| < 1e-8 (K = 1)."""
    capi = capi_mod()
    n = 256
    u0 = wl.heat_plate(n, 100.0)
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, max_iters=5000, check_every=1, tol=1e-8)
    assert ref["converged"]
    got, res = run(ctx, u0, omega=w, tol=1e-8, max_iters=5000, check_every=1, flags=capi.SOR_FLAG_EXACT_ORDER)
    assert res["converged"] and res["iterations"] == ref["iterations"]
    assert np.array_equal(got, ref["u"])
    got2, res2 = run(ctx, u0, omega=w, tol=1e-8, max_iters=5000, check_every=1)
    assert res2["converged"] and abs(res2["iterations"] - ref["iterations"]) <= 1
    from paper_1401_0763_gb300 import capi as _c
    with _c.Context(0) as mc:  # the multi-CTA rescaled path on the same plate
        mc.set_option(_c.SOR_OPT_CLUSTER, 0)
        got3, res3 = run(mc, u0, omega=w, tol=1e-8, max_iters=5000, check_every=1)
    assert res3["converged"] and abs(res3["iterations"] - ref["iterations"]) <= 1
    assert pins.rel_err(got3, ref["u"]) <= TOL64 * 10
    assert pins.rel_err(got2, ref["u"]) <= TOL64 * 10


def test_config1_harmonic_case(ctx):
    n = 256
    u0 = wl.harmonic_xx_minus_yy(n)
    w = oracle.omega_opt(n)
    got, res = run(ctx, u0, omega=w, tol=1e-13, max_iters=20000, check_every=1)
    assert res["converged"]
    c = np.arange(n + 2) / (n + 1)
    exact = c[None, :] ** 2 - c[:, None] ** 2
    assert np.max(np.abs(got - exact)) < 1e-11


@pytest.mark.parametrize("K", [1, 7, 50])
@pytest.mark.parametrize("path", PATHS)
def test_check_interval_and_resid_stop(ctxs, path, K):
    ctx = ctxs[path]
    capi = capi_mod()
    n = 100
    u0 = wl.random_edges(n, 5)
    f = wl.gaussian_source(n, 6)
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, f=f, max_iters=3000, check_every=K, tol=1e-7)
    got, res = run(ctx, u0, f, omega=w, tol=1e-7, max_iters=3000, check_every=K, flags=capi.SOR_FLAG_EXACT_ORDER)
    assert res["iterations"] == ref["iterations"] and res["converged"] == ref["converged"]
    assert np.array_equal(got, ref["u"])
    ref = oracle.sor_f64(u0, w, f=f, max_iters=3000, check_every=K, tol=1e-9, stop_mode=1)
    got, res = run(ctx, u0, f, omega=w, tol=1e-9, max_iters=3000, check_every=K, stop=capi.SOR_STOP_RESID_REL,
                   flags=capi.SOR_FLAG_EXACT_ORDER)
    assert res["iterations"] == ref["iterations"] and res["converged"] and ref["converged"]
    assert res["final_resid_rel"] == ref["final_resid_rel"]
    assert np.array_equal(got, ref["u"])


@pytest.mark.parametrize("n,inner", [(1, 3), (2, 20), (63, 20), (130, 7), (256, 20)])
def test_refine_bitwise(ctx, n, inner):
    capi = capi_mod()
    u0, f = wl.poisson_problem(n, n)
    u0 = u0 + wl.random_edges(n, n + 7)
    w = oracle.omega_opt(n)
    ref = oracle.refine(u0, w, f=f, inner_sweeps=inner, tol=1e-10, max_outer=4000 // inner)
    got, res = run(ctx, u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-10, max_iters=4000,
                   inner_sweeps=inner)
    assert res["outer_steps"] == ref["outer_steps"] and bool(res["converged"]) == ref["converged"]
    assert res["iterations"] == ref["sweeps"]
    assert res["final_resid_rel"] == ref["final_resid_rel"]
    assert np.array_equal(got, ref["u"])


def test_refine_cap_and_zero_iterations(ctx):
    capi = capi_mod()
    n = 40
    u0, f = wl.poisson_problem(n, 1)
    w = oracle.omega_opt(n)
    ref = oracle.refine(u0, w, f=f, inner_sweeps=20, tol=1e-14, max_outer=3)
    got, res = run(ctx, u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-14, max_iters=60,
                   inner_sweeps=20)
    assert res["outer_steps"] == 3 and not res["converged"] and not ref["converged"]
    assert np.array_equal(got, ref["u"])
    # zero iterations: the input comes back, residual of the input reported
    got, res = run(ctx, u0, f, omega=w, tol=1e-8, max_iters=0)
    assert res["iterations"] == 0 and np.array_equal(got, u0)
    assert res["final_resid_rel"] == oracle.resid_rel(u0, f=f)


def test_host_and_device_pointers_agree(ctx):
    n = 77
    u0 = wl.random_edges(n, 9)
    a, ra = run(ctx, u0, device=True, tol=-1.0, max_iters=30)
    b, rb = run(ctx, u0, device=False, tol=-1.0, max_iters=30)
    assert np.array_equal(a, b) and ra["iterations"] == rb["iterations"]


def test_invalid_arguments(ctx):
    capi = capi_mod()
    u0 = wl.heat_plate(8, 1.0)
    for kw in ({"omega": 2.0}, {"omega": 2.5}, {"max_iters": -1}, {"check_every": 0}, {"precision": 7},
               {"stop": 3}, {"flags": 8}, {"tol": float("nan")}, {"stall_window": -1}):
        with pytest.raises(capi.SorError) as e:
            ctx.solve(u0, **kw)
        assert e.value.status == capi.SOR_ERR_INVALID_ARG


def test_fp64_full_size_sampled(ctx):
    """4098 x 4098 with random edges (the bandwidth workload), in the launch
    configuration the benchmark times: 100 iterations compared everywhere
    with the oracle."""
    n = 4096
    u0 = wl.random_edges(n, 0)
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, max_iters=100, check_every=50, tol=-1.0)
    got, res = run(ctx, u0, omega=w, tol=-1.0, max_iters=100, check_every=50)
    assert res["iterations"] == 100
    assert pins.rel_err(got, ref["u"]) <= TOL64
    assert res["final_maxdelta"] == pytest.approx(ref["final_maxdelta"], rel=1e-9)


def test_fp64_long_strips(ctx):
    """8194^2 with a source: 32 column tiles, so the strips are about 144 rows
    long and the strip-edge pairs are formed in several groups of 32 rows;
    everything compared with the oracle after 20 iterations."""
    n = 8192
    u0 = wl.random_edges(n, 3)
    f = wl.gaussian_source(n, 4) * 10
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, f=f, max_iters=20, check_every=10, tol=-1.0)
    got, res = run(ctx, u0, f, omega=w, tol=-1.0, max_iters=20, check_every=10)
    assert res["iterations"] == 20
    assert pins.rel_err(got, ref["u"]) <= TOL64


@pytest.mark.parametrize("n,omega,K,iters,with_f", [
    (256, None, 1, 40, False),     # chunk of one iteration: every phase unscaled
    (256, None, 50, 1000, False),  # the benchmark's check interval
    (200, None, 7, 123, True),     # cap not a multiple of K, Poisson source
    (300, 0.376, 4000, 700, False),  # the paper's under-relaxation: shorter chunks (scale growth)
    (129, 1.0, 3, 90, True),       # Gauss-Seidel: alpha = 0
    (5, 1.9, 2, 31, True),
])
def test_fp64_rescaled_phases(ctx_mc, n, omega, K, iters, with_f):
    ctx = ctx_mc
    w = oracle.omega_opt(n) if omega is None else omega
    u0 = wl.random_edges(n, n + K)
    f = wl.gaussian_source(n, K) * 100 if with_f else None
    ref = oracle.sor_f64(u0, w, f=f, max_iters=iters, check_every=K, tol=-1.0)
    got, res = run(ctx, u0, f, omega=w, tol=-1.0, max_iters=iters, check_every=K)
    assert res["iterations"] == iters
    assert pins.rel_err(got, ref["u"]) <= TOL64
    assert res["final_maxdelta"] == pytest.approx(ref["final_maxdelta"], rel=1e-8, abs=1e-13)


def test_fp64_rescaled_converges_like_oracle(ctx_mc):
    ctx = ctx_mc
    n = 180
    u0 = wl.random_edges(n, 44)
    w = oracle.omega_opt(n)
    for K in (1, 10):
        ref = oracle.sor_f64(u0, w, max_iters=5000, check_every=K, tol=1e-9)
        got, res = run(ctx, u0, omega=w, tol=1e-9, max_iters=5000, check_every=K)
        assert res["converged"] and ref["converged"]
        assert abs(res["iterations"] - ref["iterations"]) <= K  # m_k near tol may cross one check apart
        assert pins.rel_err(got, ref["u"]) <= 1e-11
        refr = oracle.sor_f64(u0, w, max_iters=5000, check_every=K, tol=1e-9, stop_mode=1)
        got, res = run(ctx, u0, omega=w, tol=1e-9, max_iters=5000, check_every=K, stop=1)
        assert res["converged"] and abs(res["iterations"] - refr["iterations"]) <= K


# fused FP32 sweep kernels: (family option, depth); family 1 = tile kernels,
# 2 = wavefront kernels; depth 1 = unfused (one launch per colour phase)
FUSED = [(1, 1), (1, 2), (1, 3), (1, 4), (1, 6), (1, 8), (2, 2), (2, 3), (2, 4), (2, 5)]
FUSED_IDS = ["unfused" if d == 1 else ("tile%d" % d if k == 1 else "wave%d" % d) for k, d in FUSED]


@pytest.fixture(scope="module")
def ctx_depth():
    """Contexts with each fused-sweep kernel family and depth of the FP32 sweeps."""
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    made = {}

    def get(shape):
        family, depth = shape if isinstance(shape, tuple) else (1, shape)
        if (family, depth) not in made:
            c = capi.Context(0)
            c.set_option(capi.SOR_OPT_FUSED_KERNEL, family)
            c.set_option(capi.SOR_OPT_TEMPORAL_DEPTH, depth)
            c.set_option(capi.SOR_OPT_CLUSTER, 0)  # keep small grids on the fused-iteration kernel
            made[(family, depth)] = c
        return made[(family, depth)]
    yield get
    for c in made.values():
        c.close()


@pytest.mark.parametrize("shape", FUSED, ids=FUSED_IDS)
@pytest.mark.parametrize("n,K,iters,with_f", [(1, 1, 9, True), (2, 3, 17, False), (63, 5, 43, True),
                                               (130, 50, 200, False), (257, 7, 61, True), (600, 13, 52, True),
                                               (601, 10, 40, False)])
def test_fp32_fused_iterations_bitwise(ctx_depth, shape, n, K, iters, with_f):
    capi = capi_mod()
    depth = shape[1]
    ctx = ctx_depth(shape)
    u0 = wl.random_edges(n, n + depth)
    f = wl.gaussian_source(n, K) * 25 if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor_f32(u0, w, f=f, max_iters=iters, check_every=K, tol=-1.0)
    got, res = run(ctx, u0, f, precision=capi.SOR_FP32, omega=w, tol=-1.0, max_iters=iters, check_every=K)
    assert res["iterations"] == iters
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]


@pytest.mark.parametrize("shape", FUSED, ids=FUSED_IDS)
def test_fp32_fused_converges_like_oracle(ctx_depth, shape):
    capi = capi_mod()
    ctx = ctx_depth(shape)
    n = 150
    u0 = wl.heat_plate(n, 100.0)
    w = oracle.omega_opt(n)
    ref = oracle.sor_f32(u0, w, max_iters=4000, check_every=10, tol=1e-3)
    got, res = run(ctx, u0, precision=capi.SOR_FP32, omega=w, tol=1e-3, max_iters=4000, check_every=10)
    assert res["converged"] == ref["converged"] and res["iterations"] == ref["iterations"]
    assert np.array_equal(got, ref["u"])


@pytest.mark.parametrize("shape", FUSED, ids=FUSED_IDS)
@pytest.mark.parametrize("n,inner", [(2, 20), (63, 20), (200, 7), (129, 1), (600, 20)])
def test_refine_fused_bitwise(ctx_depth, shape, n, inner):
    capi = capi_mod()
    depth = shape[1]
    ctx = ctx_depth(shape)
    u0, f = wl.poisson_problem(n, n + depth)
    u0 = u0 + wl.random_edges(n, n)
    w = oracle.omega_opt(n)
    ref = oracle.refine(u0, w, f=f, inner_sweeps=inner, tol=1e-10, max_outer=6000 // inner)
    got, res = run(ctx, u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-10, max_iters=6000,
                   inner_sweeps=inner)
    assert res["outer_steps"] == ref["outer_steps"] and bool(res["converged"]) == ref["converged"]
    assert np.array_equal(got, ref["u"])


@pytest.mark.parametrize("shape", [(1, 6), (2, 2), (2, 4)], ids=["tile6", "wave2", "wave4"])
def test_fp32_fused_full_size(ctx_depth, shape):
    """4098^2 FP32 plate, 100 iterations (a launch of fewer iterations than the
    depth at the end of each tested chunk of 50 for depths that do not divide
    it), against the oracle."""
    capi = capi_mod()
    ctx = ctx_depth(shape)
    n = 4096
    u0 = wl.random_edges(n, 1)
    w = oracle.omega_opt(n)
    ref = oracle.sor_f32(u0, w, max_iters=100, check_every=50, tol=-1.0)
    got, res = run(ctx, u0, precision=capi.SOR_FP32, omega=w, tol=-1.0, max_iters=100, check_every=50)
    assert np.array_equal(got, ref["u"]) and res["final_maxdelta"] == ref["final_maxdelta"]


def test_autotuner_picks_a_depth_and_keeps_results(tmp_path, monkeypatch):
    """With SOR_OPT_AUTOTUNE the first FP32 / refine solve of a size bucket
    times every fused depth; results stay bit-identical to the oracle and the
    choice is written to SOR_AUTOTUNE_CACHE."""
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SOR_AUTOTUNE_CACHE", str(cache))
    n = 300
    u0 = wl.random_edges(n, 3)
    w = oracle.omega_opt(n)
    with capi.Context(0) as ctx:
        ctx.set_option(capi.SOR_OPT_AUTOTUNE, 1)
        got, res = run(ctx, u0, precision=capi.SOR_FP32, omega=w, tol=-1.0, max_iters=77, check_every=11)
        ref = oracle.sor_f32(u0, w, max_iters=77, check_every=11, tol=-1.0)
        assert np.array_equal(got, ref["u"])
        u0p, f = wl.poisson_problem(n, 4)
        got, res = run(ctx, u0p, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-10, max_iters=20000)
        refr = oracle.refine(u0p, w, f=f, inner_sweeps=20, tol=1e-10, max_outer=1000)
        assert np.array_equal(got, refr["u"]) and res["outer_steps"] == refr["outer_steps"]
        assert ctx.stats()["solves"] == 2  # tuning runs are not counted
    lines = [[int(x) for x in l.split()] for l in cache.read_text().splitlines()]
    assert {(a, b) for a, b, *_ in lines} == {(512, 0), (512, 1)}
    for _, _, family, depth, rows, chunk in lines:
        assert (family, depth) in [(0, 1)] + [(0, d) for d in (2, 3, 4, 6, 8)] + [(1, d) for d in (2, 3, 4, 5)]
        assert rows in (0, 32, 64, 128) and chunk in (0, 1, 2, 4, 8)
    refine_line = [l for l in lines if l[1] == 1][0]
    assert refine_line[5] in (1, 2, 4, 8)  # the refine solve also tuned its corrections per graph


@pytest.mark.parametrize("path", PATHS)
def test_stall_window_stops_at_the_fp64_floor(ctxs, path):
    ctx = ctxs[path]
    """A tolerance below what FP64 reaches: with stall_window the solve stops,
    not converged, once that many residual tests gave no new minimum -- at the
    same step as the oracle, with the same result bit for bit."""
    capi = capi_mod()
    n = 96
    u0, f = wl.poisson_problem(n, 7)
    w = oracle.omega_opt(n)
    ref = oracle.refine(u0, w, f=f, inner_sweeps=10, tol=1e-17, max_outer=5000, stall_window=15)
    got, res = run(ctx, u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-17, max_iters=50000,
                   inner_sweeps=10, stall_window=15)
    assert not ref["converged"] and ref["outer_steps"] < 5000
    assert res["outer_steps"] == ref["outer_steps"] and not res["converged"]
    assert np.array_equal(got, ref["u"])
    ref = oracle.sor_f64(u0, w, f=f, max_iters=50000, check_every=10, tol=1e-17, stop_mode=1, stall_window=12)
    got, res = run(ctx, u0, f, omega=w, tol=1e-17, max_iters=50000, check_every=10, stop=capi.SOR_STOP_RESID_REL,
                   stall_window=12, flags=capi.SOR_FLAG_EXACT_ORDER)
    assert not ref["converged"] and ref["iterations"] < 50000
    assert res["iterations"] == ref["iterations"] and not res["converged"]
    assert np.array_equal(got, ref["u"])


@pytest.mark.parametrize("n", [1, 2, 7, 100, 255, 384])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cluster_path_converges_like_oracle(ctx, n, precision):
    """Whole solves inside one thread-block cluster: the stop decision is taken
    on the device after each tested iteration; results equal the oracle."""
    capi = capi_mod()
    u0 = wl.random_edges(n, 5 * n + 1)
    w = oracle.omega_opt(n)
    f = wl.gaussian_source(n, n) * 10 if n % 2 else None
    if precision == "fp64":
        ref = oracle.sor_f64(u0, w, f=f, max_iters=20000, check_every=3, tol=1e-9)
        got, res = run(ctx, u0, f, omega=w, tol=1e-9, max_iters=20000, check_every=3)
    else:
        ref = oracle.sor_f32(u0, w, f=f, max_iters=20000, check_every=3, tol=2e-3)
        got, res = run(ctx, u0, f, precision=capi.SOR_FP32, omega=w, tol=2e-3, max_iters=20000, check_every=3)
    assert res["converged"] == ref["converged"] and res["iterations"] == ref["iterations"]
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]


@pytest.mark.parametrize("n", [1, 2, 4, 9, 130, 301, 384])
@pytest.mark.parametrize("K,iters,tol", [(1, 400, 1e-6), (4, 203, 1e-30), (5, 3000, 1e-7), (1000, 57, 1e-9)])
def test_grid_flow_stops_like_oracle(ctxs, n, K, iters, tol):
    """The barrier-free grid decides the stop test behind the sweeps and rolls
    each band back to its copy of the stop iteration: the iteration count,
    the last max|change| and the solution equal the oracle's, whether the
    solve stops early (K = 1 or 5), runs to a cap that is not a multiple of K,
    or has no tested iteration before the cap (K = 1000)."""
    capi = capi_mod()
    u0 = wl.random_edges(n, 11 * n + K)
    f = wl.gaussian_source(n, n + K) * 10 if n % 3 == 1 else None
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, f=f, max_iters=iters, check_every=K, tol=tol)
    for path in ("grid", "gridbar"):
        got, res = run(ctxs[path], u0, f, omega=w, tol=tol, max_iters=iters, check_every=K,
                       flags=capi.SOR_FLAG_EXACT_ORDER)
        assert res["iterations"] == ref["iterations"] and res["converged"] == ref["converged"], path
        assert res["final_maxdelta"] == ref["final_maxdelta"], path
        assert np.array_equal(got, ref["u"]), path


@pytest.mark.parametrize("n", [3, 200, 768])
def test_grid_flow_fp32_stops_like_oracle(ctx, n):
    capi = capi_mod()
    u0 = wl.random_edges(n, 7 * n)
    w = oracle.omega_opt(n)
    ref = oracle.sor_f32(u0, w, max_iters=1500, check_every=1, tol=5e-3)
    got, res = run(ctx, u0, precision=capi.SOR_FP32, omega=w, tol=5e-3, max_iters=1500, check_every=1)
    assert res["iterations"] == ref["iterations"] and res["converged"] == ref["converged"]
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    assert np.array_equal(got, ref["u"])


@pytest.fixture(scope="module")
def ctx_nochain():
    """A context whose FP64 default path launches one kernel per colour phase."""
    capi = capi_mod()
    c = capi.Context(0)
    c.set_option(capi.SOR_OPT_CLUSTER, 0)
    c.set_option(capi.SOR_OPT_FAST_CHAIN, 0)
    yield c
    c.close()


@pytest.mark.parametrize("n,iters,K,with_f,stop", [(200, 90, 10, False, 0), (513, 77, 7, True, 0),
                                                  (1000, 60, 20, True, 1), (4096, 30, 10, False, 0)])
def test_fast_chain_equals_phase_launches(ctx_mc, ctx_nochain, n, iters, K, with_f, stop):
    """A chunk in one cooperative launch (neighbour progress counters) and one
    launch per colour phase compute the same numbers bit for bit."""
    capi = capi_mod()
    if with_f:
        u0, f = wl.poisson_problem(n, n)
    else:
        u0, f = wl.random_edges(n, n), None
    kw = dict(omega=oracle.omega_opt(n), tol=-1.0 if stop == 0 else 1e-30, max_iters=iters, check_every=K,
              stop=stop)
    a, ra = run(ctx_mc, u0, f, **kw)
    b, rb = run(ctx_nochain, u0, f, **kw)
    assert ra["iterations"] == rb["iterations"] == iters
    assert np.array_equal(a, b)
    assert ra["final_maxdelta"] == rb["final_maxdelta"]
    assert ra["final_resid_rel"] == rb["final_resid_rel"]


def test_kernel_launch_count(ctx_mc):
    """Chunks of 50 iterations in one launch each: pack, ring save, 20 chunk
    launches, final residual and unpack for 1000 iterations."""
    capi = capi_mod()
    n = 1024
    u0 = wl.random_edges(n, 1)
    ctx_mc.solve(u0, omega=oracle.omega_opt(n), tol=-1.0, max_iters=1000, check_every=50)  # warm graphs
    ctx_mc.reset_stats()
    ctx_mc.solve(u0, omega=oracle.omega_opt(n), tol=-1.0, max_iters=1000, check_every=50)
    assert ctx_mc.stats()["kernel_launches"] == 2 + 20 + 2


@pytest.mark.parametrize("with_f", [False, True])
def test_residual_signed_zeros_bitwise(ctx, with_f):
    """Inputs holding -0.0 (interior and one edge): the residual pass without a
    source maps g + x to x with -0 turned into +0 on the integer units, which
    must give the oracle's bits exactly, signs of zeros included, in the
    residual stop and through the defect correction (where r~ feeds the
    sweeps and u += d)."""
    capi = capi_mod()
    n = 37
    u0 = np.full((n + 2, n + 2), -0.0)
    u0[0, :] = 50.0
    u0[:, 0] = -0.0
    u0[5:9, 5:9] = 0.0
    f = wl.gaussian_source(n, 3) if with_f else None
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, f=f, max_iters=40, check_every=5, tol=-1.0, stop_mode=1)
    got, res = run(ctx, u0, f, omega=w, tol=-1.0, max_iters=40, check_every=5, stop=capi.SOR_STOP_RESID_REL,
                   flags=capi.SOR_FLAG_EXACT_ORDER)
    assert np.array_equal(got.view(np.int64), ref["u"].view(np.int64))
    assert res["final_resid_rel"] == ref["final_resid_rel"]
    ref = oracle.refine(u0, w, f=f, inner_sweeps=20, tol=1e-9, max_outer=200)
    got, res = run(ctx, u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-9, max_iters=4000)
    assert res["outer_steps"] == ref["outer_steps"] and res["iterations"] == ref["sweeps"]
    assert np.array_equal(got.view(np.int64), ref["u"].view(np.int64))
