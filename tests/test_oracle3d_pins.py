"""Pins of the 3D oracle (7-point red-black SOR on a cube) to mathematics
that does not come from the oracle itself: the iteration written as a matrix
splitting, dense and DST-I direct solves, quadratics the 7-point operator
reproduces exactly, SOR convergence theory, and symmetry / superposition."""
import numpy as np
import pytest

import oracle
from tests import pins


def _rng(seed):
    return np.random.default_rng(seed)


def _random_cube(n, seed, with_f=True):
    g = _rng(seed)
    u0 = g.uniform(0.0, 100.0, size=(n + 2,) * 3)
    u0[1:-1, 1:-1, 1:-1] = 0.0
    f = g.uniform(-50.0, 50.0, size=(n,) * 3) if with_f else None
    return u0, f


@pytest.mark.parametrize("n,omega", [(3, 1.0), (3, 1.5), (4, 1.3), (5, 1.7)])
@pytest.mark.parametrize("with_f", [False, True])
def test_iterates_match_matrix_splitting(n, omega, with_f):
    """Every iterate equals the red-first SOR splitting (D - wL)^-1 applied to
    the dense 7-point system: pins the stencil, the colouring (i+j+k), the
    red-then-black order, omega/6 and the sign of the source."""
    u0, f = _random_cube(n, 10 * n + int(with_f), with_f)
    ref = pins.red_black_iteration3(u0, omega, 6, f=f)
    for k in (1, 2, 6):
        r = oracle.sor3d_f64(u0, omega, f=f, max_iters=k, check_every=1000, tol=0.0)
        assert r["iterations"] == k
        assert pins.rel_err3(r["u"], ref[k - 1]) < 1e-13


def test_dst_solver_matches_dense():
    """The DST-I fast solve used below is itself checked against LAPACK."""
    u0, f = _random_cube(5, 3)
    assert pins.rel_err3(pins.dst_solve3(u0, f), pins.dense_solve3(u0, f)) < 1e-12


@pytest.mark.parametrize("n", [4, 5])
def test_converges_to_dense_solution(n):
    u0, f = _random_cube(n, 40 + n)
    r = oracle.sor3d_f64(u0, oracle.omega_opt(n), f=f, max_iters=4000, tol=1e-11)
    assert r["converged"]
    assert pins.rel_err3(r["u"], pins.dense_solve3(u0, f)) < 1e-12


def test_converges_to_dst_solution_larger():
    n = 20
    u0, f = _random_cube(n, 7)
    r = oracle.sor3d_f64(u0, oracle.omega_opt(n), f=f, max_iters=5000, tol=1e-13)
    assert r["converged"]
    assert pins.rel_err3(r["u"], pins.dst_solve3(u0, f)) < 1e-11


def test_harmonic_quadratic_is_reproduced():
    """u = x^2 + y^2 - 2 z^2 is harmonic and the 7-point operator is exact on
    quadratics, so the converged iterate is the closed form to roundoff."""
    n = 14
    u0, exact = pins.cube_from(lambda x, y, z: x * x + y * y - 2.0 * z * z, n)
    r = oracle.sor3d_f64(u0, oracle.omega_opt(n), max_iters=5000, tol=1e-15)
    assert np.max(np.abs(r["u"] - exact)) < 1e-12


def test_source_sign_convention():
    """-Laplace(u) = f: u = x^2 + y^2 + z^2 needs f = -6."""
    n = 12
    u0, exact = pins.cube_from(lambda x, y, z: x * x + y * y + z * z, n)
    f = np.full((n,) * 3, -6.0)
    r = oracle.sor3d_f64(u0, oracle.omega_opt(n), f=f, max_iters=5000, tol=1e-15)
    assert np.max(np.abs(r["u"] - exact)) < 1e-12
    wrong = oracle.sor3d_f64(u0, oracle.omega_opt(n), f=-f, max_iters=5000, tol=1e-15)
    assert np.max(np.abs(wrong["u"] - exact)) > 1e-3


def _late_ratio(t, count):
    """Geometric-mean ratio m_{k+1}/m_k over the last `count` steps before the
    change reaches the rounding floor of values of size ~100."""
    last = int(np.nonzero(t > 1e-9)[0][-1])
    w = t[last - count:last + 1]
    return float(np.exp(np.mean(np.log(w[1:] / w[:-1]))))


@pytest.mark.parametrize("omega", [1.0, 1.4])
def test_rate_follows_young(omega):
    """For omega below omega_opt the change m_k decays by Young's factor with
    the Jacobi radius cos(pi h) of the 7-point operator (equal spacing)."""
    n = 10
    u0, _ = _random_cube(n, 5, with_f=False)
    r = oracle.sor3d_f64(u0, omega, max_iters=400, tol=0.0, trace=True)
    ratio = _late_ratio(r["trace"], 60)
    assert abs(ratio - pins.young_rate(omega, n)) < 2e-3


def test_rate_at_omega_opt():
    """At omega_opt the late ratio tends to omega_opt - 1 (from above, because
    of the 2 x 2 Jordan block)."""
    n = 12
    w = oracle.omega_opt(n)
    u0, _ = _random_cube(n, 9, with_f=False)
    r = oracle.sor3d_f64(u0, w, max_iters=900, tol=0.0, trace=True)
    ratio = _late_ratio(r["trace"], 40)
    assert w - 1.0 <= ratio < (w - 1.0) * 1.1


def test_residual_is_b_minus_ax():
    """r~ = b - A x and b~ = b with the dense 7-point system; rho = max|r~|/max|b|."""
    n = 4
    u0, f = _random_cube(n, 21)
    g = _rng(22)
    u = u0.copy()
    u[1:-1, 1:-1, 1:-1] = g.uniform(-10, 10, size=(n,) * 3)
    A, b = pins.dense_system3(u0, f)
    res = b - A @ u[1:-1, 1:-1, 1:-1].ravel()
    r, rm, bm = oracle.residual3d(u, f=f)
    assert np.max(np.abs(r[1:-1, 1:-1, 1:-1].ravel() - res)) < 1e-9
    assert abs(rm - np.max(np.abs(res))) < 1e-9
    assert abs(bm - np.max(np.abs(b))) < 1e-12
    assert abs(oracle.resid_rel3d(u, f=f) - rm / bm) < 1e-15
    # the exact solution has a residual at roundoff level
    assert oracle.resid_rel3d(pins.dense_solve3(u0, f), f=f) < 1e-13


def test_stop_rules():
    n = 10
    u0, _ = _random_cube(n, 2, with_f=False)
    w = oracle.omega_opt(n)
    r = oracle.sor3d_f64(u0, w, max_iters=3000, check_every=7, tol=1e-9, trace=True)
    assert r["converged"] and r["iterations"] % 7 == 0
    t = r["trace"]
    assert t[-1] < 1e-9
    # no earlier checked iteration was below tol
    assert all(t[k - 1] >= 1e-9 for k in range(7, r["iterations"], 7))
    # the cap without convergence is not an error
    c = oracle.sor3d_f64(u0, w, max_iters=5, tol=1e-30)
    assert c["iterations"] == 5 and not c["converged"]
    # residual stop
    s = oracle.sor3d_f64(u0, w, max_iters=3000, check_every=5, tol=1e-10, stop_mode=1)
    assert s["converged"] and s["iterations"] % 5 == 0 and s["final_resid_rel"] < 1e-10


def test_superposition_and_mirror_symmetry():
    n = 9
    w = oracle.omega_opt(n)
    a = np.zeros((n + 2,) * 3)
    a[0] = 100.0  # bottom face
    b = np.zeros((n + 2,) * 3)
    b[:, :, -1] = 100.0  # x = 1 face
    both = np.maximum(a, b)
    both[0, :, -1] = 100.0
    ra = oracle.sor3d_f64(a, w, max_iters=5000, tol=1e-13)["u"]
    rb = oracle.sor3d_f64(b, w, max_iters=5000, tol=1e-13)["u"]
    # the two faces share an edge; the 7-point stencil never reads shell edges,
    # so the interior of the sum equals the solve with both faces set
    rab = oracle.sor3d_f64(both, w, max_iters=5000, tol=1e-13)["u"]
    inner = (slice(1, -1),) * 3
    assert np.max(np.abs((ra + rb)[inner] - rab[inner])) < 1e-9
    # the bottom-face solution is symmetric under x -> 1-x and y -> 1-y
    assert np.max(np.abs(ra - ra[:, :, ::-1])) < 1e-9
    assert np.max(np.abs(ra - ra[:, ::-1, :])) < 1e-9


def test_f32_within_its_rounding():
    """The FP32 iteration stays within FP32 rounding of the FP64 one and
    reproduces the harmonic quadratic to FP32 accuracy."""
    n = 16
    u0, f = _random_cube(n, 31)
    w = oracle.omega_opt(n)
    a = oracle.sor3d_f64(u0, w, f=f, max_iters=200, tol=0.0)["u"]
    b = oracle.sor3d_f32(u0, w, f=f, max_iters=200, tol=0.0)["u"]
    assert pins.rel_err3(b, a) < 5e-5
    u0, exact = pins.cube_from(lambda x, y, z: x * x + y * y - 2.0 * z * z, n)
    r = oracle.sor3d_f32(u0, w, max_iters=3000, tol=1e-7)
    assert np.max(np.abs(r["u"] - exact)) < 2e-5
    # FP32 iterates are not FP64 ones: the rounding is really FP32
    assert pins.rel_err3(b, a) > 1e-9


# --- defect correction on a cube ------------------------------------------------------------------------------------

@pytest.mark.parametrize("inner", [1, 4, 20])
def test_refinement3d_with_fp64_inner_equals_plain_sor(inner):
    """u + delta_s = x* + M^s (u - x*): one outer step equals s plain sweeps,
    which pins the residual's sign, the zero start of the correction and the
    update of u against the plain iteration (itself pinned to the splitting)."""
    n = 7
    u0, f = _random_cube(n, 41)
    w = oracle.omega_opt(n)
    steps = 3
    ref = oracle.refine3d(u0, w, f=f, inner_sweeps=inner, inner_f32=False, tol=-1.0, max_outer=steps)
    plain = oracle.sor3d_f64(u0, w, f=f, max_iters=inner * steps, check_every=1000, tol=0.0)
    assert ref["outer_steps"] == steps and ref["sweeps"] == inner * steps and not ref["converged"]
    assert pins.rel_err3(ref["u"], plain["u"]) < 1e-12


def test_refinement3d_fp32_inner_tracks_plain_sor():
    """FP32 inner sweeps follow plain SOR up to single-precision rounding of
    each correction (and differ from it: the FP32 path is really taken)."""
    n = 8
    u0, f = _random_cube(n, 43)
    w = oracle.omega_opt(n)
    ref = oracle.refine3d(u0, w, f=f, inner_sweeps=6, inner_f32=True, tol=-1.0, max_outer=3)
    plain = oracle.sor3d_f64(u0, w, f=f, max_iters=18, check_every=1000, tol=0.0)
    assert 0 < pins.rel_err3(ref["u"], plain["u"]) < 1e-5


def test_refinement3d_reaches_tolerance_and_the_dst_solution():
    n = 14
    u0, f = _random_cube(n, 47)
    w = oracle.omega_opt(n)
    out = oracle.refine3d(u0, w, f=f, inner_sweeps=20, inner_f32=True, tol=1e-12, max_outer=500, trace=True)
    assert out["converged"] and out["final_resid_rel"] < 1e-12
    # the reported residual is that of the returned solution
    assert oracle.resid_rel3d(out["u"], f=f) == out["final_resid_rel"]
    # error <= cond(A) rho, cond ~ 12 / (3 pi^2 h^2) ~ 30 here
    assert pins.rel_err3(out["u"], pins.dst_solve3(u0, f)) < 1e-12 * 1e2
    tr = out["trace"]
    assert tr[-1] < 1e-12 and tr[-1] < 1e-8 * tr[0]


def test_refinement3d_caps_and_zero_steps():
    n = 5
    u0, f = _random_cube(n, 49)
    w = oracle.omega_opt(n)
    out = oracle.refine3d(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=4)
    assert out["outer_steps"] == 4 and out["sweeps"] == 12 and not out["converged"]
    out0 = oracle.refine3d(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=0)
    assert out0["outer_steps"] == 0 and np.array_equal(out0["u"], u0)
    assert out0["final_resid_rel"] == oracle.resid_rel3d(u0, f=f)


# --- the stall rule on cubes (as on the plate: for tolerances below the FP64 floor) --------------------------------

def _stall_stop(rhos, window):
    """The rule as defined (c17): the index of the residual test at which a run
    of `window` tests without a new minimum, all within 4x of it, ends."""
    best, run = np.inf, 0
    for j, r in enumerate(rhos):
        if r < best:
            best, run = r, 0
        elif r < 4.0 * best:
            run += 1
            if run >= window:
                return j
        else:
            run = 0
    return None


def test_stall_rule_on_cubes_matches_its_definition():
    """Residuals of independent runs of 5j iterations fed to the rule give
    the test at which the oracle's run with the rule stops unconverged."""
    n = 6
    u0, f = _random_cube(n, 61)
    w = oracle.omega_opt(n)
    K, window = 5, 6
    rhos = [oracle.resid_rel3d(oracle.sor3d_f64(u0, w, f=f, max_iters=K * (j + 1), check_every=10 ** 6,
                                                tol=0.0)["u"], f=f) for j in range(120)]
    j = _stall_stop(rhos, window)
    assert j is not None
    out = oracle.sor3d_f64(u0, w, f=f, max_iters=K * 120, check_every=K, tol=1e-30, stop_mode=1,
                           stall_window=window)
    assert not out["converged"] and out["iterations"] == K * (j + 1)
    off = oracle.sor3d_f64(u0, w, f=f, max_iters=K * 120, check_every=K, tol=1e-30, stop_mode=1, stall_window=0)
    assert off["iterations"] == K * 120


def test_refinement3d_stall_rule_matches_its_definition():
    """The defect correction's residual trace without the rule, fed to the
    rule as defined, gives the correction count at which the run with the
    rule stops unconverged."""
    n = 6
    u0, f = _random_cube(n, 67)
    w = oracle.omega_opt(n)
    full = oracle.refine3d(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=200, trace=True)
    j = _stall_stop(full["trace"][:200], 5)
    assert j is not None
    out = oracle.refine3d(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=200, stall_window=5)
    assert not out["converged"] and out["outer_steps"] == j
    assert oracle.refine3d(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=200)["outer_steps"] == 200
