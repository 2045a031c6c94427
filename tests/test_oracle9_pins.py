"""Pins of the four-colour 9-point SOR oracle to mathematics that does not
come from the oracle: the multi-colour SOR splitting of the dense 9-point
system, dense and DST-I direct solves, polynomials the compact 9-point
operator reproduces exactly (harmonic ones up to degree 5, which the 5-point
operator does not), the source sign, the residual as b - Ax, stop rules and
symmetry."""
import numpy as np
import pytest

import oracle
from tests import pins


def _problem(n, seed, with_f=True):
    g = np.random.default_rng(seed)
    u0 = g.uniform(0.0, 100.0, size=(n + 2, n + 2))
    u0[1:-1, 1:-1] = 0.0
    f = g.uniform(-50.0, 50.0, size=(n, n)) if with_f else None
    return u0, f


@pytest.mark.parametrize("n,omega", [(4, 1.0), (5, 1.4), (6, 1.7), (7, 1.2)])
@pytest.mark.parametrize("with_f", [False, True])
def test_iterates_match_multicolour_splitting(n, omega, with_f):
    """Pins the weights 4 / 1 / 20, the four colours and their order, w/20,
    the corner reads of the diagonal terms and the source scaling 6h^2."""
    u0, f = _problem(n, 3 * n + int(with_f), with_f)
    ref = pins.multicolour_iteration9(u0, omega, 5, f=f)
    for k in (1, 2, 5):
        r = oracle.sor9_f64(u0, omega, f=f, max_iters=k, check_every=1000, tol=0.0)
        assert r["iterations"] == k
        assert pins.rel_err(r["u"], ref[k - 1]) < 1e-13


def test_dst_solver_matches_dense():
    u0, f = _problem(7, 1)
    assert pins.rel_err(pins.dst_solve9(u0, f), pins.dense_solve9(u0, f)) < 1e-12


def test_converges_to_dense_and_dst():
    u0, f = _problem(8, 2)
    r = oracle.sor9_f64(u0, oracle.omega_opt(8), f=f, max_iters=5000, tol=1e-11)
    assert r["converged"]
    assert pins.rel_err(r["u"], pins.dense_solve9(u0, f)) < 1e-12
    n = 60
    u0, f = _problem(n, 4)
    r = oracle.sor9_f64(u0, oracle.omega_opt(n), f=f, max_iters=20000, tol=1e-11)
    assert r["converged"]
    assert pins.rel_err(r["u"], pins.dst_solve9(u0, f)) < 1e-11


@pytest.mark.parametrize("name,fn", [
    ("x2-y2", lambda x, y: x * x - y * y),
    ("x3-3xy2", lambda x, y: x ** 3 - 3.0 * x * y * y),
    ("x4-6x2y2+y4", lambda x, y: x ** 4 - 6.0 * x * x * y * y + y ** 4),
    ("x5-10x3y2+5xy4", lambda x, y: x ** 5 - 10.0 * x ** 3 * y * y + 5.0 * x * y ** 4),
])
def test_harmonic_polynomials_reproduced(name, fn):
    """The compact 9-point operator is exact on harmonic polynomials up to
    degree 5 (its error term acts through the bi-Laplacian)."""
    n = 16
    u0, exact = pins.grid_from(fn, n)
    r = oracle.sor9_f64(u0, oracle.omega_opt(n), max_iters=5000, tol=1e-15)
    assert np.max(np.abs(r["u"] - exact)) < 1e-12


def test_quartic_separates_from_5_point():
    """The same quartic harmonic is not a fixed point of the 5-point scheme:
    the agreement above is a property of the 9-point weights."""
    n = 16
    u0, exact = pins.grid_from(lambda x, y: x ** 4 - 6.0 * x * x * y * y + y ** 4, n)
    r5 = oracle.sor_f64(u0, oracle.omega_opt(n), max_iters=5000, tol=1e-15)
    assert np.max(np.abs(r5["u"] - exact)) > 1e-6


def test_source_sign_convention():
    """-Laplace(u) = f: u = x^2 + y^2 needs f = -4 (exact for the 9-point operator)."""
    n = 14
    u0, exact = pins.grid_from(lambda x, y: x * x + y * y, n)
    f = np.full((n, n), -4.0)
    r = oracle.sor9_f64(u0, oracle.omega_opt(n), f=f, max_iters=5000, tol=1e-15)
    assert np.max(np.abs(r["u"] - exact)) < 1e-12
    w = oracle.sor9_f64(u0, oracle.omega_opt(n), f=-f, max_iters=5000, tol=1e-15)
    assert np.max(np.abs(w["u"] - exact)) > 1e-3


def test_residual_is_b_minus_ax():
    n = 5
    u0, f = _problem(n, 9)
    u = u0.copy()
    u[1:-1, 1:-1] = np.random.default_rng(10).uniform(-10, 10, size=(n, n))
    A, b = pins.dense_system9(u0, f)
    res = b - A @ u[1:-1, 1:-1].ravel()
    r, rm, bm = oracle.residual9(u, f=f)
    assert np.max(np.abs(r[1:-1, 1:-1].ravel() - res)) < 1e-9
    assert abs(rm - np.max(np.abs(res))) < 1e-9
    assert abs(bm - np.max(np.abs(b))) < 1e-9
    assert oracle.resid_rel9(pins.dense_solve9(u0, f), f=f) < 1e-13


def test_stop_rules():
    n = 20
    u0, _ = _problem(n, 5, with_f=False)
    w = oracle.omega_opt(n)
    r = oracle.sor9_f64(u0, w, max_iters=5000, check_every=6, tol=1e-9, trace=True)
    assert r["converged"] and r["iterations"] % 6 == 0
    t = r["trace"]
    assert t[-1] < 1e-9 and all(t[k - 1] >= 1e-9 for k in range(6, r["iterations"], 6))
    # strict comparison: with tol equal to a tested change the loop goes on
    k0 = 6 * (len(t) // 12)
    e = oracle.sor9_f64(u0, w, max_iters=5000, check_every=6, tol=float(t[k0 - 1]))
    assert e["iterations"] > k0
    assert oracle.sor9_f64(u0, w, max_iters=5000, check_every=6, tol=float(t[k0 - 1]) * 1.0000001)["iterations"] == k0
    c = oracle.sor9_f64(u0, w, max_iters=4, tol=1e-30)
    assert c["iterations"] == 4 and not c["converged"]
    s = oracle.sor9_f64(u0, w, max_iters=5000, check_every=5, tol=1e-10, stop_mode=1)
    assert s["converged"] and s["iterations"] % 5 == 0 and s["final_resid_rel"] < 1e-10


def test_mirror_symmetry_and_superposition():
    n = 15
    w = oracle.omega_opt(n)
    a = np.zeros((n + 2, n + 2))
    a[0, :] = 100.0
    b = np.zeros((n + 2, n + 2))
    b[:, -1] = 100.0
    ra = oracle.sor9_f64(a, w, max_iters=8000, tol=1e-13)["u"]
    rb = oracle.sor9_f64(b, w, max_iters=8000, tol=1e-13)["u"]
    both = a + b
    rab = oracle.sor9_f64(both, w, max_iters=8000, tol=1e-13)["u"]
    assert np.max(np.abs((ra + rb)[1:-1, 1:-1] - rab[1:-1, 1:-1])) < 1e-9
    assert np.max(np.abs(ra - ra[:, ::-1])) < 1e-9


def test_f32_within_its_rounding():
    n = 40
    u0, f = _problem(n, 12)
    w = oracle.omega_opt(n)
    a = oracle.sor9_f64(u0, w, f=f, max_iters=150, tol=0.0)["u"]
    b = oracle.sor9_f32(u0, w, f=f, max_iters=150, tol=0.0)["u"]
    assert 1e-9 < pins.rel_err(b, a) < 5e-5


# --- defect correction with the 9-point sweeps ----------------------------------------------------------------------

@pytest.mark.parametrize("inner", [1, 3, 12])
def test_refinement9_with_fp64_inner_equals_plain_sor(inner):
    """u + delta_s = x* + M^s (u - x*): one outer step equals s plain
    four-colour iterations (pinned to the multi-colour splitting)."""
    n = 9
    u0, f = _problem(n, 51)
    w = oracle.omega_opt(n)
    steps = 3
    ref = oracle.refine9(u0, w, f=f, inner_sweeps=inner, inner_f32=False, tol=-1.0, max_outer=steps)
    plain = oracle.sor9_f64(u0, w, f=f, max_iters=inner * steps, check_every=1000, tol=0.0)
    assert ref["outer_steps"] == steps and ref["sweeps"] == inner * steps and not ref["converged"]
    assert pins.rel_err(ref["u"], plain["u"]) < 1e-12


def test_refinement9_fp32_inner_tracks_plain_sor():
    n = 12
    u0, f = _problem(n, 53)
    w = oracle.omega_opt(n)
    ref = oracle.refine9(u0, w, f=f, inner_sweeps=5, inner_f32=True, tol=-1.0, max_outer=3)
    plain = oracle.sor9_f64(u0, w, f=f, max_iters=15, check_every=1000, tol=0.0)
    assert 0 < pins.rel_err(ref["u"], plain["u"]) < 1e-5


def test_refinement9_reaches_tolerance_and_the_dst_solution():
    n = 30
    u0, f = _problem(n, 57)
    w = oracle.omega_opt(n)
    out = oracle.refine9(u0, w, f=f, inner_sweeps=20, inner_f32=True, tol=1e-12, max_outer=500, trace=True)
    assert out["converged"] and out["final_resid_rel"] < 1e-12
    assert oracle.resid_rel9(out["u"], f=f) == out["final_resid_rel"]
    assert pins.rel_err(out["u"], pins.dst_solve9(u0, f)) < 1e-12 * 1e3
    tr = out["trace"]
    assert tr[-1] < 1e-12 and tr[-1] < 1e-8 * tr[0]


def test_refinement9_caps_and_zero_steps():
    n = 6
    u0, f = _problem(n, 59)
    w = oracle.omega_opt(n)
    out = oracle.refine9(u0, w, f=f, inner_sweeps=4, tol=1e-30, max_outer=3)
    assert out["outer_steps"] == 3 and out["sweeps"] == 12 and not out["converged"]
    out0 = oracle.refine9(u0, w, f=f, inner_sweeps=4, tol=1e-30, max_outer=0)
    assert out0["outer_steps"] == 0 and np.array_equal(out0["u"], u0)
    assert out0["final_resid_rel"] == oracle.resid_rel9(u0, f=f)


# --- the stall rule with the 9-point stencil ---------------------------------------------------------------------

def test_stall_rule_9pt_matches_its_definition():
    """Residuals of independent runs of 4j iterations fed to the rule (c17)
    give the test at which the oracle's run with the rule stops."""
    n = 10
    u0, f = _problem(n, 63)
    w = oracle.omega_opt(n)
    K, window = 4, 6
    rhos = [oracle.resid_rel9(oracle.sor9_f64(u0, w, f=f, max_iters=K * (j + 1), check_every=10 ** 6,
                                              tol=0.0)["u"], f=f) for j in range(150)]
    best, run, stop = np.inf, 0, None
    for j, r in enumerate(rhos):
        if r < best:
            best, run = r, 0
        elif r < 4.0 * best:
            run += 1
            if run >= window:
                stop = j
                break
        else:
            run = 0
    assert stop is not None
    out = oracle.sor9_f64(u0, w, f=f, max_iters=K * 150, check_every=K, tol=1e-30, stop_mode=1, stall_window=window)
    assert not out["converged"] and out["iterations"] == K * (stop + 1)
    off = oracle.sor9_f64(u0, w, f=f, max_iters=K * 150, check_every=K, tol=1e-30, stop_mode=1, stall_window=0)
    assert off["iterations"] == K * 150


def test_refinement9_stall_rule_matches_its_definition():
    n = 10
    u0, f = _problem(n, 69)
    w = oracle.omega_opt(n)
    full = oracle.refine9(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=300, trace=True)
    best, run, stop = np.inf, 0, None
    for j, r in enumerate(full["trace"][:300]):
        if r < best:
            best, run = r, 0
        elif r < 4.0 * best:
            run += 1
            if run >= 5:
                stop = j
                break
        else:
            run = 0
    assert stop is not None
    out = oracle.refine9(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=300, stall_window=5)
    assert not out["converged"] and out["outer_steps"] == stop
    assert oracle.refine9(u0, w, f=f, inner_sweeps=3, tol=1e-30, max_outer=300)["outer_steps"] == 300
