"""Pins of the block two-colour SOR oracle (``oracle.sor_block_f64``), the
reading of the block-parallel SOR that Section 3.1 names beside red-black
SOR: blocks of by x bx cells coloured (I + J) mod 2, colour 0 first,
row-major order inside a block, the update of Eq. 1.

What fixes it independently of its own loops:
* 1 x 1 blocks are red-black SOR, whose oracle is pinned on its own
  (tests/test_oracle_pins.py): equal bit for bit, trace and stop included;
* any block shape equals SOR written as a matrix splitting in the order the
  definition gives (tests/pins.py), and the same splitting with the blocks
  of one colour taken in reverse order (they are independent);
* one block covering the interior is SOR in natural order, a consistently
  ordered case: Gauss-Seidel contracts by mu^2 and SOR below the optimum by
  Young's factor, as the theory of Section 2.1's method says;
* the converged iterate solves the 5-point system (dense LAPACK solve).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1401_0763_gb300 import workloads as wl
from tests import pins


def block_order(n, by, bx, reverse_colour0=False):
    """Natural interior indices in the update order the definition gives."""
    nbr, nbc = -(-n // by), -(-n // bx)
    per_colour = {0: [], 1: []}
    for I in range(nbr):
        for J in range(nbc):
            per_colour[(I + J) % 2].append((I, J))
    if reverse_colour0:
        per_colour[0] = per_colour[0][::-1]
    order = []
    for colour in (0, 1):
        for I, J in per_colour[colour]:
            for i in range(I * by, min(n, (I + 1) * by)):
                for j in range(J * bx, min(n, (J + 1) * bx)):
                    order.append(i * n + j)
    assert sorted(order) == list(range(n * n))
    return order


@pytest.mark.parametrize("n", [1, 2, 6, 13])
@pytest.mark.parametrize("with_f", [False, True])
@pytest.mark.parametrize("K,stop", [(1, 0), (4, 0), (3, 1)])
def test_unit_blocks_are_red_black(n, with_f, K, stop):
    u0 = wl.random_edges(n, seed=n)
    f = wl.rng(n + 1).uniform(-50, 50, size=(n, n)) if with_f else None
    w = 1.37
    tol = 1e-6 if stop == 0 else 1e-5
    a = oracle.sor_f64(u0, w, f=f, max_iters=400, check_every=K, tol=tol, stop_mode=stop, trace=True)
    b = oracle.sor_block_f64(u0, w, by=1, bx=1, f=f, max_iters=400, check_every=K, tol=tol, stop_mode=stop,
                             trace=True)
    assert np.array_equal(a["u"], b["u"])
    assert np.array_equal(a["trace"], b["trace"])
    for key in ("iterations", "converged", "final_maxdelta", "final_resid_rel"):
        assert a[key] == b[key], key


@pytest.mark.parametrize("n", [5, 7])
@pytest.mark.parametrize("by,bx", [(2, 3), (3, 2), (1, 4), (4, 1), (2, 2), (7, 7), (3, 7)])
@pytest.mark.parametrize("omega", [0.7, 1.0, 1.6])
def test_iterates_match_ordered_splitting(n, by, bx, omega):
    u0 = wl.random_edges(n, seed=3)
    f = wl.rng(4).uniform(-10, 10, size=(n, n))
    ref = pins.ordered_sor_iteration(u0, omega, 4, block_order(n, by, bx), f)
    for k in (1, 2, 4):
        out = oracle.sor_block_f64(u0, omega, by=by, bx=bx, f=f, max_iters=k, tol=-1.0, trace=True)
        assert out["iterations"] == k and not out["converged"]
        assert pins.rel_err(out["u"], ref[k - 1]) < 1e-13
    # m_k: the largest change between successive iterates
    out = oracle.sor_block_f64(u0, omega, by=by, bx=bx, f=f, max_iters=4, tol=-1.0, trace=True)
    for k in range(4):
        prev = u0 if k == 0 else ref[k - 1]
        mk = np.max(np.abs(ref[k] - prev))
        assert abs(out["trace"][k] - mk) <= 1e-12 * max(mk, 1.0)


def test_blocks_of_a_colour_are_independent():
    n, by, bx, w = 9, 2, 3, 1.4
    u0 = wl.random_edges(n, seed=11)
    f = wl.rng(12).uniform(-10, 10, size=(n, n))
    fwd = pins.ordered_sor_iteration(u0, w, 3, block_order(n, by, bx), f)
    rev = pins.ordered_sor_iteration(u0, w, 3, block_order(n, by, bx, reverse_colour0=True), f)
    out = oracle.sor_block_f64(u0, w, by=by, bx=bx, f=f, max_iters=3, tol=-1.0)
    assert pins.rel_err(fwd[2], rev[2]) < 1e-13
    assert pins.rel_err(out["u"], rev[2]) < 1e-13


def test_colour_order_matters_for_larger_blocks():
    """Colour 1 first is a different iteration (the pin above would catch a
    swapped colour)."""
    n, by, bx, w = 6, 2, 2, 1.2
    u0 = wl.random_edges(n, seed=5)
    order = block_order(n, by, bx)
    nb0 = sum(1 for I in range(3) for J in range(3) if (I + J) % 2 == 0) * by * bx
    swapped = order[nb0:] + order[:nb0]
    a = pins.ordered_sor_iteration(u0, w, 1, order)[0]
    b = pins.ordered_sor_iteration(u0, w, 1, swapped)[0]
    out = oracle.sor_block_f64(u0, w, by=by, bx=bx, max_iters=1, tol=-1.0)
    assert pins.rel_err(out["u"], a) < 1e-13
    assert pins.rel_err(a, b) > 1e-6


def _late_ratio(trace, k0, k1):
    t = np.asarray(trace)
    return float(np.exp((np.log(t[k1]) - np.log(t[k0])) / (k1 - k0)))


def test_one_block_gauss_seidel_rate_is_mu_squared():
    n = 31
    u0 = wl.heat_plate(n, 100.0)
    out = oracle.sor_block_f64(u0, 1.0, by=n, bx=n, max_iters=3000, tol=-1.0, trace=True)
    mu = np.cos(np.pi / (n + 1))
    t = out["trace"]
    k1 = int(np.nonzero(t > 1e-10)[0][-1])
    assert _late_ratio(t, k1 - 500, k1) == pytest.approx(mu * mu, rel=1e-4)


@pytest.mark.parametrize("omega", [1.3, 1.6])
def test_one_block_young_rate_below_optimum(omega):
    n = 31
    u0 = wl.heat_plate(n, 100.0)
    out = oracle.sor_block_f64(u0, omega, by=n, bx=n, max_iters=3000, tol=-1.0, trace=True)
    t = out["trace"]
    k1 = int(np.nonzero(t > 1e-10)[0][-1])
    assert _late_ratio(t, k1 - 150, k1) == pytest.approx(pins.young_rate(omega, n), rel=2e-3)


@pytest.mark.parametrize("by,bx", [(3, 5), (1, 12), (4, 4)])
def test_converged_matches_dense_solve(by, bx):
    n = 12
    u0 = wl.random_edges(n, seed=21)
    f = wl.rng(22).uniform(-100, 100, size=(n, n))
    out = oracle.sor_block_f64(u0, 1.5, by=by, bx=bx, f=f, max_iters=20000, tol=1e-11)
    assert out["converged"]
    ref = pins.dense_solve(u0, f)
    assert pins.rel_err(out["u"], ref) < 1e-11
    assert out["final_resid_rel"] < 1e-12


@pytest.mark.parametrize("K", [1, 5, 7])
def test_stops_at_first_passing_check(K):
    n = 10
    u0 = wl.heat_plate(n, 100.0)
    full = oracle.sor_block_f64(u0, 1.5, by=3, bx=4, max_iters=500, tol=-1.0, trace=True)
    tol = 1e-4
    out = oracle.sor_block_f64(u0, 1.5, by=3, bx=4, max_iters=500, check_every=K, tol=tol)
    passing = [k for k in range(K, 501, K) if full["trace"][k - 1] < tol]
    assert out["converged"] and out["iterations"] == passing[0]
    assert out["final_maxdelta"] == full["trace"][passing[0] - 1]


def test_bad_arguments_rejected():
    u0 = wl.heat_plate(4, 1.0)
    for kw in (dict(by=0, bx=1), dict(by=1, bx=0)):
        with pytest.raises(ValueError):
            oracle.sor_block_f64(u0, 1.0, max_iters=1, **kw)


# --- the FP32 form ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 4, 11])
@pytest.mark.parametrize("with_f", [False, True])
@pytest.mark.parametrize("K", [1, 3])
def test_fp32_unit_blocks_are_red_black_fp32(n, with_f, K):
    """1 x 1 blocks in FP32 are the FP32 red-black oracle (pinned on its own), bit for bit."""
    u0 = wl.random_edges(n, seed=40 + n)
    f = wl.rng(41 + n).uniform(-50, 50, size=(n, n)) if with_f else None
    a = oracle.sor_f32(u0, 1.45, f=f, max_iters=300, check_every=K, tol=1e-4, trace=True)
    b = oracle.sor_block_f32(u0, 1.45, by=1, bx=1, f=f, max_iters=300, check_every=K, tol=1e-4, trace=True)
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["trace"], b["trace"])
    for key in ("iterations", "converged", "final_maxdelta"):
        assert a[key] == b[key], key


@pytest.mark.parametrize("by,bx", [(2, 3), (5, 5), (1, 7), (4, 2)])
def test_fp32_tracks_fp64_within_single_precision(by, bx):
    """The FP32 iterate stays within a few single-precision units (relative to the data) of the FP64 one
    of the same block ordering, itself pinned to the ordered SOR splitting."""
    n = 10
    u0 = wl.random_edges(n, seed=50)
    f = wl.rng(51).uniform(-100, 100, size=(n, n))
    for k in (1, 5, 40):
        a = oracle.sor_block_f64(u0, 1.5, by=by, bx=bx, f=f, max_iters=k, tol=-1.0)
        b = oracle.sor_block_f32(u0, 1.5, by=by, bx=bx, f=f, max_iters=k, tol=-1.0)
        scale = max(1.0, float(np.max(np.abs(a["u"]))))
        assert float(np.max(np.abs(a["u"] - b["u"]))) <= 64 * 2.0 ** -24 * scale * k


def test_fp32_converges_to_dense_solve_in_single_precision():
    n = 12
    u0 = wl.random_edges(n, seed=52)
    f = wl.rng(53).uniform(-100, 100, size=(n, n))
    out = oracle.sor_block_f32(u0, 1.5, by=3, bx=4, f=f, max_iters=5000, tol=1e-4)  # FP32 floor of the change: ~1e-5 at |u| ~ 100
    assert out["converged"]
    ref = pins.dense_solve(u0, f)
    assert float(np.max(np.abs(out["u"] - ref))) <= 1e-4 * max(1.0, float(np.max(np.abs(ref))))
