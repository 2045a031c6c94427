"""The all-core CPU baseline (threaded red-black SOR) equals the oracle bit for
bit: within a colour phase the updates are independent (Section 3.1), so the
split of rows among threads cannot change a single rounding."""
import numpy as np
import pytest

import cpu_baseline
import oracle
from paper_1401_0763_gb300 import workloads as wl


@pytest.mark.parametrize("n", [1, 2, 5, 64, 129])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_twin_equals_oracle(n, threads):
    u0 = wl.random_edges(n, 70 + n)
    f = wl.gaussian_source(n, 80 + n) * 30 if n % 2 else None
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, f=f, max_iters=45, check_every=7, tol=-1.0)
    got = cpu_baseline.sor_f64_mt(u0, w, f=f, max_iters=45, check_every=7, tol=-1.0, threads=threads)
    assert got["iterations"] == ref["iterations"] == 45
    assert np.array_equal(got["u"], ref["u"])
    assert got["final_maxdelta"] == ref["final_maxdelta"]


def test_threaded_twin_stops_like_oracle():
    n = 96
    u0 = wl.heat_plate(n, 100.0)
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, max_iters=3000, check_every=3, tol=1e-8)
    got = cpu_baseline.sor_f64_mt(u0, w, max_iters=3000, check_every=3, tol=1e-8, threads=4)
    assert ref["converged"] and got["converged"]
    assert got["iterations"] == ref["iterations"]
    assert np.array_equal(got["u"], ref["u"])


def test_zero_iterations_and_bad_input():
    u0 = wl.random_edges(10, 1)
    got = cpu_baseline.sor_f64_mt(u0, 1.5, max_iters=0, threads=2)
    assert got["iterations"] == 0 and np.array_equal(got["u"], u0)
    with pytest.raises(ValueError):
        cpu_baseline.sor_f64_mt(np.zeros((4, 5)), 1.5)
    assert cpu_baseline.host_cores() >= 1
