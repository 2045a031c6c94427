"""Continuous batching through sor_batch_submit / sor_poll / sor_wait.

Each request's result must be the same alone (sor_solve) and in the mix,
bit for bit: slots never interact and every slot runs the same arithmetic
as a lone solve.  A small budget forces queueing and admission as memory
frees up.
"""
import numpy as np
import pytest

import oracle
from paper_1401_0763_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def capi_mod():
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    return capi


def make_requests(capi, seed=0, count=14):
    g = wl.rng(seed)
    reqs = []
    for k in range(count):
        n = int(g.integers(20, 260))
        kind = k % 7
        if kind < 5:
            u0 = wl.random_edges(n, seed * 100 + k)
            f = wl.gaussian_source(n, seed * 100 + k + 1)
            kw = dict(precision=capi.SOR_FP32_REFINE, omega=oracle.omega_opt(n),
                      tol=float(np.exp(g.uniform(np.log(1e-10), np.log(1e-6)))), max_iters=20000,
                      inner_sweeps=20)
        elif kind == 5:
            u0, f = wl.heat_plate(n, 100.0), None
            kw = dict(precision=capi.SOR_FP64, omega=oracle.omega_opt(n), tol=1e-8, max_iters=3000, check_every=3,
                      flags=capi.SOR_FLAG_EXACT_ORDER)
        else:
            u0, f = wl.random_edges(n, k), None
            kw = dict(precision=capi.SOR_FP32, omega=oracle.omega_opt(n), tol=1e-3, max_iters=400, check_every=10)
        reqs.append((u0, f, kw))
    return reqs


@pytest.mark.parametrize("budget_mb", [0, 24])
def test_alone_equals_in_the_mix(budget_mb):
    capi = capi_mod()
    reqs = make_requests(capi, seed=budget_mb)
    alone = []
    with capi.Context(0) as solo:
        for u0, f, kw in reqs:
            alone.append(solo.solve(u0, f, **kw))
    with capi.Context(0, budget_bytes=budget_mb << 20) as ctx:
        tickets = [ctx.submit(u0, f, **kw) for u0, f, kw in reqs]
        for (t, out), (ref, rres), (u0, f, kw) in zip(tickets, alone, reqs):
            st, res = ctx.wait(t, 120.0)
            assert st == capi.SOR_OK, (st, ctx.last_error())
            assert res["iterations"] == rres["iterations"] and res["converged"] == rres["converged"]
            assert res["outer_steps"] == rres["outer_steps"]
            assert np.array_equal(out, ref), kw
            assert res["final_resid_rel"] == rres["final_resid_rel"]
            if kw["precision"] == capi.SOR_FP32_REFINE:
                assert res["converged"] and res["final_resid_rel"] < kw["tol"]
        st = ctx.stats()
        assert st["batch_completed"] == len(reqs)
        if budget_mb:
            assert st["bytes_peak"] <= budget_mb << 20


def test_device_buffers_and_late_arrivals():
    capi = capi_mod()
    with capi.Context(0) as ctx:
        n = 300
        u0, f = wl.poisson_problem(n, 9)
        big_t, big_out = ctx.submit(torch.from_numpy(u0).cuda(), torch.from_numpy(f).cuda(),
                                    precision=capi.SOR_FP32_REFINE, omega=oracle.omega_opt(n), tol=1e-10,
                                    max_iters=50000)
        # requests arriving while the first is on the device
        small = []
        for k in range(5):
            m = 40 + 10 * k
            a, b = wl.poisson_problem(m, k)
            small.append((ctx.submit(a, b, precision=capi.SOR_FP32_REFINE, omega=oracle.omega_opt(m), tol=1e-9,
                                     max_iters=50000), a, b, m))
        for (t, out), a, b, m in small:
            st, res = ctx.wait(t, 60.0)
            assert st == capi.SOR_OK
            ref = oracle.refine(a, oracle.omega_opt(m), f=b, inner_sweeps=20, tol=1e-9, max_outer=2500)
            assert np.array_equal(out, ref["u"]) and res["outer_steps"] == ref["outer_steps"]
        st, res = ctx.wait(big_t, 120.0)
        assert st == capi.SOR_OK and res["converged"]
        torch.cuda.synchronize()
        ref = oracle.refine(u0, oracle.omega_opt(n), f=f, inner_sweeps=20, tol=1e-10, max_outer=2500)
        assert np.array_equal(big_out.cpu().numpy(), ref["u"])


def test_ticket_errors_and_timeouts():
    capi = capi_mod()
    with capi.Context(0) as ctx:
        st, _ = ctx.poll(12345)
        assert st == capi.SOR_ERR_UNKNOWN_TICKET
        n = 1024
        u0, f = wl.poisson_problem(n, 2)
        t, out = ctx.submit(u0, f, precision=capi.SOR_FP32_REFINE, omega=oracle.omega_opt(n), tol=1e-12,
                            max_iters=200000)
        st, _ = ctx.wait(t, 0.001)
        assert st == capi.SOR_ERR_TIMEOUT
        st, _ = ctx.poll(t)
        assert st in (capi.SOR_NOT_READY, capi.SOR_OK)
        st, res = ctx.wait(t, 300.0)
        assert st == capi.SOR_OK
        st, _ = ctx.poll(t)  # collected once: unknown now
        assert st == capi.SOR_ERR_UNKNOWN_TICKET
        # a request larger than the whole budget is refused at submit
    with capi.Context(0, budget_bytes=1 << 20) as small:
        with pytest.raises(capi.SorError) as e:
            small.submit(*wl.poisson_problem(512, 0), precision=capi.SOR_FP32_REFINE)
        assert e.value.status == capi.SOR_ERR_BUDGET


def test_destroy_with_pending_work():
    capi = capi_mod()
    ctx = capi.Context(0)
    n = 2048
    u0, f = wl.poisson_problem(n, 3)
    for _ in range(3):
        ctx.submit(u0, f, precision=capi.SOR_FP32_REFINE, omega=oracle.omega_opt(n), tol=1e-12, max_iters=100000)
    ctx.close()  # cancels queued and running work, frees everything
    # the device is still usable
    with capi.Context(0) as again:
        out, res = again.solve(wl.heat_plate(16, 1.0), tol=1e-8)
        assert res["converged"]


@pytest.mark.parametrize("family,depth", [(1, 2), (1, 6), (2, 2), (2, 3), (2, 5)])
def test_mixed_inner_sweeps_share_the_fused_sweeps(family, depth):
    """Slots with different inner sweep counts in one batch: the fused sweeps
    run for the largest count, each slot stops at its own (the kernel takes
    min(depth, inner - sweep) per slot) and its correction is read from the
    buffer its own count ends in; every result equals the oracle's defect
    correction with that slot's count, bit for bit."""
    capi = capi_mod()
    counts = [7, 20, 13, 1, 4, 20, 9]
    with capi.Context(0) as ctx:
        ctx.set_option(capi.SOR_OPT_FUSED_KERNEL, family)
        ctx.set_option(capi.SOR_OPT_TEMPORAL_DEPTH, depth)
        jobs = []
        for k, inner in enumerate(counts):
            n = 60 + 37 * k
            u0, f = wl.poisson_problem(n, 40 + k)
            u0 = u0 + wl.random_edges(n, 50 + k)
            w = oracle.omega_opt(n)
            t, out = ctx.submit(u0, f, precision=capi.SOR_FP32_REFINE, omega=w, tol=1e-9, max_iters=60000,
                                inner_sweeps=inner)
            jobs.append((t, out, u0, f, w, inner))
        for t, out, u0, f, w, inner in jobs:
            st, res = ctx.wait(t, 300.0)
            assert st == capi.SOR_OK, ctx.last_error()
            ref = oracle.refine(u0, w, f=f, inner_sweeps=inner, tol=1e-9, max_outer=60000 // inner)
            assert res["outer_steps"] == ref["outer_steps"] and bool(res["converged"]) == ref["converged"]
            assert np.array_equal(out, ref["u"]), inner


@pytest.mark.parametrize("step", [0, 5, 64])
def test_plain_step_length_changes_no_result(step):
    """Plain (FP64 exact-order and FP32) batch slots step a number of
    iterations per scheduler round that is tuned online (step 0: 8, 16, 32, 64
    tried, the fastest kept) or fixed by SOR_OPT_BATCH_PLAIN_STEP; every slot
    stops on the device at its own tested iteration, so results equal the
    lone solves bit for bit whatever the length."""
    capi = capi_mod()
    reqs = []
    for k in range(12):
        n = 50 + 23 * k
        if k % 2:
            reqs.append((wl.heat_plate(n, 100.0), dict(precision=capi.SOR_FP64, omega=oracle.omega_opt(n), tol=1e-7,
                                                       max_iters=4000, check_every=3,
                                                       flags=capi.SOR_FLAG_EXACT_ORDER)))
        else:
            reqs.append((wl.random_edges(n, k), dict(precision=capi.SOR_FP32, omega=oracle.omega_opt(n), tol=1e-3,
                                                     max_iters=3000, check_every=10)))
    with capi.Context(0) as solo:
        alone = [solo.solve(u0, None, **kw) for u0, kw in reqs]
    with capi.Context(0) as ctx:
        ctx.set_option(capi.SOR_OPT_BATCH_PLAIN_STEP, step)
        tickets = [ctx.submit(u0, None, **kw) for u0, kw in reqs]
        for (t, out), (ref, rres) in zip(tickets, alone):
            st, res = ctx.wait(t, 300.0)
            assert st == capi.SOR_OK, ctx.last_error()
            assert res["iterations"] == rres["iterations"] and res["converged"] == rres["converged"]
            assert np.array_equal(out, ref)
        used = ctx.stats()["batch_plain_step"]
        assert used == step if step else used in (8, 16, 32, 64)
