"""Input magnitudes and relaxation factors at the edges of the legal range.

Eq. 1 (Section 2.1) holds for any 0 < omega < 2 and any finite data.  The
FP64 default phases store each colour rescaled inside a chunk of iterations
(scale up to (4/omega)^(2L-2) on the plate, (6/omega)^(2L-2) on the cube),
so the chunk length they may use depends on how large the inputs are and on
omega; inputs near the top or the bottom of the normal range take the
exact-order phases.  Each case runs a chunk-sized iteration count through the
C ABI and compares with the oracle: exact order bit for bit, the default
path within 1e-12 (normwise), or bit for bit where it must have taken the
exact order.
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
def ctx_mc():
    """Context with the single-cluster path for small plates switched off, so
    the plate cases run the chunked multi-CTA kernels."""
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    c = capi.Context(0)
    c.set_option(capi.SOR_OPT_CLUSTER, 0)
    yield c
    c.close()


def capi_mod():
    from paper_1401_0763_gb300 import capi
    return capi


def on_device(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (name, ring scale, source scale or None, omega or None for omega_opt,
#  default path expected to take the exact order)
PLATE_CASES = [
    ("ring_1e200", 1e198, None, None, False),
    ("source_1e250", 1.0, 1e250, None, False),
    ("omega_1e-3", 1.0, 20.0, 1e-3, False),
    ("omega_1.999", 1.0, 20.0, 1.999, False),
    ("omega_1e-3_ring_1e250", 1e248, None, 1e-3, False),
    ("ring_1e300_exact", 1e298, None, None, True),
    ("ring_1e-300_exact", 1e-302, None, None, True),
]


@pytest.mark.parametrize("name,uscale,fscale,omega,exact_route", PLATE_CASES, ids=[c[0] for c in PLATE_CASES])
def test_plate_extreme_magnitudes(ctx_mc, name, uscale, fscale, omega, exact_route):
    capi = capi_mod()
    n = 300  # two column tiles, ragged strips
    iters = 200  # one chunk as long as the omega-only cap allows (197 at omega_opt)
    u0 = wl.random_edges(n, 41) * uscale
    f = wl.gaussian_source(n, 42) * fscale if fscale is not None else None
    w = oracle.omega_opt(n) if omega is None else omega
    ref = oracle.sor_f64(u0, w, f=f, max_iters=iters, check_every=iters, tol=-1.0)
    assert np.all(np.isfinite(ref["u"]))
    out, res = ctx_mc.solve(on_device(u0), on_device(f), omega=w, tol=-1.0, max_iters=iters, check_every=iters,
                            flags=capi.SOR_FLAG_EXACT_ORDER)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert res["iterations"] == iters
    assert np.array_equal(got, ref["u"])
    assert res["final_maxdelta"] == ref["final_maxdelta"]
    out, res = ctx_mc.solve(on_device(u0), on_device(f), omega=w, tol=-1.0, max_iters=iters, check_every=iters)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert res["iterations"] == iters
    assert np.all(np.isfinite(got)), name
    if exact_route:
        assert np.array_equal(got, ref["u"]), pins.rel_err(got, ref["u"])
        assert res["final_maxdelta"] == ref["final_maxdelta"]
    else:
        assert pins.rel_err(got, ref["u"]) <= TOL64, pins.rel_err(got, ref["u"])


def test_plate_extreme_host_buffers(ctx_mc):
    """The same guard when the inputs come from host memory (staged copies)."""
    n = 260
    iters = 150
    u0 = wl.random_edges(n, 43) * 1e198
    w = oracle.omega_opt(n)
    ref = oracle.sor_f64(u0, w, max_iters=iters, check_every=iters, tol=-1.0)
    got, res = ctx_mc.solve(np.ascontiguousarray(u0), None, omega=w, tol=-1.0, max_iters=iters, check_every=iters)
    assert res["iterations"] == iters and np.all(np.isfinite(got))
    assert pins.rel_err(got, ref["u"]) <= TOL64


CUBE_CASES = [
    ("ring_1e200", 1e198, None, None, False),
    ("source_1e250", 1.0, 1e250, None, False),
    ("omega_1e-3", 1.0, 20.0, 1e-3, False),
    ("omega_1.999", 1.0, None, 1.999, False),
    ("ring_1e300_unscaled_chunks", 1e298, None, None, False),  # room for L = 1 (no scale) only
    ("ring_1e303_exact", 1e301, None, None, True),
]


@pytest.mark.parametrize("name,uscale,fscale,omega,exact_route", CUBE_CASES, ids=[c[0] for c in CUBE_CASES])
def test_cube_extreme_magnitudes(name, uscale, fscale, omega, exact_route):
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    n = 40
    iters = 120  # longer than the chunk the guard allows for the large inputs (omega-only cap: 118)
    u0 = wl.random_shell(n, 44) * uscale
    f = wl.gaussian_source3(n, 45) * fscale if fscale is not None else None
    w = oracle.omega_opt(n) if omega is None else omega
    ref = oracle.sor3d_f64(u0, w, f=f, max_iters=iters, check_every=iters, tol=-1.0)
    assert np.all(np.isfinite(ref["u"]))
    with capi.Context(0) as ctx:
        out, res = ctx.solve3d(on_device(u0), on_device(f), omega=w, tol=-1.0, max_iters=iters, check_every=iters,
                               precision=capi.SOR_FP64, flags=capi.SOR_FLAG_EXACT_ORDER)
        got = out.cpu().numpy()
        assert res["iterations"] == iters and np.array_equal(got, ref["u"])
        out, res = ctx.solve3d(on_device(u0), on_device(f), omega=w, tol=-1.0, max_iters=iters, check_every=iters,
                               precision=capi.SOR_FP64)
        got = out.cpu().numpy()
    assert res["iterations"] == iters and np.all(np.isfinite(got)), name
    if exact_route:
        assert np.array_equal(got, ref["u"]), pins.rel_err3(got, ref["u"])
    else:
        assert pins.rel_err3(got, ref["u"]) <= TOL64, pins.rel_err3(got, ref["u"])
