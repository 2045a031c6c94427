"""Accuracy of the precision workload's solution against the exact discrete
solution (DST-I fast Poisson solve of the same 5-point system): the 4098^2
Poisson plate with the 8-Gaussian source, FP32 inner sweeps inside FP64
defect correction, stopped at a relative residual of 1e-8.  The residual
stop bounds the error only through the condition number (about 7e6 here),
so the bar is empirical: the stored FP64 solution is expected within 1e-9
of the exact discrete one (measured: a few 1e-12)."""
import numpy as np
import pytest

from paper_1401_0763_gb300 import workloads as wl
from tests import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_poisson4096_refine_error_against_exact_solution():
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    n = 4096
    u0, f = wl.poisson_problem(n, 0)
    exact = pins.dst_solve(u0, f)
    with capi.Context(0) as ctx:
        out, res = ctx.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(f).cuda(),
                             precision=capi.SOR_FP32_REFINE, omega=capi.sor_omega_opt(n), tol=1e-8,
                             max_iters=400000, inner_sweeps=20, stall_window=50)
        got = out.cpu().numpy()
    assert res["converged"] and res["final_resid_rel"] < 1e-8
    err = pins.rel_err(got, exact)
    print(f"relative error against the DST-I solution: {err:.3e}")
    assert err < 1e-9
