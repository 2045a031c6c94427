"""The FP64 rate probe (sor_diag_fp64_rate): the measured peak the FP64 colour
phases are reported against.  It must report a rate of the right order for
a GPU of 152 SMs with 2 FP64 lanes per clock each (6.3e11 lane operations/s
at 2.07 GHz): positive, not above the nominal rate by more than the clock
could explain, and refuse unknown kinds."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_0763_gb300 import _build, capi
    _build.build()
    c = capi.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_fp64_rate_probe_reports_a_plausible_rate(ctx, kind):
    props = torch.cuda.get_device_properties(0)
    rate = ctx.diag_fp64_rate(kind)
    # at most 2 FP64 lanes per clock per SM at a clock of at most 2.2 GHz
    # (an upper bound for GB300; other parts need not pass this check)
    assert 0.0 < rate <= props.multi_processor_count * 2 * 2.2e9 * 1.05, rate


def test_fp64_rate_probe_rejects_unknown_kind(ctx):
    from paper_1401_0763_gb300 import capi
    with pytest.raises(capi.SorError):
        ctx.diag_fp64_rate(2)
