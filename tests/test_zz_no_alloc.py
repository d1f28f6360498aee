"""The allocation-free totals entry point (alb_totals_noalloc).

Some callers cannot allocate device memory (another component owns every
allocation, or cudaMalloc is not allowed where they run). alb_totals_noalloc
gives them the global totals of caller-owned conserved fields with scratch
taken from a static device array. This file checks, through the C ABI, that
two calls in a row agree with alb_totals (which uses handle-owned scratch) on
the same state, and that sizes beyond the static scratch are refused before
anything is launched. It is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12  # same tolerance as the totals tests of the parity suite


@pytest.fixture(scope="module")
def alb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13426_gb300 import alb as A
    A.lib()
    return A


@pytest.mark.parametrize("nx,ny,precision", [(300, 300, 0), (270, 260, 1), (1, 1, 0)])
def test_noalloc_totals_match_alb_totals_twice(alb, nx, ny, precision):
    fields = flows.isentropic_vortex(nx, ny, radius=max(1.5, min(nx, ny) / 15), mach=0.8)
    fl = alb.Flow(nx, ny, precision=precision)
    fl.init(*fields)
    fl.step(4)
    fl.sync()
    ref = fl.totals()
    n = nx * ny
    dev = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4)]
    alb.alb_moments(fl.h, dev)
    fl.sync()
    for _ in range(2):  # the second call reuses the scratch the first one left
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        alb.alb_totals_noalloc(*dev, n, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=TOL, atol=0)
    fl.close()


def test_noalloc_totals_refuses_oversized_input(alb):
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(alb.AlbError) as ei:
        alb.alb_totals_noalloc(x, x, x, x, 4096 * 65536 + 1, out)
    assert ei.value.code == alb.ALB_EINVAL
    assert "exceeds" in alb.alb_last_error()
    with pytest.raises(alb.AlbError):
        alb.alb_totals_noalloc(x, x, x, x, -1, out)
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == 0).all()  # nothing was launched
