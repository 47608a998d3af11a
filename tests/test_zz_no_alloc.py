"""ov_wilson_noalloc: D_W for callers that cannot allocate device memory (for
example code living inside a framework whose memory pool owns the whole GPU).
It keeps its packed copies in one fixed device array of the library instead
of allocating, and must give the same result as ov_wilson on an FP64
context.  Two calls in a row with different inputs check that nothing left in
the shared array from the previous call leaks into the next result."""
import numpy as np
import pytest

from oracle import wilson
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, OverlapError, ov_last_error, ov_wilson_noalloc
from tests.gpu_util import dev, host, need_gpu, rel, torch

pytestmark = pytest.mark.gpu

TOL = 1e-13  # FP64 stencil tolerance of the other GPU tests


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _reference(dims, links, psi, antiperiodic):
    with Ctx(dims, dev(links), "fp64", antiperiodic_t=antiperiodic) as c:
        return host(c.wilson(dev(psi)))


def test_noalloc_matches_ov_wilson_twice():
    cases = [((8, 8, 8, 8), False, 1, np.complex128, 9001),
             ((6, 4, 4, 10), True, 2, np.complex64, 9002)]
    for dims, antiperiodic, nrhs, dtype, seed in cases:
        links = inputs.gauge_links(dims, seed=seed)
        psi = inputs.gaussian_source(dims, seed=seed + 1, nrhs=nrhs).astype(dtype)
        want = _reference(dims, links, psi, antiperiodic)
        out = torch.empty(psi.shape, dtype=torch.complex128 if dtype == np.complex128 else torch.complex64,
                          device="cuda")
        ov_wilson_noalloc(dims, dev(links), dev(psi), out, nrhs, antiperiodic_t=antiperiodic)
        got = host(out)
        tol = TOL if dtype == np.complex128 else 1e-6
        assert rel(got, want) < tol
        # and against the oracle directly
        oracle_out = np.stack([wilson.wilson(links, p.astype(np.complex128), antiperiodic) for p in psi])
        assert rel(got, oracle_out) < tol


def test_noalloc_rejects_oversize_and_host_memory():
    dims = (16, 16, 16, 16)  # 65536 sites: beyond the 32 MiB scratch
    links = torch.zeros((4, 16, 16, 16, 16, 3, 3), dtype=torch.complex128, device="cuda")
    psi = torch.zeros((1, 16, 16, 16, 16, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(OverlapError) as e:
        ov_wilson_noalloc(dims, links, psi, torch.empty_like(psi), 1)
    assert e.value.status == 1 and "32 MiB" in ov_last_error(None)
    small = (4, 4, 4, 4)
    lk = inputs.gauge_links(small, seed=9003)
    ps = inputs.gaussian_source(small, seed=9004)
    with pytest.raises(OverlapError):
        ov_wilson_noalloc(small, lk, ps, np.empty_like(ps), 1)  # host arrays
