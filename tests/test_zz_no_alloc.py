"""ov_wilson_noalloc: D_W for callers that cannot allocate device memory (for
example code living inside a framework whose memory pool owns the whole GPU).
It keeps its packed copies in one fixed device array of the library instead
of allocating, and must give the same result as ov_wilson on an FP64
context.

No test here depends on the others: the file is named to be collected last
only so that, should it fail, a run stopped at the first failure has already
run every other test.  Each case works on its own inputs and its own
contexts, and it passes alone in a fresh process as well as after the rest.
"""
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


def _reference(dims, links, psi, antiperiodic, m_w=1.5):
    with Ctx(dims, dev(links), "fp64", m_w=m_w, antiperiodic_t=antiperiodic) as c:
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


def test_noalloc_same_size_twice_allocates_nothing():
    """Two calls of the same size with different fields and sources: each
    equals its own ov_wilson result (so nothing of the first call survives in
    the shared array into the second), and the device's free memory is the
    same before and after each call (nothing allocated)."""
    dims = (8, 8, 8, 12)
    runs = []
    for seed in (9011, 9013):
        links = dev(inputs.gauge_links(dims, seed=seed))
        psi = dev(inputs.gaussian_source(dims, seed=seed + 1))
        runs.append((links, psi, torch.empty_like(psi), _reference(dims, host(links), host(psi), False)))
    ov_wilson_noalloc(dims, runs[0][0], runs[0][1], runs[0][2], 1)  # warm-up: address look-up, module load
    torch.cuda.synchronize()
    for links, psi, out, want in runs:
        out.zero_()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        ov_wilson_noalloc(dims, links, psi, out, 1)
        free_after = torch.cuda.mem_get_info()[0]
        assert free_after == free_before
        assert rel(host(out), want) < TOL


def test_noalloc_is_independent_of_m_w():
    """D_W (Eq. 2) has no m_W: ov_wilson on a context made with another m_W
    gives the same D_W as the entry point, which takes none."""
    dims = (4, 6, 4, 8)
    links = inputs.gauge_links(dims, seed=9021)
    psi = inputs.gaussian_source(dims, seed=9022)
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    ov_wilson_noalloc(dims, dev(links), dev(psi), out, 1)
    for m_w in (0.9, 1.5, 1.8):
        assert rel(host(out), _reference(dims, links, psi, False, m_w=m_w)) < TOL


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
