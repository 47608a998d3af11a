"""The failure path of the two kernels that wait on their own asynchronous
work, exercised without any fault: with ov_test_wait_expiry, each wait of
their copy / MMA pipelines first waits (for 20000 cycles) on a device flag
that nothing sets, so it runs out.  The kernel then records its error flag,
drains its own copies and MMAs with the normal bound, frees its tensor memory
and returns; the call must report OV_ERR_CUDA, and the next call on the same
context, with the hook off, must give the result of a context that never
failed."""
import numpy as np
import pytest

from oracle import chebyshev, overlap, wilson
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import OV_ERR_CUDA, Ctx, OverlapError, ov_last_error, ov_test_wait_expiry
from tests.gpu_util import dev, host, need_gpu, rel, torch
from tests.oracle_fixtures import field_shape

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _orthonormal(dims, n, seed):
    rng = np.random.default_rng(seed)
    vol = inputs.volume(dims)
    m = rng.standard_normal((12 * vol, n)) + 1j * rng.standard_normal((12 * vol, n))
    q, _ = np.linalg.qr(m)
    return np.ascontiguousarray(q.T).reshape((n,) + field_shape(dims))


def test_tensor_core_projection_gives_up_and_recovers():
    """sign(K) of 4 right-hand sides on an FP32 context (deflation projection on
    the tensor cores), 8^4, 6 orthonormal deflation vectors, order 16."""
    dims = (8, 8, 8, 8)
    links = inputs.gauge_links(dims, seed=9701)
    psi = inputs.gaussian_source(dims, seed=9702, nrhs=4)
    evecs = _orthonormal(dims, 6, 9703)
    evals = np.array([0.5, -0.52, 0.55, -0.57, 0.6, -0.61])
    a, b, order = 0.65, 6.6, 16
    with Ctx(dims, dev(links), "fp32") as c:
        c.sign_config(order, a, b, evals, dev(evecs))
        want = c.sign(dev(psi))
        launches = c.stats()["tc_gemm_launches"]
        assert launches >= 1  # the projection ran on the tensor cores
        ov_test_wait_expiry(c.handle, 20000)
        with pytest.raises(OverlapError) as e:
            c.sign(dev(psi))
        assert e.value.status == OV_ERR_CUDA and "bounded wait" in ov_last_error(c.handle)
        ov_test_wait_expiry(c.handle, 0)
        again = c.sign(dev(psi))
        assert c.stats()["tc_gemm_launches"] == launches + 2
    assert torch.equal(want, again)
    cfg = overlap.SignConfig(chebyshev.coefficients(order, a, b), a, b, evals, evecs)
    ref = np.stack([overlap.sign_apply(links, p, cfg) for p in psi])
    assert rel(host(again), ref) < 1e-5


def test_slab_stencil_gives_up_and_recovers(monkeypatch):
    """D_W through the slab kernel (FP16, 8 x 4 x 4 x 6: one 32-site plane per
    item, bulk copies into the shared-memory ring)."""
    monkeypatch.setenv("OV_STENCIL", "slab")
    dims = (8, 4, 4, 6)
    links = inputs.gauge_links(dims, seed=9711)
    psi = inputs.gaussian_source(dims, seed=9712, nrhs=2)
    with Ctx(dims, dev(links), "fp16") as c:
        assert c.stats()["stencil_slab"] > 0
        want = c.wilson(dev(psi))
        ov_test_wait_expiry(c.handle, 20000)
        with pytest.raises(OverlapError) as e:
            c.wilson(dev(psi))
        assert e.value.status == OV_ERR_CUDA and "bulk copy" in ov_last_error(c.handle)
        ov_test_wait_expiry(c.handle, 0)
        again = c.wilson(dev(psi))
    assert torch.equal(want, again)
    ref = np.stack([wilson.wilson(links, p) for p in psi])
    assert rel(host(again), ref) < 2e-3
