"""GPU adjoint of S = chi^dagger P(K) chi against the oracle's reverse sweep and
against finite differences along random su(3) directions."""
import numpy as np
import pytest

from oracle import chebyshev, force
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, ov_set_grad_memory, ov_sign_poly_grad
from tests.gpu_util import dev, host, need_gpu, rel, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _gpu_grad(dims, links, chi, order, a, b, prec, antiperiodic=False, grad_mem=-1, kept=None):
    out = torch.zeros(links.shape, dtype=torch.complex128, device="cuda")
    with Ctx(dims, dev(links), prec, antiperiodic_t=antiperiodic) as c:
        ov_set_grad_memory(c.handle, grad_mem)
        ov_sign_poly_grad(c.handle, order, a, b, dev(chi), out)
        if kept is not None:
            assert c.stats()["grad_kept_terms"] == kept
    return host(out)


@pytest.mark.parametrize("order", [1, 2, 15, 16, 17, 40])
@pytest.mark.parametrize("antiperiodic", [False, True])
@pytest.mark.parametrize("keep_all", [True, False])
@pytest.mark.parametrize("dims", [(4, 2, 4, 2), (4, 4, 4, 2), (8, 4, 2, 2)])
def test_grad_matches_oracle(order, antiperiodic, keep_all, dims):
    """Both sweeps: every recurrence term kept (default allowance) and
    checkpoints every 16 terms with recomputation (allowance 0).  4x2x4x2 runs
    the per-site force kernel in both precisions; the shared-memory tiled one
    runs for FP64 (box 4x4x2x2) on 4x4x4x2 and 8x4x2x2 and for FP32 (box
    8x2x2x2: two blocks, the z and t faces wrapping onto the box) on 8x4x2x2."""
    links = inputs.gauge_links(dims, seed=7001)
    chi = inputs.gaussian_source(dims, seed=7002)
    a, b = 0.4, 6.6
    c = chebyshev.coefficients(order, a, b)
    want = force.gradient(links, chi[0], c, a, b, antiperiodic_t=antiperiodic)
    mem, kept = (-1, 2 * order + 1) if keep_all else (0, 2 * (order // 16 + 2))
    got = _gpu_grad(dims, links, chi, order, a, b, "fp64", antiperiodic, mem, kept)
    assert rel(got, want) < 1e-12
    got32 = _gpu_grad(dims, links, chi.astype(np.complex64), order, a, b, "fp32", antiperiodic, mem, kept)
    assert rel(got32, want) < 2e-5


def test_grad_sweeps_agree_8x8x8x8():
    """The kept-terms and recomputing sweeps run the same FP64 arithmetic on the
    same vectors, so their gradients agree to rounding (order 100, 8^4)."""
    dims = (8, 8, 8, 8)
    links = inputs.gauge_links(dims, seed=7201)
    chi = inputs.gaussian_source(dims, seed=7202)
    g_all = _gpu_grad(dims, links, chi, 100, 0.45, 6.5, "fp64", grad_mem=-1, kept=201)
    g_ck = _gpu_grad(dims, links, chi, 100, 0.45, 6.5, "fp64", grad_mem=0, kept=2 * (100 // 16 + 2))
    assert rel(g_all, g_ck) < 1e-13


def test_grad_finite_difference_4x4():
    """dS/deps along random su(3) directions from the GPU gradient equals central
    finite differences of the oracle's S (Richardson), 4^4, order 32."""
    dims = (4, 4, 4, 4)
    links = inputs.gauge_links(dims, seed=7101)
    chi = inputs.gaussian_source(dims, seed=7102)
    a, b, order = 0.4, 6.5, 32
    c = chebyshev.coefficients(order, a, b)
    grad = _gpu_grad(dims, links, chi, order, a, b, "fp64")
    for seed in (inputs.SEED_DIRECTIONS, inputs.SEED_DIRECTIONS + 1):
        x_dir = inputs.su3_directions(dims, seed=seed)
        from_grad = np.sum(np.einsum("...ab,...ab->...", x_dir.conj(), grad)).real
        fd = force.finite_difference(links, chi[0], c, a, b, x_dir, eps=1e-3)
        assert abs(from_grad - fd) < 1e-8 * abs(fd)
