"""SignPolyQuad (torch.autograd.Function) for S = chi^dagger P(K) chi, P(K) the
undeflated polynomial of Eq. 3: its value and the gradients torch.autograd
returns for the links (the su(3) link derivative) and for chi (2 P(K) chi),
against the FP64 oracle's action, reverse sweep, polynomial and Richardson
finite differences."""
import numpy as np
import pytest

from oracle import chebyshev, force
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.autograd import sign_poly_quad
from tests.gpu_util import dev, host, need_gpu, rel, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("antiperiodic", [False, True])
def test_value_and_gradients_match_the_oracle(prec, tol, antiperiodic):
    dims = (4, 2, 4, 2)
    order, a, b = 17, 0.4, 6.6
    links = inputs.gauge_links(dims, seed=7301)
    chi = inputs.gaussian_source(dims, seed=7302)
    cf = chebyshev.coefficients(order, a, b)
    s_want = force.action(links, chi[0], cf, a, b, antiperiodic_t=antiperiodic)
    g_want = force.gradient(links, chi[0], cf, a, b, antiperiodic_t=antiperiodic)
    p_chi = chebyshev.poly_apply(links, chi[0], cf, a, b, antiperiodic_t=antiperiodic)

    lt = dev(links).requires_grad_(True)
    ct = dev(chi if prec == "fp64" else chi.astype(np.complex64)).requires_grad_(True)
    s = sign_poly_quad(lt, ct, dims, order, a, b, prec=prec, antiperiodic_t=antiperiodic)
    assert s.dtype == torch.float64 and s.dim() == 0
    assert abs(s.item() - s_want) < tol * abs(s_want)
    # a scaled loss: the incoming gradient multiplies both results
    g_links, g_chi = torch.autograd.grad(3.0 * s, [lt, ct])
    assert rel(host(g_links) / 3.0, g_want) < tol
    assert rel(host(g_chi)[0] / 6.0, p_chi) < tol


def test_link_gradient_against_finite_differences_4x4():
    """Sum Re tr(X^dagger F) with F from backward equals the oracle's Richardson
    central difference of S along two random su(3) directions (4^4, order 32)."""
    dims = (4, 4, 4, 4)
    order, a, b = 32, 0.4, 6.5
    links = inputs.gauge_links(dims, seed=7401)
    chi = inputs.gaussian_source(dims, seed=7402)
    cf = chebyshev.coefficients(order, a, b)
    lt = dev(links).requires_grad_(True)
    s = sign_poly_quad(lt, dev(chi), dims, order, a, b)
    (g_links,) = torch.autograd.grad(s, [lt])
    grad = host(g_links)
    for seed in (inputs.SEED_DIRECTIONS + 10, inputs.SEED_DIRECTIONS + 11):
        x_dir = inputs.su3_directions(dims, seed=seed)
        from_grad = np.sum(np.einsum("...ab,...ab->...", x_dir.conj(), grad)).real
        fd = force.finite_difference(links, chi[0], cf, a, b, x_dir, eps=1e-3)
        assert abs(from_grad - fd) < 1e-8 * abs(fd)


def test_chi_gradient_passes_gradcheck():
    """torch.autograd.gradcheck of S as a function of chi alone (FP64, 2^4):
    the backward gradient against torch's own finite differences."""
    dims = (2, 2, 2, 2)
    links = dev(inputs.gauge_links(dims, seed=7501))
    chi = dev(inputs.gaussian_source(dims, seed=7502)).requires_grad_(True)

    def f(x):
        return sign_poly_quad(links, x, dims, 12, 0.45, 6.6)

    assert torch.autograd.gradcheck(f, (chi,), eps=1e-6, atol=1e-7, rtol=1e-6, fast_mode=True)


def test_no_gradient_requested_still_returns_the_value():
    dims = (4, 2, 4, 2)
    links = inputs.gauge_links(dims, seed=7601)
    chi = inputs.gaussian_source(dims, seed=7602)
    cf = chebyshev.coefficients(9, 0.4, 6.6)
    with torch.no_grad():
        s = sign_poly_quad(dev(links), dev(chi), dims, 9, 0.4, 6.6)
    assert abs(s.item() - force.action(links, chi[0], cf, 0.4, 6.6)) < 1e-12 * abs(s.item())
