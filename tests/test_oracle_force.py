"""Pins of the oracle's link derivative of S = chi^dagger P(K) chi."""
import numpy as np
import pytest

from oracle import chebyshev, force
from paper_1510_06897_gb300 import inputs

DIMS = (3, 2, 4, 2)


@pytest.mark.parametrize("antiperiodic", [False, True])
def test_gradient_tangent_and_fd_agree(antiperiodic):
    links = inputs.gauge_links(DIMS, seed=3101)
    chi = inputs.gaussian_source(DIMS, seed=3102)[0]
    x_dir = inputs.su3_directions(DIMS, seed=inputs.SEED_DIRECTIONS)
    a, b, order = 0.4, 6.6, 8
    c = chebyshev.coefficients(order, a, b)
    grad = force.gradient(links, chi, c, a, b, antiperiodic_t=antiperiodic)
    # the gradient lies in su(3)
    herm = grad + np.conj(np.swapaxes(grad, -1, -2))
    assert np.max(np.abs(herm)) < 1e-12
    assert np.max(np.abs(np.trace(grad, axis1=-2, axis2=-1))) < 1e-12
    from_grad = np.sum(np.einsum("...ab,...ab->...", x_dir.conj(), grad)).real
    tangent = force.directional_derivative(links, chi, c, a, b, x_dir, antiperiodic_t=antiperiodic)
    fd = force.finite_difference(links, chi, c, a, b, x_dir, eps=1e-3, antiperiodic_t=antiperiodic)
    scale = abs(fd)
    assert abs(tangent - fd) < 1e-8 * scale
    assert abs(from_grad - fd) < 1e-8 * scale
    assert abs(from_grad - tangent) < 1e-11 * scale


def test_gradient_single_link_direction():
    """A direction supported on one link in t picks out that link's gradient."""
    links = inputs.gauge_links(DIMS, seed=3201)
    chi = inputs.gaussian_source(DIMS, seed=3202)[0]
    a, b, order = 0.4, 6.6, 5
    c = chebyshev.coefficients(order, a, b)
    grad = force.gradient(links, chi, c, a, b)
    x_dir = np.zeros_like(links)
    x_dir[3, 1, 2, 1, 0] = inputs.su3_directions((1, 1, 1, 1), seed=5)[0, 0, 0, 0, 0]
    want = force.finite_difference(links, chi, c, a, b, x_dir, eps=1e-3)
    got = np.sum(np.einsum("...ab,...ab->...", x_dir.conj(), grad)).real
    assert abs(got - want) < 1e-8 * abs(want)
