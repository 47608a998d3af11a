"""Pins of the oracle's Chebyshev polynomial and deflated sign(K) (Eq. 3)."""
import numpy as np
import pytest

from oracle import chebyshev, dense, overlap, wilson
from paper_1510_06897_gb300 import inputs
from tests.oracle_fixtures import DIMS_4, field_shape, small_problem


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("order,a,b", [(8, 0.5, 6.5), (64, 0.3, 6.5), (200, 0.05, 7.0)])
def test_coefficients_interpolate_at_nodes(order, a, b):
    """f_N equals y^{-1/2} at the N + 1 Chebyshev-Gauss nodes (interpolation)."""
    c = chebyshev.coefficients(order, a, b)
    n1 = order + 1
    x = np.cos(np.pi * (np.arange(n1) + 0.5) / n1)
    y = ((b * b - a * a) * x + b * b + a * a) / 2
    assert np.max(np.abs(chebyshev.f_scalar(c, a, b, y) * np.sqrt(y) - 1)) < 1e-11


def test_sign_error_decays_geometrically():
    """The Chebyshev error of y^{-1/2} on [a^2, b^2] decays like rho^{-N},
    rho = (b + a)/(b - a) (the Bernstein ellipse through the pole at y = 0)."""
    a, b = 0.5, 6.5
    rho = (b + a) / (b - a)
    errs = [chebyshev.sign_error(chebyshev.coefficients(n, a, b), a, b) for n in (16, 32, 48)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 0.5 * rho ** 16 < r1 < 2 * rho ** 16
    assert 0.5 * rho ** 16 < r2 < 2 * rho ** 16


@pytest.mark.parametrize("n", [(1, 0, 0, 0), (0, 2, 1, 3), (2, 2, 2, 2)])
def test_free_field_polynomial_closed_form(n):
    """U = 1: K(p)^2 = (A^2 + s^2) 1 is scalar, so P(K) psi_p = f_N(A^2 + s^2) K(p) psi_p."""
    dims = DIMS_4
    rng = np.random.default_rng(3)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    p = [2 * np.pi * k / 4 for k in n]
    t, z, y, x = np.meshgrid(*(np.arange(4),) * 4, indexing="ij")
    psi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None, None] * u
    links = inputs.unit_links(dims)
    a, b, order = 0.5, 6.5, 24
    c = chebyshev.coefficients(order, a, b)
    got = chebyshev.poly_apply(links, psi, c, a, b)
    big_a = sum(1 - np.cos(pm) for pm in p) - wilson.M_W
    s2 = sum(np.sin(pm) ** 2 for pm in p)
    kp = wilson.GAMMA5 @ (big_a * np.eye(4) + 1j * sum(wilson.GAMMA[mu] * np.sin(p[mu]) for mu in range(4)))
    want = chebyshev.f_scalar(c, a, b, big_a ** 2 + s2) * np.einsum("st,...ta->...sa", kp, psi)
    assert _rel(got, want) < 1e-13


@pytest.fixture(scope="module")
def prob():
    return small_problem()


def test_polynomial_matches_spectral_form(prob):
    """Forward recurrence == V diag(lambda f_N(lambda^2)) V^dagger on the dense K."""
    order = 64
    c = chebyshev.coefficients(order, prob["a"], prob["b"])
    psi = inputs.gaussian_source(DIMS_4, seed=2001)[0]
    got = chebyshev.poly_apply(prob["links"], psi, c, prob["a"], prob["b"])
    w, v = np.linalg.eigh(prob["kmat"])
    pw = chebyshev.p_scalar(c, prob["a"], prob["b"], w)
    want = ((v * pw) @ (v.conj().T @ psi.ravel())).reshape(psi.shape)
    assert _rel(got, want) < 1e-12


def _cfg(prob, order=64):
    c = chebyshev.coefficients(order, prob["a"], prob["b"])
    return overlap.SignConfig(c, prob["a"], prob["b"], prob["evals"], prob["evecs"])


def test_sign_matches_dense_within_chebyshev_error(prob):
    """||S_cheb psi - sign(K) psi|| <= eps_cheb ||psi|| with sign(K) from eigh."""
    cfg = _cfg(prob)
    eps = chebyshev.sign_error(cfg.coeffs, cfg.a, cfg.b)
    psi = inputs.gaussian_source(DIMS_4, seed=2001)[0]
    got = overlap.sign_apply(prob["links"], psi, cfg)
    want = dense.apply_matrix(dense.exact_sign(prob["kmat"]), psi)
    err = np.linalg.norm(got - want) / np.linalg.norm(psi)
    assert err <= eps * 1.0001 + 1e-13
    assert err > 1e-3 * eps  # the approximation error is really there
    # with more terms the error shrinks accordingly
    cfg2 = _cfg(prob, order=128)
    got2 = overlap.sign_apply(prob["links"], psi, cfg2)
    assert np.linalg.norm(got2 - want) / np.linalg.norm(psi) < 1e-8


def test_deflated_modes_exact(prob):
    """sign(K) phi_i = sign(lambda_i) phi_i for the deflated eigenvectors."""
    cfg = _cfg(prob)
    for i in range(len(cfg.evals)):
        phi = cfg.evecs[i]
        got = overlap.sign_apply(prob["links"], phi, cfg)
        assert np.linalg.norm(got - np.sign(cfg.evals[i]) * phi) < 1e-12


def test_literal_equals_projected(prob):
    """Eq. 3 as printed == the projected form, for exact eigenvectors."""
    cfg = _cfg(prob)
    psi = inputs.gaussian_source(DIMS_4, seed=2002)[0]
    a = overlap.sign_apply(prob["links"], psi, cfg)
    b = overlap.sign_apply_literal(prob["links"], psi, cfg)
    assert _rel(a, b) < 1e-12


def test_sign_is_hermitian_and_involutive(prob):
    cfg = _cfg(prob, order=128)
    phi = inputs.gaussian_source(DIMS_4, seed=2003)[0]
    psi = inputs.gaussian_source(DIMS_4, seed=2004)[0]
    s_psi = overlap.sign_apply(prob["links"], psi, cfg)
    lhs = np.vdot(phi, s_psi)
    rhs = np.vdot(overlap.sign_apply(prob["links"], phi, cfg), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    s2 = overlap.sign_apply(prob["links"], s_psi, cfg)
    assert _rel(s2, psi) < 1e-8


@pytest.mark.parametrize("order,a,b", [(8, 0.3, 6.5), (40, 0.45, 6.5), (256, 0.2, 6.6)])
def test_coefficients_match_numpy_chebinterpolate(order, a, b):
    """The coefficients equal NumPy's interpolant at the Chebyshev points of
    the first kind in z (NumPy keeps c_0 whole; the oracle's series halves it)."""
    from numpy.polynomial import chebyshev as npcheb
    c = chebyshev.coefficients(order, a, b)
    f = lambda z: (((b * b - a * a) * z + b * b + a * a) / 2) ** -0.5  # noqa: E731
    want = npcheb.chebinterpolate(f, order)
    assert np.max(np.abs(c[1:] - want[1:])) < 1e-13
    assert abs(c[0] / 2 - want[0]) < 1e-13
