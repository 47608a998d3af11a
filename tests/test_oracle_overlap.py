"""Pins of the oracle's D[mu] (Eq. 1) and CG on D^dagger D."""
import numpy as np
import pytest

from oracle import cg, chebyshev, dense, overlap
from paper_1510_06897_gb300 import inputs
from tests.oracle_fixtures import DIMS_4, field_shape, small_problem


def _cfg(prob, order):
    c = chebyshev.coefficients(order, prob["a"], prob["b"])
    return overlap.SignConfig(c, prob["a"], prob["b"], prob["evals"], prob["evecs"])


def _spectral_sign(prob, cfg):
    """Dense sign(K) of Eq. 3 built from the eigendecomposition: sign(lambda)
    on the deflated modes, P(lambda) = lambda f_N(lambda^2) on all others."""
    w, v = dense.sorted_eigh(prob["kmat"])
    n_ev = len(cfg.evals)
    s = chebyshev.p_scalar(cfg.coeffs, cfg.a, cfg.b, w)
    s[:n_ev] = np.where(w[:n_ev] >= 0, 1.0, -1.0)
    return (v * s) @ v.conj().T


@pytest.fixture(scope="module")
def prob():
    return small_problem()


def test_ginsparg_wilson_within_chebyshev_error(prob):
    """{gamma5, D} - 2 D gamma5 D = -1/2 gamma5 (S^2 - 1) at mu = 0, and
    ||S^2 - 1|| <= max_{a<=|l|<=b} |P(l)^2 - 1| (0 on deflated modes)."""
    cfg = _cfg(prob, 32)
    links = prob["links"]
    psi = inputs.gaussian_source(DIMS_4, seed=2101)[0]
    g5 = overlap.gamma5

    def d(v):
        return overlap.overlap(links, v, 0.0, cfg)

    lhs = g5(d(psi)) + d(g5(psi)) - 2 * d(g5(d(psi)))
    lam = np.linspace(cfg.a, cfg.b, 20001)
    bound = 0.5 * np.max(np.abs(chebyshev.p_scalar(cfg.coeffs, cfg.a, cfg.b, lam) ** 2 - 1))
    rel = np.linalg.norm(lhs) / np.linalg.norm(psi)
    assert rel <= bound * 1.0001 + 1e-13
    assert bound > 1e-6           # order 32: the violation is visible ...
    assert rel > 1e-3 * bound     # ... and the oracle really shows it
    cfg_hi = _cfg(prob, 128)

    def d_hi(v):
        return overlap.overlap(links, v, 0.0, cfg_hi)

    lhs_hi = g5(d_hi(psi)) + d_hi(g5(psi)) - 2 * d_hi(g5(d_hi(psi)))
    assert np.linalg.norm(lhs_hi) / np.linalg.norm(psi) < 1e-8


def test_overlap_adjoint(prob):
    """<phi, D psi> = <D^dagger phi, psi> and gamma5 D gamma5 = D^dagger."""
    cfg = _cfg(prob, 32)
    links = prob["links"]
    phi = inputs.gaussian_source(DIMS_4, seed=2102)[0]
    psi = inputs.gaussian_source(DIMS_4, seed=2103)[0]
    mu = 0.05
    lhs = np.vdot(phi, overlap.overlap(links, psi, mu, cfg))
    rhs = np.vdot(overlap.overlap_dag(links, phi, mu, cfg), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    g5 = overlap.gamma5
    a = g5(overlap.overlap(links, g5(psi), mu, cfg))
    b = overlap.overlap_dag(links, psi, mu, cfg)
    assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(b)


def test_sign_matches_spectral_construction(prob):
    """The operator sign_apply builds equals Eq. 3 evaluated on the dense spectrum."""
    cfg = _cfg(prob, 64)
    psi = inputs.gaussian_source(DIMS_4, seed=2104)[0]
    got = overlap.sign_apply(prob["links"], psi, cfg)
    want = dense.apply_matrix(_spectral_sign(prob, cfg), psi)
    assert np.linalg.norm(got - want) < 1e-12 * np.linalg.norm(want)


def test_spectrum_on_gw_circle():
    """Eigenvalues of D[mu] (columns of the oracle operator, 2^4) lie on the circle
    |z - (1+mu)/2| = (1-mu)/2 up to the Chebyshev error."""
    prob2 = small_problem((2, 2, 2, 2), seed=1500, n_ev=4)
    cfg = _cfg(prob2, 48)
    eps = chebyshev.sign_error(cfg.coeffs, cfg.a, cfg.b)
    mu = 0.1
    n = 12 * inputs.volume(prob2["dims"])
    shape = field_shape(prob2["dims"])
    dmat = np.empty((n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1
        dmat[:, k] = overlap.overlap(prob2["links"], e.reshape(shape), mu, cfg).ravel()
    z = np.linalg.eigvals(dmat)
    dist = np.abs(np.abs(z - 0.5 * (1 + mu)) - 0.5 * (1 - mu))
    assert np.max(dist) <= 0.5 * (1 - mu) * eps + 1e-12


def test_cg_matches_dense_solve(prob):
    """CG on D^dagger D x = D^dagger b agrees with a dense solve of the same system."""
    cfg = _cfg(prob, 16)
    mu = 0.1
    b = inputs.gaussian_source(DIMS_4, seed=2105)[0]
    x, iters, res = cg.cg_normal(prob["links"], b, mu, cfg, tol=1e-11, maxit=500)
    s = _spectral_sign(prob, cfg)
    vol = inputs.volume(DIMS_4)
    dmat = 0.5 * ((1 + mu) * np.eye(12 * vol) + (1 - mu) * dense.gamma5_matrix(vol) @ s)
    x_ref = np.linalg.solve(dmat, b.ravel()).reshape(b.shape)
    assert res <= 1e-11
    assert 10 < iters < 500
    assert np.linalg.norm(x - x_ref) < 1e-9 * np.linalg.norm(x_ref)
