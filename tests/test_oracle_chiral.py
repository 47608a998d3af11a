"""Pins of the oracle's chiral-sector normal operator (one sign function
application per CG iteration instead of two).  The identities are algebraic,
so they are checked on the 2^3 x 4 lattice (4 deflated pairs), where the
dense matrices are 384 x 384."""
import numpy as np
import pytest

from oracle import cg, chebyshev, dense, overlap
from paper_1510_06897_gb300 import inputs
from tests.oracle_fixtures import small_problem

DIMS = (2, 2, 2, 4)
N_EV = 4


def _problem():
    return small_problem(DIMS, n_ev=N_EV)


def _dense_overlap(smat, mu, vol):
    return 0.5 * ((1 + mu) * np.eye(12 * vol) + (1 - mu) * dense.gamma5_matrix(vol) @ smat)


def _proj_matrix(vol, chirality):
    g5 = dense.gamma5_matrix(vol)
    return 0.5 * (np.eye(12 * vol) + chirality * g5)


@pytest.mark.parametrize("chirality", [1, -1])
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_chiral_operator_equals_projected_normal_with_exact_sign(chirality, mu):
    """With the exact dense sign (S^2 = 1): A = P D^dagger D P, built here from
    dense matrices independently of the oracle's operator code."""
    prob = _problem()
    vol = inputs.volume(prob["dims"])
    s_exact = dense.exact_sign(prob["kmat"])
    d = _dense_overlap(s_exact, mu, vol)
    pm = _proj_matrix(vol, chirality)
    want_mat = pm @ d.conj().T @ d @ pm
    psi = inputs.gaussian_source(prob["dims"], seed=9101)[0]
    got = overlap.chiral_normal_op(prob["links"], psi, mu, None, chirality,
                                   sign=lambda v: dense.apply_matrix(s_exact, v))
    want = dense.apply_matrix(want_mat, psi)
    assert np.linalg.norm(got - want) < 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("chirality", [1, -1])
def test_chiral_operator_with_polynomial_sign_within_chebyshev_error(chirality):
    """With the order-64 polynomial sign the identity holds up to the sign's
    own error (S^2 - 1 on the spectrum), measured here directly."""
    prob = _problem()
    mu = 0.05
    cfg = overlap.SignConfig(chebyshev.coefficients(64, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    psi = overlap.chiral_project(inputs.gaussian_source(prob["dims"], seed=9102)[0], chirality)
    got = overlap.chiral_normal_op(prob["links"], psi, mu, cfg, chirality)
    want = overlap.chiral_project(overlap.normal_op(prob["links"], psi, mu, cfg), chirality)
    s2 = overlap.sign_apply(prob["links"], overlap.sign_apply(prob["links"], psi, cfg), cfg)
    eps = np.linalg.norm(s2 - psi) / np.linalg.norm(psi)       # |S^2 - 1| on this vector
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 0.25 * (1 - mu) ** 2 * eps * 1.01 + 1e-14
    assert err > 0.0


@pytest.mark.parametrize("chirality", [1, -1])
def test_chiral_cg_matches_dense_solve(chirality):
    prob = _problem()
    mu = 0.05
    cfg = overlap.SignConfig(chebyshev.coefficients(48, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    b = inputs.gaussian_source(prob["dims"], seed=9103)[0]
    x, it, res = cg.cg_chiral(prob["links"], b, mu, cfg, chirality, tol=1e-12)
    assert res <= 1e-12
    # dense: the operator's matrix on the sector, from the polynomial sign's spectral form
    vol = inputs.volume(prob["dims"])
    w, v = dense.sorted_eigh(prob["kmat"])
    n_ev = len(cfg.evals)
    s = chebyshev.p_scalar(cfg.coeffs, cfg.a, cfg.b, w)
    s[:n_ev] = np.where(w[:n_ev] >= 0, 1.0, -1.0)
    smat = (v * s) @ v.conj().T
    pm = _proj_matrix(vol, chirality)
    c0 = 0.25 * ((1 + mu) ** 2 + (1 - mu) ** 2)
    amat = c0 * pm + 0.5 * chirality * (1 - mu * mu) * pm @ smat @ pm
    pb = overlap.chiral_project(b, chirality).ravel()
    # A vanishes off the sector: solve on the sector's own indices
    idx = np.where(np.diag(pm).real > 0.5)[0]
    want = np.zeros_like(pb)
    want[idx] = np.linalg.solve(amat[np.ix_(idx, idx)], pb[idx])
    want = want.reshape(b.shape)
    assert np.linalg.norm(x - want) < 1e-9 * np.linalg.norm(want)
    assert np.allclose(overlap.chiral_project(x, -chirality), 0.0)


def test_chiral_coefficient_mistakes_are_caught(monkeypatch):
    """A planted sign error in the chirality term, or (1 - mu) for (1 + mu) in
    the diagonal, makes the exact-sign pin fail."""
    prob = _problem()
    vol = inputs.volume(prob["dims"])
    mu, chirality = 0.3, 1
    s_exact = dense.exact_sign(prob["kmat"])
    d = _dense_overlap(s_exact, mu, vol)
    pm = _proj_matrix(vol, chirality)
    psi = inputs.gaussian_source(prob["dims"], seed=9104)[0]
    want = dense.apply_matrix(pm @ d.conj().T @ d @ pm, psi)
    sgn_fn = lambda v: dense.apply_matrix(s_exact, v)  # noqa: E731

    def ok():
        got = overlap.chiral_normal_op(prob["links"], psi, mu, None, chirality, sign=sgn_fn)
        return np.linalg.norm(got - want) < 1e-12 * np.linalg.norm(want)

    assert ok()
    def flipped(links, psi_, mu_, cfg, chi, m_w=1.5, antiperiodic_t=False, sign=None):
        p = overlap.chiral_project(psi_, chi)
        return (0.25 * ((1 + mu_) ** 2 + (1 - mu_) ** 2) * p
                - 0.5 * chi * (1 - mu_ * mu_) * overlap.chiral_project(sign(p), chi))
    monkeypatch.setattr(overlap, "chiral_normal_op", flipped)
    assert not ok()

    def diag_swap(links, psi_, mu_, cfg, chi, m_w=1.5, antiperiodic_t=False, sign=None):
        p = overlap.chiral_project(psi_, chi)
        return (0.5 * (1 - mu_) ** 2 * p
                + 0.5 * chi * (1 - mu_ * mu_) * overlap.chiral_project(sign(p), chi))
    monkeypatch.setattr(overlap, "chiral_normal_op", diag_swap)
    assert not ok()
