"""Pins of the SUMR / GMRESR oracle (oracle/sumr.py) against brute force and
dense linear algebra:

  * for an exactly unitary matrix the SUMR iterate after k products equals
    the minimal residual iterate over the Krylov space (least squares on an
    explicit QR-orthonormalised Krylov basis), and 1/sqrt(s_k) equals the true
    relative residual;
  * the same for U = gamma5 sign(K) with the exact dense sign of a 2^3 x 4
    lattice, and the converged iterate solves the dense D[mu] x = b;
  * with the polynomial sign (not unitary) the normalised recursion still
    converges to the dense solve of the polynomial operator, and the stencil
    form (overlap_sumr) equals the dense-matrix form;
  * GCR with the identity preconditioner equals the minimal residual iterate
    of the matrix itself (GMRES), and with the exact inverse ends in one step;
  * GMRESR with a relaxed (low-order) inner sign converges to the dense
    solve of the accurate polynomial operator;
  * planted mistakes (a conjugated coefficient, a dropped shift term, the
    wrong sign of the shift, GCR without orthogonalisation) each fail one of
    these.
"""
import numpy as np
import pytest

import oracle.sumr as sumr_mod
from oracle import chebyshev, dense, overlap, sumr
from paper_1510_06897_gb300 import inputs
from tests.oracle_fixtures import small_problem

DIMS = (2, 2, 2, 4)
N_EV = 4


def _random_unitary(n, seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _min_res(a, b, k, krylov_op):
    """argmin over K_k(krylov_op, b) of |b - a x|, by least squares on an
    orthonormalised explicit Krylov basis."""
    cols = [b]
    for _ in range(k - 1):
        cols.append(krylov_op(cols[-1]))
    q, _ = np.linalg.qr(np.stack(cols, axis=1))
    y = np.linalg.lstsq(a @ q, b, rcond=None)[0]
    return q @ y


def _rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def _sumr_unitary_ok(n=64, seed=7):
    u = _random_unitary(n, seed)
    b = np.random.default_rng(seed + 1).standard_normal(n) + 0j
    for zeta in (-1.3, 0.4 + 0.2j, -1.05):
        a = u - zeta * np.eye(n)
        for k in (1, 2, 5, 12):
            x, it, est = sumr.sumr(lambda v: u @ v, zeta, b, k)
            want = _min_res(a, b, k, lambda v: u @ v)
            res = np.linalg.norm(b - a @ x) / np.linalg.norm(b)
            if it != k or _rel(x, want) > 1e-9 or abs(est - res) > 1e-9 * res:
                return False
    return True


def test_sumr_is_minimal_residual_for_unitary():
    assert _sumr_unitary_ok()


@pytest.fixture(scope="module")
def prob():
    return small_problem(dims=DIMS, n_ev=N_EV)


def _unitary_exact(prob):
    vol = inputs.volume(DIMS)
    return dense.gamma5_matrix(vol) @ dense.exact_sign(prob["kmat"])


def _sign_poly_matrix(prob, order):
    w, v = dense.sorted_eigh(prob["kmat"])
    c = chebyshev.coefficients(order, prob["a"], prob["b"])
    s = chebyshev.p_scalar(c, prob["a"], prob["b"], w)
    s[:N_EV] = np.where(w[:N_EV] >= 0, 1.0, -1.0)
    return (v * s) @ v.conj().T, c


def _source(seed):
    return inputs.gaussian_source(DIMS, seed=seed)[0]


def _exact_sign_ok(prob, mu=0.02):
    u = _unitary_exact(prob)
    n = u.shape[0]
    zeta = sumr.zeta_of(mu)
    b = _source(9401).ravel()
    rhs = 2.0 * b / (1.0 - mu)
    for k in (3, 8):
        x, _, est = sumr.sumr(lambda v: u @ v, zeta, rhs, k)
        want = _min_res(u - zeta * np.eye(n), rhs, k, lambda v: u @ v)
        if _rel(x, want) > 1e-9:
            return False
    d = 0.5 * ((1 + mu) * np.eye(n) + (1 - mu) * u)
    x, _, est = sumr.sumr(lambda v: u @ v, zeta, rhs, 500, 1e-12)
    return est <= 1e-12 and _rel(x, np.linalg.solve(d, b)) < 1e-9


def test_sumr_overlap_exact_sign(prob):
    assert _exact_sign_ok(prob)


def test_sumr_polynomial_sign_converges(prob):
    """Polynomial sign (order 16: U^dagger U - 1 ~ 0.2) with the normalised
    recursion: the iterate solves the dense polynomial D[mu] and the estimate
    tracks the true residual; the stencil form gives the same iterates."""
    mu = 0.05
    vol = inputs.volume(DIMS)
    smat, c = _sign_poly_matrix(prob, 16)
    u = dense.gamma5_matrix(vol) @ smat
    n = u.shape[0]
    assert np.linalg.norm(u.conj().T @ u - np.eye(n), 2) > 0.1
    b = _source(9402)
    zeta = sumr.zeta_of(mu)
    d = 0.5 * ((1 + mu) * np.eye(n) + (1 - mu) * u)
    x, it, est = sumr.sumr(lambda v: u @ v, zeta, 2.0 * b.ravel() / (1.0 - mu), 2000, 1e-11)
    res = np.linalg.norm(b.ravel() - d @ x) / np.linalg.norm(b)
    assert est <= 1e-11 and res <= 1e-10
    assert _rel(x, np.linalg.solve(d, b.ravel())) < 1e-8

    cfg = overlap.SignConfig(c, prob["a"], prob["b"], prob["evals"], prob["evecs"])
    for k in (1, 4, 9):
        xs, _, est_s = sumr.overlap_sumr(prob["links"], b, mu, cfg, k)
        xd, _, est_d = sumr.sumr(lambda v: u @ v, zeta, 2.0 * b.ravel() / (1.0 - mu), k)
        assert _rel(xs.ravel(), xd) < 1e-11
        assert abs(est_s - est_d) < 1e-11


def _gcr_identity_ok(n=50, seed=11):
    rng = np.random.default_rng(seed)
    a = 3.0 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for k in (1, 3, 7):
        x, it, _ = sumr.gcr(lambda v: a @ v, lambda r: r.copy(), b, 0.0, k)
        if it != k or _rel(x, _min_res(a, b, k, lambda v: a @ v)) > 1e-10:
            return False
    return True


def test_gcr_identity_preconditioner_is_gmres():
    assert _gcr_identity_ok()


def test_gcr_exact_preconditioner_one_step():
    rng = np.random.default_rng(12)
    n = 30
    a = 2.0 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    ainv = np.linalg.inv(a)
    b = rng.standard_normal(n) + 0j
    x, it, rel = sumr.gcr(lambda v: a @ v, lambda r: ainv @ r, b, 1e-12, 10)
    assert it == 1 and rel < 1e-12
    assert _rel(x, np.linalg.solve(a, b)) < 1e-12


def test_gmresr_relaxed_inner_matches_dense_solve(prob):
    """GMRESR on D[mu] with the order-40 sign, inner SUMR with the order-12
    sign (20% sign error) to 10%: converges to the dense solve of the
    order-40 operator."""
    mu = 0.05
    smat, c = _sign_poly_matrix(prob, 40)
    _, c_in = _sign_poly_matrix(prob, 12)
    vol = inputs.volume(DIMS)
    n = 12 * vol
    d = 0.5 * ((1 + mu) * np.eye(n) + (1 - mu) * dense.gamma5_matrix(vol) @ smat)
    cfg = overlap.SignConfig(c, prob["a"], prob["b"], prob["evals"], prob["evecs"])
    cfg_in = overlap.SignConfig(c_in, prob["a"], prob["b"], prob["evals"], prob["evecs"])
    b = _source(9403)
    x, outer, n_inner, res = sumr.gmresr_overlap(prob["links"], b, mu, cfg, cfg_in, 0.1, tol=1e-10)
    assert res <= 1e-10
    assert outer >= 2 and n_inner > outer
    assert _rel(x.ravel(), np.linalg.solve(d, b.ravel())) < 1e-8


# ---- planted mistakes -------------------------------------------------------

def test_planted_conjugated_coefficient_fails(monkeypatch):
    """<u, v> taken as <v, u> (conj(alpha) in place of alpha and so on)."""
    monkeypatch.setattr(sumr_mod, "inner", lambda u, v: np.vdot(v.ravel(), u.ravel()))
    assert not _sumr_unitary_ok()
    assert not _gcr_identity_ok()


def test_planted_dropped_shift_term_fails(monkeypatch):
    """D_{j+1} built without the zeta D_j term."""
    def bad(v, d, dt, m, zeta, rho, rho_t):
        return (v - m * dt) / rho, (dt - np.conj(m) * v) / rho_t
    monkeypatch.setattr(sumr_mod, "_divided_step", bad)
    assert not _sumr_unitary_ok()


def test_planted_shift_sign_fails(monkeypatch, prob):
    """zeta = +(1 + mu)/(1 - mu): the iterate no longer solves D[mu] x = b."""
    assert _exact_sign_ok(prob)
    monkeypatch.setattr(sumr_mod, "zeta_of", lambda mu: (1.0 + mu) / (1.0 - mu))
    mu = 0.1
    u = _unitary_exact(prob)
    n = u.shape[0]
    b = _source(9404).ravel()
    x, _, _ = sumr_mod.sumr(lambda v: u @ v, sumr_mod.zeta_of(mu), 2.0 * b / (1.0 - mu), 400, 1e-12)
    d = 0.5 * ((1 + mu) * np.eye(n) + (1 - mu) * u)
    assert _rel(x, np.linalg.solve(d, b)) > 1e-3


def test_planted_missing_orthogonalisation_fails(monkeypatch):
    """GCR without the Gram-Schmidt step against the kept directions."""
    monkeypatch.setattr(sumr_mod, "_orthogonalise", lambda c, u, us, cs: (c, u))
    assert not _gcr_identity_ok()
