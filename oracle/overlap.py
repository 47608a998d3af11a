"""Deflated sign(K) and the overlap operator, FP64 (test infrastructure).

  sign(K) = sum_m alpha_m T_m(K) + sum_i phi_i phi_i^dagger [sign(lambda_i) - sum_m alpha_m T_m(lambda_i)]   (Eq. 3)
  D[mu]   = 1/2 (1 + mu + (1 - mu) gamma5 sign(K))                                                      (Eq. 1)

(phi_i, lambda_i) are the lowest-|lambda| eigenpairs of K (Sec. 2).  The
polynomial part is P(K) = K f_N(K^2) (see chebyshev.py for that reading).

Two forms of Eq. 3 are implemented:
  * projected (used everywhere): psi_perp = (1 - Phi Phi^dagger) psi,
    sign(K) psi = P(K) psi_perp + sum_i sign(lambda_i) phi_i (phi_i^dagger psi);
  * literal: P(K) psi + sum_i phi_i [sign(lambda_i) - P(lambda_i)] (phi_i^dagger psi).
They agree when the phi_i are exact orthonormal eigenvectors; the projected
form is the one that stays stable when the undeflated polynomial would
amplify modes below a.  sign(0) is taken as +1.

D[mu]^dagger = 1/2 (1 + mu + (1 - mu) sign(K) gamma5), since K and sign(K)
are Hermitian.

Pinned by: dense sign(K) within eps_cheb, exactness on deflated modes,
literal == projected, Ginsparg-Wilson bound, spectrum on the GW circle,
gamma5 D gamma5 = D^dagger (tests/test_oracle_sign.py, tests/test_oracle_overlap.py);
the chiral-sector operator against P D^dagger D P built from dense matrices
with the exact sign, and against it with the polynomial sign within the
Chebyshev error (tests/test_oracle_chiral.py).
"""
import numpy as np

from .chebyshev import apply_fn, p_scalar
from .wilson import M_W, gamma5, kernel_k


def sgn(lam):
    lam = np.asarray(lam, dtype=np.float64)
    return np.where(lam >= 0, 1.0, -1.0)


def inner(u, v):
    """<u, v> = sum over sites, spin and colour of conj(u) v."""
    return np.vdot(u.ravel(), v.ravel())


def project(evecs, psi):
    """c_i = phi_i^dagger psi."""
    return np.array([inner(phi, psi) for phi in evecs], dtype=np.complex128)


class SignConfig:
    """Everything Eq. 3 needs besides K: polynomial coefficients and interval,
    and the deflated eigenpairs."""

    def __init__(self, coeffs, a, b, evals=None, evecs=None):
        self.coeffs = np.asarray(coeffs, dtype=np.float64)
        self.a, self.b = float(a), float(b)
        if evals is None:
            evals = np.zeros(0)
            evecs = None
        self.evals = np.asarray(evals, dtype=np.float64)
        self.evecs = evecs


def sign_apply(links, psi, cfg, m_w=M_W, antiperiodic_t=False):
    """sign(K) psi, projected form of Eq. 3."""
    def kop(w):
        return kernel_k(links, w, m_w, antiperiodic_t)

    n_ev = len(cfg.evals)
    psi_perp = psi.copy()
    low = np.zeros_like(psi)
    if n_ev:
        c = project(cfg.evecs, psi)
        for i in range(n_ev):
            psi_perp = psi_perp - c[i] * cfg.evecs[i]
            low = low + sgn(cfg.evals[i]) * c[i] * cfg.evecs[i]
    return kop(apply_fn(kop, cfg.coeffs, cfg.a, cfg.b, psi_perp)) + low


def sign_apply_literal(links, psi, cfg, m_w=M_W, antiperiodic_t=False):
    """sign(K) psi exactly as Eq. 3 is printed: undeflated polynomial plus the
    eigenvalue correction on each deflated mode."""
    def kop(w):
        return kernel_k(links, w, m_w, antiperiodic_t)

    out = kop(apply_fn(kop, cfg.coeffs, cfg.a, cfg.b, psi))
    for i in range(len(cfg.evals)):
        phi = cfg.evecs[i]
        corr = sgn(cfg.evals[i]) - p_scalar(cfg.coeffs, cfg.a, cfg.b, cfg.evals[i])
        out = out + phi * (corr * inner(phi, psi))
    return out


def overlap(links, psi, mu, cfg, m_w=M_W, antiperiodic_t=False):
    """D[mu] psi = 1/2 ((1 + mu) psi + (1 - mu) gamma5 sign(K) psi), Eq. 1."""
    s = sign_apply(links, psi, cfg, m_w, antiperiodic_t)
    return 0.5 * ((1 + mu) * psi + (1 - mu) * gamma5(s))


def overlap_dag(links, psi, mu, cfg, m_w=M_W, antiperiodic_t=False):
    """D[mu]^dagger psi = 1/2 ((1 + mu) psi + (1 - mu) sign(K) gamma5 psi)."""
    s = sign_apply(links, gamma5(psi), cfg, m_w, antiperiodic_t)
    return 0.5 * ((1 + mu) * psi + (1 - mu) * s)


def normal_op(links, psi, mu, cfg, m_w=M_W, antiperiodic_t=False):
    """D[mu]^dagger D[mu] psi."""
    return overlap_dag(links, overlap(links, psi, mu, cfg, m_w, antiperiodic_t),
                       mu, cfg, m_w, antiperiodic_t)


def chiral_project(psi, chirality):
    """P psi = (1 + chirality gamma5) / 2 psi: keeps spins 0, 1 (chirality +1)
    or spins 2, 3 (chirality -1) of the chiral basis, gamma5 = diag(1, 1, -1, -1)."""
    out = np.zeros_like(psi)
    keep = slice(0, 2) if chirality > 0 else slice(2, 4)
    out[..., keep, :] = psi[..., keep, :]
    return out


def chiral_normal_op(links, psi, mu, cfg, chirality, m_w=M_W, antiperiodic_t=False, sign=None):
    """D[mu]^dagger D[mu] inside one chiral sector, written with a single sign
    function application:

      A psi = 1/4 [(1 + mu)^2 + (1 - mu)^2] P psi + chirality/2 (1 - mu^2) P S P psi.

    From D^dagger D = 1/4 [(1+mu)^2 + (1-mu)^2 S^2 + (1-mu^2)(gamma5 S + S gamma5)]
    (Eq. 1, S Hermitian): on chiral vectors the anticommutator becomes
    2 chirality P S P, and S^2 = 1 turns the middle term into (1-mu)^2.  With
    the polynomial S of Eq. 3, S^2 = 1 only up to the Chebyshev error, so A
    differs from P D^dagger D P by that much; A itself is Hermitian and, for
    |mu| < 1, positive definite on the sector.  sign: optional callable
    replacing sign_apply (for pins with the exact dense sign)."""
    p = chiral_project(psi, chirality)
    s = sign(p) if sign is not None else sign_apply(links, p, cfg, m_w, antiperiodic_t)
    c0 = 0.25 * ((1 + mu) ** 2 + (1 - mu) ** 2)
    c1 = 0.5 * chirality * (1 - mu * mu)
    return c0 * p + c1 * chiral_project(s, chirality)
