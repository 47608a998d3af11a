"""Conjugate gradient on the normal equations D^dagger D x = D^dagger b, FP64
(test infrastructure).

The paper inverts the overlap operator with GMRESR variants (Sec. 2); the
solver on this path is plain CG on the normal equations.  Reading used: the
stopping test is the normal-equation residual ||D^dagger b - D^dagger D x|| /
||D^dagger b|| <= tol, recomputed from scratch at the end, with D the same
approximate operator (same order, interval and deflated pairs).

cg_chiral: the same CG on the chiral-sector operator A of
overlap.chiral_normal_op, A x = P b, stopping on ||P b - A x|| / ||P b||.

Pinned by: dense linear solves at 4^4 (tests/test_oracle_overlap.py,
tests/test_oracle_chiral.py).
"""
import numpy as np

from .overlap import chiral_normal_op, chiral_project, inner, normal_op, overlap_dag
from .wilson import M_W


def cg_normal(links, b, mu, cfg, tol=1e-10, maxit=1000, m_w=M_W, antiperiodic_t=False):
    """Returns (x, iterations, true relative residual)."""
    def a_op(v):
        return normal_op(links, v, mu, cfg, m_w, antiperiodic_t)

    rhs = overlap_dag(links, b, mu, cfg, m_w, antiperiodic_t)
    rhs_norm = np.sqrt(inner(rhs, rhs).real)
    x = np.zeros_like(b)
    r = rhs.copy()
    p = r.copy()
    rr = inner(r, r).real
    it = 0
    while it < maxit and np.sqrt(rr) > tol * rhs_norm:
        q = a_op(p)
        alpha = rr / inner(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = inner(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    true_r = rhs - a_op(x)
    return x, it, float(np.sqrt(inner(true_r, true_r).real) / rhs_norm)


def _cg(a_op, rhs, tol, maxit):
    rhs_norm = np.sqrt(inner(rhs, rhs).real)
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = inner(r, r).real
    it = 0
    while it < maxit and np.sqrt(rr) > tol * rhs_norm:
        q = a_op(p)
        alpha = rr / inner(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = inner(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    true_r = rhs - a_op(x)
    return x, it, float(np.sqrt(inner(true_r, true_r).real) / rhs_norm)


def cg_chiral(links, b, mu, cfg, chirality, tol=1e-10, maxit=1000, m_w=M_W, antiperiodic_t=False):
    """A x = P b on one chiral sector (one sign apply per iteration).
    Returns (x, iterations, true relative residual)."""
    def a_op(v):
        return chiral_normal_op(links, v, mu, cfg, chirality, m_w, antiperiodic_t)

    return _cg(a_op, chiral_project(b, chirality), tol, maxit)
