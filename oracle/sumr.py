"""Shifted-unitary minimal residual (SUMR) and the GMRESR outer loop for the
overlap operator, FP64 (test infrastructure: only tests/, smoke() and the CPU
legs of bench.py use this module).

Sec. 2 inverts the overlap operator with GMRESR(eigSUMR): a recursive GMRES
(GCR) outer loop whose preconditioner is a low-accuracy SUMR solve with a
relaxed sign function.  The paper gives no formulas; the readings used here:

SUMR.  With U = gamma5 sign(K) (unitary for the exact sign), Eq. 1 reads

    D[mu] = (1 - mu)/2 (U - zeta),   zeta = -(1 + mu)/(1 - mu),

so D x = b is the shifted unitary system (U - zeta) x = b' with
b' = 2 b / (1 - mu).  The minimal residual iterate over the Krylov space
K_k(U, b') is built from the Szego recursion of the orthonormal polynomials
phi_j of the spectral measure of U at v_0 = b'/|b'| (phi_j^* the reversed
ones, alpha_j the recursion coefficients, rho_j = rho~_j = sqrt(1 - |alpha_j|^2)
for unitary U):

    m        = <v~_j, U v_j>                     (= conj(alpha_j))
    v_{j+1}  = (U v_j - m v~_j) / rho_j          v~_{j+1} = (v~_j - conj(m) U v_j) / rho~_j

The residual polynomial of the minimal residual iterate is the normalised
reproducing kernel at zeta,
    p_k(z) = sum_{j<=k} conj(phi_j(zeta)) phi_j(z) / s_k,   s_k = sum_{j<=k} |phi_j(zeta)|^2,
so |r_k| = |b'| / sqrt(s_k) for unitary U, and
    x_k = -(|b'| / s_k) sum_{j<=k} conj(phi_j(zeta)) D_j,
with D_j = d_j(U) v_0 the divided differences d_j(z) = (phi_j(z) - phi_j(zeta))/(z - zeta).
Because (U - zeta) D_j = v_j - phi_j(zeta) v_0, the D_j and their reversed
partners D~_j obey a recursion that needs no further product with U:

    D_{j+1}  = (v_j + zeta D_j - m D~_j) / rho_j      D~_{j+1} = (D~_j - conj(m) (v_j + zeta D_j)) / rho~_j
    phi_{j+1}(zeta) = (zeta phi_j(zeta) - m phi_j^*(zeta)) / rho_j
    phi^*_{j+1}(zeta) = (phi_j^*(zeta) - conj(m) zeta phi_j(zeta)) / rho~_j

(D_0 = D~_0 = 0, phi_0 = phi_0^* = 1): one product with U per iteration and
six vectors.

Normalisation.  For exactly unitary U the new vectors have norm rho_j.  With
the polynomial sign U is unitary only to the Chebyshev error, and dividing by
sqrt(1 - |m|^2) lets the vector norms grow geometrically until the recursion
breaks down (already at 1e-5 non-unitarity, and in FP64 rounding at small mu).
Reading used here: v_{j+1} and v~_{j+1} are divided by their own computed
norms rho_j and rho~_j, and the scalar and divided-difference recursions use
the same divisors (rho_j for the phi / D line, rho~_j for the phi^* / D~
line).  The updates stay polynomial identities for whatever coefficients are
used, so b' - (U - zeta) x_k = |b'|/s_k sum_j conj(phi_j(zeta)) v_j holds
exactly; for unitary U the divisors equal sqrt(1 - |m|^2) and the iterate is
the minimal residual one; otherwise the v_j stay unit vectors and the
estimate |b'|/sqrt(s_k) keeps tracking the true residual.

GMRESR.  GCR on D[mu] with a variable preconditioner (the inner SUMR solve
of D u = r with the relaxed operator): u_k = M_k(r_k), c_k = D u_k,
c_k and u_k orthogonalised against the previous c_i (modified Gram-Schmidt,
the same combination applied to u), normalised, then x += <c_k, r> u_k and
r -= <c_k, r> c_k.  The outer operator is the accurate one, so the updated
residual tracks the true one.

Pinned by: the SUMR iterate equals the brute-force minimal residual iterate
(least squares over an explicit Krylov basis) for a dense unitary matrix and
for gamma5 times the exact dense sign(K), its residual estimate equals the
true residual there, GCR with the identity preconditioner equals the same
brute-force minimum, and GMRESR with a relaxed inner sign converges to the
dense solve of the accurate polynomial operator (tests/test_oracle_sumr.py).
"""
import numpy as np

from .overlap import inner, sign_apply
from .wilson import M_W, gamma5


def zeta_of(mu):
    """Shift of the unitary form: D[mu] = (1 - mu)/2 (U - zeta)."""
    return -(1.0 + mu) / (1.0 - mu)


def _divided_step(v, d, dt, m, zeta, rho, rho_t):
    """Next pair (D_{j+1}, D~_{j+1}) of divided-difference vectors."""
    t = v + zeta * d
    return (t - m * dt) / rho, (dt - np.conj(m) * t) / rho_t


def sumr(apply_u, zeta, rhs, maxit, tol=0.0):
    """Solves (U - zeta) x = rhs by the short recurrences above.

    Stops after maxit products with U or when the estimate 1/sqrt(s_k) of the
    relative residual is <= tol.  Returns (x, iterations, estimate)."""
    nb = np.sqrt(inner(rhs, rhs).real)
    x = np.zeros_like(rhs)
    if nb == 0.0:
        return x, 0, 0.0
    v = rhs / nb
    vt = v.copy()
    d = np.zeros_like(rhs)
    dt = np.zeros_like(rhs)
    acc = np.zeros_like(rhs)  # sum_j conj(phi_j(zeta)) D_j
    phi, phis, s = 1.0 + 0j, 1.0 + 0j, 1.0
    it = 0
    while it < maxit and 1.0 / np.sqrt(s) > tol:
        w = apply_u(v)
        m = inner(vt, w)
        v_new = w - m * vt
        vt_new = vt - np.conj(m) * w
        rho = np.sqrt(inner(v_new, v_new).real)
        rho_t = np.sqrt(inner(vt_new, vt_new).real)
        if not min(rho, rho_t) > 1e-7:
            break  # the Krylov space is (numerically) invariant
        d, dt = _divided_step(v, d, dt, m, zeta, rho, rho_t)
        v, vt = v_new / rho, vt_new / rho_t
        phi, phis = (zeta * phi - m * phis) / rho, (phis - np.conj(m) * zeta * phi) / rho_t
        s += abs(phi) ** 2
        acc = acc + np.conj(phi) * d
        it += 1
    return -(nb / s) * acc, it, float(1.0 / np.sqrt(s))


def overlap_unitary(links, psi, cfg, m_w=M_W, antiperiodic_t=False):
    """U psi = gamma5 sign(K) psi (sign of Eq. 3)."""
    return gamma5(sign_apply(links, psi, cfg, m_w, antiperiodic_t))


def overlap_sumr(links, b, mu, cfg, maxit, tol=0.0, m_w=M_W, antiperiodic_t=False):
    """SUMR for D[mu] x = b (Eq. 1) with the sign of cfg.  Returns
    (x, iterations, estimate of |b - D x| / |b|)."""
    def u_op(v):
        return overlap_unitary(links, v, cfg, m_w, antiperiodic_t)

    return sumr(u_op, zeta_of(mu), 2.0 * b / (1.0 - mu), maxit, tol)


def _orthogonalise(c, u, us, cs):
    """Modified Gram-Schmidt of c against the kept c_i, the same combination
    applied to u."""
    for ui, ci in zip(us, cs):
        beta = inner(ci, c)
        c = c - beta * ci
        u = u - beta * ui
    return c, u


def gcr(apply_a, precond, b, tol, max_outer, max_dirs=None):
    """GCR with a (possibly varying) preconditioner precond(r) ~ A^{-1} r.

    Returns (x, outer iterations, relative updated residual)."""
    nb = np.sqrt(inner(b, b).real)
    x = np.zeros_like(b)
    r = b.copy()
    us, cs = [], []
    k = 0
    while k < max_outer and np.sqrt(inner(r, r).real) > tol * nb:
        u = precond(r)
        c, u = _orthogonalise(apply_a(u), u, us, cs)
        n = np.sqrt(inner(c, c).real)
        c, u = c / n, u / n
        g = inner(c, r)
        x = x + g * u
        r = r - g * c
        us.append(u)
        cs.append(c)
        if max_dirs is not None and len(us) >= max_dirs:
            us, cs = [], []
        k += 1
    return x, k, float(np.sqrt(inner(r, r).real) / nb)


def gmresr_overlap(links, b, mu, cfg, cfg_inner, inner_tol, tol=1e-10, max_outer=50, inner_maxit=10000,
                   m_w=M_W, antiperiodic_t=False):
    """GMRESR(SUMR): GCR on D[mu] with the sign of cfg, each direction an
    inner SUMR solve with the (relaxed) sign of cfg_inner to relative
    estimate inner_tol.  Returns (x, outer iterations, inner iterations,
    true relative residual |b - D x| / |b|)."""
    zeta = zeta_of(mu)
    n_inner = [0]

    def d_op(v):
        return 0.5 * ((1 + mu) * v + (1 - mu) * overlap_unitary(links, v, cfg, m_w, antiperiodic_t))

    def u_lo(v):
        return overlap_unitary(links, v, cfg_inner, m_w, antiperiodic_t)

    def precond(r):
        u, it, _ = sumr(u_lo, zeta, 2.0 * r / (1.0 - mu), inner_maxit, inner_tol)
        n_inner[0] += it
        return u

    x, k, _ = gcr(d_op, precond, b, tol, max_outer)
    rt = b - d_op(x)
    return x, k, n_inner[0], float(np.sqrt(inner(rt, rt).real / inner(b, b).real))
