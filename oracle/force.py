"""Link derivative of S(U) = chi^dagger P(K) chi, FP64 (test infrastructure).

P(K) = K f_N(K^2) is the undeflated polynomial part of Eq. 3 (reading in
chebyshev.py).  The derivative is taken along U_mu(x) -> exp(eps X_mu(x)) U_mu(x)
with X_mu(x) anti-Hermitian traceless; the gradient F_mu(x) is the su(3)
matrix with

    dS/deps |_0 = sum_{x,mu} Re tr(X_mu(x)^dagger F_mu(x)).

Only the hopping term of D_W (Eq. 2) depends on the links:
    dK = gamma5 dD_W,
    dD_W psi(x) = -1/2 sum_mu [(1 - gamma_mu) dU_mu(x) psi(x+mu^) + (1 + gamma_mu) dU_mu(x-mu^)^dagger psi(x-mu^)].

Two independent evaluations:
  * ``gradient``: reverse sweep through the forward three-term recurrence,
    storing every T_j, collecting (u, v) pairs with dS = sum w u^dagger dK v,
    and turning each pair into colour outer products per link;
  * ``directional_derivative``: forward-mode tangent (T_j, dT_j) along one
    direction X, no pairs, no outer products.
Both are pinned against central finite differences of S with Richardson
extrapolation (tests/test_oracle_force.py).
"""
import numpy as np

from .chebyshev import apply_fn
from .overlap import inner
from .wilson import GAMMA, M_W, ONE4, gamma5, hopping, kernel_k, shift, spin_mul


def action(links, chi, coeffs, a, b, m_w=M_W, antiperiodic_t=False):
    """S = chi^dagger P(K) chi (real: P(K) is Hermitian)."""
    def kop(w):
        return kernel_k(links, w, m_w, antiperiodic_t)
    return inner(chi, kop(apply_fn(kop, coeffs, a, b, chi))).real


def project_ta(m):
    """Anti-Hermitian traceless part of a 3x3 matrix field."""
    ah = 0.5 * (m - np.conj(np.swapaxes(m, -1, -2)))
    tr = np.trace(ah, axis1=-2, axis2=-1) / 3.0
    return ah - tr[..., None, None] * np.eye(3)


def _outer(a, b):
    """sum_s a_s b_s^dagger for spinor fields a, b: a 3x3 colour matrix per site."""
    return np.einsum("...sa,...sb->...ab", a, b.conj())


def _pair_matrix(links, u, v, antiperiodic_t=False):
    """G_mu(x) with u^dagger dK v = sum_{x,mu} tr(X_mu(x) G_mu(x)) for dU = X U."""
    lt = u.shape[0]
    ubar = gamma5(u)
    g = np.zeros(links.shape, dtype=np.complex128)
    for mu in range(4):
        uv_fwd = np.einsum("...ab,...sb->...sa", links[mu], shift(v, mu, +1))
        proj_b = spin_mul(ONE4 + GAMMA[mu], shift(ubar, mu, +1))
        u_proj_b = np.einsum("...ab,...sb->...sa", links[mu], proj_b)
        if antiperiodic_t and mu == 3:
            sign = np.ones(lt)
            sign[lt - 1] = -1.0
            sign = sign.reshape(lt, 1, 1, 1, 1, 1)
            uv_fwd = uv_fwd * sign
            u_proj_b = u_proj_b * sign
        m_a = _outer(uv_fwd, spin_mul(ONE4 - GAMMA[mu], ubar))
        m_b = _outer(v, u_proj_b)
        g[mu] = -0.5 * (m_a - m_b)
    return g


def gradient(links, chi, coeffs, a, b, m_w=M_W, antiperiodic_t=False):
    """F_mu(x) of S = chi^dagger P(K) chi, shape (4, Lt, Lz, Ly, Lx, 3, 3)."""
    def kop(w):
        return kernel_k(links, w, m_w, antiperiodic_t)

    alpha = 2.0 / (b * b - a * a)
    beta = -(b * b + a * a) / (b * b - a * a)

    def zop(w):
        return alpha * kop(kop(w)) + beta * w

    n = len(coeffs) - 1
    # forward recurrence, keeping every T_j
    t = [chi, zop(chi)]
    for j in range(1, n):
        t.append(2 * zop(t[j]) - t[j - 1])
    cp = np.array(coeffs, dtype=np.float64)
    cp[0] *= 0.5
    g_vec = sum(cp[j] * t[j] for j in range(n + 1))

    # pairs (weight, u, v) of dK, and (weight, u, v) of dZ
    dk_pairs = [(1.0, chi, g_vec)]
    dz_pairs = []
    gbar = kop(chi)
    tbar = [cp[j] * gbar for j in range(n + 1)]
    for m in range(n, 1, -1):
        dz_pairs.append((2.0, tbar[m], t[m - 1]))
        tbar[m - 1] = tbar[m - 1] + 2 * zop(tbar[m])
        tbar[m - 2] = tbar[m - 2] - tbar[m]
    dz_pairs.append((1.0, tbar[1], chi))
    for w, u, v in dz_pairs:
        dk_pairs.append((alpha * w, u, kop(v)))
        dk_pairs.append((alpha * w, kop(u), v))

    g = np.zeros(links.shape, dtype=np.complex128)
    for w, u, v in dk_pairs:
        g += w * _pair_matrix(links, u, v, antiperiodic_t)
    # dS/deps = Re sum tr(X G) = sum Re tr(X^dagger P_TA(G^dagger))
    return project_ta(np.conj(np.swapaxes(g, -1, -2)))


def directional_derivative(links, chi, coeffs, a, b, x_dir, m_w=M_W, antiperiodic_t=False):
    """dS/deps along U -> exp(eps X) U by forward-mode propagation of (T_j, dT_j)."""
    def kop(w):
        return kernel_k(links, w, m_w, antiperiodic_t)

    dlinks = np.einsum("...ab,...bc->...ac", x_dir, links)

    def dkop(w):
        return gamma5(-0.5 * hopping(dlinks, w, antiperiodic_t))

    alpha = 2.0 / (b * b - a * a)
    beta = -(b * b + a * a) / (b * b - a * a)

    def zop(w):
        return alpha * kop(kop(w)) + beta * w

    def dzop(w):
        return alpha * (dkop(kop(w)) + kop(dkop(w)))

    n = len(coeffs) - 1
    t_prev, t_cur = chi, zop(chi)
    dt_prev, dt_cur = np.zeros_like(chi), dzop(chi)
    g = 0.5 * coeffs[0] * t_prev + coeffs[1] * t_cur
    dg = coeffs[1] * dt_cur
    for j in range(1, n):
        t_next = 2 * zop(t_cur) - t_prev
        dt_next = 2 * (dzop(t_cur) + zop(dt_cur)) - dt_prev
        t_prev, t_cur = t_cur, t_next
        dt_prev, dt_cur = dt_cur, dt_next
        g = g + coeffs[j + 1] * t_cur
        dg = dg + coeffs[j + 1] * dt_cur
    return (inner(chi, dkop(g)) + inner(chi, kop(dg))).real


def exp_su3(x):
    """exp of an anti-Hermitian 3x3 field via eigh of the Hermitian -i X."""
    h = -1j * x
    h = 0.5 * (h + np.conj(np.swapaxes(h, -1, -2)))
    w, v = np.linalg.eigh(h)
    return np.einsum("...ik,...k,...jk->...ij", v, np.exp(1j * w), v.conj())


def finite_difference(links, chi, coeffs, a, b, x_dir, eps=1e-3, m_w=M_W, antiperiodic_t=False):
    """Central differences at eps and eps/2 combined by Richardson extrapolation."""
    def s_at(e):
        u = np.einsum("...ab,...bc->...ac", exp_su3(e * x_dir), links)
        return action(u, chi, coeffs, a, b, m_w, antiperiodic_t)

    d1 = (s_at(eps) - s_at(-eps)) / (2 * eps)
    d2 = (s_at(eps / 2) - s_at(-eps / 2)) / eps
    return (4 * d2 - d1) / 3
