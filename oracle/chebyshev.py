"""Chebyshev approximation of sign(K), FP64 (test infrastructure).

Eq. 3 writes the polynomial part of sign(K) as sum_m alpha_m T_m(K) with
"appropriate coefficients" and does not say how they are built.  Reading used
here (and by the library): the polynomial is P(K) = K f_N(K^2), where f_N is
the degree-N Chebyshev interpolant of f(y) = y^{-1/2} on [a^2, b^2], with
a = |lambda_{n+1}| (first undeflated eigenvalue of K) and b >= lambda_max.
P is odd in K, so it is a series in odd T_m(K / b) as Eq. 3 writes it.
"Order N" is the highest Chebyshev index of f_N: N + 1 coefficients,
degree 2N + 1 in K.

  nodes        x_k = cos(pi (k + 1/2) / (N + 1)),  k = 0..N
  mapped       y_k = ((b^2 - a^2) x_k + b^2 + a^2) / 2
  coefficients c_j = 2/(N + 1) sum_k f(y_k) T_j(x_k)
  series       f_N(y) = c_0/2 + sum_{j>=1} c_j T_j(z),  z = (2y - b^2 - a^2)/(b^2 - a^2)

The vector evaluation uses the FORWARD three-term recurrence of the T_j
(Eq. 3's "short three vector recurrence", Sec. 2), deliberately a different
evaluation order from the library's backward (Clenshaw) sweep:
  T_0 = v,  T_1 = Z v,  T_{j+1} = 2 Z T_j - T_{j-1},  Z = alpha K^2 + beta,
  alpha = 2/(b^2 - a^2),  beta = -(b^2 + a^2)/(b^2 - a^2).

Pinned by: interpolation at the nodes, NumPy's Chebyshev interpolation of
the same function, the free-field scalar closed form, and dense
eigendecomposition within the scalar error bound (tests/test_oracle_sign.py).
"""
import numpy as np

from .wilson import M_W, kernel_k


def coefficients(order, a, b):
    """c_0..c_N of the Chebyshev interpolant of y^{-1/2} on [a^2, b^2]."""
    if order < 1 or not (0 < a < b):
        raise ValueError("need order >= 1 and 0 < a < b")
    n1 = order + 1
    theta = np.pi * (np.arange(n1) + 0.5) / n1
    x = np.cos(theta)
    y = ((b * b - a * a) * x + b * b + a * a) / 2
    fy = y ** -0.5
    c = np.empty(n1)
    for j in range(n1):
        c[j] = 2.0 / n1 * np.sum(fy * np.cos(j * theta))
    return c


def z_map(y, a, b):
    return (2 * y - b * b - a * a) / (b * b - a * a)


def f_scalar(c, a, b, y):
    """f_N(y) for scalar / array y by the forward recurrence of T_j(z)."""
    z = z_map(np.asarray(y, dtype=np.float64), a, b)
    t_prev, t_cur = np.ones_like(z), z
    acc = 0.5 * c[0] * t_prev + c[1] * t_cur
    for j in range(1, len(c) - 1):
        t_prev, t_cur = t_cur, 2 * z * t_cur - t_prev
        acc = acc + c[j + 1] * t_cur
    return acc


def p_scalar(c, a, b, lam):
    """P(lambda) = lambda f_N(lambda^2): the polynomial part of sign on a scalar."""
    lam = np.asarray(lam, dtype=np.float64)
    return lam * f_scalar(c, a, b, lam * lam)


def sign_error(c, a, b, samples=20001):
    """eps_cheb = max_{a <= |lambda| <= b} |P(lambda) - sign(lambda)|, sampled densely."""
    lam = np.linspace(a, b, samples)
    return float(np.max(np.abs(p_scalar(c, a, b, lam) - 1.0)))


def apply_fn(kop, c, a, b, v):
    """f_N(K^2) v with the forward recurrence; kop(v) applies K."""
    alpha = 2.0 / (b * b - a * a)
    beta = -(b * b + a * a) / (b * b - a * a)

    def zop(w):
        return alpha * kop(kop(w)) + beta * w

    t_prev = v
    t_cur = zop(v)
    g = 0.5 * c[0] * t_prev + c[1] * t_cur
    for j in range(1, len(c) - 1):
        t_prev, t_cur = t_cur, 2 * zop(t_cur) - t_prev
        g = g + c[j + 1] * t_cur
    return g


def poly_apply(links, v, c, a, b, m_w=M_W, antiperiodic_t=False):
    """P(K) v = K f_N(K^2) v (undeflated)."""
    def kop(w):
        return kernel_k(links, w, m_w, antiperiodic_t)
    return kop(apply_fn(kop, c, a, b, v))
