"""Wilson-Dirac operator and the sign-function kernel, FP64 (test infrastructure).

  (D_W psi)(x) = 4 psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu^)
                                        + (1 + gamma_mu) U_mu(x-mu^)^dagger psi(x-mu^) ]   (Eq. 2)
  K = gamma5 (D_W - m_W),  m_W = 1.5                                                       (Sec. 2)

Reading of Eq. 2: the printed "4 - 1/2 sum ..." drops the psi(x) of the
diagonal term; the standard r = 1 Wilson operator 4 psi(x) - ... is meant.
The paper does not fix a gamma basis; the chiral (DeGrand-Rossi) basis below
is used, with gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1, 1, -1, -1).
Boundary conditions are periodic, optionally antiperiodic in t.

Neighbours are taken with np.roll on arrays shaped (Lt, Lz, Ly, Lx, 4, 3);
links are (4, Lt, Lz, Ly, Lx, 3, 3) with U[mu] on the link x -> x + mu^.

Pinned by: free-field plane-wave closed form, gamma5-hermiticity of D_W,
gauge covariance, dense column build vs direct stencil (tests/test_oracle_wilson.py).
"""
import numpy as np

M_W = 1.5

_I = 1j
# Hermitian Euclidean gamma matrices, chiral (DeGrand-Rossi) basis; index 0..3 = x, y, z, t.
GAMMA = np.array([
    [[0, 0, 0, _I], [0, 0, _I, 0], [0, -_I, 0, 0], [-_I, 0, 0, 0]],
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    [[0, 0, _I, 0], [0, 0, 0, -_I], [-_I, 0, 0, 0], [0, _I, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=np.complex128)

# Direction mu -> axis of a (Lt, Lz, Ly, Lx, ...) field.
_AXIS = (3, 2, 1, 0)


def shift(field, mu, step):
    """field(x + step * mu^) with periodic wrap (step = +1 or -1)."""
    return np.roll(field, -step, axis=_AXIS[mu])


def _t_boundary_sign(lt, forward):
    """Sign picked up by a hop in t that wraps around the lattice when the
    fermion boundary condition in t is antiperiodic: the forward hop out of
    t = Lt-1 and the backward hop out of t = 0."""
    s = np.ones(lt)
    s[lt - 1 if forward else 0] = -1.0
    return s.reshape(lt, 1, 1, 1, 1, 1)


def colour_mul(u, psi):
    """(U psi)(x)_s,a = sum_b U(x)_ab psi(x)_s,b."""
    return np.einsum("...ab,...sb->...sa", u, psi)


def colour_mul_dag(u, psi):
    """(U^dagger psi)(x)_s,a = sum_b conj(U(x)_ba) psi(x)_s,b."""
    return np.einsum("...ba,...sb->...sa", u.conj(), psi)


def spin_mul(m, psi):
    """(M psi)(x)_s,a = sum_t M_st psi(x)_t,a."""
    return np.einsum("st,...ta->...sa", m, psi)


def gamma5(psi):
    return spin_mul(GAMMA5, psi)


def hopping(links, psi, antiperiodic_t=False):
    """sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu^) + (1 + gamma_mu) U_mu(x-mu^)^dagger psi(x-mu^) ]."""
    out = np.zeros_like(psi)
    lt = psi.shape[0]
    for mu in range(4):
        fwd = colour_mul(links[mu], shift(psi, mu, +1))
        bwd = shift(colour_mul_dag(links[mu], psi), mu, -1)
        if antiperiodic_t and mu == 3:
            fwd = fwd * _t_boundary_sign(lt, True)
            bwd = bwd * _t_boundary_sign(lt, False)
        out += spin_mul(ONE4 - GAMMA[mu], fwd) + spin_mul(ONE4 + GAMMA[mu], bwd)
    return out


def wilson(links, psi, antiperiodic_t=False):
    """D_W psi, Eq. 2."""
    return 4.0 * psi - 0.5 * hopping(links, psi, antiperiodic_t)


def kernel_k(links, psi, m_w=M_W, antiperiodic_t=False):
    """K psi = gamma5 (D_W - m_W) psi, Sec. 2."""
    return gamma5(wilson(links, psi, antiperiodic_t) - m_w * psi)
