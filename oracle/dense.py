"""Dense matrices on tiny lattices (2^4, 4^4), FP64 (test infrastructure).

  * wilson_matrix: D_W of Eq. 2 assembled block by block from the stencil
    (12 x 12 blocks kron(spin, colour) per site pair), an independent
    construction from the np.roll form in wilson.py;
  * kernel_matrix: K = gamma5 (D_W - m_W) (Sec. 2);
  * eigenpairs of K sorted by |lambda| (ties by lambda, then index), the
    deflation input of Eq. 3 (Sec. 2 computes them with Lanczos; on 2^4 and
    4^4 a dense Hermitian eigensolver gives them exactly);
  * exact sign(K) = V sign(Lambda) V^dagger, the quantity Eq. 3 approximates.

Vector flattening: index = site * 12 + spin * 3 + colour, the row-major
flattening of a (Lt, Lz, Ly, Lx, 4, 3) field.
"""
import numpy as np

from .wilson import GAMMA, GAMMA5, M_W, ONE4


def _site(coord, dims):
    x, y, z, t = coord
    lx, ly, lz, lt = dims
    return ((t * lz + z) * ly + y) * lx + x


def wilson_matrix(links, antiperiodic_t=False):
    """12V x 12V matrix of D_W, from the stencil of Eq. 2."""
    lt, lz, ly, lx = links.shape[1:5]
    dims = (lx, ly, lz, lt)
    vol = lx * ly * lz * lt
    m = np.zeros((12 * vol, 12 * vol), dtype=np.complex128)
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    coord = [x, y, z, t]
                    s = _site(coord, dims)
                    m[12 * s:12 * s + 12, 12 * s:12 * s + 12] += 4.0 * np.eye(12)
                    for mu in range(4):
                        fw = list(coord)
                        fw[mu] = (fw[mu] + 1) % dims[mu]
                        bw = list(coord)
                        bw[mu] = (bw[mu] - 1) % dims[mu]
                        sf, sb = _site(fw, dims), _site(bw, dims)
                        phase_f = phase_b = 1.0
                        if antiperiodic_t and mu == 3:
                            phase_f = -1.0 if t == lt - 1 else 1.0
                            phase_b = -1.0 if t == 0 else 1.0
                        u_here = links[mu, t, z, y, x]
                        u_back = links[mu, bw[3], bw[2], bw[1], bw[0]]
                        m[12 * s:12 * s + 12, 12 * sf:12 * sf + 12] += \
                            -0.5 * phase_f * np.kron(ONE4 - GAMMA[mu], u_here)
                        m[12 * s:12 * s + 12, 12 * sb:12 * sb + 12] += \
                            -0.5 * phase_b * np.kron(ONE4 + GAMMA[mu], u_back.conj().T)
    return m


def gamma5_matrix(vol):
    return np.kron(np.eye(vol), np.kron(GAMMA5, np.eye(3)))


def kernel_matrix(links, m_w=M_W, antiperiodic_t=False):
    dw = wilson_matrix(links, antiperiodic_t)
    vol = dw.shape[0] // 12
    return gamma5_matrix(vol) @ (dw - m_w * np.eye(12 * vol))


def sorted_eigh(kmat):
    """Eigenpairs of the Hermitian K, ordered by |lambda|, ties by lambda."""
    w, v = np.linalg.eigh(kmat)
    order = np.lexsort((np.arange(len(w)), w, np.abs(w)))
    return w[order], v[:, order]


def eigenpairs_as_fields(kmat, n_ev, field_shape):
    """(evals[:n_ev], evecs shaped (n_ev,) + field_shape) of K."""
    w, v = sorted_eigh(kmat)
    evecs = np.ascontiguousarray(v[:, :n_ev].T).reshape((n_ev,) + tuple(field_shape))
    return w[:n_ev].copy(), evecs, w


def exact_sign(kmat):
    w, v = np.linalg.eigh(kmat)
    s = np.where(w >= 0, 1.0, -1.0)
    return (v * s) @ v.conj().T


def apply_matrix(m, field):
    return (m @ field.ravel()).reshape(field.shape)
