"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random numbers and shapes them into gauge links,
sources and Lie-algebra directions; it holds none of the overlap method's
arithmetic.  The paper measured on stout-smeared dynamical ensembles
(Sec. 2, Table 2); those configurations are not available, so seeded
near-identity SU(3) fields stand in for them at the same volumes.

Array conventions (shared by every interface of the library):
  * lattice dims are (Lx, Ly, Lz, Lt); the site index is
    ((t*Lz + z)*Ly + y)*Lx + x, so a NumPy field has shape (Lt, Lz, Ly, Lx, ...)
  * links:   complex128 (4, Lt, Lz, Ly, Lx, 3, 3), U[mu] is the link x -> x+mu^,
             mu = 0, 1, 2, 3 for x, y, z, t, colour matrix row-major
  * spinors: complex128 (nrhs, Lt, Lz, Ly, Lx, 4, 3), [spin][colour] per site
"""
import numpy as np

# Gell-Mann matrices lambda_1..lambda_8 (the standard su(3) basis).
_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1], _GELL_MANN[1][1, 0] = -1j, 1j
_GELL_MANN[2][0, 0], _GELL_MANN[2][1, 1] = 1, -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2], _GELL_MANN[4][2, 0] = -1j, 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2], _GELL_MANN[6][2, 1] = -1j, 1j
_GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)

SEED_LINKS = 1000
SEED_SOURCE = 2000
SEED_DIRECTIONS = 3000


def volume(dims):
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt


def _field_shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def random_hermitian_traceless(rng, shape):
    """H = sum_a h_a lambda_a / 2 with h_a ~ N(0, 1)."""
    h = rng.standard_normal(shape + (8,))
    return np.einsum("...a,aij->...ij", h, _GELL_MANN) / 2


def _project_su3(u):
    """Gram-Schmidt the first two rows, rebuild the third as conj(r0 x r1)
    so that every link is unitary with unit determinant to rounding."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(r0.conj() * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.cross(r0, r1).conj()
    return np.stack([r0, r1, r2], axis=-2)


def gauge_links(dims, seed=SEED_LINKS, eps=0.3):
    """U = exp(i * eps * H) per link, H seeded Gaussian traceless Hermitian 3x3."""
    rng = np.random.default_rng(seed)
    shape = (4,) + _field_shape(dims)
    h = random_hermitian_traceless(rng, shape)
    w, v = np.linalg.eigh(h)
    u = np.einsum("...ik,...k,...jk->...ij", v, np.exp(1j * eps * w), v.conj())
    return np.ascontiguousarray(_project_su3(u))


def unit_links(dims):
    """The free field U = 1."""
    shape = (4,) + _field_shape(dims) + (3, 3)
    return np.broadcast_to(np.eye(3, dtype=np.complex128), shape).copy()


def gaussian_source(dims, seed=SEED_SOURCE, nrhs=1):
    """Re and Im of every spinor component ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    shape = (nrhs,) + _field_shape(dims) + (4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def point_sources(dims, site=0):
    """The 12 spin-colour point sources e_{s,c} delta_{x,site}: (12, ..., 4, 3)."""
    shape = (12,) + _field_shape(dims) + (4, 3)
    out = np.zeros(shape, dtype=np.complex128)
    flat = out.reshape(12, -1, 4, 3)
    for s in range(4):
        for c in range(3):
            flat[3 * s + c, site, s, c] = 1.0
    return out


def su3_directions(dims, seed=SEED_DIRECTIONS):
    """X_mu(x) = i * sum_a omega_a lambda_a / 2, omega ~ N(0, 1): a random
    anti-Hermitian traceless direction per link."""
    rng = np.random.default_rng(seed)
    shape = (4,) + _field_shape(dims)
    return 1j * random_hermitian_traceless(rng, shape)


def gauge_transform(dims, seed):
    """A random SU(3) matrix per site, g(x) = exp(i H(x))."""
    rng = np.random.default_rng(seed)
    h = random_hermitian_traceless(rng, _field_shape(dims))
    w, v = np.linalg.eigh(h)
    g = np.einsum("...ik,...k,...jk->...ij", v, np.exp(1j * w), v.conj())
    return _project_su3(g)
