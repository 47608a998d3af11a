"""Pins of the oracle's D_W (Eq. 2) and K = gamma5 (D_W - m_W) (Sec. 2)."""
import numpy as np
import pytest

from oracle import dense, wilson
from paper_1510_06897_gb300 import inputs

DIMS_ASYM = (4, 2, 3, 6)   # Lx, Ly, Lz, Lt all different: catches axis mix-ups


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_gamma_algebra():
    g = wilson.GAMMA
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
    assert np.allclose(wilson.GAMMA5, np.diag([1, 1, -1, -1]))


def _plane_wave(dims, n, u, antiperiodic_t=False):
    lx, ly, lz, lt = dims
    p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
         (2 * n[3] + (1 if antiperiodic_t else 0)) * np.pi / lt]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return p, phase[..., None, None] * u


@pytest.mark.parametrize("antiperiodic", [False, True])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 1, 2, 1), (3, 0, 1, 5), (2, 1, 1, 3)])
def test_free_field_plane_wave(n, antiperiodic):
    """U = 1: D_W e^{ipx} u = [sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu] e^{ipx} u."""
    rng = np.random.default_rng(7)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    p, psi = _plane_wave(DIMS_ASYM, n, u, antiperiodic)
    links = inputs.unit_links(DIMS_ASYM)
    got = wilson.wilson(links, psi, antiperiodic)
    mom = sum(1 - np.cos(pm) for pm in p) * np.eye(4) + 1j * sum(
        wilson.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    want = np.einsum("st,...ta->...sa", mom, psi)
    assert np.linalg.norm(got - want) < 1e-14 * np.linalg.norm(psi)


def test_free_field_spectrum_bounds():
    """At 4^4 periodic, U = 1: |lambda(K)| = sqrt(A^2 + s^2), A = sum(1 - cos p) - 1.5,
    s^2 = sum sin^2 p, so min |lambda| = 0.5 (one p component = pi) and max = 6.5."""
    links = inputs.unit_links((4, 4, 4, 4))
    w = np.linalg.eigvalsh(dense.kernel_matrix(links))
    assert abs(np.min(np.abs(w)) - 0.5) < 1e-12
    assert abs(np.max(np.abs(w)) - 6.5) < 1e-12


@pytest.mark.parametrize("antiperiodic", [False, True])
def test_gamma5_hermiticity(antiperiodic):
    """<phi, K psi> = <K phi, psi> for a random gauge field."""
    links = inputs.gauge_links(DIMS_ASYM, seed=11)
    phi = inputs.gaussian_source(DIMS_ASYM, seed=12)[0]
    psi = inputs.gaussian_source(DIMS_ASYM, seed=13)[0]
    lhs = np.vdot(phi, wilson.kernel_k(links, psi, antiperiodic_t=antiperiodic))
    rhs = np.vdot(wilson.kernel_k(links, phi, antiperiodic_t=antiperiodic), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and the non-trivial part: D_W itself is not Hermitian
    lhs_w = np.vdot(phi, wilson.wilson(links, psi))
    rhs_w = np.vdot(wilson.wilson(links, phi), psi)
    assert abs(lhs_w - rhs_w) > 1e-3 * abs(lhs_w)


@pytest.mark.parametrize("antiperiodic", [False, True])
def test_gauge_covariance(antiperiodic):
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger, psi -> g psi  =>  D_W psi -> g D_W psi."""
    links = inputs.gauge_links(DIMS_ASYM, seed=21)
    psi = inputs.gaussian_source(DIMS_ASYM, seed=22)[0]
    g = inputs.gauge_transform(DIMS_ASYM, seed=23)
    links_g = np.empty_like(links)
    for mu in range(4):
        g_fwd = wilson.shift(g, mu, +1)
        links_g[mu] = np.einsum("...ab,...bc,...dc->...ad", g, links[mu], g_fwd.conj())
    psi_g = np.einsum("...ab,...sb->...sa", g, psi)
    got = wilson.wilson(links_g, psi_g, antiperiodic)
    want = np.einsum("...ab,...sb->...sa", g, wilson.wilson(links, psi, antiperiodic))
    assert _rel(got, want) < 1e-13


@pytest.mark.parametrize("dims,antiperiodic", [((2, 2, 2, 2), False), ((2, 3, 2, 4), True)])
def test_dense_stencil_matches_columns(dims, antiperiodic):
    """The block-assembled matrix equals D_W applied to every unit vector."""
    links = inputs.gauge_links(dims, seed=31)
    m = dense.wilson_matrix(links, antiperiodic)
    vol = inputs.volume(dims)
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    cols = np.empty_like(m)
    for k in range(12 * vol):
        e = np.zeros(12 * vol, dtype=np.complex128)
        e[k] = 1
        cols[:, k] = wilson.wilson(links, e.reshape(shape), antiperiodic).ravel()
    assert np.max(np.abs(cols - m)) < 1e-14


def test_links_are_su3():
    links = inputs.gauge_links((2, 2, 2, 4), seed=41)
    uu = np.einsum("...ab,...cb->...ac", links, links.conj())
    assert np.max(np.abs(uu - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(links) - 1)) < 1e-14
