"""The oracle pins must catch plausible mistakes.  Each case plants one error
in the oracle (monkeypatched, CPU only) and checks that the corresponding
closed-form / invariant / dense check then fails."""
import numpy as np
import pytest

import oracle.chebyshev as cheb
import oracle.overlap as ovl
import oracle.wilson as wil
from oracle import dense
from paper_1510_06897_gb300 import inputs

DIMS = (4, 2, 3, 6)


def _free_field_ok():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    n = (1, 1, 2, 1)
    lx, ly, lz, lt = DIMS
    p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, 2 * np.pi * n[3] / lt]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    psi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None, None] * u
    got = wil.wilson(inputs.unit_links(DIMS), psi)
    mom = sum(1 - np.cos(pm) for pm in p) * np.eye(4) + 1j * sum(wil.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    want = np.einsum("st,...ta->...sa", mom, psi)
    return np.linalg.norm(got - want) < 1e-12 * np.linalg.norm(psi)


def _hermiticity_ok():
    links = inputs.gauge_links(DIMS, seed=11)
    phi = inputs.gaussian_source(DIMS, seed=12)[0]
    psi = inputs.gaussian_source(DIMS, seed=13)[0]
    lhs = np.vdot(phi, wil.kernel_k(links, psi))
    rhs = np.vdot(wil.kernel_k(links, phi), psi)
    return abs(lhs - rhs) < 1e-12 * abs(lhs)


def _gauge_covariance_ok():
    links = inputs.gauge_links(DIMS, seed=21)
    psi = inputs.gaussian_source(DIMS, seed=22)[0]
    g = inputs.gauge_transform(DIMS, seed=23)
    links_g = np.empty_like(links)
    for mu in range(4):
        links_g[mu] = np.einsum("...ab,...bc,...dc->...ad", g, links[mu], wil.shift(g, mu, +1).conj())
    got = wil.wilson(links_g, np.einsum("...ab,...sb->...sa", g, psi))
    want = np.einsum("...ab,...sb->...sa", g, wil.wilson(links, psi))
    return np.linalg.norm(got - want) < 1e-12 * np.linalg.norm(want)


def _wilson_pins_ok():
    return _free_field_ok() and _hermiticity_ok() and _gauge_covariance_ok()


def _nodes_ok():
    a, b, order = 0.3, 6.5, 40
    c = cheb.coefficients(order, a, b)
    n1 = order + 1
    xk = np.cos(np.pi * (np.arange(n1) + 0.5) / n1)
    y = ((b * b - a * a) * xk + b * b + a * a) / 2
    return np.max(np.abs(cheb.f_scalar(c, a, b, y) * np.sqrt(y) - 1)) < 1e-11


_SMALL = {}


def _small():
    if not _SMALL:
        dims = (2, 2, 2, 4)
        links = inputs.gauge_links(dims, seed=31)
        km = dense.kernel_matrix(links)
        shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
        ev, evec, w_all = dense.eigenpairs_as_fields(km, 4, shape)
        _SMALL.update(dims=dims, links=links, km=km, ev=ev, evec=evec, a=float(abs(w_all[4])),
                      b=float(np.max(np.abs(w_all))), psi=inputs.gaussian_source(dims, seed=32)[0])
    return _SMALL


def _polynomial_ok():
    s = _small()
    c = cheb.coefficients(24, s["a"], s["b"])
    got = cheb.poly_apply(s["links"], s["psi"], c, s["a"], s["b"])
    w, v = np.linalg.eigh(s["km"])
    want = ((v * cheb.p_scalar(c, s["a"], s["b"], w)) @ (v.conj().T @ s["psi"].ravel())).reshape(s["psi"].shape)
    return np.linalg.norm(got - want) < 1e-12 * np.linalg.norm(want)


def _deflation_ok():
    s = _small()
    cfg = ovl.SignConfig(cheb.coefficients(24, s["a"], s["b"]), s["a"], s["b"], s["ev"], s["evec"])
    return all(np.linalg.norm(ovl.sign_apply(s["links"], s["evec"][i], cfg) - np.sign(s["ev"][i]) * s["evec"][i])
               < 1e-12 for i in range(len(s["ev"])))


def _gw_circle_ok():
    s = _small()
    cfg = ovl.SignConfig(cheb.coefficients(40, s["a"], s["b"]), s["a"], s["b"], s["ev"], s["evec"])
    eps = cheb.sign_error(cfg.coeffs, cfg.a, cfg.b)
    mu = 0.1
    n = s["psi"].size
    cols = []
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1
        cols.append(ovl.overlap(s["links"], e.reshape(s["psi"].shape), mu, cfg).ravel())
    z = np.linalg.eigvals(np.array(cols).T)
    return np.max(np.abs(np.abs(z - 0.5 * (1 + mu)) - 0.5 * (1 - mu))) <= 0.5 * (1 - mu) * eps + 1e-12


def test_unmutated_oracle_passes_every_check():
    assert _wilson_pins_ok() and _nodes_ok() and _polynomial_ok() and _deflation_ok() and _gw_circle_ok()


def _wrong_hopping_projector(links, psi, antiperiodic_t=False):
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = wil.colour_mul(links[mu], wil.shift(psi, mu, +1))
        bwd = wil.shift(wil.colour_mul_dag(links[mu], psi), mu, -1)
        out += wil.spin_mul(wil.ONE4 + wil.GAMMA[mu], fwd) + wil.spin_mul(wil.ONE4 - wil.GAMMA[mu], bwd)
    return out


def _wrong_backward_link(links, psi, antiperiodic_t=False):
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = wil.colour_mul(links[mu], wil.shift(psi, mu, +1))
        bwd = wil.shift(wil.colour_mul(links[mu], psi), mu, -1)  # U instead of U^dagger
        out += wil.spin_mul(wil.ONE4 - wil.GAMMA[mu], fwd) + wil.spin_mul(wil.ONE4 + wil.GAMMA[mu], bwd)
    return out


def _wrong_link_site(links, psi, antiperiodic_t=False):
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = wil.colour_mul(links[mu], wil.shift(psi, mu, +1))
        bwd = wil.colour_mul_dag(links[mu], wil.shift(psi, mu, -1))  # U(x) instead of U(x - mu)
        out += wil.spin_mul(wil.ONE4 - wil.GAMMA[mu], fwd) + wil.spin_mul(wil.ONE4 + wil.GAMMA[mu], bwd)
    return out


def _swapped_axes_shift(field, mu, step):
    return np.roll(field, -step, axis=(0, 1, 2, 3)[mu])  # x <-> t mix-up


@pytest.mark.parametrize("name,target,attr,replacement", [
    ("projector sign", wil, "hopping", _wrong_hopping_projector),
    ("U instead of U^dagger backward", wil, "hopping", _wrong_backward_link),
    ("backward link at the wrong site", wil, "hopping", _wrong_link_site),
    ("axis order", wil, "shift", _swapped_axes_shift),
    ("dropped diagonal 4 psi", wil, "wilson", lambda links, psi, ap=False: -0.5 * wil.hopping(links, psi, ap)),
])
def test_wilson_mutations_are_caught(monkeypatch, name, target, attr, replacement):
    monkeypatch.setattr(target, attr, replacement)
    assert not _wilson_pins_ok(), name


def test_chebyshev_node_offset_is_caught(monkeypatch):
    orig = cheb.coefficients

    def wrong(order, a, b):
        n1 = order + 1
        theta = np.pi * np.arange(n1) / n1          # k instead of k + 1/2
        y = ((b * b - a * a) * np.cos(theta) + b * b + a * a) / 2
        return np.array([2.0 / n1 * np.sum(y ** -0.5 * np.cos(j * theta)) for j in range(n1)])

    monkeypatch.setattr(cheb, "coefficients", wrong)
    assert not _nodes_ok()
    monkeypatch.setattr(cheb, "coefficients", orig)


def test_recurrence_sign_is_caught(monkeypatch):
    def wrong_apply_fn(kop, c, a, b, v):
        alpha = 2.0 / (b * b - a * a)
        beta = -(b * b + a * a) / (b * b - a * a)

        def zop(w):
            return alpha * kop(kop(w)) + beta * w

        t_prev, t_cur = v, zop(v)
        g = 0.5 * c[0] * t_prev + c[1] * t_cur
        for j in range(1, len(c) - 1):
            t_prev, t_cur = t_cur, 2 * zop(t_cur) + t_prev   # + instead of -
            g = g + c[j + 1] * t_cur
        return g

    monkeypatch.setattr(cheb, "apply_fn", wrong_apply_fn)
    assert not _polynomial_ok()


def test_deflation_sign_is_caught(monkeypatch):
    monkeypatch.setattr(ovl, "sgn", lambda lam: -np.where(np.asarray(lam) >= 0, 1.0, -1.0))
    assert not _deflation_ok()


def test_overlap_mass_swap_is_caught(monkeypatch):
    def wrong(links, psi, mu, cfg, m_w=wil.M_W, antiperiodic_t=False):
        s = ovl.sign_apply(links, psi, cfg, m_w, antiperiodic_t)
        return 0.5 * ((1 - mu) * psi + (1 + mu) * ovl.gamma5(s))
    monkeypatch.setattr(ovl, "overlap", wrong)
    assert not _gw_circle_ok()
