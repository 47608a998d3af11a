"""Pins of the over-improved stout smearing oracle (oracle/smear.py):

  * rho = 0 leaves the field unchanged; the free field stays free;
  * gauge covariance: smearing U^g gives (smeared U)^g;
  * the smeared links are SU(3); plain stout raises the average plaquette
    step by step, the over-improved staple on its first step;
  * diagonal (abelian) fields: the update equals the closed form
    theta' = theta + Im Omega_kk - mean_k Im Omega_kk, with every staple's
    phase written out by hand as a sum of link angles;
  * the staple weights: for a small transverse abelian plane wave of
    momentum k the relative update is -rho [k^2 - eps/12 k^4 + O(k^6)]
    (normalised to the continuum Laplacian; the O(a^2) term proportional to
    eps, zero at the tree-level Symanzik eps = 0 and -k^4/12 for plain stout
    at eps = 1), which fixes both weights;
  * planted mistakes (rectangle weight sign, a missing rectangle staple, the
    trace term dropped) each fail one of these.
"""
import numpy as np
import pytest

import oracle.smear as sm
from paper_1510_06897_gb300 import inputs

DIMS = (4, 3, 2, 5)  # asymmetric, so that an axis mix-up shows
_AX = (3, 2, 1, 0)


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def test_rho_zero_is_identity():
    links = inputs.gauge_links(DIMS, seed=601)
    out = sm.stout_smear(links, rho=0.0, eps=-0.25, steps=2)
    assert np.max(np.abs(out - links)) < 1e-14


def test_free_field_stays_free():
    links = inputs.unit_links(DIMS)
    out = sm.stout_smear(links, rho=0.1, eps=-0.25, steps=3)
    assert np.max(np.abs(out - links)) < 1e-14


def _gauge_ok(eps=-0.25):
    links = inputs.gauge_links(DIMS, seed=602)
    g = inputs.gauge_transform(DIMS, seed=603)
    gl = np.empty_like(links)
    for mu in range(4):
        gl[mu] = g @ links[mu] @ _dag(np.roll(g, -1, axis=_AX[mu]))
    a = sm.stout_smear(gl, 0.1, eps, 1)
    b = sm.stout_smear(links, 0.1, eps, 1)
    for mu in range(4):
        b[mu] = g @ b[mu] @ _dag(np.roll(g, -1, axis=_AX[mu]))
    return np.max(np.abs(a - b)) < 1e-13


def test_gauge_covariance():
    assert _gauge_ok(-0.25) and _gauge_ok(1.0)


def _su3_ok():
    links = inputs.gauge_links(DIMS, seed=604)
    out = sm.stout_smear(links, 0.1, -0.25, 3)
    unit = np.max(np.abs(out @ _dag(out) - np.eye(3)))
    det = np.max(np.abs(np.linalg.det(out) - 1.0))
    return unit < 1e-13 and det < 1e-13


def test_output_is_su3():
    assert _su3_ok()


def test_plaquette_rises():
    """Plain stout (eps = 1) smooths monotonically; the over-improved staple
    at rho = 0.1 damps the shortest wavelength only by a factor
    1 - rho (16 - 4 eps) = -0.7 per step (see the small-k response below),
    so on these rough fields only its first step is sure to raise the
    plaquette."""
    links = inputs.gauge_links(DIMS, seed=605)
    p = [sm.average_plaquette(links)]
    for _ in range(3):
        links = sm.stout_step(links, 0.1, 1.0)
        p.append(sm.average_plaquette(links))
    assert all(b > a for a, b in zip(p, p[1:])), p
    links = inputs.gauge_links(DIMS, seed=605)
    assert sm.average_plaquette(sm.stout_step(links, 0.1, -0.25)) > p[0] + 0.1


# ---- abelian closed form ----------------------------------------------------

def _shift(f, off):
    for mu in range(4):
        if off[mu]:
            f = np.roll(f, -off[mu], axis=_AX[mu])
    return f


def _e(mu, k=1):
    o = [0, 0, 0, 0]
    o[mu] = k
    return o


def _add(*offs):
    return [sum(c) for c in zip(*offs)]


def _staple_phases(th, mu, nu, s):
    """Phases of the plaquette staple and the three rectangle staples of
    U_mu in the (mu, nu) plane on the side s, written as link-angle sums.
    th[d] is the angle field of the links in direction d."""
    def t(d, off):
        return _shift(th[d], off)
    m, n = _e(mu), _e(nu, s)
    n2, mm, nm, zero = _e(nu, 2 * s), _e(mu, -1), _e(nu, -s), [0, 0, 0, 0]
    if s > 0:
        plaq = t(nu, zero) + t(mu, n) - t(nu, m)
        r12 = t(nu, zero) + t(nu, n) + t(mu, n2) - t(nu, _add(m, n)) - t(nu, m)
        r21a = t(nu, zero) + t(mu, n) + t(mu, _add(m, n)) - t(nu, _e(mu, 2)) - t(mu, m)
        r21b = -t(mu, mm) + t(nu, mm) + t(mu, _add(mm, n)) + t(mu, n) - t(nu, m)
    else:
        plaq = -t(nu, n) + t(mu, n) + t(nu, _add(n, m))
        r12 = -t(nu, n) - t(nu, n2) + t(mu, n2) + t(nu, _add(n2, m)) + t(nu, _add(n, m))
        r21a = -t(nu, n) + t(mu, n) + t(mu, _add(n, m)) + t(nu, _add(n, _e(mu, 2))) - t(mu, m)
        r21b = -t(mu, mm) - t(nu, _add(mm, n)) + t(mu, _add(mm, n)) + t(mu, n) + t(nu, _add(n, m))
    del nm
    return plaq, (r12, r21a, r21b)


def _abelian_links(theta):
    """diag(e^{i th0}, e^{i th1}, e^{-i (th0 + th1)}) per link; theta: (2, 4, ...)."""
    links = np.zeros(theta.shape[1:] + (3, 3), dtype=np.complex128)
    links[..., 0, 0] = np.exp(1j * theta[0])
    links[..., 1, 1] = np.exp(1j * theta[1])
    links[..., 2, 2] = np.exp(-1j * (theta[0] + theta[1]))
    return links


def _abelian_expected(theta, rho, eps):
    wp, wr = (5.0 - 2.0 * eps) / 3.0, -(1.0 - eps) / 12.0
    comps = [theta[0], theta[1], -(theta[0] + theta[1])]
    out = np.empty((3,) + theta.shape[1:])
    for mu in range(4):
        im = []
        for th in comps:
            c = 0.0
            for nu in range(4):
                if nu == mu:
                    continue
                for s in (1, -1):
                    plaq, rects = _staple_phases(th, mu, nu, s)
                    c = c + wp * np.exp(1j * plaq) + wr * sum(np.exp(1j * r) for r in rects)
            im.append(np.imag(rho * c * np.exp(-1j * th[mu])))
        mean = sum(im) / 3.0
        for k in range(3):
            out[k, mu] = comps[k][mu] + im[k] - mean
    return out


def _abelian_ok(eps):
    rng = np.random.default_rng(607)
    shape = (2, 4) + (DIMS[3], DIMS[2], DIMS[1], DIMS[0])
    theta = rng.uniform(-0.6, 0.6, size=shape)
    out = sm.stout_step(_abelian_links(theta), 0.1, eps)
    want = _abelian_expected(theta, 0.1, eps)
    got = np.stack([np.angle(out[..., k, k]) for k in range(3)])
    off = out.copy()
    for k in range(3):
        off[..., k, k] = 0.0
    return np.max(np.abs(off)) < 1e-14 and np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("eps", [-0.25, 0.0, 1.0])
def test_abelian_closed_form(eps):
    assert _abelian_ok(eps)


# ---- the staple weights from the small-k response ---------------------------

def _k4_coefficient(eps, amp=1e-3, length=64):
    """(R(k) - k^2)/k^4 extrapolated to k -> 0 (Richardson on k, 2k), with
    R(k) = -(theta' - theta) / (rho theta) for theta_x(x) = amp sin(k y)."""
    dims = (2, length, 2, 2)
    rho = 0.1
    r = {}
    for n in (1, 2):
        k = 2 * np.pi * n / length
        theta = np.zeros((2, 4, dims[3], dims[2], dims[1], dims[0]))
        y = np.arange(length)
        theta[0, 0] = amp * np.sin(k * y)[None, None, :, None]   # links in x vary along y
        theta[1, 0] = -theta[0, 0]
        out = sm.stout_step(_abelian_links(theta), rho, eps)
        yi = length // (4 * n)  # sin(k y) = 1
        th, th2 = theta[0, 0][0, 0, yi, 0], np.angle(out[0][0, 0, yi, 0, 0, 0])
        rk = -(th2 - th) / (rho * th)
        r[n] = (rk, k)
    c = {n: (rk - k * k) / k ** 4 for n, (rk, k) in r.items()}
    k1 = r[1][1]
    return (4 * c[1] - c[2]) / 3, r[1][0] / (k1 * k1)


def _weights_ok(eps):
    c4, norm = _k4_coefficient(eps)
    return abs(norm - 1.0) < 1e-2 and abs(c4 + eps / 12.0) < 1e-4


@pytest.mark.parametrize("eps", [-0.25, 0.0, 1.0])
def test_small_k_response_fixes_the_weights(eps):
    assert _weights_ok(eps)


# ---- planted mistakes -------------------------------------------------------

def test_planted_rectangle_weight_sign_fails(monkeypatch):
    monkeypatch.setattr(sm, "staple_weights", lambda eps: ((5.0 - 2.0 * eps) / 3.0, (1.0 - eps) / 12.0))
    assert not _weights_ok(-0.25)
    assert not _abelian_ok(-0.25)


def test_planted_missing_rectangle_fails(monkeypatch):
    full = sm.rectangle_paths
    monkeypatch.setattr(sm, "rectangle_paths", lambda mu: [p for i, p in enumerate(full(mu)) if i % 3 != 2])
    assert not _weights_ok(-0.25)
    assert not _abelian_ok(-0.25)


def test_planted_trace_term_dropped_fails(monkeypatch):
    monkeypatch.setattr(sm, "antihermitian_traceless", lambda om: 0.5 * (om - _dag(om)))
    assert not _su3_ok()
