"""Over-improved stout smearing of the gauge links, FP64 (test infrastructure:
only tests/, smoke() and the CPU legs of bench.py use this module).

Sec. 3 prepares its ensembles with 3 steps of over-improved stout smearing,
rho = 0.1, epsilon = -0.25 (stout smearing of Morningstar and Peardon with
the over-improved staple of Moran and Leinweber, both cited there).  The
paper prints no formulas; the reading used:

  C_mu(x)  = rho sum_{nu != mu, +-} [ (5 - 2 eps)/3 (plaquette staple)
                                      - (1 - eps)/12 (the three rectangle staples) ]
  Omega    = C_mu(x) U_mu(x)^dagger
  Q        = i/2 (Omega^dagger - Omega) - i/6 tr(Omega^dagger - Omega)       (traceless Hermitian)
  U'_mu(x) = exp(i Q) U_mu(x),

all links updated at once from the old field.  A staple is the parallel
transporter from x to x + mu^ along a path of links: the plaquette staple
goes x -> x+nu' -> x+nu'+mu -> x+mu (nu' = +-nu); the rectangle staples
are the three 5-link paths that close a 1x2 or 2x1 rectangle with the link:
out 2 along nu', long side along mu starting at x, long side along mu
starting at x-mu.  A step along -nu from y uses U_nu(y - nu^)^dagger.
eps = 1 gives plain stout smearing, eps = 0 the tree-level Symanzik staple.
exp(iQ) is computed from the eigendecomposition of the Hermitian Q.

Pinned by: rho = 0 leaves the field unchanged, the free field stays free,
gauge covariance, the output is SU(3), the average plaquette rises, and for
diagonal (abelian) fields the closed form of the phase update written with
angles (tests/test_oracle_smear.py).
"""
import numpy as np

# direction mu -> axis of a (Lt, Lz, Ly, Lx, ...) field
_AXIS = (3, 2, 1, 0)


def _at(field, off):
    """field(x + off) for an integer offset off = (dx, dy, dz, dt), periodic."""
    out = field
    for mu in range(4):
        if off[mu]:
            out = np.roll(out, -off[mu], axis=_AXIS[mu])
    return out


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _step_link(links, d, off):
    """Link matrix of the step d (+-(mu + 1)) taken from x + off."""
    mu = abs(d) - 1
    if d > 0:
        return _at(links[mu], off)
    back = list(off)
    back[mu] -= 1
    return _dag(_at(links[mu], back))


def transporter(links, steps):
    """U_{d1}(x) U_{d2}(x + d1) ... along the signed directions in steps."""
    off = [0, 0, 0, 0]
    out = None
    for d in steps:
        m = _step_link(links, d, off)
        out = m if out is None else out @ m
        off[abs(d) - 1] += 1 if d > 0 else -1
    return out


def plaquette_paths(mu):
    """Signed-direction paths (1-based) of the plaquette staples of U_mu."""
    m = mu + 1
    return [[s * (nu + 1), m, -s * (nu + 1)] for nu in range(4) if nu != mu for s in (1, -1)]


def rectangle_paths(mu):
    """The three rectangle staples per (nu, sign) of U_mu."""
    m = mu + 1
    out = []
    for nu in range(4):
        if nu == mu:
            continue
        for s in (1, -1):
            n = s * (nu + 1)
            out.append([n, n, m, -n, -n])   # 1x2, out 2 along nu'
            out.append([n, m, m, -n, -m])   # 2x1, the link first on the long side
            out.append([-m, n, m, m, -n])   # 2x1, the link second on the long side
    return out


def staple_weights(eps):
    """(plaquette weight, rectangle weight) of the over-improved staple."""
    return (5.0 - 2.0 * eps) / 3.0, -(1.0 - eps) / 12.0


def antihermitian_traceless(omega):
    """i Q = 1/2 (Omega - Omega^dagger) - 1/6 tr(Omega - Omega^dagger)."""
    a = 0.5 * (omega - _dag(omega))
    tr = np.trace(a, axis1=-2, axis2=-1)[..., None, None]
    return a - tr / 3.0 * np.eye(3)


def expm_antihermitian(a):
    """exp(A) for anti-Hermitian A = iQ, from the eigendecomposition of Q."""
    w, v = np.linalg.eigh(-1j * a)
    return np.einsum("...ik,...k,...jk->...ij", v, np.exp(1j * w), v.conj())


def stout_step(links, rho, eps):
    """One over-improved stout step of every link (old field on the right)."""
    wp, wr = staple_weights(eps)
    out = np.empty_like(links)
    for mu in range(4):
        c = np.zeros_like(links[mu])
        for p in plaquette_paths(mu):
            c = c + wp * transporter(links, p)
        if wr != 0.0:
            for p in rectangle_paths(mu):
                c = c + wr * transporter(links, p)
        omega = rho * c @ _dag(links[mu])
        out[mu] = expm_antihermitian(antihermitian_traceless(omega)) @ links[mu]
    return out


def stout_smear(links, rho=0.1, eps=-0.25, steps=3):
    """steps over-improved stout steps (Sec. 3: rho = 0.1, eps = -0.25, 3 steps)."""
    out = links
    for _ in range(steps):
        out = stout_step(out, rho, eps)
    return out


def average_plaquette(links):
    """(1/3) Re tr of the plaquette, averaged over sites and the 6 planes."""
    total = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            p = transporter(links, [mu + 1, nu + 1, -(mu + 1), -(nu + 1)])
            total += np.trace(p, axis1=-2, axis2=-1).real.mean() / 3.0
    return total / 6.0
