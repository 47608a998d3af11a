"""sign(K), D[mu] and D[mu]^dagger on an 8^3 x 32 lattice (the smaller of the
paper's two volumes, Sec. 3) in the launch shape the autotuner picks for this
lattice (V = 16384: the tuner runs at context creation), Chebyshev order 64.

Against the FP64 oracle, the deflation vectors are seeded orthonormal vectors
with chosen sgn(lambda): the projected form of Eq. 3 is defined for any
orthonormal set, and no oracle input may come from the CUDA path, so the
eigenpairs ov_eigs finds cannot serve here.  The realistic case (pairs from
ov_eigs, interval [|lambda_13|, lambda_max]) is checked CUDA against CUDA:
every storage precision against the FP64 path with the same pairs, which the
oracle comparison pins.  The 16-bit paths are checked on the whole field and
site by site (site_rel), which an error confined to a boundary plane or to
the tail blocks of a launch would fail."""
import numpy as np
import pytest

from oracle import chebyshev, overlap, wilson
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, ov_eigs
from tests.gpu_util import dev, host, need_gpu, rel, site_rel, torch
from tests.oracle_fixtures import field_shape

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 32)
N_EV, ORDER, MU = 12, 64, 0.05
SIGN_TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-2, "bf16": 6e-2}
SITE_FACTOR = 2.5


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def problem():
    need_gpu()
    links = inputs.gauge_links(DIMS, seed=4601)
    rng = np.random.default_rng(4604)
    vol = inputs.volume(DIMS)
    m = rng.standard_normal((12 * vol, N_EV)) + 1j * rng.standard_normal((12 * vol, N_EV))
    q, _ = np.linalg.qr(m)
    ev = np.ascontiguousarray(q.T).reshape((N_EV,) + field_shape(DIMS))
    evals = np.array([0.11, -0.13, 0.16, -0.18, 0.2, -0.22, 0.25, -0.27, 0.3, -0.31, 0.33, -0.35])
    a, b = 0.4, 6.6
    cfg = overlap.SignConfig(chebyshev.coefficients(ORDER, a, b), a, b, evals, ev)
    psi = inputs.gaussian_source(DIMS, seed=4602)
    want = {"sign": overlap.sign_apply(links, psi[0], cfg)[None],
            "D": overlap.overlap(links, psi[0], MU, cfg)[None],
            "Ddag": overlap.overlap_dag(links, psi[0], MU, cfg)[None]}
    return dict(links=links, evals=evals, evecs=ev, a=a, b=b, psi=psi, want=want)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_sign_and_overlap_tuned_8x8x8x32(problem, prec):
    p = problem
    with Ctx(DIMS, dev(p["links"]), prec) as c:
        st = c.stats()
        assert st["stencil_tpb"] > 0  # the tuned shape this context runs
        c.sign_config(ORDER, p["a"], p["b"], p["evals"], dev(p["evecs"]))
        got = {"sign": host(c.sign(dev(p["psi"]))),
               "D": host(c.overlap(dev(p["psi"]), MU)),
               "Ddag": host(c.overlap(dev(p["psi"]), MU, dagger=True))}
    for k, want in p["want"].items():
        err, serr = rel(got[k], want), site_rel(got[k], want)
        print(f"{prec} {k}: field {err:.2e}, worst site {serr:.2e}, stencil {st['stencil_tpb']},"
              f"{st['stencil_minb']},{st['stencil_lrec']} async {st['stencil_async']} brick {st['stencil_brick']}")
        assert err < SIGN_TOL[prec], k
        assert serr < SITE_FACTOR * SIGN_TOL[prec], k


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("bf16", 1.5e-2)])
def test_stencil_site_errors_8x8x8x32(problem, prec, tol):
    """K on 3 right-hand sides in the tuned 1- and 3-RHS shapes: whole field and
    worst site against the oracle."""
    p = problem
    psi = inputs.gaussian_source(DIMS, seed=4603, nrhs=3)
    want = np.stack([wilson.kernel_k(p["links"], x) for x in psi])
    with Ctx(DIMS, dev(p["links"]), prec) as c:
        got1 = host(c.kernel(dev(psi[:1])))
        got3 = host(c.kernel(dev(psi)))
    assert rel(got1, want[:1]) < tol and site_rel(got1, want[:1]) < SITE_FACTOR * tol
    assert rel(got3, want) < tol and site_rel(got3, want) < SITE_FACTOR * tol


def test_sign_with_eigs_pairs_8x8x8x32(problem):
    """Pairs from ov_eigs (13 found, 12 deflated, interval [|lambda_13|,
    lambda_max]): FP32, FP16 and BF16 against the FP64 path on the same pairs."""
    p = problem
    shape = (N_EV + 1,) + field_shape(DIMS)
    evecs = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    with Ctx(DIMS, dev(p["links"]), "fp32") as c:
        evals, lmax = ov_eigs(c.handle, N_EV + 1, 2e-5, 3000, evecs, allow_not_converged=True)
    a, b = float(abs(evals[N_EV])), float(lmax)
    ev = evecs[:N_EV].contiguous()
    out = {}
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        with Ctx(DIMS, dev(p["links"]), prec) as c:
            c.sign_config(ORDER, a, b, evals[:N_EV], ev)
            out[prec] = (host(c.sign(dev(p["psi"]))), host(c.overlap(dev(p["psi"]), MU)))
    for prec in ("fp32", "fp16", "bf16"):
        for k in range(2):
            assert rel(out[prec][k], out["fp64"][k]) < SIGN_TOL[prec], (prec, k)
            assert site_rel(out[prec][k], out["fp64"][k]) < SITE_FACTOR * SIGN_TOL[prec], (prec, k)
