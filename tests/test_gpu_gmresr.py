"""GPU SUMR (ov_sumr) and GMRESR (ov_solve_gmresr) against the FP64 oracle on
4^4 with 8 deflated pairs:

  * ov_sumr on an FP64 context equals the oracle's SUMR iterate after a fixed
    number of iterations (same polynomial sign, same recursion), and its
    estimate equals the oracle's;
  * ov_sumr run to a tolerance solves D[mu] x = b for the oracle's operator
    (FP64, FP32 contexts);
  * ov_solve_gmresr in every precision returns x with ||b - D x|| / ||b|| <=
    1e-10 recomputed by the ORACLE's operator and equal to the dense solve of
    the same polynomial operator; restarts (max_dirs 2) and an explicit
    relaxed order converge too.
"""
import numpy as np
import pytest

from oracle import chebyshev, dense, overlap, sumr
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, OverlapError, ov_set_gmresr_params
from tests.gpu_util import dev, host, need_gpu
from tests.oracle_fixtures import small_problem

pytestmark = pytest.mark.gpu

ORDER, MU = 48, 0.05


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def setup():
    prob = small_problem()
    cfg = overlap.SignConfig(chebyshev.coefficients(ORDER, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    return prob, cfg


@pytest.fixture(scope="module")
def dense_d(setup):
    """D[mu] of the order-48 deflated polynomial sign as a dense matrix."""
    prob, cfg = setup
    vol = inputs.volume(prob["dims"])
    w, v = dense.sorted_eigh(prob["kmat"])
    s = chebyshev.p_scalar(cfg.coeffs, cfg.a, cfg.b, w)
    s[:8] = np.where(w[:8] >= 0, 1.0, -1.0)
    smat = (v * s) @ v.conj().T
    return 0.5 * ((1 + MU) * np.eye(12 * vol) + (1 - MU) * dense.gamma5_matrix(vol) @ smat)


def _ctx(prob, prec):
    c = Ctx(prob["dims"], dev(prob["links"]), prec)
    c.sign_config(ORDER, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
    return c


def test_sumr_fp64_matches_oracle_iterates(setup):
    prob, cfg = setup
    b = inputs.gaussian_source(prob["dims"], seed=9501, nrhs=2)
    k = 12
    with _ctx(prob, "fp64") as c:
        x, it, est = c.sumr(dev(b), MU, 0.0, k)
        st = c.stats()
    x = host(x)
    assert it == k
    assert st["sign_applies"] == 2 * k  # one per RHS per iteration
    ests = []
    for r in range(2):
        want, _, e = sumr.overlap_sumr(prob["links"], b[r], MU, cfg, k)
        ests.append(e)
        assert np.linalg.norm(x[r] - want) <= 1e-10 * np.linalg.norm(want), r
    assert abs(est - max(ests)) <= 1e-10 * max(ests)


@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-10, 2e-10), ("fp32", 1e-7, 1e-4)])
def test_sumr_solves_overlap(setup, prec, tol, bound):
    prob, cfg = setup
    b = inputs.gaussian_source(prob["dims"], seed=9502)
    with _ctx(prob, prec) as c:
        x, it, est = c.sumr(dev(b), MU, tol, 2000)
    x = host(x)
    assert est <= tol and it < 2000
    r = b[0] - overlap.overlap(prob["links"], x[0], MU, cfg)
    assert np.linalg.norm(r) <= bound * np.linalg.norm(b[0])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_gmresr_matches_oracle(setup, dense_d, prec):
    prob, cfg = setup
    b = inputs.gaussian_source(prob["dims"], seed=9503, nrhs=2)
    with _ctx(prob, prec) as c:
        x, it, res = c.solve_gmresr(dev(b), MU)
        st = c.stats()
    x = host(x)
    print(f"{prec}: {it} SUMR iterations, {st['gcr_iterations']} GCR steps, {st['outer_iterations']} FP64 passes, "
          f"{st['sign_applies']} sign applies, residual {res:.1e}")
    assert res <= 1e-10
    assert st["gcr_iterations"] >= 1 and st["outer_iterations"] >= 1 and it >= st["gcr_iterations"]
    for r in range(2):
        rr = b[r] - overlap.overlap(prob["links"], x[r], MU, cfg)
        assert np.linalg.norm(rr) <= 2e-10 * np.linalg.norm(b[r]), r
        want = np.linalg.solve(dense_d, b[r].ravel())
        assert np.linalg.norm(x[r].ravel() - want) <= 1e-8 * np.linalg.norm(want), r


def test_gmresr_restarts_and_explicit_order(setup):
    prob, cfg = setup
    b = inputs.gaussian_source(prob["dims"], seed=9504)
    with _ctx(prob, "fp32") as c:
        ov_set_gmresr_params(c.handle, inner_order=12, inner_tol=0.3, inner_maxit=200, max_dirs=2)
        x, it, res = c.solve_gmresr(dev(b), MU)
        st = c.stats()
    assert res <= 1e-10 and st["gcr_iterations"] > 2
    rr = b[0] - overlap.overlap(prob["links"], host(x)[0], MU, cfg)
    assert np.linalg.norm(rr) <= 2e-10 * np.linalg.norm(b[0])


def test_gmresr_rejects_bad_arguments(setup):
    prob, _ = setup
    b = dev(inputs.gaussian_source(prob["dims"], seed=9505))
    with Ctx(prob["dims"], dev(prob["links"]), "fp32") as c:
        with pytest.raises(OverlapError) as e:
            c.solve_gmresr(b, MU)
        assert e.value.status == 5  # OV_ERR_STATE: no sign configuration
        c.sign_config(16, prob["a"], prob["b"])
        for mu in (1.0, -1.0, float("nan")):
            with pytest.raises(OverlapError) as e:
                c.solve_gmresr(b, mu)
            assert e.value.status == 1
        for args in ((-1, 0.1, 10, 4), (0, 1.0, 10, 4), (0, 0.1, 0, 4), (0, 0.1, 10, 0), (0, 0.1, 10, 65)):
            with pytest.raises(OverlapError) as e:
                ov_set_gmresr_params(c.handle, *args)
            assert e.value.status == 1


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_gmresr_ragged_antiperiodic_three_rhs(prec):
    """3x2x5x4 (volume not a multiple of any block), antiperiodic t, 6 dense
    eigenpairs deflated, order 20, 3 right-hand sides in one call."""
    prob = small_problem((3, 2, 5, 4), seed=4301, n_ev=6, antiperiodic=True)
    order, mu = 20, 0.05
    cfg = overlap.SignConfig(chebyshev.coefficients(order, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    vol = inputs.volume(prob["dims"])
    w, v = dense.sorted_eigh(prob["kmat"])
    s = chebyshev.p_scalar(cfg.coeffs, cfg.a, cfg.b, w)
    s[:6] = np.where(w[:6] >= 0, 1.0, -1.0)
    dmat = 0.5 * ((1 + mu) * np.eye(12 * vol) + (1 - mu) * dense.gamma5_matrix(vol) @ ((v * s) @ v.conj().T))
    b = inputs.gaussian_source(prob["dims"], seed=9506, nrhs=3)
    with Ctx(prob["dims"], dev(prob["links"]), prec, antiperiodic_t=True) as c:
        c.sign_config(order, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
        x, it, res = c.solve_gmresr(dev(b), mu)
    x = host(x)
    assert res <= 1e-10
    for r in range(3):
        rr = b[r] - overlap.overlap(prob["links"], x[r], mu, cfg, antiperiodic_t=True)
        assert np.linalg.norm(rr) <= 2e-10 * np.linalg.norm(b[r]), r
        want = np.linalg.solve(dmat, b[r].ravel())
        assert np.linalg.norm(x[r].ravel() - want) <= 1e-8 * np.linalg.norm(want), r


def test_sumr_fp64_three_rhs_larger_mu(setup):
    """Same iterates as the oracle for 3 RHS at mu = 0.3 after 8 steps (FP64
    batched deflation path)."""
    prob, cfg = setup
    b = inputs.gaussian_source(prob["dims"], seed=9507, nrhs=3)
    mu, k = 0.3, 8
    with _ctx(prob, "fp64") as c:
        x, it, est = c.sumr(dev(b), mu, 0.0, k)
    x = host(x)
    assert it == k
    for r in range(3):
        want, _, _ = sumr.overlap_sumr(prob["links"], b[r], mu, cfg, k)
        assert np.linalg.norm(x[r] - want) <= 1e-10 * np.linalg.norm(want), r
