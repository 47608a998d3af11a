"""GPU CG on D^dagger D against the oracle: the true residual of the GPU solution
is recomputed by the ORACLE operator (one D^dagger D application in FP64 on the
CPU), and the solution is compared with a dense solve of the same system."""
import numpy as np
import pytest

from oracle import chebyshev, dense, overlap
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, ov_set_solver_params
from tests.gpu_util import dev, host, need_gpu, torch
from tests.oracle_fixtures import small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _dense_x(prob, cfg, mu, b):
    w, v = dense.sorted_eigh(prob["kmat"])
    n_ev = len(cfg.evals)
    s = chebyshev.p_scalar(cfg.coeffs, cfg.a, cfg.b, w)
    s[:n_ev] = np.where(w[:n_ev] >= 0, 1.0, -1.0)
    smat = (v * s) @ v.conj().T
    vol = inputs.volume(prob["dims"])
    dmat = 0.5 * ((1 + mu) * np.eye(12 * vol) + (1 - mu) * dense.gamma5_matrix(vol) @ smat)
    return np.linalg.solve(dmat, b.ravel()).reshape(b.shape)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_solve_true_residual(prec):
    prob = small_problem()
    order, mu, tol = 48, 0.05, 1e-10
    cfg = overlap.SignConfig(chebyshev.coefficients(order, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    b = inputs.gaussian_source(prob["dims"], seed=5001, nrhs=2)
    with Ctx(prob["dims"], dev(prob["links"]), prec) as c:
        c.sign_config(order, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
        x, iters, res = c.solve(dev(b), mu, tol=tol, maxit=20000)
        stats = c.stats()
    x = host(x)
    print(prec, iters, res, stats)
    assert res <= tol
    for r in range(b.shape[0]):
        rhs = overlap.overlap_dag(prob["links"], b[r], mu, cfg)
        true_r = rhs - overlap.normal_op(prob["links"], x[r], mu, cfg)
        assert np.linalg.norm(true_r) / np.linalg.norm(rhs) <= 2 * tol
        x_ref = _dense_x(prob, cfg, mu, b[r])
        # error <= cond(D^dag D) * residual
        assert np.linalg.norm(x[r] - x_ref) / np.linalg.norm(x_ref) < 4e-7
    if prec != "fp64":
        assert stats["outer_iterations"] >= 2


def test_solve_maxit_reports_not_converged():
    prob = small_problem()
    b = dev(inputs.gaussian_source(prob["dims"], seed=5101))
    with Ctx(prob["dims"], dev(prob["links"]), "fp64") as c:
        c.sign_config(16, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
        from paper_1510_06897_gb300.binding import ov_solve
        x = torch.empty_like(b)
        it, res = ov_solve(c.handle, 0.05, 1e-12, 5, b, x, 1, allow_not_converged=True)
        assert it <= 5 and res > 1e-12
        assert np.all(np.isfinite(host(x)))
