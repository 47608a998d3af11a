"""GPU chiral-sector solve (ov_solve_chiral) against the FP64 oracle: the
solution of A x = P b with A = c0 P + chirality c1 P S P (one sign(K)
application per CG iteration) compared with a dense solve of the same
operator on the sector, its true residual recomputed by the ORACLE's
operator, and its opposite-chirality part exactly zero; every precision,
both chiralities, 4^4 with 8 deflated pairs."""
import numpy as np
import pytest

from oracle import chebyshev, dense, overlap
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, OverlapError
from tests.gpu_util import dev, host, need_gpu
from tests.oracle_fixtures import small_problem

pytestmark = pytest.mark.gpu

ORDER, MU = 48, 0.05


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _dense_sector_solve(prob, cfg, b, chirality):
    vol = inputs.volume(prob["dims"])
    w, v = dense.sorted_eigh(prob["kmat"])
    n_ev = len(cfg.evals)
    s = chebyshev.p_scalar(cfg.coeffs, cfg.a, cfg.b, w)
    s[:n_ev] = np.where(w[:n_ev] >= 0, 1.0, -1.0)
    smat = (v * s) @ v.conj().T
    pm = 0.5 * (np.eye(12 * vol) + chirality * dense.gamma5_matrix(vol))
    c0 = 0.25 * ((1 + MU) ** 2 + (1 - MU) ** 2)
    amat = c0 * pm + 0.5 * chirality * (1 - MU * MU) * pm @ smat @ pm
    pb = overlap.chiral_project(b, chirality).ravel()
    idx = np.where(np.diag(pm).real > 0.5)[0]
    x = np.zeros_like(pb)
    x[idx] = np.linalg.solve(amat[np.ix_(idx, idx)], pb[idx])
    return x.reshape(b.shape)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("chirality", [1, -1])
def test_chiral_solve_matches_oracle(prec, chirality):
    prob = small_problem()
    cfg = overlap.SignConfig(chebyshev.coefficients(ORDER, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    b = inputs.gaussian_source(prob["dims"], seed=9201, nrhs=2)
    with Ctx(prob["dims"], dev(prob["links"]), prec) as c:
        c.sign_config(ORDER, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
        x, it, res = c.solve_chiral(dev(b), MU, chirality)
        st = c.stats()
    x = host(x)
    assert res <= 1e-10
    # one sign apply per RHS per inner iteration (+ the FP64 outer residuals);
    # the D^dagger D solve needs two
    assert st["sign_applies"] <= 2 * (it + 12)
    for r in range(2):
        assert np.all(overlap.chiral_project(x[r], -chirality) == 0)
        ax = overlap.chiral_normal_op(prob["links"], x[r], MU, cfg, chirality)
        pb = overlap.chiral_project(b[r], chirality)
        assert np.linalg.norm(pb - ax) <= 2e-10 * np.linalg.norm(pb)
        want = _dense_sector_solve(prob, cfg, b[r], chirality)
        assert np.linalg.norm(x[r] - want) <= 1e-8 * np.linalg.norm(want)


def test_chiral_solve_rejects_bad_arguments():
    prob = small_problem()
    b = dev(inputs.gaussian_source(prob["dims"], seed=9202))
    with Ctx(prob["dims"], dev(prob["links"]), "fp32") as c:
        c.sign_config(16, prob["a"], prob["b"])
        for chi, mu in ((0, 0.1), (2, 0.1), (1, 1.0), (-1, -1.5)):
            with pytest.raises(OverlapError) as e:
                c.solve_chiral(b, mu, chi)
            assert e.value.status == 1
