"""GMRESR with the FP32 GCR level of a 16-bit context against the FP64 oracle
on 4^4 with 8 deflated pairs: same solution (dense solve of the polynomial
operator, the oracle's residual), no more FP64 passes than GCR in the
storage precision (ov_set_gmresr_fp32_level off), whether the FP32 copy is
made by ov_enable_fp32_operator before or after the sign configuration or by
the solver itself on its first call (the default); a no-op on FP32 contexts.
Every case builds its own contexts, so the tests depend on no other test."""
import numpy as np
import pytest

from oracle import chebyshev, dense, overlap
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, ov_enable_fp32_operator, ov_set_gmresr_fp32_level
from tests.gpu_util import dev, host, need_gpu
from tests.oracle_fixtures import small_problem

pytestmark = pytest.mark.gpu

ORDER, MU = 48, 0.05


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def problem():
    prob = small_problem()
    cfg = overlap.SignConfig(chebyshev.coefficients(ORDER, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    vol = inputs.volume(prob["dims"])
    w, v = dense.sorted_eigh(prob["kmat"])
    s = chebyshev.p_scalar(cfg.coeffs, cfg.a, cfg.b, w)
    s[:8] = np.where(w[:8] >= 0, 1.0, -1.0)
    dmat = 0.5 * ((1 + MU) * np.eye(12 * vol) + (1 - MU) * dense.gamma5_matrix(vol) @ ((v * s) @ v.conj().T))
    return prob, cfg, dmat


def _solve(prob, b, prec, fp32_level, enable_first=True, automatic=False):
    with Ctx(prob["dims"], dev(prob["links"]), prec) as c:
        if not fp32_level:
            ov_set_gmresr_fp32_level(c.handle, 0)
        elif enable_first and not automatic:
            ov_enable_fp32_operator(c.handle, dev(prob["links"]))
        c.sign_config(ORDER, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
        if fp32_level and not enable_first and not automatic:
            ov_enable_fp32_operator(c.handle, prob["links"])  # host links
        x, it, res = c.solve_gmresr(dev(b), MU)
        return host(x), res, c.stats()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("enable_first", [True, False])
def test_gmresr_fp32_gcr_level(problem, prec, enable_first):
    prob, cfg, dmat = problem
    b = inputs.gaussian_source(prob["dims"], seed=9508, nrhs=2)
    x, res, st = _solve(prob, b, prec, True, enable_first)
    _, res0, st0 = _solve(prob, b, prec, False)
    print(f"{prec}: FP64 passes {st['outer_iterations']} with the FP32 level, {st0['outer_iterations']} without; "
          f"GCR steps {st['gcr_iterations']} / {st0['gcr_iterations']}")
    assert res <= 1e-10 and res0 <= 1e-10
    assert st["outer_iterations"] <= st0["outer_iterations"]
    for r in range(2):
        rr = b[r] - overlap.overlap(prob["links"], x[r], MU, cfg)
        assert np.linalg.norm(rr) <= 2e-10 * np.linalg.norm(b[r]), r
        want = np.linalg.solve(dmat, b[r].ravel())
        assert np.linalg.norm(x[r].ravel() - want) <= 1e-8 * np.linalg.norm(want), r


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_fp32_level_is_the_default(problem, prec):
    """Without any call, the solver builds the FP32 copy from the context's own
    FP64 links: the result equals, bit for bit, that of a context given the
    FP32 copy by ov_enable_fp32_operator (4^4: no stencil tuning, so both
    contexts run the same launch shapes)."""
    prob, _, _ = problem
    b = inputs.gaussian_source(prob["dims"], seed=9510, nrhs=2)
    x_auto, res_auto, st_auto = _solve(prob, b, prec, True, automatic=True)
    x_exp, res_exp, st_exp = _solve(prob, b, prec, True)
    assert res_auto <= 1e-10
    assert st_auto["outer_iterations"] == st_exp["outer_iterations"]
    assert np.array_equal(x_auto, x_exp)


def test_fp32_operator_is_a_no_op_on_fp32_contexts(problem):
    prob, _, _ = problem
    b = inputs.gaussian_source(prob["dims"], seed=9509)
    x0, res0, _ = _solve(prob, b, "fp32", False)
    x1, res1, _ = _solve(prob, b, "fp32", True)
    # each context tunes its own stencil shape, so the two agree to the solve's accuracy, not bitwise
    assert res0 <= 1e-10 and res1 <= 1e-10
    assert np.linalg.norm(x1 - x0) <= 1e-8 * np.linalg.norm(x0)
