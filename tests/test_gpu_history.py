"""Residual history of the solvers (ov_get_residual_history): one entry per
FP64 pass, the last equal to the residual the solve returns, the sequence
falling; 4^4, FP16 storage, both ov_solve and ov_solve_gmresr."""
import pytest

from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, ov_get_residual_history
from tests.gpu_util import dev, need_gpu
from tests.oracle_fixtures import small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("solver", ["cg", "gmresr"])
def test_residual_history(solver):
    prob = small_problem()
    b = dev(inputs.gaussian_source(prob["dims"], seed=9701))
    with Ctx(prob["dims"], dev(prob["links"]), "fp16") as c:
        c.sign_config(48, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
        _, _, res = c.solve(b, 0.05) if solver == "cg" else c.solve_gmresr(b, 0.05)
        hist = ov_get_residual_history(c.handle)
        outer = c.stats()["outer_iterations"]
    assert len(hist) == outer >= 2
    assert hist[-1] == res and res <= 1e-10
    assert all(b_ < a_ for a_, b_ in zip(hist, hist[1:])), hist
