"""Output checks (ov_set_checks): a finite output passes unchanged, a NaN or
Inf in the output is reported as OV_ERR_NONFINITE, and with checks off the
non-finite values come back as computed.  4^4, FP32 context."""
import numpy as np
import pytest

from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, OverlapError, ov_set_checks
from tests.gpu_util import dev, need_gpu, torch
from tests.oracle_fixtures import small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def test_output_checks():
    prob = small_problem()
    b = inputs.gaussian_source(prob["dims"], seed=9601)
    bad = b.copy()
    bad[0, 1, 2, 3, 0, 0, 1] = np.nan
    inf = b.copy()
    inf[0, 0, 0, 0, 2, 1, 0] = np.inf
    with Ctx(prob["dims"], dev(prob["links"]), "fp32") as c:
        c.sign_config(16, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
        ref = c.overlap(dev(b), 0.05)
        ov_set_checks(c.handle, 1)
        again = c.overlap(dev(b), 0.05)
        assert torch.equal(ref, again)  # the scan leaves the result alone, bit for bit
        for x in (bad, inf):
            with pytest.raises(OverlapError) as e:
                c.overlap(dev(x), 0.05)
            assert e.value.status == 6
            with pytest.raises(OverlapError) as e:
                c.wilson(dev(x))
            assert e.value.status == 6
        ov_set_checks(c.handle, 0)
        out = c.overlap(dev(bad), 0.05)
        assert not torch.isfinite(out).all()
