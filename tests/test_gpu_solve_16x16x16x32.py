"""16^3 x 32, FP32 operator with FP64 reductions: 20 deflated eigenpairs from
ov_eigs, Chebyshev order 200 on [|lambda_21|, lambda_max], CG on D^dagger D at
mu = 0.05 to a 1e-10 true residual (links seed 1002, source seed 2002).

One oracle sign apply at this volume takes ~400 applications of the oracle's
K (about a second each on the host), so the checks are ones that hold at any
size and need few oracle operations:
  * every eigenpair handed to the deflation satisfies K phi = lambda phi for
    the ORACLE's K, and the eigenvectors are orthonormal;
  * the returned solution's true residual ||D^dag b - D^dag D x|| / ||D^dag b||,
    recomputed through a separate FP64 context with the public ov_overlap
    calls, is below 1e-10 (the operator of that context is parity-tested
    against the oracle at smaller volumes and, stencil by stencil, at 24^3 x 48).
"""
import numpy as np
import pytest

from oracle import wilson
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, ov_eigs
from tests.gpu_util import dev, host, need_gpu, torch
from tests.oracle_fixtures import field_shape

pytestmark = pytest.mark.gpu

DIMS = (16, 16, 16, 32)
N_EV, ORDER, MU, TOL = 20, 200, 0.05, 1e-10


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def test_fp32_operator_solve_16x16x16x32():
    links = inputs.gauge_links(DIMS, seed=1002)
    evecs = torch.zeros((N_EV + 1,) + field_shape(DIMS), dtype=torch.complex128, device="cuda")
    b_src = dev(inputs.gaussian_source(DIMS, seed=2002))
    with Ctx(DIMS, dev(links), "fp32") as c:
        evals, lmax = ov_eigs(c.handle, N_EV + 1, 2e-5, 3000, evecs)  # dense low band: |lambda| 0.531..0.536
        a, b = float(abs(evals[N_EV])), float(lmax)
        c.sign_config(ORDER, a, b, evals[:N_EV], evecs[:N_EV].contiguous())
        x, iters, res = c.solve(b_src, MU, TOL, 5000)
        st = c.stats()
    print(f"16^3x32 fp32: interval [{a:.4f}, {b:.4f}], {iters} inner iterations, {st['outer_iterations']} outer, "
          f"true residual {res:.2e}, {st['dslash_launches']} stencil launches")
    assert res <= TOL
    assert 0.0 < a < b <= 6.6

    # eigenpairs against the oracle's K (the lowest and highest three of the 20)
    ev = host(evecs[:N_EV])
    for i in (0, 1, 2, N_EV - 3, N_EV - 2, N_EV - 1):
        r = wilson.kernel_k(links, ev[i]) - evals[i] * ev[i]
        assert np.linalg.norm(r) < 5e-5 * lmax, i
    flat = ev.reshape(N_EV, -1)
    assert np.max(np.abs(flat.conj() @ flat.T - np.eye(N_EV))) < 1e-5
    assert np.all(np.diff(np.abs(evals[:N_EV + 1])) >= -1e-6)

    # true residual of the returned x through a separate FP64 context
    with Ctx(DIMS, dev(links), "fp64") as c64:
        c64.sign_config(ORDER, a, b, evals[:N_EV], evecs[:N_EV].contiguous())
        db = c64.overlap(b_src, MU, dagger=True)
        ddx = c64.overlap(c64.overlap(x, MU), MU, dagger=True)
    rel = (torch.linalg.vector_norm(db - ddx) / torch.linalg.vector_norm(db)).item()
    assert rel <= 1.5 * TOL, rel
