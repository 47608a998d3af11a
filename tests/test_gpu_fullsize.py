"""Full-size (24^3 x 48) checks in the launch configuration bench.py times
(autotuned stencil, 16-bit links persisting in L2): the stencil against the
oracle on the whole field, and sign(K) with 40 deflated pairs (from ov_eigs)
through properties that hold at any size."""
import numpy as np
import pytest

from oracle import wilson
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, ov_eigs
from tests.gpu_util import dev, host, need_gpu, rel, torch

pytestmark = pytest.mark.gpu

DIMS = (24, 24, 24, 48)
SHAPE = (48, 24, 24, 24, 4, 3)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def links():
    return inputs.gauge_links(DIMS, seed=1003)


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("fp32", 1e-6)])
def test_stencil_full_size(links, prec, tol):
    psi = inputs.gaussian_source(DIMS, seed=2003)
    with Ctx(DIMS, dev(links), prec) as c:
        got = host(c.kernel(dev(psi)))
    want = wilson.kernel_k(links, psi[0])[None]
    assert rel(got, want) < tol


@pytest.mark.parametrize("prec,tol_h,tol_inv", [("fp32", 1e-6, 1e-5), ("fp16", 2e-3, 2e-2)])
def test_sign_full_size_properties(links, prec, tol_h, tol_inv):
    """<phi, S psi> = <S phi, psi> (S Hermitian) and S(S psi) = psi up to the
    Chebyshev error and storage rounding, order 256, 40 deflated pairs."""
    n_ev = 40
    ld = dev(links)
    evecs = torch.zeros((n_ev + 1,) + SHAPE, dtype=torch.complex128, device="cuda")
    with Ctx(DIMS, ld, "fp32") as c32:
        evals, lmax = ov_eigs(c32.handle, n_ev + 1, 2e-5, 300, evecs)
    a, b = float(abs(evals[n_ev])), float(lmax)
    phi = dev(inputs.gaussian_source(DIMS, seed=2004))
    psi = dev(inputs.gaussian_source(DIMS, seed=2005))
    with Ctx(DIMS, ld, prec) as c:
        c.sign_config(256, a, b, evals[:n_ev], evecs[:n_ev].contiguous())
        s_psi = c.sign(psi)
        s_phi = c.sign(phi)
        ss_psi = c.sign(s_psi)
    lhs = torch.vdot(phi.flatten(), s_psi.flatten()).item()
    rhs = torch.vdot(s_phi.flatten(), psi.flatten()).item()
    assert abs(lhs - rhs) < tol_h * np.linalg.norm(host(phi)) * np.linalg.norm(host(psi))
    assert rel(host(ss_psi), host(psi)) < tol_inv
