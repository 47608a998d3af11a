"""GPU eigensolver (deflation input of Eq. 3) against dense eigh / the oracle K."""
import numpy as np
import pytest

from oracle import wilson
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx, ov_eigs
from tests.gpu_util import dev, host, need_gpu, torch
from tests.oracle_fixtures import field_shape, small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def test_eigs_match_dense_4x4():
    prob = small_problem()
    n_ev = 8
    evecs = torch.zeros((n_ev,) + field_shape(prob["dims"]), dtype=torch.complex128, device="cuda")
    with Ctx(prob["dims"], dev(prob["links"]), "fp64") as c:
        evals, lmax = ov_eigs(c.handle, n_ev, 1e-11, 400, evecs)
    ev = host(evecs)
    assert lmax >= np.max(np.abs(prob["w_all"]))
    assert np.max(np.abs(evals - prob["w_all"][:n_ev])) < 1e-9
    for i in range(n_ev):
        r = wilson.kernel_k(prob["links"], ev[i]) - evals[i] * ev[i]
        assert np.linalg.norm(r) < 1e-9
    gram = np.einsum("ia,ja->ij", ev.reshape(n_ev, -1).conj(), ev.reshape(n_ev, -1))
    assert np.max(np.abs(gram - np.eye(n_ev))) < 1e-10
    # same invariant subspace as the dense eigenvectors
    pd = prob["evecs"].reshape(n_ev, -1)
    overlap = np.abs(np.einsum("ia,ja->ij", pd.conj(), ev.reshape(n_ev, -1))) ** 2
    assert np.allclose(overlap.sum(axis=1), 1.0, atol=1e-9)


def test_eigs_fp32_8x8_residuals():
    dims = (8, 8, 8, 8)
    links = inputs.gauge_links(dims, seed=6001)
    n_ev = 12
    evecs = torch.zeros((n_ev,) + field_shape(dims), dtype=torch.complex128, device="cuda")
    with Ctx(dims, dev(links), "fp32") as c:
        evals, lmax = ov_eigs(c.handle, n_ev, 2e-5, 400, evecs)
    ev = host(evecs)
    assert np.all(np.diff(np.abs(evals)) >= -1e-6)
    for i in range(n_ev):
        r = wilson.kernel_k(links, ev[i]) - evals[i] * ev[i]
        assert np.linalg.norm(r) < 5e-5 * lmax
    gram = np.einsum("ia,ja->ij", ev.reshape(n_ev, -1).conj(), ev.reshape(n_ev, -1))
    assert np.max(np.abs(gram - np.eye(n_ev))) < 1e-5


def test_eigs_block_wider_than_one_gram_tile():
    """30 pairs: a block of 75 vectors, so every Gram matrix of the iteration is
    assembled from 64-vector tiles (4^4, FP64, against dense eigh)."""
    prob = small_problem()
    n_ev = 30
    evecs = torch.zeros((n_ev,) + field_shape(prob["dims"]), dtype=torch.complex128, device="cuda")
    with Ctx(prob["dims"], dev(prob["links"]), "fp64") as c:
        evals, lmax = ov_eigs(c.handle, n_ev, 1e-10, 600, evecs)
    ev = host(evecs).reshape(n_ev, -1)
    w = prob["w_all"]
    # the 30 smallest |lambda|; a degenerate pair may straddle the cut, so compare |lambda|
    assert np.max(np.abs(np.abs(evals) - np.abs(w[:n_ev]))) < 1e-8
    for i in range(n_ev):
        r = wilson.kernel_k(prob["links"], ev[i].reshape(field_shape(prob["dims"]))) - evals[i] * ev[i].reshape(
            field_shape(prob["dims"]))
        assert np.linalg.norm(r) < 1e-8
    gram = ev.conj() @ ev.T
    assert np.max(np.abs(gram - np.eye(n_ev))) < 1e-9
