"""GPU over-improved stout smearing (ov_stout_smear) against the FP64 oracle:

  * element by element on whole lattices (asymmetric 4x3x2x5 with length-2
    wrap-around, 8^4 spanning many thread blocks), the paper's parameters
    (rho = 0.1, eps = -0.25, 3 steps) and plain stout (eps = 1);
  * in place (links_out = links_in) equals out of place; steps = 0 copies;
  * at 24^3 x 48 (3 steps, the paper's parameters), properties that hold at
    any size: the output is SU(3), smearing commutes with a random gauge
    transformation, and sampled links equal the oracle run on a periodic
    window cut around them (the smeared link depends on links within
    distance 6 of its site, so a 16^4 window centred on it is exact).
"""
import numpy as np
import pytest

from oracle import smear
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import OverlapError, ov_stout_smear
from tests.gpu_util import dev, host, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("dims", [(4, 3, 2, 5), (8, 8, 8, 8)])
@pytest.mark.parametrize("eps", [-0.25, 1.0])
def test_smear_matches_oracle(dims, eps):
    links = inputs.gauge_links(dims, seed=611)
    want = smear.stout_smear(links, 0.1, eps, 3)
    d_in = dev(links)
    d_out = torch.empty_like(d_in)
    ov_stout_smear(dims, d_in, d_out, 0.1, eps, 3)
    got = host(d_out)
    assert np.max(np.abs(got - want)) < 1e-13
    assert np.array_equal(host(d_in), links)  # input untouched


def test_smear_in_place_and_zero_steps():
    dims = (4, 4, 4, 4)
    links = inputs.gauge_links(dims, seed=612)
    a = dev(links)
    b = torch.empty_like(a)
    ov_stout_smear(dims, a, b, 0.1, -0.25, 2)
    ov_stout_smear(dims, a, a, 0.1, -0.25, 2)
    assert torch.equal(a, b)
    c = torch.zeros_like(b)
    ov_stout_smear(dims, b, c, 0.1, -0.25, 0)
    assert torch.equal(b, c)


def test_smear_rejects_host_pointers():
    dims = (2, 2, 2, 2)
    links = inputs.gauge_links(dims, seed=613)
    with pytest.raises(OverlapError) as e:
        ov_stout_smear(dims, links, links.copy(), 0.1, -0.25, 1)
    assert e.value.status == 1


def _gauge(u, g, mu):
    """g(x) U_mu(x) g(x + mu)^dagger on the device (axes t, z, y, x)."""
    gs = torch.roll(g, shifts=-1, dims=(3, 2, 1, 0)[mu])
    return g @ u @ gs.conj().transpose(-1, -2)


def test_smear_fullsize_properties():
    dims = (24, 24, 24, 48)
    links = inputs.gauge_links(dims, seed=1003)
    d = dev(links)
    out = torch.empty_like(d)
    ov_stout_smear(dims, d, out, 0.1, -0.25, 3)
    eye = torch.eye(3, dtype=out.dtype, device=out.device)
    unit = (out @ out.conj().transpose(-1, -2) - eye).abs().max().item()
    det = (torch.linalg.det(out) - 1).abs().max().item()
    assert unit < 1e-13 and det < 1e-13

    # gauge covariance
    g = dev(inputs.gauge_transform(dims, seed=1004))
    dg = torch.stack([_gauge(d[mu], g, mu) for mu in range(4)])
    del d
    outg = torch.empty_like(dg)
    ov_stout_smear(dims, dg, outg, 0.1, -0.25, 3)
    want = torch.stack([_gauge(out[mu], g, mu) for mu in range(4)])
    assert (outg - want).abs().max().item() < 1e-12
    del dg, outg, want, g

    # sampled links against the oracle on 16^4 windows (periodic on the
    # window; exact at its centre, which sees only links within distance 6)
    w = 16
    res = host(out)
    rng = np.random.default_rng(1005)
    for _ in range(2):
        x0 = [int(rng.integers(0, n)) for n in dims]  # x, y, z, t
        idx = [np.arange(x0[a] - w // 2, x0[a] + w // 2) % dims[a] for a in range(4)]
        win = links[:, idx[3]][:, :, idx[2]][:, :, :, idx[1]][:, :, :, :, idx[0]]
        sm = smear.stout_smear(np.ascontiguousarray(win), 0.1, -0.25, 3)
        c = w // 2
        for mu in range(4):
            got = res[mu, x0[3], x0[2], x0[1], x0[0]]
            assert np.max(np.abs(got - sm[mu, c, c, c, c])) < 1e-13
