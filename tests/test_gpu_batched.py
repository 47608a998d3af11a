"""Batched right-hand sides: every compiled stencil variant (threads per block,
register cap, right-hand sides per thread) pinned through OV_STENCIL, the
12 spin-colour point sources through sign(K) with batched deflation, D and
D^dagger, and a multi-RHS solve, all against the FP64 oracle."""
import os

import numpy as np
import pytest

from oracle import chebyshev, overlap, wilson
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx
from tests.gpu_util import dev, host, need_gpu, rel, torch
from tests.oracle_fixtures import field_shape, small_problem

pytestmark = pytest.mark.gpu

VARIANTS = [(128, 2, 1), (192, 3, 1), (256, 4, 1), (64, 5, 1), (128, 2, 2), (192, 3, 2), (96, 1, 3), (128, 2, 3),
            (64, 1, 4), (256, 2, 4), (64, 1, 6)]
TOL = {"fp64": 1e-13, "fp32": 1e-6, "fp16": 2e-3, "bf16": 1.5e-2}


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture
def pin(monkeypatch):
    def _pin(tpb, minb, rt, lrec=12):
        monkeypatch.setenv("OV_STENCIL", f"{tpb},{minb},{lrec},{rt}")
    return _pin


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_stencil_variants(pin, prec, variant):
    tpb, minb, rt = variant
    if prec == "fp64" and rt > 1:
        pytest.skip("FP64 is compiled with one RHS per thread")
    pin(tpb, minb, rt, lrec=18 if prec == "bf16" else 12)
    dims = (8, 6, 4, 10)
    links = inputs.gauge_links(dims, seed=8001)
    psi = inputs.gaussian_source(dims, seed=8002, nrhs=5)   # ragged against rt = 2 and 4
    with Ctx(dims, dev(links), prec, antiperiodic_t=True) as c:
        got = host(c.kernel(dev(psi)))
        assert c.stats()["stencil_tpb"] == tpb
    want = np.stack([wilson.kernel_k(links, p, antiperiodic_t=True) for p in psi])
    assert rel(got, want) < TOL[prec]


ASYNC_VARIANTS = [(64, 4, 1), (64, 3, 2), (96, 3, 1), (128, 4, 2), (256, 3, 1)]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("variant", ASYNC_VARIANTS)
def test_staged_stencil_variants(monkeypatch, prec, variant):
    """The shared-memory staged kernel (asynchronous copies, spinors and links or
    spinors only) pinned: D_W and K on a ragged plane (48 sites against 64- to
    256-thread blocks) with an antiperiodic t boundary, against the oracle and
    bit for bit against the gather kernel, which does the same arithmetic in
    the same order."""
    tpb, minb, staged = variant
    dims = (8, 6, 4, 10)
    links = inputs.gauge_links(dims, seed=8031)
    psi = inputs.gaussian_source(dims, seed=8032, nrhs=3)
    results = {}
    for name, pin in (("gather", f"{tpb},{minb},12,1"), ("staged", f"{tpb},{minb},12,1,{staged}")):
        monkeypatch.setenv("OV_STENCIL", pin)
        with Ctx(dims, dev(links), prec, antiperiodic_t=True) as c:
            assert c.stats()["stencil_async"] == (staged if name == "staged" else 0)
            results[name] = (c.wilson(dev(psi)), c.kernel(dev(psi)))
    assert torch.equal(results["gather"][0], results["staged"][0])
    assert torch.equal(results["gather"][1], results["staged"][1])
    want_w = np.stack([wilson.wilson(links, p, True) for p in psi])
    want_k = np.stack([wilson.kernel_k(links, p, antiperiodic_t=True) for p in psi])
    assert rel(host(results["staged"][0]), want_w) < TOL[prec]
    assert rel(host(results["staged"][1]), want_k) < TOL[prec]


BRICK_VARIANTS = [("64,4,{l},1,0", "fp16"), ("96,3,{l},1,0", "fp32"), ("192,3,{l},2,0", "bf16"), ("64,3,12,1,1", "fp16"),
                  ("128,4,12,1,2", "bf16"), ("64,4,12,1,0", "fp64"), ("128,2,{l},3,0", "fp16")]


@pytest.mark.parametrize("pin,prec", BRICK_VARIANTS)
def test_brick_mapping(monkeypatch, pin, prec):
    """Blocks mapped onto 8 x 4 x (tpb / 32) bricks of sites (8 x 4 x 12 x 6
    lattice: 2 to 6 brick layers in z, antiperiodic t): D_W and K against the
    oracle and bit for bit against the plane mapping of the same variant."""
    lrec = 18 if prec == "bf16" else 12
    pin = pin.format(l=lrec)
    dims = (8, 4, 12, 6)
    links = inputs.gauge_links(dims, seed=8051)
    psi = inputs.gaussian_source(dims, seed=8052, nrhs=3)
    res = {}
    for bk in (0, 1):
        monkeypatch.setenv("OV_STENCIL", f"{pin},{bk}")
        with Ctx(dims, dev(links), prec, antiperiodic_t=True) as c:
            assert c.stats()["stencil_brick"] == bk
            res[bk] = (c.wilson(dev(psi)), c.kernel(dev(psi)))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    want_w = np.stack([wilson.wilson(links, p, True) for p in psi])
    want_k = np.stack([wilson.kernel_k(links, p, antiperiodic_t=True) for p in psi])
    assert rel(host(res[1][0]), want_w) < TOL[prec]
    assert rel(host(res[1][1]), want_k) < TOL[prec]


@pytest.mark.parametrize("staged", [1, 2])
def test_staged_sign_and_overlap(monkeypatch, staged):
    """sign(K), D[mu] and D[mu]^dagger through the staged kernel: every
    epilogue form of the recurrence (three staged vectors), the deflation
    correction and the FP32 assembly, 8 deflated pairs at 4^4, order 24, FP16;
    bit for bit against the gather kernel and within the FP16 bound of the
    oracle."""
    prob = small_problem()
    psi = inputs.gaussian_source(prob["dims"], seed=8041, nrhs=2)
    order, mu = 24, 0.1
    cfg = overlap.SignConfig(chebyshev.coefficients(order, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    out = {}
    for name, pin in (("gather", "64,4,12,1"), ("staged", f"64,4,12,1,{staged}")):
        monkeypatch.setenv("OV_STENCIL", pin)
        with Ctx(prob["dims"], dev(prob["links"]), "fp16") as c:
            c.sign_config(order, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
            out[name] = (c.sign(dev(psi)), c.overlap(dev(psi), mu), c.overlap(dev(psi), mu, dagger=True))
    for g, s in zip(out["gather"], out["staged"]):
        assert torch.equal(g, s)
    want = [np.stack([overlap.sign_apply(prob["links"], p, cfg) for p in psi]),
            np.stack([overlap.overlap(prob["links"], p, mu, cfg) for p in psi]),
            np.stack([overlap.overlap_dag(prob["links"], p, mu, cfg) for p in psi])]
    for got, w in zip(out["staged"], want):
        assert rel(host(got), w) < 1e-2


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("dims,nrhs", [((8, 4, 5, 6), 3), ((8, 4, 6, 16), 4), ((32, 2, 2, 2), 1)])
def test_slab_stencil(monkeypatch, prec, dims, nrhs):
    """The slab kernel pinned: D_W and K on several right-hand sides, with more
    (rhs, slice) items than CTAs in the second case (each CTA cycles through
    both shared-memory buffers several times) and Lz = Lt = 2 in the third
    (the +mu and -mu planes coincide)."""
    monkeypatch.setenv("OV_STENCIL", "slab")
    links = inputs.gauge_links(dims, seed=8011)
    psi = inputs.gaussian_source(dims, seed=8012, nrhs=nrhs)
    with Ctx(dims, dev(links), prec, antiperiodic_t=True) as c:
        assert c.stats()["stencil_slab"] > 0
        got_w = host(c.wilson(dev(psi)))
        got_k = host(c.kernel(dev(psi)))
    want_w = np.stack([wilson.wilson(links, p, True) for p in psi])
    want_k = np.stack([wilson.kernel_k(links, p, antiperiodic_t=True) for p in psi])
    assert rel(got_w, want_w) < TOL[prec]
    assert rel(got_k, want_k) < TOL[prec]


def test_slab_sign_and_overlap(monkeypatch):
    """sign(K) and D[mu] through the slab kernel (every epilogue form of the
    recurrence and the FP32 assembly), 8 x 4 x 4 x 6, order 24, undeflated."""
    monkeypatch.setenv("OV_STENCIL", "slab")
    dims = (8, 4, 4, 6)
    links = inputs.gauge_links(dims, seed=8021)
    psi = inputs.gaussian_source(dims, seed=8022, nrhs=2)
    a, b, order, mu = 0.2, 6.6, 24, 0.1
    cfg = overlap.SignConfig(chebyshev.coefficients(order, a, b), a, b)
    want_s = np.stack([overlap.sign_apply(links, p, cfg) for p in psi])
    want_d = np.stack([overlap.overlap(links, p, mu, cfg) for p in psi])
    with Ctx(dims, dev(links), "fp16") as c:
        assert c.stats()["stencil_slab"] > 0
        c.sign_config(order, a, b)
        got_s = host(c.sign(dev(psi)))
        got_d = host(c.overlap(dev(psi), mu))
    assert rel(got_s, want_s) < 1e-2
    assert rel(got_d, want_d) < 1e-2


def _random_orthonormal(dims, n, seed):
    rng = np.random.default_rng(seed)
    vol = inputs.volume(dims)
    m = rng.standard_normal((12 * vol, n)) + 1j * rng.standard_normal((12 * vol, n))
    q, _ = np.linalg.qr(m)
    return np.ascontiguousarray(q.T).reshape((n,) + field_shape(dims))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("fp16", 1e-2)])
def test_point_sources_batched_sign_and_overlap(prec, tol):
    """8^4, 12 point sources, 6 orthonormal deflation vectors, order 24: the
    projected form of Eq. 3 is evaluated identically by both sides."""
    dims = (8, 8, 8, 8)
    links = inputs.gauge_links(dims, seed=8101)
    src = inputs.point_sources(dims)
    evecs = _random_orthonormal(dims, 6, 8102)
    evals = np.array([0.3, -0.31, 0.4, -0.45, 0.5, 0.52])
    a, b, order, mu = 0.5, 6.5, 24, 0.05
    cfg = overlap.SignConfig(chebyshev.coefficients(order, a, b), a, b, evals, evecs)
    with Ctx(dims, dev(links), prec) as c:
        c.sign_config(order, a, b, evals, dev(evecs))
        got_s = host(c.sign(dev(src)))
        got_d = host(c.overlap(dev(src), mu))
        got_dd = host(c.overlap(dev(src), mu, dagger=True))
        single = host(c.sign(dev(src[3:4])))
    want_s = np.stack([overlap.sign_apply(links, p, cfg) for p in src])
    want_d = np.stack([overlap.overlap(links, p, mu, cfg) for p in src])
    want_dd = np.stack([overlap.overlap_dag(links, p, mu, cfg) for p in src])
    assert rel(got_s, want_s) < tol
    assert rel(got_d, want_d) < tol
    assert rel(got_dd, want_dd) < tol
    assert rel(single, got_s[3:4]) < (1e-13 if prec == "fp64" else tol)


def test_batched_solve_three_rhs():
    prob = small_problem()
    order, mu, tol = 32, 0.05, 1e-10
    cfg = overlap.SignConfig(chebyshev.coefficients(order, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    b = inputs.gaussian_source(prob["dims"], seed=8201, nrhs=3)
    with Ctx(prob["dims"], dev(prob["links"]), "fp32") as c:
        c.sign_config(order, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
        x, iters, res = c.solve(dev(b), mu, tol=tol, maxit=20000)
    x = host(x)
    assert res <= tol
    for r in range(3):
        rhs = overlap.overlap_dag(prob["links"], b[r], mu, cfg)
        true_r = rhs - overlap.normal_op(prob["links"], x[r], mu, cfg)
        assert np.linalg.norm(true_r) / np.linalg.norm(rhs) <= 2 * tol


@pytest.mark.parametrize("dims,n_ev,nrhs", [((8, 8, 8, 8), 40, 12), ((3, 3, 3, 5), 20, 7), ((4, 4, 4, 8), 64, 16),
                                            ((4, 4, 4, 8), 65, 3), ((6, 6, 6, 6), 128, 16)])
def test_tensor_core_projection(monkeypatch, dims, n_ev, nrhs):
    """The tcgen05 projection (TF32 split products) against the CUDA-core
    FP64-sum Gram kernel on the same inputs, through sign(K) and D^dagger
    (gamma5 on the input), including a K tail that is not a multiple of the
    64-float chunk; n_ev <= 64 packs the hi and lo parts of the eigenvectors
    into one tile, 65..128 uses two tiles; 16 right-hand sides fill the B tile."""
    links = inputs.gauge_links(dims, seed=8301)
    src = inputs.gaussian_source(dims, seed=8302, nrhs=nrhs)
    evecs = _random_orthonormal(dims, n_ev, 8303)
    evals = np.linspace(-0.5, 0.5, n_ev) + 0.01
    a, b, order, mu = 0.5, 6.5, 12, 0.1
    outs = {}
    for mode in ("tc", "cuda"):
        monkeypatch.setenv("OV_DEFL_GEMM", mode)
        with Ctx(dims, dev(links), "fp32") as c:
            c.sign_config(order, a, b, evals, dev(evecs))
            s = host(c.sign(dev(src)))
            d = host(c.overlap(dev(src), mu, dagger=True))
            outs[mode] = (s, d, c.stats()["tc_gemm_launches"])
    assert outs["tc"][2] == 2 and outs["cuda"][2] == 0
    assert rel(outs["tc"][0], outs["cuda"][0]) < 1e-6
    assert rel(outs["tc"][1], outs["cuda"][1]) < 1e-6
    cfg = overlap.SignConfig(chebyshev.coefficients(order, a, b), a, b, evals, evecs)
    want = np.stack([overlap.sign_apply(links, p, cfg) for p in src])
    assert rel(outs["tc"][0], want) < 2e-5
