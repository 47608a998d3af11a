"""Error of every result against the FP64 oracle, per precision (4^4 lattice,
8 deflated dense eigenpairs, order 64, mu = 0.05; solve to 1e-10).  The
measured values are printed, written to $OV_REPORT_DIR/precision_report.md
when that variable names a directory, and bounded by the tolerances of the
parity tests."""
import os

import numpy as np
import pytest

from oracle import chebyshev, dense, overlap, wilson
from paper_1510_06897_gb300 import inputs
from paper_1510_06897_gb300.binding import Ctx
from tests.gpu_util import dev, host, need_gpu, rel
from tests.oracle_fixtures import small_problem

pytestmark = pytest.mark.gpu

BOUND = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-2, "bf16": 6e-2}


def test_precision_report():
    need_gpu()
    prob = small_problem()
    order, mu = 64, 0.05
    cfg = overlap.SignConfig(chebyshev.coefficients(order, prob["a"], prob["b"]), prob["a"], prob["b"],
                             prob["evals"], prob["evecs"])
    psi = inputs.gaussian_source(prob["dims"], seed=9101)
    want = {
        "D_W": wilson.wilson(prob["links"], psi[0])[None],
        "sign(K)": overlap.sign_apply(prob["links"], psi[0], cfg)[None],
        "D[mu]": overlap.overlap(prob["links"], psi[0], mu, cfg)[None],
        "D[mu]^dag": overlap.overlap_dag(prob["links"], psi[0], mu, cfg)[None],
    }
    exact_sign = dense.apply_matrix(dense.exact_sign(prob["kmat"]), psi[0])[None]
    rows = []
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        with Ctx(prob["dims"], dev(prob["links"]), prec) as c:
            c.sign_config(order, prob["a"], prob["b"], prob["evals"], dev(prob["evecs"]))
            got = {"D_W": host(c.wilson(dev(psi))), "sign(K)": host(c.sign(dev(psi))),
                   "D[mu]": host(c.overlap(dev(psi), mu)), "D[mu]^dag": host(c.overlap(dev(psi), mu, dagger=True))}
            x, iters, res = c.solve(dev(psi), mu, tol=1e-10, maxit=20000)
        x = host(x)
        rhs = overlap.overlap_dag(prob["links"], psi[0], mu, cfg)
        true_res = np.linalg.norm(rhs - overlap.normal_op(prob["links"], x[0], mu, cfg)) / np.linalg.norm(rhs)
        errs = {k: rel(got[k], want[k]) for k in want}
        errs["sign(K) vs exact"] = rel(got["sign(K)"], exact_sign)
        rows.append((prec, errs, iters, true_res))
        for k in want:
            assert errs[k] < BOUND[prec], (prec, k)
        assert true_res <= 2e-10
    lines = ["| precision | D_W | sign(K) | D[mu] | D[mu]^dag | sign(K) vs exact sign | solve: iterations, oracle true residual |",
             "|---|---|---|---|---|---|---|"]
    for prec, e, it, tr in rows:
        lines.append(f"| {prec} | {e['D_W']:.1e} | {e['sign(K)']:.1e} | {e['D[mu]']:.1e} | {e['D[mu]^dag']:.1e} | "
                     f"{e['sign(K) vs exact']:.1e} | {it}, {tr:.1e} |")
    text = "\n".join(lines)
    print("\n" + text)
    out_dir = os.environ.get("OV_REPORT_DIR")
    if out_dir and os.path.isdir(out_dir):
        with open(os.path.join(out_dir, "precision_report.md"), "w") as f:
            f.write(text + "\n")
