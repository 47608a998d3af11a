"""Shared small-lattice fixtures for the oracle pins and the GPU parity tests:
the 4^4 plain-FP64 workload (links exp(i 0.3 H), 8 deflated dense eigenpairs,
Chebyshev order 64 on [|lambda_9|, lambda_max])."""
import functools

import numpy as np

from oracle import dense
from paper_1510_06897_gb300 import inputs

DIMS_4 = (4, 4, 4, 4)


def field_shape(dims):
    return (dims[3], dims[2], dims[1], dims[0], 4, 3)


@functools.lru_cache(maxsize=None)
def small_problem(dims=DIMS_4, seed=inputs.SEED_LINKS + 1, n_ev=8, antiperiodic=False):
    """Links, dense K, its full sorted spectrum, n_ev eigenpairs and (a, b)."""
    links = inputs.gauge_links(dims, seed=seed)
    kmat = dense.kernel_matrix(links, antiperiodic_t=antiperiodic)
    evals, evecs, w_all = dense.eigenpairs_as_fields(kmat, n_ev, field_shape(dims))
    a = float(abs(w_all[n_ev]))
    b = float(np.max(np.abs(w_all)))
    return dict(dims=dims, links=links, kmat=kmat, evals=evals, evecs=evecs,
                w_all=w_all, a=a, b=b, antiperiodic=antiperiodic)
