"""SignPolyQuad: S = chi^dagger P(K) chi as a differentiable torch operation.

P(K) = K f_N(K^2) is the undeflated Chebyshev polynomial of Eq. 3 (order N
on [lo^2, hi^2]); K = gamma5 (D_W - m_W) with D_W of Eq. 2.  Forward and
backward both run in the library's kernels through the C ABI
(ov_sign_poly_quad, ov_sign_poly_grad); this module only marshals tensors
and applies the chain rule's scalar factor.

Gradients delivered by backward (times the incoming scalar gradient):

* links: the su(3)-valued link derivative F_mu(x) of ov_sign_poly_grad,
  defined by dS/deps = sum_{x,mu} Re tr(X_mu(x)^dagger F_mu(x)) along
  U_mu(x) -> exp(eps X_mu(x)) U_mu(x), X in su(3).  This is the force a gauge
  update (molecular dynamics, gradient flow) consumes; it is the derivative
  along the group manifold, not with respect to the 18 unconstrained real
  entries of each matrix (those directions leave SU(3), where the
  reconstruct-12 storage of the operator is not defined).
* chi: 2 P(K) chi, the derivative of the real S in torch's convention for
  complex inputs (dS/d Re chi + i dS/d Im chi).

The operator context is created from `links` in forward (FP64 or FP32
storage) and kept until backward has run.
"""
import torch

from .binding import Ctx, ov_sign_poly_grad, ov_sign_poly_quad


class SignPolyQuad(torch.autograd.Function):
    """S = Re chi^dagger P(K) chi (a 0-dim float64 tensor on links.device).

    links: complex128 (4, Lt, Lz, Ly, Lx, 3, 3) on the GPU, SU(3) matrices.
    chi:   complex128 (FP64) or complex64 (FP32) spinor (1, Lt, Lz, Ly, Lx, 4, 3).
    dims:  (Lx, Ly, Lz, Lt); order, lo, hi: the polynomial of Eq. 3;
    prec:  "fp64" or "fp32" operator storage.
    """

    @staticmethod
    def forward(ctx, links, chi, dims, order, lo, hi, prec="fp64", m_w=1.5, antiperiodic_t=False):
        if prec not in ("fp64", "fp32"):
            raise ValueError("SignPolyQuad runs on an fp64 or fp32 operator")
        opc = Ctx(dims, links.detach().contiguous(), prec, m_w, antiperiodic_t)
        chi_c = chi.detach().contiguous()
        p_chi = torch.empty_like(chi_c) if ctx.needs_input_grad[1] else None
        try:
            s = ov_sign_poly_quad(opc.handle, order, lo, hi, chi_c, p_chi)
        except Exception:
            opc.close()
            raise
        if ctx.needs_input_grad[0]:
            ctx.opc = opc
        else:
            opc.close()
            ctx.opc = None
        ctx.poly = (int(order), float(lo), float(hi))
        ctx.links_shape = links.shape
        ctx.save_for_backward(chi_c, p_chi)
        return torch.tensor(s, dtype=torch.float64, device=links.device)

    @staticmethod
    def backward(ctx, grad_s):
        chi_c, p_chi = ctx.saved_tensors
        order, lo, hi = ctx.poly
        g_links = g_chi = None
        if ctx.needs_input_grad[0]:
            grad = torch.empty(ctx.links_shape, dtype=torch.complex128, device=chi_c.device)
            try:
                ov_sign_poly_grad(ctx.opc.handle, order, lo, hi, chi_c, grad)
            finally:
                ctx.opc.close()
                ctx.opc = None
            g_links = grad * grad_s
        if ctx.needs_input_grad[1]:
            g_chi = p_chi * (2.0 * grad_s).to(p_chi.real.dtype)
        return g_links, g_chi, None, None, None, None, None, None, None


def sign_poly_quad(links, chi, dims, order, lo, hi, prec="fp64", m_w=1.5, antiperiodic_t=False):
    """S = chi^dagger P(K) chi, differentiable in links (su(3) force) and chi."""
    return SignPolyQuad.apply(links, chi, tuple(int(d) for d in dims), order, lo, hi, prec, m_w, antiperiodic_t)
