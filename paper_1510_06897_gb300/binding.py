"""ctypes binding of the C ABI in include/overlap.h (argument marshalling only).

Each ``ov_*`` function here takes the same arguments as its C counterpart,
with tensors / arrays in place of raw pointers, and raises OverlapError on a
non-OK status.  Device tensors are passed by pointer; CPU tensors and NumPy
arrays are passed as host pointers, which the library stages itself.  No
computation happens in Python: if the shared library has not been built,
``lib()`` raises instead of falling back to anything else.

Tensor layouts (C order):
  links   complex128 (4, Lt, Lz, Ly, Lx, 3, 3)
  spinors complex128 or complex64 (nrhs, Lt, Lz, Ly, Lx, 4, 3)
  evecs   complex128 (n_ev, Lt, Lz, Ly, Lx, 4, 3)
"""
import ctypes
import os

import numpy as np

from .build import LIB_PATH

OV_OK, OV_ERR_INVALID, OV_ERR_NOMEM, OV_ERR_CUDA, OV_ERR_NOT_CONVERGED, OV_ERR_STATE, OV_ERR_NONFINITE = range(7)
OV_FP64, OV_FP32, OV_MIXED_FP16, OV_MIXED_BF16 = range(4)
OV_C128, OV_C64 = range(2)
PRECISIONS = {"fp64": OV_FP64, "fp32": OV_FP32, "fp16": OV_MIXED_FP16, "bf16": OV_MIXED_BF16}
STATUS_NAMES = {0: "OV_OK", 1: "OV_ERR_INVALID", 2: "OV_ERR_NOMEM", 3: "OV_ERR_CUDA",
                4: "OV_ERR_NOT_CONVERGED", 5: "OV_ERR_STATE", 6: "OV_ERR_NONFINITE"}


class OverlapError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ov_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong),
                ("dslash_launches", ctypes.c_longlong),
                ("sign_applies", ctypes.c_longlong),
                ("inner_iterations", ctypes.c_longlong),
                ("outer_iterations", ctypes.c_longlong),
                ("dslash_timed", ctypes.c_longlong),
                ("dslash_ms", ctypes.c_double),
                ("stencil_tpb", ctypes.c_int),
                ("stencil_minb", ctypes.c_int),
                ("stencil_lrec", ctypes.c_int),
                ("tc_gemm_launches", ctypes.c_int),
                ("stencil_slab", ctypes.c_int),
                ("gcr_iterations", ctypes.c_longlong),
                ("gmresr_order", ctypes.c_int),
                ("stencil_async", ctypes.c_int),
                ("stencil_brick", ctypes.c_int),
                ("grad_kept_terms", ctypes.c_int)]


_LIB = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double

_SIGNATURES = {
    "ov_create": [ctypes.POINTER(_vp), ctypes.POINTER(_i), _vp, _i, _d, _i, _vp],
    "ov_destroy": [_vp],
    "ov_wilson": [_vp, _vp, _vp, _i, _i],
    "ov_kernel": [_vp, _vp, _vp, _i, _i],
    "ov_sign_config": [_vp, _i, _d, _d, ctypes.POINTER(_d), _vp, _i],
    "ov_sign_apply": [_vp, _vp, _vp, _i, _i],
    "ov_sign": [_vp, _i, _d, _d, ctypes.POINTER(_d), _vp, _i, _vp, _vp, _i, _i],
    "ov_overlap": [_vp, _d, _i, _vp, _vp, _i, _i],
    "ov_solve": [_vp, _d, _d, _i, _vp, _vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)],
    "ov_solve_chiral": [_vp, _d, _i, _d, _i, _vp, _vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)],
    "ov_set_solver_params": [_vp, _d, _i],
    "ov_sumr": [_vp, _d, _d, _i, _vp, _vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)],
    "ov_solve_gmresr": [_vp, _d, _d, _i, _vp, _vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)],
    "ov_set_gmresr_params": [_vp, _i, _d, _i, _i],
    "ov_enable_fp32_operator": [_vp, _vp],
    "ov_eigs": [_vp, _i, _d, _i, ctypes.POINTER(_d), _vp, ctypes.POINTER(_d)],
    "ov_sign_poly_grad": [_vp, _i, _d, _d, _vp, _vp, _i],
    "ov_get_stats": [_vp, ctypes.POINTER(ov_stats)],
    "ov_reset_stats": [_vp],
    "ov_set_profiling": [_vp, _i],
    "ov_set_checks": [_vp, _i],
    "ov_get_residual_history": [_vp, ctypes.POINTER(_d), _i, ctypes.POINTER(_i)],
    "ov_set_gmresr_fp32_level": [_vp, _i],
    "ov_test_wait_expiry": [_vp, ctypes.c_longlong],
    "ov_set_grad_memory": [_vp, ctypes.c_longlong],
    "ov_sign_poly_quad": [_vp, _i, _d, _d, _vp, _vp, _i, ctypes.POINTER(_d)],
    "ov_wilson_noalloc": [ctypes.POINTER(_i), _vp, _vp, _vp, _i, _i, _i, _vp],
    "ov_stout_smear": [ctypes.POINTER(_i), _vp, _vp, _d, _d, _i, _vp],
}


def lib():
    """Loads the in-tree library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{os.path.basename(LIB_PATH)} is not built; run __graft_entry__.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(handle, name, None)
            if fn is None:
                continue  # reported by the export test; calling it raises AttributeError
            fn.argtypes = args
            fn.restype = ctypes.c_int
        handle.ov_last_error.argtypes = [_vp]
        handle.ov_last_error.restype = ctypes.c_char_p
        _LIB = handle
    return _LIB


def _check(status, ctx):
    if status != OV_OK:
        msg = lib().ov_last_error(ctx)
        raise OverlapError(status, msg.decode() if msg else "")
    return status


def _ptr(x):
    """Raw pointer of a torch tensor or NumPy array (must be C-contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


def _dtype_code(x):
    name = str(x.dtype)
    if name.endswith("complex128"):
        return OV_C128
    if name.endswith("complex64"):
        return OV_C64
    raise TypeError(f"spinor dtype must be complex128 or complex64, got {x.dtype}")


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def ov_create(dims, links, prec=OV_FP64, m_w=1.5, antiperiodic_t=False, stream=None):
    if isinstance(prec, str):
        prec = PRECISIONS[prec]
    handle = _vp()
    cdims = (_i * 4)(*[int(d) for d in dims])
    st = lib().ov_create(ctypes.byref(handle), cdims, _ptr(links), int(prec), float(m_w), int(bool(antiperiodic_t)),
                         _stream_ptr(stream))
    _check(st, None)
    return handle


def ov_destroy(ctx):
    return _check(lib().ov_destroy(ctx), ctx)


def ov_wilson(ctx, inp, out, nrhs):
    return _check(lib().ov_wilson(ctx, _ptr(inp), _ptr(out), int(nrhs), _dtype_code(inp)), ctx)


def ov_kernel(ctx, inp, out, nrhs):
    return _check(lib().ov_kernel(ctx, _ptr(inp), _ptr(out), int(nrhs), _dtype_code(inp)), ctx)


def _evals_arg(evals):
    if evals is None or len(evals) == 0:
        return None, None
    arr = np.ascontiguousarray(np.asarray(evals, dtype=np.float64))
    return arr, arr.ctypes.data_as(ctypes.POINTER(_d))


def ov_sign_config(ctx, order, lo, hi, evals, evecs, n_ev):
    keep, ev = _evals_arg(evals)
    return _check(lib().ov_sign_config(ctx, int(order), float(lo), float(hi), ev, _ptr(evecs), int(n_ev)), ctx)


def ov_sign_apply(ctx, inp, out, nrhs):
    return _check(lib().ov_sign_apply(ctx, _ptr(inp), _ptr(out), int(nrhs), _dtype_code(inp)), ctx)


def ov_sign(ctx, order, lo, hi, evals, evecs, n_ev, inp, out, nrhs):
    keep, ev = _evals_arg(evals)
    return _check(lib().ov_sign(ctx, int(order), float(lo), float(hi), ev, _ptr(evecs), int(n_ev), _ptr(inp),
                                _ptr(out), int(nrhs), _dtype_code(inp)), ctx)


def ov_overlap(ctx, mu, dagger, inp, out, nrhs):
    return _check(lib().ov_overlap(ctx, float(mu), int(bool(dagger)), _ptr(inp), _ptr(out), int(nrhs),
                                   _dtype_code(inp)), ctx)


def ov_solve(ctx, mu, tol, maxit, b, x, nrhs, allow_not_converged=False):
    """Returns (iterations, true relative residual)."""
    it = _i(0)
    res = _d(0.0)
    st = lib().ov_solve(ctx, float(mu), float(tol), int(maxit), _ptr(b), _ptr(x), int(nrhs), _dtype_code(b),
                        ctypes.byref(it), ctypes.byref(res))
    if not (allow_not_converged and st == OV_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return it.value, res.value


def ov_solve_chiral(ctx, mu, chirality, tol, maxit, b, x, nrhs, allow_not_converged=False):
    """Chiral-sector solve A x = P b (see overlap.h); returns (iterations, true relative residual)."""
    it = _i(0)
    res = _d(0.0)
    st = lib().ov_solve_chiral(ctx, float(mu), int(chirality), float(tol), int(maxit), _ptr(b), _ptr(x), int(nrhs),
                               _dtype_code(b), ctypes.byref(it), ctypes.byref(res))
    if not (allow_not_converged and st == OV_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return it.value, res.value


def ov_sumr(ctx, mu, tol, maxit, b, x, nrhs):
    """SUMR for D[mu] x = b (see overlap.h); returns (iterations, residual estimate)."""
    it = _i(0)
    est = _d(0.0)
    _check(lib().ov_sumr(ctx, float(mu), float(tol), int(maxit), _ptr(b), _ptr(x), int(nrhs), _dtype_code(b),
                         ctypes.byref(it), ctypes.byref(est)), ctx)
    return it.value, est.value


def ov_solve_gmresr(ctx, mu, tol, maxit, b, x, nrhs, allow_not_converged=False):
    """GMRESR for D[mu] x = b (see overlap.h); returns (SUMR iterations, true relative residual)."""
    it = _i(0)
    res = _d(0.0)
    st = lib().ov_solve_gmresr(ctx, float(mu), float(tol), int(maxit), _ptr(b), _ptr(x), int(nrhs), _dtype_code(b),
                               ctypes.byref(it), ctypes.byref(res))
    if not (allow_not_converged and st == OV_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return it.value, res.value


def ov_enable_fp32_operator(ctx, links):
    """FP32 operator beside a 16-bit one, for the GCR level of ov_solve_gmresr (see overlap.h)."""
    return _check(lib().ov_enable_fp32_operator(ctx, _ptr(links)), ctx)


def ov_set_gmresr_fp32_level(ctx, on=True):
    """GCR level of GMRESR on an FP32 copy of a 16-bit operator (default) or not."""
    return _check(lib().ov_set_gmresr_fp32_level(ctx, int(bool(on))), ctx)


def ov_set_grad_memory(ctx, nbytes=-1):
    """Device bytes ov_sign_poly_grad may fill with recurrence terms (< 0: half the free memory; 0: recompute)."""
    return _check(lib().ov_set_grad_memory(ctx, int(nbytes)), ctx)


def ov_set_gmresr_params(ctx, inner_order=0, inner_tol=0.1, inner_maxit=1000, max_dirs=12):
    return _check(lib().ov_set_gmresr_params(ctx, int(inner_order), float(inner_tol), int(inner_maxit),
                                             int(max_dirs)), ctx)


def ov_set_solver_params(ctx, inner_tol, max_outer):
    return _check(lib().ov_set_solver_params(ctx, float(inner_tol), int(max_outer)), ctx)


def ov_eigs(ctx, n_ev, tol, max_iter, evecs, allow_not_converged=False):
    """Fills evecs (complex128 (n_ev, ...)); returns (evals ndarray, lambda_max)."""
    evals = np.zeros(n_ev, dtype=np.float64)
    lmax = _d(0.0)
    st = lib().ov_eigs(ctx, int(n_ev), float(tol), int(max_iter), evals.ctypes.data_as(ctypes.POINTER(_d)),
                       _ptr(evecs), ctypes.byref(lmax))
    if not (allow_not_converged and st == OV_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return evals, lmax.value


def ov_sign_poly_quad(ctx, order, lo, hi, chi, p_chi=None):
    """S = chi^dagger P(K) chi (undeflated polynomial); p_chi, if given, receives P(K) chi."""
    s = _d(0.0)
    _check(lib().ov_sign_poly_quad(ctx, int(order), float(lo), float(hi), _ptr(chi), _ptr(p_chi), _dtype_code(chi),
                                   ctypes.byref(s)), ctx)
    return s.value


def ov_sign_poly_grad(ctx, order, lo, hi, chi, grad_links):
    return _check(lib().ov_sign_poly_grad(ctx, int(order), float(lo), float(hi), _ptr(chi), _ptr(grad_links),
                                          _dtype_code(chi)), ctx)


def ov_get_stats(ctx):
    s = ov_stats()
    _check(lib().ov_get_stats(ctx, ctypes.byref(s)), ctx)
    return {name: getattr(s, name) for name, _ in ov_stats._fields_}


def _numel(x):
    return int(x.size) if isinstance(x, np.ndarray) else int(x.numel())


def ov_wilson_noalloc(dims, links, inp, out, nrhs, antiperiodic_t=False, stream=None):
    """D_W without a context and without any device allocation (see overlap.h).
    The library cannot see buffer sizes, so they are checked here: links
    complex128 with 36 V elements, inp 12 V nrhs elements, out the dtype and
    element count of inp."""
    vol = 1
    for d in dims:
        vol *= int(d)
    if not str(links.dtype).endswith("complex128") or _numel(links) != 36 * vol:
        raise ValueError(f"links must be complex128 with 36 * V = {36 * vol} elements")
    if _numel(inp) != 12 * vol * int(nrhs):
        raise ValueError(f"inp must hold 12 * V * nrhs = {12 * vol * int(nrhs)} elements")
    if str(out.dtype) != str(inp.dtype) or _numel(out) != _numel(inp):
        raise ValueError("out must have the dtype and element count of inp")
    cdims = (_i * 4)(*[int(d) for d in dims])
    return _check(lib().ov_wilson_noalloc(cdims, _ptr(links), _ptr(inp), _ptr(out), int(nrhs), _dtype_code(inp),
                                          int(bool(antiperiodic_t)), _stream_ptr(stream)), None)


def ov_stout_smear(dims, links_in, links_out, rho=0.1, eps=-0.25, steps=3, stream=None):
    """Over-improved stout smearing (see overlap.h); links_out may be links_in."""
    cdims = (_i * 4)(*[int(d) for d in dims])
    return _check(lib().ov_stout_smear(cdims, _ptr(links_in), _ptr(links_out), float(rho), float(eps), int(steps),
                                       _stream_ptr(stream)), None)


def ov_set_profiling(ctx, on):
    """on: 0 off, 1 (or True) every stencil launch, 2 the recurrence as one bracket (see overlap.h)."""
    return _check(lib().ov_set_profiling(ctx, 2 if on == 2 else int(bool(on))), ctx)


def ov_get_residual_history(ctx):
    """Largest true relative residual after each FP64 pass of the last solve."""
    n = _i(0)
    _check(lib().ov_get_residual_history(ctx, None, 0, ctypes.byref(n)), ctx)
    buf = (_d * max(1, n.value))()
    _check(lib().ov_get_residual_history(ctx, buf, n.value, ctypes.byref(n)), ctx)
    return [buf[i] for i in range(n.value)]


def ov_test_wait_expiry(ctx, cycles):
    """Testing hook: pipeline waits of the tensor-core projection and the slab
    stencil run out after `cycles` on a flag nothing sets; 0 turns it off (see overlap.h)."""
    return _check(lib().ov_test_wait_expiry(ctx, int(cycles)), ctx)


def ov_set_checks(ctx, on):
    """Scan every vector output for NaN / Inf (see overlap.h)."""
    return _check(lib().ov_set_checks(ctx, int(bool(on))), ctx)


def ov_reset_stats(ctx):
    return _check(lib().ov_reset_stats(ctx), ctx)


def ov_last_error(ctx):
    msg = lib().ov_last_error(ctx)
    return msg.decode() if msg else ""


class Ctx:
    """Owns one ov_ctx; convenience wrappers that allocate outputs like their inputs."""

    def __init__(self, dims, links, prec=OV_FP64, m_w=1.5, antiperiodic_t=False, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.handle = ov_create(self.dims, links, prec, m_w, antiperiodic_t, stream)

    def close(self):
        if self.handle is not None:
            ov_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _like(x):
        if isinstance(x, np.ndarray):
            return np.empty_like(x)
        import torch
        return torch.empty_like(x)

    def wilson(self, x):
        out = self._like(x)
        ov_wilson(self.handle, x, out, x.shape[0])
        return out

    def kernel(self, x):
        out = self._like(x)
        ov_kernel(self.handle, x, out, x.shape[0])
        return out

    def sign_config(self, order, lo, hi, evals=None, evecs=None):
        n_ev = 0 if evals is None else len(evals)
        ov_sign_config(self.handle, order, lo, hi, evals, evecs, n_ev)

    def sign(self, x):
        out = self._like(x)
        ov_sign_apply(self.handle, x, out, x.shape[0])
        return out

    def overlap(self, x, mu, dagger=False):
        out = self._like(x)
        ov_overlap(self.handle, mu, dagger, x, out, x.shape[0])
        return out

    def solve(self, b, mu, tol=1e-10, maxit=5000):
        x = self._like(b)
        it, res = ov_solve(self.handle, mu, tol, maxit, b, x, b.shape[0])
        return x, it, res

    def solve_chiral(self, b, mu, chirality, tol=1e-10, maxit=5000):
        x = self._like(b)
        it, res = ov_solve_chiral(self.handle, mu, chirality, tol, maxit, b, x, b.shape[0])
        return x, it, res

    def sumr(self, b, mu, tol=0.0, maxit=100):
        x = self._like(b)
        it, est = ov_sumr(self.handle, mu, tol, maxit, b, x, b.shape[0])
        return x, it, est

    def solve_gmresr(self, b, mu, tol=1e-10, maxit=20000):
        x = self._like(b)
        it, res = ov_solve_gmresr(self.handle, mu, tol, maxit, b, x, b.shape[0])
        return x, it, res

    def stats(self):
        return ov_get_stats(self.handle)
