"""Host-only checks of the C ABI: the library builds, loads without a GPU and
exports every function include/overlap.h declares; argument validation that
happens before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1510_06897_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "overlap.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ov_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("ov_create", "ov_destroy", "ov_wilson", "ov_sign", "ov_overlap", "ov_solve", "ov_eigs",
               "ov_sign_poly_grad", "ov_last_error"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(build.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(raw, n)]
    assert not missing, missing


@pytest.mark.parametrize("dims", [(1, 4, 4, 4), (4, 4, 0, 4), (4, 4, 4, -2)])
def test_create_rejects_bad_dims_before_device_work(lib, dims):
    links = np.zeros((4, 1, 1, 1, 1, 3, 3), dtype=np.complex128)
    with pytest.raises(binding.OverlapError) as e:
        binding.ov_create(dims, links)
    assert e.value.status == binding.OV_ERR_INVALID
    assert "extent" in binding.ov_last_error(None)


@pytest.mark.parametrize("dims,msg", [((2, 2, 256, 512), "Lz * Lt"), ((1024, 1024, 16, 16), "too large")])
def test_create_rejects_oversize_lattices_before_device_work(lib, dims, msg):
    """More (z, t) slices than the stencil grid's y dimension holds, or more
    than 2^27 sites: rejected on the host (no device allocation, no GPU needed)."""
    links = np.zeros((4, 1, 1, 1, 1, 3, 3), dtype=np.complex128)
    with pytest.raises(binding.OverlapError) as e:
        binding.ov_create(dims, links)
    assert e.value.status == binding.OV_ERR_INVALID
    assert msg in binding.ov_last_error(None)


def test_create_rejects_bad_precision_and_null(lib):
    links = np.zeros((4, 2, 2, 2, 2, 3, 3), dtype=np.complex128)
    with pytest.raises(binding.OverlapError):
        binding.ov_create((2, 2, 2, 2), links, prec=7)
    handle = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(2, 2, 2, 2)
    assert lib.ov_create(ctypes.byref(handle), dims, None, 0, 1.5, 0, None) == binding.OV_ERR_INVALID
    assert lib.ov_create(None, dims, links.ctypes.data, 0, 1.5, 0, None) == binding.OV_ERR_INVALID


def test_null_context_calls(lib):
    assert lib.ov_destroy(None) == binding.OV_OK
    assert lib.ov_wilson(None, None, None, 1, 0) == binding.OV_ERR_INVALID
    assert lib.ov_sign_apply(None, None, None, 1, 0) == binding.OV_ERR_INVALID
    assert lib.ov_solve(None, 0.1, 1e-10, 10, None, None, 1, 0, None, None) == binding.OV_ERR_INVALID
    assert lib.ov_solve_chiral(None, 0.1, 1, 1e-10, 10, None, None, 1, 0, None, None) == binding.OV_ERR_INVALID
    assert lib.ov_sumr(None, 0.1, 1e-10, 10, None, None, 1, 0, None, None) == binding.OV_ERR_INVALID
    assert lib.ov_solve_gmresr(None, 0.1, 1e-10, 10, None, None, 1, 0, None, None) == binding.OV_ERR_INVALID
    assert lib.ov_set_gmresr_params(None, 0, 0.1, 100, 8) == binding.OV_ERR_INVALID
    assert lib.ov_enable_fp32_operator(None, None) == binding.OV_ERR_INVALID
    assert lib.ov_set_grad_memory(None, 0) == binding.OV_ERR_INVALID


def test_stout_smear_rejects_bad_arguments_before_device_work(lib):
    dims = (ctypes.c_int * 4)(4, 4, 4, 4)
    links = np.zeros((4, 4, 4, 4, 4, 3, 3), dtype=np.complex128)
    p = links.ctypes.data
    assert lib.ov_stout_smear(None, p, p, 0.1, -0.25, 3, None) == binding.OV_ERR_INVALID
    assert lib.ov_stout_smear(dims, None, p, 0.1, -0.25, 3, None) == binding.OV_ERR_INVALID
    bad = (ctypes.c_int * 4)(4, 1, 4, 4)
    assert lib.ov_stout_smear(bad, p, p, 0.1, -0.25, 3, None) == binding.OV_ERR_INVALID
    assert lib.ov_stout_smear(dims, p, p, 0.1, -0.25, -1, None) == binding.OV_ERR_INVALID
    assert lib.ov_stout_smear(dims, p, p, float("nan"), -0.25, 3, None) == binding.OV_ERR_INVALID
    assert b"extent" in lib.ov_last_error(None) or b"steps" in lib.ov_last_error(None)
    assert lib.ov_get_stats(None, None) == binding.OV_ERR_INVALID
    assert lib.ov_set_checks(None, 1) == binding.OV_ERR_INVALID
    assert lib.ov_get_residual_history(None, None, 0, None) == binding.OV_ERR_INVALID


def test_binding_dtype_codes():
    assert binding._dtype_code(np.zeros(2, np.complex128)) == binding.OV_C128
    assert binding._dtype_code(np.zeros(2, np.complex64)) == binding.OV_C64
    with pytest.raises(TypeError):
        binding._dtype_code(np.zeros(2, np.float64))
    with pytest.raises(ValueError):
        binding._ptr(np.zeros((4, 4), np.complex128)[:, ::2])


def _prototypes():
    """name -> list of parameter declarations, parsed from include/overlap.h."""
    text = open(os.path.join(ROOT, "include", "overlap.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = {}
    for m in re.finditer(r"\b(?:ov_status|const char\s*\*)\s*(ov_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", text):
        params = [p.strip() for p in m.group(2).replace("\n", " ").split(",") if p.strip() and p.strip() != "void"]
        out[m.group(1)] = params
    return out


def _kind(decl):
    """'p' for a pointer parameter (including arrays), 'd' for double, 'l' for
    long long, 'i' for int / enum."""
    if "*" in decl or "[" in decl:
        return "p"
    if re.search(r"\bdouble\b", decl):
        return "d"
    if re.search(r"\blong\s+long\b", decl):
        return "l"
    return "i"


def _ctype_kind(t):
    if t is ctypes.c_void_p or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "p"
    if t is ctypes.c_double:
        return "d"
    if t is ctypes.c_longlong:
        return "l"
    return "i"


def test_binding_signatures_match_the_header():
    protos = _prototypes()
    assert len(protos) >= len(binding._SIGNATURES)
    for name, args in binding._SIGNATURES.items():
        assert name in protos, name
        want = [_kind(p) for p in protos[name]]
        got = [_ctype_kind(t) for t in args]
        assert got == want, (name, got, want)


def test_stats_struct_matches_the_header():
    text = open(os.path.join(ROOT, "include", "overlap.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct\s*\{([^}]*)\}\s*ov_stats\s*;", text).group(1)
    fields = re.findall(r"(long long|double|int)\s+([a-z_0-9]+)\s*;", body)
    ctypes_of = {"long long": ctypes.c_longlong, "double": ctypes.c_double, "int": ctypes.c_int}
    assert [(n, ctypes_of[t]) for t, n in fields] == list(binding.ov_stats._fields_)


def test_noalloc_binding_checks_buffer_sizes():
    """The C entry point cannot see buffer sizes; the binding refuses links,
    inputs and outputs whose dtype or element count does not fit the lattice
    before anything reaches the library."""
    dims = (4, 4, 4, 4)
    vol = 256
    links = np.zeros((4, 4, 4, 4, 4, 3, 3), dtype=np.complex128)
    psi = np.zeros((1, 4, 4, 4, 4, 4, 3), dtype=np.complex128)
    bad = [
        (links.astype(np.complex64), psi, psi.copy()),           # links in the wrong dtype
        (links[:3], psi, psi.copy()),                              # links too small
        (links, psi[:, :3], psi[:, :3].copy()),                    # input too small
        (links, psi, np.zeros_like(psi, dtype=np.complex64)),      # output dtype differs
        (links, psi, np.zeros(12 * vol - 1, dtype=np.complex128)),  # output too small
    ]
    for lk, x, out in bad:
        with pytest.raises(ValueError):
            binding.ov_wilson_noalloc(dims, lk, x, out, 1)
    with pytest.raises(ValueError):
        binding.ov_wilson_noalloc(dims, links, psi, psi.copy(), 2)  # nrhs larger than the input
