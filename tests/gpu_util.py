"""Helpers for the GPU parity tests: device tensors from the seeded NumPy inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def site_rel(got, want):
    """Largest error of one site (over sites and right-hand sides), relative to
    the RMS site norm of want: |got(s) - want(s)| / rms_s |want(s)|.  Unlike the
    whole-field norm it is not diluted when an error is confined to a few
    sites (a boundary plane, a tail block)."""
    g = np.asarray(got).reshape(-1, 12)
    w = np.asarray(want).reshape(-1, 12)
    err = np.linalg.norm(g - w, axis=1)
    rms = np.sqrt(np.mean(np.sum(np.abs(w) ** 2, axis=1)))
    return float(err.max() / rms)
