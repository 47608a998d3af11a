"""Save and reload the expensive state of an overlap computation: gauge
fields, deflation eigenpairs of K, sign(K) intervals and solutions.

One checkpoint is one ``.npz`` file holding named arrays plus a JSON header
(``__meta__``) with the format version, caller metadata (lattice, seeds,
interval, order, ...) and the SHA-256 digest, dtype and shape of every array.
Writes go to a temporary file in the same directory that is renamed over
the target only when complete, so a crash never leaves a half-written
checkpoint under the final name.  ``load`` recomputes every digest and
raises ``CheckpointError`` on any mismatch, a missing array, or a format
version it does not know.

Arrays may be NumPy arrays or torch tensors (copied to host memory); they are
returned as NumPy arrays.  Eigenpairs of K for deflation (ov_eigs output) go
through ``save_eigenpairs`` / ``load_eigenpairs``, which also check that the
stored lattice and pair count match what the caller expects.
"""
import hashlib
import json
import os
import tempfile
import zipfile

import numpy as np

FORMAT = "overlap-checkpoint"
VERSION = 1
_META_KEY = "__meta__"


class CheckpointError(RuntimeError):
    pass


def _host(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a)
    if hasattr(a, "detach"):  # torch tensor
        return np.ascontiguousarray(a.detach().cpu().numpy())
    return np.ascontiguousarray(np.asarray(a))


def _digest(a):
    return hashlib.sha256(memoryview(np.ascontiguousarray(a)).cast("B")).hexdigest()


def save(path, arrays, meta=None):
    """Writes arrays (name -> array) and meta (JSON-serialisable dict) to path."""
    if not arrays:
        raise CheckpointError("nothing to save")
    host = {}
    for name, a in arrays.items():
        if name == _META_KEY or not name.isidentifier():
            raise CheckpointError(f"bad array name {name!r}")
        host[name] = _host(a)
    header = {"format": FORMAT, "version": VERSION, "meta": meta or {},
              "arrays": {n: {"sha256": _digest(a), "dtype": a.dtype.str, "shape": list(a.shape)}
                         for n, a in host.items()}}
    blob = np.frombuffer(json.dumps(header, sort_keys=True).encode(), dtype=np.uint8)
    path = os.fspath(path)
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".ckpt-", suffix=".npz", dir=d)
    try:
        with os.fdopen(fd, "wb") as f:
            np.savez(f, **host, **{_META_KEY: blob})
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise
    return path


def load(path, verify=True):
    """Returns (arrays, meta).  Raises CheckpointError if the file is not a
    checkpoint of a known version or an array does not match its digest."""
    try:
        with np.load(os.fspath(path), allow_pickle=False) as z:
            if _META_KEY not in z.files:
                raise CheckpointError(f"{path}: no checkpoint header")
            header = json.loads(bytes(z[_META_KEY]).decode())
            if header.get("format") != FORMAT or header.get("version") != VERSION:
                raise CheckpointError(f"{path}: unknown format {header.get('format')!r} "
                                      f"version {header.get('version')!r}")
            arrays = {}
            for name, info in header["arrays"].items():
                if name not in z.files:
                    raise CheckpointError(f"{path}: array {name!r} missing")
                a = z[name]
                if a.dtype.str != info["dtype"] or list(a.shape) != info["shape"]:
                    raise CheckpointError(f"{path}: array {name!r} has dtype/shape {a.dtype.str}/{list(a.shape)}, "
                                          f"header says {info['dtype']}/{info['shape']}")
                if verify and _digest(a) != info["sha256"]:
                    raise CheckpointError(f"{path}: array {name!r} does not match its SHA-256 digest")
                arrays[name] = a
    except CheckpointError:
        raise
    except (OSError, ValueError, KeyError, json.JSONDecodeError, zipfile.BadZipFile) as e:
        raise CheckpointError(f"{path}: unreadable checkpoint ({e})") from e
    return arrays, header["meta"]


def save_eigenpairs(path, dims, evals, evecs, lambda_max=None, **meta):
    """Eigenpairs of K (ascending |lambda|) for deflation, with the lattice
    they belong to and any caller metadata (seeds, tolerance, ...)."""
    evals = _host(evals).astype(np.float64)
    m = dict(meta, kind="eigenpairs", dims=[int(d) for d in dims], n_ev=int(evals.shape[0]))
    if lambda_max is not None:
        m["lambda_max"] = float(lambda_max)
    return save(path, {"evals": evals, "evecs": evecs}, m)


def load_eigenpairs(path, dims, n_ev=None, **expect):
    """Returns (evals, evecs, meta); CheckpointError unless the file holds
    eigenpairs of this lattice (and at least n_ev of them, of which the first
    n_ev are returned) with meta entries equal to ``expect``."""
    arrays, meta = load(path)
    if meta.get("kind") != "eigenpairs":
        raise CheckpointError(f"{path}: not an eigenpair checkpoint")
    if meta.get("dims") != [int(d) for d in dims]:
        raise CheckpointError(f"{path}: lattice {meta.get('dims')} != {list(dims)}")
    for k, v in expect.items():
        if meta.get(k) != v:
            raise CheckpointError(f"{path}: {k} = {meta.get(k)!r}, expected {v!r}")
    evals, evecs = arrays["evals"], arrays["evecs"]
    if evecs.shape[0] != evals.shape[0]:
        raise CheckpointError(f"{path}: {evals.shape[0]} eigenvalues but {evecs.shape[0]} eigenvectors")
    if n_ev is not None:
        if evals.shape[0] < n_ev:
            raise CheckpointError(f"{path}: holds {evals.shape[0]} pairs, {n_ev} requested")
        evals, evecs = evals[:n_ev], evecs[:n_ev]
    return evals, evecs, meta
