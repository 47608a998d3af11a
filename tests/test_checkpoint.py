"""Checkpoint files (paper_1510_06897_gb300/checkpoint.py): round trips,
integrity and metadata checks, atomic replacement.  CPU only."""
import os

import numpy as np
import pytest

from paper_1510_06897_gb300 import checkpoint as ck
from paper_1510_06897_gb300 import inputs

DIMS = (4, 3, 2, 5)


def test_round_trip_numpy_and_torch(tmp_path):
    torch = pytest.importorskip("torch")
    links = inputs.gauge_links(DIMS, seed=701)
    src = torch.from_numpy(inputs.gaussian_source(DIMS, seed=702, nrhs=2))
    p = ck.save(tmp_path / "state.npz", {"links": links, "x": src}, {"dims": list(DIMS), "mu": 0.02})
    arrays, meta = ck.load(p)
    assert meta == {"dims": list(DIMS), "mu": 0.02}
    assert np.array_equal(arrays["links"], links) and arrays["links"].dtype == np.complex128
    assert np.array_equal(arrays["x"], src.numpy())


def test_eigenpairs_round_trip_and_checks(tmp_path):
    rng = np.random.default_rng(703)
    evals = np.sort(rng.uniform(0.4, 0.6, 6)) * np.array([1, -1, 1, -1, 1, -1])
    evecs = rng.standard_normal((6, 5, 2, 3, 4, 4, 3)) + 0j
    p = tmp_path / "eig.npz"
    ck.save_eigenpairs(p, DIMS, evals, evecs, lambda_max=6.5, seed=1003, tol=2e-5)
    ev, vec, meta = ck.load_eigenpairs(p, DIMS, n_ev=4, seed=1003)
    assert np.array_equal(ev, evals[:4]) and np.array_equal(vec, evecs[:4])
    assert meta["lambda_max"] == 6.5 and meta["n_ev"] == 6
    with pytest.raises(ck.CheckpointError, match="lattice"):
        ck.load_eigenpairs(p, (4, 4, 4, 4))
    with pytest.raises(ck.CheckpointError, match="requested"):
        ck.load_eigenpairs(p, DIMS, n_ev=7)
    with pytest.raises(ck.CheckpointError, match="seed"):
        ck.load_eigenpairs(p, DIMS, seed=1004)


def test_corruption_is_detected(tmp_path):
    a = np.arange(4096, dtype=np.float64)
    p = ck.save(tmp_path / "c.npz", {"a": a})
    # a flipped byte in the file: the archive's CRC catches it
    raw = bytearray(open(p, "rb").read())
    i = raw.find(a[1000:1001].tobytes())
    assert i > 0
    raw[i] ^= 0x01
    bad = tmp_path / "flipped.npz"
    bad.write_bytes(bytes(raw))
    with pytest.raises(ck.CheckpointError):
        ck.load(bad)
    # a consistent archive whose array differs from the header's digest
    with np.load(p) as z:
        header = z["__meta__"]
    b = a.copy()
    b[1000] += 1.0
    swapped = tmp_path / "swapped.npz"
    np.savez(swapped, a=b, __meta__=header)
    with pytest.raises(ck.CheckpointError, match="digest"):
        ck.load(swapped)
    arrays, _ = ck.load(swapped, verify=False)
    assert arrays["a"][1000] == 1001.0


def test_not_a_checkpoint_and_bad_names(tmp_path):
    p = tmp_path / "plain.npz"
    np.savez(p, a=np.zeros(3))
    with pytest.raises(ck.CheckpointError, match="header"):
        ck.load(p)
    (tmp_path / "junk.npz").write_bytes(b"not a zip file")
    with pytest.raises(ck.CheckpointError, match="unreadable"):
        ck.load(tmp_path / "junk.npz")
    with pytest.raises(ck.CheckpointError):
        ck.save(tmp_path / "x.npz", {"__meta__": np.zeros(1)})
    with pytest.raises(ck.CheckpointError):
        ck.save(tmp_path / "x.npz", {})


def test_failed_write_keeps_the_old_file(tmp_path, monkeypatch):
    p = tmp_path / "keep.npz"
    ck.save(p, {"a": np.ones(3)})

    def boom(*args, **kwargs):
        raise OSError("disk full")
    monkeypatch.setattr(np, "savez", boom)
    with pytest.raises(OSError):
        ck.save(p, {"a": np.zeros(3)})
    monkeypatch.undo()
    arrays, _ = ck.load(p)
    assert np.array_equal(arrays["a"], np.ones(3))
    assert [f for f in os.listdir(tmp_path) if f.startswith(".ckpt-")] == []
