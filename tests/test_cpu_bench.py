"""bench.py's byte accounting and its link to the committed ncu summary (CPU)."""
import os
import shutil

import pytest

import bench


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("order", [1, 2, 17, 256])
def test_recurrence_bytes_hand_count(prec, order):
    """N K-steps (links + in + out) and N recurrence steps (links + in +
    b_{k+1} + b_{k+2} + psi_perp + out), the first of which has no b_{k+2}
    and b_{k+1} = psi_perp: 2N link reads and 7N - 2 spinor passes."""
    vol = 1000
    want = vol * (2 * order * bench.LINK_B[prec] + (7 * order - 2) * bench.SPIN_B[prec])
    assert bench.recurrence_bytes(prec, order, vol) == want


def test_fp16_average_bytes_per_launch():
    avg = bench.recurrence_bytes("fp16", 256, 1) / 512
    assert abs(avg - 264.0) < 0.2


def test_stencil_metrics_arithmetic():
    vol, launch_s, peak = 663552, 42e-6, 6785.5
    m = bench.stencil_metrics("fp16", vol, launch_s, peak)
    assert m["t_min_over_t"] == pytest.approx(bench.MIN_B["fp16"] * vol / (peak * 1e9) / launch_s)
    assert m["effective_GBps_no_reuse"] == pytest.approx(bench.NO_REUSE_B["fp16"] * vol / launch_s / 1e9)
    traffic = bench.ncu_traffic("fp16")
    if traffic is not None:
        assert m["dram_GBps_ncu_traffic"] == pytest.approx(traffic * vol / launch_s / 1e9)


def test_ncu_traffic_is_keyed_to_the_stencil_sources(tmp_path, monkeypatch):
    """The traffic figure is used only while the stencil sources hash to the
    value recorded beside it."""
    import hashlib
    root = tmp_path / "repo"
    csrc = root / "paper_1510_06897_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (root / "profiles").mkdir()
    h = hashlib.sha256()
    for name in ("dslash_kernel.cuh", "spin.cuh", "common.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_1510_06897_gb300", "csrc", name), csrc / name)
        h.update((csrc / name).read_bytes())
    (root / "profiles" / "dslash_24x24x24x48.md").write_text(
        f"    source_sha256_16: {h.hexdigest()[:16]}\n    traffic_bytes_per_site_fp16: 123.4\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_traffic("fp16") == pytest.approx(123.4)
    assert bench.ncu_traffic("fp32") is None  # no line for it
    with open(csrc / "spin.cuh", "a") as f:
        f.write("\n// changed\n")
    assert bench.ncu_traffic("fp16") is None
