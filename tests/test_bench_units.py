"""Host arithmetic of bench.py's roofline block (no GPU): the per-unit
fractions scale the 16-view ncu counters to the timed launch and name the
unit closest to its peak; a kernel whose sources changed since the capture
reports nothing."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_units_scale_and_binding(monkeypatch):
    prof = {"sha": "abc", "dram_read": 1.0e9, "dram_write": 0.5e9, "lts_bytes": 20e9, "warp_inst": 2e9,
            "l1_wavefronts": 1e9, "l1_pct": 90.0, "issue_pct": 55.0, "ncu_ms": 4.0}
    monkeypatch.setitem(bench.NCU_PROFILE, "fx", prof)
    u = bench.measured_units("fx", "abc", launch_ms=50.0, n_views=200, sm_mhz=2000.0, l2_peak=20000.0,
                             hbm_peak=8000.0)
    scale = 200 / bench.NCU_VIEWS
    assert u["dram"]["bytes_per_launch"] == round(1.5e9 * scale)
    assert abs(u["dram"]["frac"] - round(1.5e9 * scale / 0.05 / 1e9 / 8000.0, 4)) < 1e-12
    assert abs(u["l2"]["frac"] - round(20e9 * scale / 0.05 / 1e9 / 20000.0, 4)) < 1e-12
    peak_i = 152 * 4 * 2000e6
    assert abs(u["issue"]["frac"] - round(2e9 * scale / 0.05 / peak_i, 4)) < 1e-12
    assert u["l1_data_pipe"]["frac"] == 0.9
    fr = {k: v["frac"] for k, v in u.items() if isinstance(v, dict) and "frac" in v}
    assert u["binding"] == max(fr, key=fr.get)
    # without the L2 probe or the clock the unit is left out, not guessed
    u2 = bench.measured_units("fx", "abc", 50.0, 200, None, None, 8000.0)
    assert "l2" not in u2 and "issue" not in u2


def test_units_none_for_changed_or_unknown_kernel(monkeypatch):
    monkeypatch.setitem(bench.NCU_PROFILE, "fx", {"sha": "abc"})
    assert bench.measured_units("fx", "other", 50.0, 200, 2000.0, 1.0, 1.0) is None
    assert bench.measured_units("nope", "abc", 50.0, 200, 2000.0, 1.0, 1.0) is None


def test_kernel_sha_covers_the_render_sources():
    sha = bench.kernel_sha()
    assert len(sha) == 16 and all(c in "0123456789abcdef" for c in sha)
    for f in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_2103_14024_gb300", f))


def test_pinned_d2h_rate_is_none_without_a_gpu():
    """The copy-rate figure beside the end-to-end number is measured, never
    guessed: without a CUDA device it is None."""
    import torch
    if torch.cuda.is_available():
        return
    assert bench.pinned_d2h_gbs(torch, torch.empty(16)) is None
