"""Host-side arithmetic of bench.py's roofline fields (no GPU)."""
import bench


def test_issue_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "profile_entry", lambda k: {"warp_inst_per_voxel": 16.0})
    r = bench.issue_roofline({"fused_compose": {"avg_launch_ms": 0.2}}, 1_000_000, 2000.0)
    peak = 152 * 4 * 2000e6
    assert r["peak"] == peak
    k = r["kernels"]["fused_compose"]
    assert k["achieved"] == 16.0 * 1_000_000 / 0.2e-3
    assert k["frac"] == round(16.0 * 1_000_000 / 0.2e-3 / peak, 4)


def test_stale_profile_gives_no_figures(monkeypatch):
    monkeypatch.setattr(bench, "profile_entry", lambda k: None)
    assert bench.traffic_from_profile("fused_compose", 10) is None
    assert bench.issue_roofline({"fused_compose": {"avg_launch_ms": 0.2}}, 10, None)["kernels"] == {}
