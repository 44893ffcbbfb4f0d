"""Host-side arithmetic of bench.py (no GPU): the roofline figures, the
whole-job throughput, the pose schedule and the digest that keys the
captured DRAM bytes."""
import os

import pytest

import bench


def _stats(vis, pairs, evals):
    return [{"n_visible": vis, "n_pairs": pairs, "raster_evals": evals}]


def test_roofline_figures_follow_the_stated_bytes_and_ops():
    n, vis, pairs, evals = 1_000_000, 3_000_000, 4_000_000, 350_000_000
    stage_ms = {"project": 0.2, "partition": 0.1, "sort": 0.15, "raster": 0.6, "merge": 0.03}
    pk = {"hbm_gbs": 6795.8, "sm_max_mhz": 2070.0}
    top, out = bench.roofline(stage_ms, _stats(vis, pairs, evals), n, pk, 2070.0, 152)
    assert top == "raster"
    vis_bits = bench.VIEWS * ((n + 31) // 32) * 4
    # projection: 236 bytes read per gaussian, 68 written per visible entry
    proj = n * 236 + vis * 68 + vis_bits
    assert out["project"]["achieved"] == pytest.approx(proj / 0.2e-3 / 1e9, abs=0.01)
    assert out["project"]["frac"] == pytest.approx(out["project"]["achieved"] / 6795.8, abs=1e-4)
    part = vis * 32 + vis_bits * 2 + pairs * 8
    assert out["partition"]["achieved"] == pytest.approx(part / 0.1e-3 / 1e9, abs=0.01)
    assert out["sort"]["achieved"] == pytest.approx(pairs * 16 / 0.15e-3 / 1e9, abs=0.01)
    # rasteriser: FP32-pipe ops against 152 SMs x 128 lanes x the maximum clock
    peak = 152 * 128 * 2070e6 / 1e12
    assert out["raster"]["peak"] == pytest.approx(peak, abs=0.05)
    ops = evals * bench.RASTER_OPS_PER_EVAL
    assert out["raster"]["achieved"] == pytest.approx(ops / 0.6e-3 / 1e12, abs=0.01)
    assert out["raster"]["frac"] == pytest.approx(out["raster"]["achieved"] / peak, abs=1e-3)
    assert {v["bound"] for v in out.values()} == {"hbm", "alu"}
    # the SM count is the device's, not a constant
    _, out148 = bench.roofline(stage_ms, _stats(vis, pairs, evals), n, pk, 2070.0, 148)
    assert out148["raster"]["peak"] == pytest.approx(148 * 128 * 2070e6 / 1e12, abs=0.05)


def test_captured_traffic_only_for_the_sources_it_was_taken_on(monkeypatch):
    monkeypatch.setattr(bench, "sources_digest", lambda: bench.MEASURED_TRAFFIC["digest"])
    assert bench.measured_traffic("raster") == bench.MEASURED_TRAFFIC["bytes"]["raster"]
    monkeypatch.setattr(bench, "sources_digest", lambda: "0" * 16)
    assert bench.measured_traffic("raster") is None


def test_digest_covers_the_forward_sources_only(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2606_00352_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("raster.cu", "blend.cuh", "internal.h", "backward.cu", "serve.cu", "notes.txt"):
        (csrc / f).write_text(f"// {f}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.sources_digest()
    (csrc / "backward.cu").write_text("// changed\n")
    (csrc / "serve.cu").write_text("// changed\n")
    (csrc / "notes.txt").write_text("changed\n")
    assert bench.sources_digest() == d0
    (csrc / "blend.cuh").write_text("// changed\n")
    d1 = bench.sources_digest()
    assert d1 != d0
    (csrc / "raster.cu").write_text("// changed\n")
    assert bench.sources_digest() != d1
    assert set(bench.FORWARD_INDEPENDENT) >= {"backward.cu", "train.cu", "serve.cu"}
    # the real tree: every listed file exists, so the list names real sources
    real = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_00352_gb300", "csrc")
    for f in bench.FORWARD_INDEPENDENT:
        assert os.path.exists(os.path.join(real, f)), f


def test_job_throughput_single_rank():
    value, ms = bench.job_throughput(40.0, 80, 1)
    assert ms == 40.0 and value == pytest.approx(2000.0)


def test_pose_schedule():
    cams = list(range(bench.N_POSES))
    b0 = bench.pose_batch(cams, 0, 0)
    assert b0 == list(range(bench.VIEWS))
    # consecutive steps take consecutive poses, wrapping around the orbit
    steps = [bench.pose_batch(cams, k, 0) for k in range(bench.N_POSES // bench.VIEWS + 1)]
    assert steps[-1] == b0
    # ranks start at different poses
    assert bench.pose_batch(cams, 0, 1) != b0
