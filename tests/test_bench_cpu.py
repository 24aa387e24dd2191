"""The benchmark's host-side helpers (no GPU): the DRAM traffic of the step
kernel is taken from the committed ncu summary only while the summary's
source hash matches the kernel sources, scaled by the sites per launch; the
JSON line's arithmetic; the CPU-baseline helpers."""
import bench


def _summary(tmp_path, sha, nbytes, sites=8192 * 8192):
    p = tmp_path / "summary.md"
    p.write_text(f"# step\n\nkernel_source_sha256: {sha}\ndram_bytes_per_launch: {nbytes}\n"
                 f"sites_per_launch: {sites}\n")
    return str(p)


def test_traffic_follows_the_source_hash_and_scales_by_sites(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha256()
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", _summary(tmp_path, sha, 1.1e9))
    assert bench.traffic_from_profile(8192 * 8192) == 1.1e9
    assert abs(bench.traffic_from_profile(16384 * 16384) - 4.4e9) < 1.0
    other = ("0" if sha[0] != "0" else "1") + sha[1:]
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", _summary(tmp_path, other, 1.1e9))
    assert bench.traffic_from_profile(8192 * 8192) is None
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.traffic_from_profile(8192 * 8192) is None


def test_kernel_hash_covers_the_step_kernel_sources():
    names = [p.rsplit("/", 1)[-1] for p in bench.KERNEL_SOURCES]
    assert names == ["lbm_kernels.cu", "lbm_rows.cuh", "lbm_internal.cuh", "lbm_crack.cuh"]
    assert len(bench.kernel_source_sha256()) == 64


def test_replica_value_is_whole_job_throughput():
    # 4 ranks, 268 M sites each, 20 steps in 0.7 ms x 20: 4 x 383 GLUPS
    v = bench.replica_value(4, 16384 * 16384, 20, 20 * 0.7e-3)
    assert abs(v - 4 * 16384 * 16384 / 0.7e-3 / 1e9) < 1e-6


def test_round_to_four_digits():
    assert bench.r4(374.59845685655915) == 374.6
    assert bench.r4(0.0008753047756) == 0.0008753
    assert bench.r4(None) is None


def test_oracle_band_is_a_row_band_of_the_headline_workload():
    p = bench.oracle_band(64)
    assert (p["nx"], p["ny"]) == (16384, 64)
    assert p["crack"]["y"] == 32.0 and p["crack"]["mode"] == "prescribed" and p["crack"]["v_rel"] == 0.5
    assert p["crack"]["x_tip"] == 2048.0


def test_oracle_timing_sample_is_bounded(oracle_mod):
    from paper_2206_12412_gb300 import workloads as W
    mlups, n, dt, used = bench.oracle_mlups(W.plain_fp64("macroscopic"), 2, 0.3)
    assert mlups > 0 and n >= 2 and dt < 5.0 and used in (1, 2)


def test_committed_summary_names_its_sites():
    text = open(bench.PROFILE_SUMMARY).read()
    assert "sites_per_launch: 67108864" in text and "dram_bytes_per_launch:" in text
    nbytes = float(text.split("dram_bytes_per_launch:")[1].split()[0])
    # the full-size figure is the per-launch bytes scaled by 4, or none while
    # the kernel sources differ from the ones the summary was taken on
    assert bench.traffic_from_profile(16384 * 16384) in (None, 4 * nbytes)
