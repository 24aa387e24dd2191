"""The benchmark's host-side helpers (no GPU): the DRAM traffic of the step
kernel is taken from the committed ncu summary only while the summary's
source hash matches the kernel sources, and the JSON line's arithmetic."""
import bench


def _summary(tmp_path, sha, nbytes):
    p = tmp_path / "summary.md"
    p.write_text(f"# step\n\nkernel_source_sha256: {sha}\ndram_bytes_per_launch: {nbytes}\n")
    return str(p)


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha256()
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", _summary(tmp_path, sha, 81395968))
    assert bench.traffic_from_profile() == 81395968.0
    other = ("0" if sha[0] != "0" else "1") + sha[1:]
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", _summary(tmp_path, other, 81395968))
    assert bench.traffic_from_profile() is None
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.traffic_from_profile() is None


def test_kernel_hash_covers_the_step_kernel_sources():
    names = [p.rsplit("/", 1)[-1] for p in bench.KERNEL_SOURCES]
    assert names == ["lbm_kernels.cu", "lbm_rows.cuh", "lbm_internal.cuh", "lbm_crack.cuh"]
    assert len(bench.kernel_source_sha256()) == 64


def test_replica_value_is_whole_job_throughput():
    # 4 ranks, 8.39 M sites each, 200 steps in 22.5 ms x 200: 4 x 373 GLUPS
    v = bench.replica_value(4, 4096 * 2048, 200, 200 * 22.5e-6)
    assert abs(v - 4 * 4096 * 2048 / 22.5e-6 / 1e9) < 1e-9
