"""Host logic of bench.py on CPU: the DRAM traffic of an ncu summary is reported only for the collision code
and layout it was captured on; the clock samplers fail over cleanly without NVML or nvidia-smi; the
percentile helper; the oracle timing of the uneven batch."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, sha, variant, traffic=1234567):
    p = tmp_path / "summary.md"
    p.write_text(f"# a capture\n\ntraffic_bytes_per_launch: {traffic}\ncollide_variant: {variant}\n"
                 f"collide_code_sha256: {sha}\n")
    return str(p)


def test_traffic_only_for_the_captured_code_and_layout(tmp_path, monkeypatch):
    sha = bench.collide_code_sha256()
    monkeypatch.setitem(bench.PROFILE_NOTES, 6, _summary(tmp_path, sha, 6))
    assert bench.traffic_from_profile(6) == 1234567.0
    monkeypatch.setitem(bench.PROFILE_NOTES, 6, _summary(tmp_path, "0" * 64, 6))
    assert bench.traffic_from_profile(6) is None              # the kernels changed since the capture
    monkeypatch.setitem(bench.PROFILE_NOTES, 6, _summary(tmp_path, sha, 5))
    assert bench.traffic_from_profile(6) is None              # captured on another layout
    assert bench.traffic_from_profile(3) is None              # no summary for this layout


def test_code_hash_ignores_comments_only(tmp_path, monkeypatch):
    a, b = tmp_path / "a.cu", tmp_path / "b.cu"
    a.write_text("int f() { return 1; }  // one\n\n// a note\nint g();\n")
    b.write_text("int f() { return 1; }  // changed words\nint g();\n")
    monkeypatch.setattr(bench, "COLLIDE_SRC", [str(a)])
    ha = bench.collide_code_sha256()
    monkeypatch.setattr(bench, "COLLIDE_SRC", [str(b)])
    assert bench.collide_code_sha256() == ha
    b.write_text("int f() { return 2; }\nint g();\n")
    assert bench.collide_code_sha256() != ha


def test_clock_samplers_fail_over(monkeypatch):
    import ctypes
    real = ctypes.CDLL

    def no_nvml(name, *args, **kw):
        if "nvidia-ml" in str(name):
            raise OSError("not found")
        return real(name, *args, **kw)

    monkeypatch.setattr(ctypes, "CDLL", no_nvml)
    with pytest.raises(OSError):
        bench.NvmlClocks(None, 0)
    c = bench.Clocks(0)
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: (_ for _ in ()).throw(OSError("no smi")))
    c.start()
    out = c.stop()
    assert out["samples"] == 0 and out["sm_mhz"] is None and out["reasons"]


def test_percentiles():
    v = list(range(1, 101))
    assert bench.pct(v, 50) == 50 and bench.pct(v, 99) == 99 and bench.pct(v, 100) == 100
    assert bench.pct([], 50) is None


def test_oracle_batch_sample_extrapolates():
    """The uneven batch's oracle timing: a sample of whole scenarios and trajectory pairs, timed on one
    thread and on every core, extrapolated to the batch's pose tests (small sizes here)."""
    from paper_2005_06773_gb300 import scenarios as S
    batch = S.batch_scenarios(seed=3, count=6)
    r = bench.cpu_oracle_batch(batch, target_tests=2e5, n_scen=2)
    assert 1e5 <= r["tests"] <= 3e5
    assert r["batch_tests"] == sum(sc.n_tests() for sc in batch)
    assert r["one_thread_tests_per_s"] > 0 and r["all_cores_tests_per_s"] > 0 and r["cores"] >= 1
    assert r["batch_s_one_thread"] >= r["batch_tests"] / r["one_thread_tests_per_s"]
    assert r["batch_s_all_cores"] >= r["batch_tests"] / r["all_cores_tests_per_s"]
