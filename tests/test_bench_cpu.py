"""The benchmark's host-side bookkeeping on the CPU: the DRAM traffic figure is
taken from the committed ncu summary only while the kernel sources it was
measured on are unchanged, and the configuration block names the storage
form and the bytes per node it is measured against."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _profile(tmp_path, sha, traffic="123456789"):
    p = tmp_path / "profile.md"
    p.write_text(f"# summary\n\nkernel_source_sha: {sha}\ntraffic_bytes_per_launch: {traffic}\n")
    return str(p)


def test_traffic_only_for_the_sources_it_was_measured_on(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE", _profile(tmp_path, bench.kernel_sources_hash()))
    assert bench.profiled_traffic("f32") == 123456789.0
    assert bench.profiled_traffic("f16") is None  # the summary covers FP32 storage only
    monkeypatch.setattr(bench, "PROFILE", _profile(tmp_path, "0" * 16))
    assert bench.profiled_traffic("f32") is None
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic("f32") is None


def test_source_hash_follows_the_kernel_sources(tmp_path, monkeypatch):
    h = bench.kernel_sources_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    copy = tmp_path / "repo"
    for rel in bench.KERNEL_SOURCES:
        dst = copy / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(copy))
    assert bench.kernel_sources_hash() == h
    with open(copy / bench.KERNEL_SOURCES[0], "ab") as f:
        f.write(b"\n")
    assert bench.kernel_sources_hash() != h


def test_configuration_block():
    c32, c16 = bench.config_block("f32"), bench.config_block("f16")
    assert c32["storage"] == "f32" and "offsets" in c16["storage"]
    assert "range replay" in c32["l2"] and "range replay" not in c16["l2"]
    assert c32["grid"] == [2048, 1024] and c32["instances"] == 5
    assert bench.BYTES_PER_LUP == {"f32": 72, "f16": 36, "bf16": 36, "f16sr": 36, "bf16sr": 36}
