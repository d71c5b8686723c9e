"""Host-side helpers of the benchmark: profile figures are attached to the JSON line only while
the kernel source still hashes to the one the ncu capture was taken on."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _layout(tmp_path, source_text: bytes, digest: str):
    csrc = tmp_path / "paper_2509_16079_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.md").write_text(
        "summary\n\ntraffic_bytes_per_launch: 123456 source %s\n"
        "pipes_pct: fma 61.5 xu 30.0 fp64 6.0 issue 78.5 source %s\n" % (digest, digest))


def test_profile_figures_follow_the_source_hash(tmp_path, monkeypatch):
    text = b"__global__ void k() {}\n"
    _layout(tmp_path, text, hashlib.sha256(text).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k.md", "k.cu") == 123456
    pipes = bench.profiled_pipes("k.md", "k.cu")
    assert pipes["fma_pipe_pct"] == 61.5 and pipes["mufu_pipe_pct"] == 30.0
    assert pipes["fp64_pipe_pct"] == 6.0 and pipes["issue_active_pct"] == 78.5
    # the source changes: both figures are withdrawn
    (tmp_path / "paper_2509_16079_b300" / "csrc" / "k.cu").write_bytes(text + b"// edit\n")
    assert bench.profiled_traffic("k.md", "k.cu") is None
    assert bench.profiled_pipes("k.md", "k.cu") is None


def test_profile_figures_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("missing.md", "missing.cu") is None
    assert bench.profiled_pipes("missing.md", "missing.cu") is None
