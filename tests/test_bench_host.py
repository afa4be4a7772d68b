"""Host-side pieces of bench.py (CPU only): the algorithmic bytes per pass,
and the DRAM traffic record read only when it was taken on the current
kernel sources."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_pass_bytes_at_256():
    n = 256
    nvox = n ** 3
    spec = 6 * n * n * (n // 2 + 1) * 8
    assert bench._pass_bytes(n, "y_fwd") == 2 * spec
    assert bench._pass_bytes(n, "x_inv") == spec + 5 * 6 * nvox * 4
    assert bench._pass_bytes(n, "xfwd_tangent") == 6 * nvox * 4 + 5 * nvox + spec
    # one CG iteration's product: 342.5 B/voxel
    total = sum(bench._pass_bytes(n, k) for k in bench.HV_PASSES)
    assert abs(total / nvox - 342.5) < 0.05
    assert bench._pass_bytes(n, "nonexistent") is None


def test_traffic_record_is_keyed_to_the_sources(tmp_path, monkeypatch):
    rec = {"kernel_hash": bench._kernel_hash(), "kernels": {"x_inv@256": {"dram_bytes_per_launch": 123.0}}}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_hash", lambda: rec["kernel_hash"])
    assert bench._traffic("x_inv", 256) == 123.0
    assert bench._traffic("z_proj", 256) is None
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "0" * 16)
    assert bench._traffic("x_inv", 256) is None


def test_kernel_hash_ignores_host_only_and_separate_files():
    h = bench._kernel_hash()
    assert len(h) == 16 and h == bench._kernel_hash()
