"""Host logic of bench.py that decides what a measurement line reports: the
per-domain check interval of the batch comparison (reading A18: about eight
crossings of the domain at the preconditioned convection speed U / gamma, a
multiple of the batch's tick), the DRAM-traffic lookup (a committed ncu
summary counts only for the kernel sources and work decomposition it was
taken on)."""
import os

import bench
import workloads as wl


def test_check_interval_is_eight_transits_rounded_up_to_the_tick():
    K = 10000
    for n, g in ((64, 0.2), (96, 0.9), (512, 0.5), (1024, 1.0), (1024, 0.25)):
        c = wl.cavity(n, 500.0, 0.1, g)
        k = bench.check_interval(c, K)
        t = 8.0 * n * g / 0.1
        assert k % K == 0 and k >= K
        assert k >= t and k - t < K, (n, g, k, t)
    ch = wl.channel_obstacle(nx=4 * 256, ny=256, D=16, Re=40.0, U0=0.05, gamma=0.5, xc=128)
    assert bench.check_interval(ch, 1000) >= 8 * 1024 * 0.5 / 0.05   # the longer side, its own U


def _write_profile(root, storage, n, h, rows):
    d = os.path.join(root, "profiles")
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, f"stream_collide_{storage}_cavity{n}.txt"), "w") as f:
        f.write("# comment: with colon\n")
        f.write(f"kernel_sources_sha256: {h}\n")
        f.write("dram_bytes_per_launch: 1215859584\n")
        if rows is not None:
            f.write(f"rows_per_item: {rows}\n")


def test_traffic_lookup_needs_the_same_sources_and_decomposition(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "abc123")
    assert bench.profiled_traffic("f32", 4096, 14) is None                  # no summary
    _write_profile(str(tmp_path), "f32", 4096, "abc123", 14)
    assert bench.profiled_traffic("f32", 4096, 14) == 1215859584
    assert bench.profiled_traffic("f32", 4096, 16) is None                  # other work items
    assert bench.profiled_traffic("f16", 4096, 14) is None                  # other storage
    monkeypatch.setattr(bench, "kernel_hash", lambda: "def456")
    assert bench.profiled_traffic("f32", 4096, 14) is None                  # other sources
    _write_profile(str(tmp_path), "f32", 4096, "def456", None)
    assert bench.profiled_traffic("f32", 4096, 16) == 1215859584            # no decomposition recorded

