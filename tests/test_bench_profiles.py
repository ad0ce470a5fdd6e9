"""Host logic of bench.py's roofline `traffic`: DRAM bytes come from a committed ncu summary
only while that summary's kernel hash matches the current kernel sources."""
import os

import bench


def _summary(tmp_path, name, hash_, per_cell):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / (name + ".txt")).write_text(
        "# a summary\n# Command: ncu ... (comment lines are skipped: a: b)\n"
        "dram_bytes_per_cell: %s\nkernel_hash: %s\n" % (per_cell, hash_))


def test_traffic_scales_the_per_cell_bytes_when_the_hash_matches(tmp_path, monkeypatch):
    h = bench._kernel_hash()
    monkeypatch.setattr(bench, "_kernel_hash", lambda: h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _summary(tmp_path, "k", h, "28.64")
    assert bench._profiled_traffic("k", 1000) == 28640


def test_traffic_is_null_for_a_stale_or_missing_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "0123456789abcdef")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _summary(tmp_path, "k", "fedcba9876543210", "28.64")
    assert bench._profiled_traffic("k", 1000) is None          # taken on other sources
    assert bench._profiled_traffic("absent", 1000) is None
    _summary(tmp_path, "bad", "0123456789abcdef", "n/a")
    assert bench._profiled_traffic("bad", 1000) is None        # unreadable figure


def test_kernel_hash_covers_the_kernel_sources(tmp_path, monkeypatch):
    # a copy of the three files that hold the timed kernels hashes alike; a change to any
    # one of them changes the hash
    import shutil
    src = os.path.join(bench.ROOT, "paper_2604_18886_b300", "csrc")
    dst = tmp_path / "paper_2604_18886_b300" / "csrc"
    dst.mkdir(parents=True)
    files = ("kernels.cuh", "octet.cuh", "ocg_api.cu")
    for f in files:
        shutil.copy(os.path.join(src, f), dst / f)
    h0 = bench._kernel_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._kernel_hash() == h0
    seen = {h0}
    for f in files:
        with open(dst / f, "ab") as fh:
            fh.write(b"\n")
        h = bench._kernel_hash()
        assert h not in seen, f
        seen.add(h)
