"""Host-side pieces of bench.py that need no GPU."""
import os
import shutil

import pytest


def _copy_sources(bench, dst):
    src = os.path.join(bench.ROOT, "paper_1902_11193_gb300", "csrc")
    out = os.path.join(dst, "paper_1902_11193_gb300", "csrc")
    os.makedirs(out)
    for name in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, name), out)
    return out


def test_kernel_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The measured-traffic line stays valid across comment edits and is
    dropped after a code edit."""
    import bench

    out = _copy_sources(bench, str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    path = os.path.join(out, bench.KERNEL_SOURCES[0])
    text = open(path).read()
    with open(path, "w") as fh:
        fh.write("// a new comment line\n/* and a block\n   comment */\n\n" + text + "\n// trailing\n")
    assert bench.kernel_source_hash() == h0
    with open(path, "w") as fh:
        fh.write(text.replace("256u", "257u", 1))
    assert bench.kernel_source_hash() != h0


def test_measured_traffic_needs_matching_sources(tmp_path, monkeypatch):
    import bench

    _copy_sources(bench, str(tmp_path))
    prof = os.path.join(str(tmp_path), "profiles")
    os.makedirs(prof)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    with open(os.path.join(prof, "stream_collide_sparse_fp32.md"), "w") as fh:
        fh.write(f"bench-traffic: layout=sparse precision=fp32 kernel_src={h} "
                 "bytes_per_fluid_node=150.0\n")
    assert bench.measured_traffic("sparse", "fp32", 1000) == pytest.approx(150000.0)
    with open(os.path.join(prof, "stream_collide_sparse_fp32.md"), "w") as fh:
        fh.write("bench-traffic: layout=sparse precision=fp32 kernel_src=0000000000000000 "
                 "bytes_per_fluid_node=150.0\n")
    assert bench.measured_traffic("sparse", "fp32", 1000) is None
