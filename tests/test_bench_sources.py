"""bench.py's record of the dominant kernel's DRAM traffic applies only while
the kernel's sources are those the counters were taken on.  The sources of
a kernel are its translation unit and the project headers it includes,
transitively; a header the unit does not include does not invalidate it."""
import os

import bench


def test_include_closure_follows_the_includes():
    grep = bench.include_closure("k_gauge_rep.cu")
    assert grep[0] == "k_gauge_rep.cu"
    assert {"lgf_common.cuh", "lgf_kernels.cuh", "lgf_reduce.cuh", "lgf_gstep.cuh"} <= set(grep)
    assert "fft_reg.cuh" not in grep  # the gradient uses no FFT code
    zt = bench.include_closure("k_fft_zt.cu")
    assert zt[0] == "k_fft_zt.cu" and "fft_reg.cuh" in zt and "lgf_common.cuh" in zt


def test_source_hash_changes_with_an_included_header_only(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1208_1186_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k_a.cu").write_text('#include "h1.cuh"\n')
    (csrc / "h1.cuh").write_text('#include "h2.cuh"\nint a;\n')
    (csrc / "h2.cuh").write_text("int b;\n")
    (csrc / "other.cuh").write_text("int c;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SOURCES, "probe", "k_a.cu")
    assert bench.include_closure("k_a.cu") == ["k_a.cu", "h1.cuh", "h2.cuh"]
    h0 = bench.kernel_source_hash("probe", False)
    (csrc / "other.cuh").write_text("int c2;\n")
    assert bench.kernel_source_hash("probe", False) == h0
    (csrc / "h2.cuh").write_text("int b2;\n")
    assert bench.kernel_source_hash("probe", False) != h0


def test_every_kernel_source_exists():
    csrc = os.path.join(bench.ROOT, "paper_1208_1186_gb300", "csrc")
    for name in set(bench.KERNEL_SOURCES.values()) | {"k_gauge_rep.cu"}:
        assert os.path.exists(os.path.join(csrc, name)), name
