"""CPU checks of the benchmark's roofline bookkeeping (no GPU): which roofline binds a kernel,
the fractions it reports, and that DRAM traffic is taken from an ncu summary only while the
summary was captured from the current kernel sources."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1800.0,
         "source": "measured"}


def test_hbm_bound_kernel_reports_bytes_against_the_copy_peak():
    # 12 GB in 4 ms = 3000 GB/s, no products: HBM-bound at half the measured copy peak
    st = {"total_ms": 4.0, "launches": 2, "bytes": 12e9, "flops": 0.0}
    r = bench.roofline_record("stream", st, PEAKS, True, 6.1e9)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(3000.0)
    assert r["frac"] == pytest.approx(0.5)
    assert r["traffic"] == 6.1e9
    assert r["ms_per_launch"] == pytest.approx(2.0)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(6e9)


def test_tensor_bound_kernel_reports_products_against_the_sustained_peak():
    # 1 GB and 9 TFLOP in 10 ms: ideal times 0.17 ms (HBM) against 5 ms (tensor at the
    # sustained 1800 TFLOP/s), so the tensor roofline binds: 900 / 1800 = 0.5
    st = {"total_ms": 10.0, "launches": 1, "bytes": 1e9, "flops": 9e12}
    r = bench.roofline_record("gram_split", st, PEAKS, True, None)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(1800.0)
    assert r["frac"] == pytest.approx(0.5)
    assert r["hbm_frac"] == pytest.approx(100.0 / 6000.0)
    # a kernel timed alone takes the burst peak
    r2 = bench.roofline_record("gram_split", st, PEAKS, False, None)
    assert r2["peak"] == pytest.approx(2000.0) and r2["frac"] == pytest.approx(0.45)


def test_e4m3_products_count_against_twice_the_bf16_peak():
    st = {"total_ms": 1.0, "launches": 1, "bytes": 1e6, "flops": 1.8e12}
    r = bench.roofline_record("gram_fp8", st, PEAKS, True, None)
    assert r["peak"] == pytest.approx(3600.0)
    assert r["frac"] == pytest.approx(0.5)


def test_low_intensity_gram_is_hbm_bound():
    # 100 flop per byte is below the ridge (1800e12 / 6000e9 = 300 flop/B): HBM binds
    st = {"total_ms": 2.0, "launches": 1, "bytes": 6e9, "flops": 6e11}
    r = bench.roofline_record("gram_fp8", st, PEAKS, True, None)
    assert r["bound"] == "hbm"
    assert r["frac"] == pytest.approx(0.5)
    assert r["tensor_frac"] == pytest.approx(300.0 / 3600.0)


def test_traffic_only_from_summaries_of_the_current_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2512_15187_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("__global__ void k() {}\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_sources_sha16()
    (prof / "gram_kernel_x.md").write_text(
        f"# x\n\nsource_sha256_16: {sha}\n\ndram_bytes_per_full_launch: 2.5e+11\n")
    (prof / "stream_kernel_y.md").write_text(
        "# y\n\nsource_sha256_16: 0000000000000000\n\ndram_bytes_per_full_launch: 1e+10\n")
    assert bench.ncu_traffic("gram_kernel_x") == pytest.approx(2.5e11)
    assert bench.ncu_traffic("stream_kernel_y") is None      # captured from other sources
    assert bench.ncu_traffic("bands_kernel") is None          # no summary at all
    (csrc / "k.cu").write_text("__global__ void k() { }\n")   # any source edit
    assert bench.ncu_traffic("gram_kernel_x") is None


def test_committed_summaries_describe_the_committed_sources():
    """Every ncu summary under profiles/ was captured from the kernel sources as they are, so
    the benchmark's traffic figures come from the kernels it times."""
    sha = bench.kernel_sources_sha16()
    prof = os.path.join(ROOT, "profiles")
    stamps = {}
    for name in sorted(os.listdir(prof)):
        if name.endswith(".md"):
            txt = open(os.path.join(prof, name)).read()
            line = [ln for ln in txt.splitlines() if ln.startswith("source_sha256_16:")]
            stamps[name] = line[0].split(":")[1].strip() if line else None
    assert stamps, "no ncu summaries"
    assert all(v == sha for v in stamps.values()), stamps


def test_step_hbm_rate_sums_every_launch_over_the_step_time():
    prof = {"stream": {"launches": 10, "bytes": 20e9, "total_ms": 5.0, "flops": 0.0},
            "gram": {"launches": 0, "bytes": 0.0, "total_ms": 0.0, "flops": 0.0},
            "gram_split": {"launches": 2, "bytes": 400e9, "total_ms": 80.0, "flops": 1e12}}
    r = bench.step_hbm_record(prof, 2, 200.0, PEAKS)      # 2 steps in 200 ms
    assert r["algorithmic_gb_per_step"] == pytest.approx(210.0)
    assert r["achieved_gbs"] == pytest.approx(2100.0)
    assert r["frac"] == pytest.approx(2100.0 / 6000.0)
