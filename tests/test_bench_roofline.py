"""The bench's roofline arithmetic on synthetic sweep statistics (CPU only):
the dominant sweep is the one with the most device time; HBM-bound sweeps
report algorithmic bytes over the mean launch time against the copy
bandwidth; tensor-core block products report the bf16 work they issue
(3 products per term for the two-term split, 36 and 10 digit pairs for the
complex128 and complex64 integer-slice products) against the sustained bf16
peak; complex128 sweeps on the FP64 pipe report FP64 flops against the
measured FP64 rate, the fixed-point complex128 row sweep bytes against the
copy bandwidth."""
import pytest

import bench
from paper_1208_4869_gb300 import ccg


def test_hbm_sweep_is_bytes_over_time():
    n = 8192
    stats = {(ccg.C64, 0): (100, 8.25, n * n * 8.0),      # A x: 100 launches, 82.5 us each
             (ccg.C64, 1): (10, 1.0, n * n * 8.0)}        # less total time
    r = bench.roofline(ccg, stats, n)
    assert r["kernel"] == "gemv_n_rows_c64" and r["bound"] == "hbm"
    gbs = n * n * 8.0 / 82.5e-6 / 1e9
    assert r["achieved"] == pytest.approx(gbs)
    assert r["frac"] == pytest.approx(gbs / r["peak"])
    assert r["avg_launch_ms"] == pytest.approx(0.0825)
    assert r["sweeps"]["gemv_n_rows_c64"]["tflops"] == pytest.approx(8.0 * n * n / 82.5e-6 / 1e12)


def test_fused_sweep_counts_two_products():
    n = 4096
    stats = {(ccg.C64, 2): (4, 0.4, n * n * 8.0)}
    r = bench.roofline(ccg, stats, n)
    assert r["kernel"] == "gemv_tile_both_c64"
    assert r["sweeps"]["gemv_tile_both_c64"]["tflops"] == pytest.approx(2 * 8.0 * n * n / 0.1e-3 / 1e12)


@pytest.mark.parametrize("kind,prec,name,products", [
    (4, ccg.C64, "gemm_bf16_split_c64", 3),
    (5, ccg.C128, "ozaki_gemm_c128", 36),
    (5, ccg.C64, "ozaki_gemm_c64", 10)])
def test_tensor_products_report_issued_bf16_work(kind, prec, name, products):
    n, k = 8192, 256
    stats = {(prec, kind): (6, 6 * 4.0, 1.0)}             # 4 ms per product
    r = bench.roofline(ccg, stats, n, nrhs=k)
    assert r["kernel"] == name and r["bound"] == "tensor"
    equiv = 8.0 * n * n * k / 4.0e-3 / 1e12               # complex-equivalent TFLOP/s
    assert r["achieved"] == pytest.approx(equiv * products)
    assert r["products_per_term"] == products
    assert r["frac"] == pytest.approx(equiv * products / r["peak"])


def test_complex128_fp64_sweeps_use_the_measured_rate():
    n = 8192
    stats = {(ccg.C128, 1): (10, 4.67, n * n * 16.0)}     # A^H x on the FP64 pipe
    r = bench.roofline(ccg, stats, n, rates={"fp64_fma_tflops": 1.254}, fx=False)
    assert r["kernel"] == "gemv_tile_c_c128" and r["bound"] == "alu" and r["peak"] == 1.254
    assert r["achieved"] == pytest.approx(8.0 * n * n / 0.467e-3 / 1e12)
    assert "measured" in r["peak_source"]
    # without a measurement: the datasheet rate, said so
    r = bench.roofline(ccg, stats, n, fx=False)
    assert r["peak"] == bench.FP64_NOMINAL_TFLOPS and "nominal" in r["peak_source"]
    # the FP64-pipe row sweep (fixed-point sweep switched off)
    r = bench.roofline(ccg, {(ccg.C128, 0): (10, 4.67, n * n * 16.0)}, n, rates={"fp64_fma_tflops": 1.25}, fx=False)
    assert r["kernel"] == "gemv_n_rows_c128" and r["bound"] == "alu"


@pytest.mark.parametrize("kind,tag", [(0, "gemv_fx_rows_c128"), (1, "gemv_fx_tile_c_c128"),
                                      (2, "gemv_fx_tile_both_c128")])
def test_fixed_point_sweeps_are_tagged_hbm_bound(kind, tag):
    n = 4096
    r = bench.roofline(ccg, {(ccg.C128, kind): (4, 0.4, n * n * 16.0)}, n, rates={"fp64_fma_tflops": 1.25})
    assert r["kernel"] == tag and r["bound"] == "hbm"


def test_fixed_point_row_sweep_is_hbm_bound():
    """The default complex128 row sweep reads 16 bytes of digits per element
    on the integer pipe: bytes over time against the copy bandwidth."""
    n = 8192
    stats = {(ccg.C128, 0): (10, 1.9, n * n * 16.0)}
    r = bench.roofline(ccg, stats, n, rates={"fp64_fma_tflops": 1.254})
    assert r["kernel"] == "gemv_fx_rows_c128" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(n * n * 16.0 / 0.19e-3 / 1e9)


def test_no_sweeps_gives_none():
    assert bench.roofline(ccg, {(ccg.C64, 0): (0, 0.0, 1.0)}, 256) is None
