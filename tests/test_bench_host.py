"""bench.py's host-side arithmetic (CPU only): the roofline's binding unit
and fraction, and the DRAM-traffic record keyed by the kernel source's hash."""
import hashlib
import json
import os

import pytest

import bench

PEAKS = {"bf16_tflops": 1908.7}


def test_tensor_bound_for_one_weight_vector():
    # 1M x 64 workload: 12.5e9 pairs, the kernel in 6.12 ms
    P, sec = 12.499349438e9, 6.12e-3
    roof = bench.roofline(P, 64, 1, "fp16x3", sec, PEAKS, 2070.0)
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(P * 3 * 2 * 64 / sec / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 1908.7)
    assert "of measured" in roof["peak_source"]


def test_fma_bound_for_sixteen_weight_vectors():
    # r = 16: 18 FMAs a pair outweigh 384 tensor flops and one ex2
    P, sec = 4.392e11, 1.166
    roof = bench.roofline(P, 64, 16, "fp16x3", sec, PEAKS, 2070.0)
    assert roof["bound"] == "alu" and roof["unit"] == "Tfma/s"
    assert roof["peak"] == pytest.approx(152 * 128 * 2070e6 / 1e12)
    assert roof["achieved"] == pytest.approx(P * 18 / sec / 1e12)


def test_mufu_bound_when_the_contraction_is_short():
    # d = 4: three split products of length 4 take less than one ex2
    roof = bench.roofline(1e9, 4, 1, "fp16x3", 1e-3, PEAKS, 2070.0)
    assert roof["bound"] == "alu" and roof["unit"] == "Tex2/s"
    assert roof["peak"] == pytest.approx(152 * 32 * 2070e6 / 1e12)


def test_tensor_bound_at_d64_with_the_full_ex2_rate():
    # 384 tensor flops a pair at the measured bf16 rate outlast one ex2 at 32/clk/SM
    roof = bench.roofline(12.5e9, 64, 1, "fp16x3", 3.5e-3, PEAKS, 2070.0, arg_on_tensor=True)
    assert roof["bound"] == "tensor"


def test_long_timed_regions_take_the_sustained_peak():
    # 1M x 1000: 5.15e10 pairs in 176 ms per launch, timed inside seconds-long steps
    peaks = {"bf16_tflops": 1896.9, "bf16_tflops_sustained": 1726.1}
    burst = bench.roofline(5.15e10, 1000, 1, "fp16x3", 0.176, peaks, 2070.0)
    sus = bench.roofline(5.15e10, 1000, 1, "fp16x3", 0.176, peaks, 2070.0, sustained=True)
    assert burst["peak"] == 1896.9 and sus["peak"] == 1726.1
    assert sus["achieved"] == burst["achieved"] and "sustained" in sus["peak_source"]
    # without a sustained figure the burst one stands
    assert bench.roofline(5.15e10, 1000, 1, "fp16x3", 0.176, PEAKS, 2070.0, sustained=True)["peak"] == 1908.7
    # 1M x 64 steps (4.4 ms) are short; 8M and 1M x 1000 Evaluates (290-380 ms) are long
    assert not bench.long_step(4.4) and bench.long_step(290.0) and bench.long_step(380.0)


def test_tf32_peak_and_plain_fp32():
    roof = bench.roofline(1e10, 64, 1, "tf32x3", 1e-2, PEAKS, 2070.0)
    assert roof["peak"] == pytest.approx(1908.7 * 1.1 / 2.25)
    roof = bench.roofline(1e10, 64, 1, "simt_fp32", 1e-1, None, 2070.0)
    assert roof["bound"] == "alu" and roof["achieved"] == pytest.approx(1e10 * 128 / 1e-1 / 1e12)


def test_traffic_record_follows_the_kernel_source():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for kernel, r in rec.items():
        src = open(os.path.join(bench.ROOT, r["source"]), "rb").read()
        current = hashlib.sha256(src).hexdigest() == r["source_sha256"]
        got = bench.measured_traffic(kernel, r["workload"])
        assert got == (r["bytes_per_launch"] if current else None)
        assert bench.measured_traffic(kernel, r["workload"] + " (another size)") is None


def test_fma_count_when_the_tensor_cores_form_the_argument():
    # the global-centered kernel: only the r weight FMAs remain in the epilogue
    P, sec = 4.392e11, 0.9
    roof = bench.roofline(P, 64, 16, "fp16x3", sec, PEAKS, 2070.0, arg_on_tensor=True)
    assert roof["bound"] == "alu" and roof["achieved"] == pytest.approx(P * 16 / sec / 1e12)


def test_mean_request_targets_matches_the_request_stream():
    """The sustained serving rate divides capacity by the mean request size:
    the closed form must agree with the stream's own draws."""
    from paper_1410_0260_gb300 import workloads as wl
    N = 1 << 21
    spec = wl.request_stream(100_000, 200.0, seed=3)
    sample = sum(N * s if k == "weights" else s for _, k, s in spec) / len(spec)
    assert bench._mean_request_targets(N) == pytest.approx(sample, rel=0.02)


def test_weight_sums_on_the_tensor_cores():
    # r = 16 with the weight MMA: 3 x 2 x (64 + 16) tensor flops a pair, no FMAs
    P, sec = 4.392e11, 0.44
    roof = bench.roofline(P, 64, 16, "fp16x3", sec, PEAKS, 2070.0, arg_on_tensor=True, weights_on_tensor=True)
    assert roof["bound"] == "tensor"
    assert roof["achieved"] == pytest.approx(P * 3 * 2 * 80 / sec / 1e12)
