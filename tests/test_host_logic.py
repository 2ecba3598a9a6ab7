"""Host-side logic that needs no GPU: the binding's layout helpers, the batch plan's input
checks, and the benchmark's clock-record parsing (against fake nvidia-smi lines)."""
import importlib.util
import os

import numpy as np
import pytest
import torch

import paper_2104_05877_gb300 as skel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_colmajor_keeps_column_major_views_and_copies_others():
    A = torch.arange(12.0).reshape(3, 4)                 # row-major 3 x 4
    C, ld = skel._colmajor(A)
    assert C.stride(0) == 1 and ld == 3 and torch.equal(C, A)
    F = A.t().contiguous().t()                           # already column-major
    C2, ld2 = skel._colmajor(F)
    assert C2.data_ptr() == F.data_ptr() and ld2 == 3
    big = torch.zeros(5, 4).t().contiguous().t()         # column-major with lda 5, view of 3 rows
    V = big[:3]
    C3, ld3 = skel._colmajor(V)
    assert C3.data_ptr() == V.data_ptr() and ld3 == 5
    with pytest.raises(ValueError):
        skel._colmajor(torch.zeros(3))


def test_rowmajor_and_pad16():
    X = torch.arange(10.0).reshape(2, 5)
    R, ld = skel._rowmajor(X)
    assert ld == 5 and torch.equal(R, X)
    R2, ld2 = skel._rowmajor(X.t())                      # transposed view: copied row-major
    assert R2.is_contiguous() and ld2 == 2 and torch.equal(R2, X.t())
    A = torch.randn(7, 3, dtype=torch.float32).t().contiguous().t()   # lda = 7: not a multiple of 4
    P, ldp = skel._pad16(A)
    assert ldp == 8 and P.shape == A.shape and torch.equal(P, A) and P.stride() == (1, 8)


def test_binding_rejects_non_cuda_batch_blocks():
    with pytest.raises(ValueError):
        skel.BatchPlan([torch.zeros(64, 64)], 8)


def test_clock_summary_flags_throttle_reasons():
    """The benchmark's clock record: median SM clock, max clock and the throttle reasons that
    were active in any sample, parsed from nvidia-smi's CSV (fields: sm, max sm, power,
    active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap)."""
    b = _bench()
    cs = b.ClockSampler(0)
    cs.lines = ["2070, 2070, 800.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                "2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                "2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage line"]
    sm = cs.summary()
    assert sm["sm_mhz"] == 2070.0 and sm["sm_max_mhz"] == 2070.0 and sm["samples"] == 3
    assert sm["reasons"] == ["sw_power_cap"]
    cs.lines = ["1500, 2070, 700.0, 0x40, Not Active, Active, Not Active, Not Active"]
    assert cs.summary()["reasons"] == ["hw_thermal_slowdown"]
    cs.lines = []
    assert cs.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_peaks_fallback_and_workload_config():
    b = _bench()
    hbm, bf16, src = b.load_peaks()
    assert hbm > 1000 and bf16 > 100 and src in ("measured", "fallback")
    cfg = b.workload_config("dense_8192x8192", 256, 16, "tf32")
    assert cfg["m"] == cfg["n"] == 8192 and cfg["l"] == 272 and "workload" in cfg
    cfg = b.workload_config("dense_65536x32768", 1024, 76, "bf16")
    assert (cfg["m"], cfg["n"], cfg["k"], cfg["l"]) == (65536, 32768, 1024, 1100)
    assert b.tensor_peak("tf32", {"bf16_tflops": 2250.0, "bf16_tflops_sustained": 1800.0}, False) == pytest.approx(1100.0)
    assert b.tensor_peak("fp8", {"bf16_tflops": 2250.0, "bf16_tflops_sustained": 1800.0}, True) == pytest.approx(3600.0)


def test_recorded_traffic_is_the_algorithmic_bytes():
    """The DRAM traffic the bench line reports for its sketch kernels (ncu captures, scaled from a
    slice at 65536 x 32768) is within 1% of the algorithmic bytes: A read once by the TF32
    sketch (4 m n), A8 and Gamma's e4m3 normals read once by the FP8 GEMM (m n + l_pad m),
    the 8192^2 sketch reading A once."""
    b = _bench()
    m, n, l = 65536, 32768, 1100
    lpad = (l + 127) // 128 * 128
    t5 = b.TRAFFIC_PER_LAUNCH["dense_65536x32768"]
    assert t5["sketch_tc_tf32"] == pytest.approx(4.0 * m * n, rel=0.01)
    assert t5["sketch_fp8_fp8"] == pytest.approx(1.0 * m * n + lpad * m, rel=0.01)
    assert b.TRAFFIC_PER_LAUNCH["dense_8192x8192"]["sketch_tc"] == pytest.approx(4.0 * 8192 * 8192, rel=0.02)
