"""The C ABI library loads and exports every entry point include/skel.h declares; host-side
argument checks reject bad calls without touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_2104_05877_gb300 as skel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:skel_status|const char\*|int|void|uint64_t)\s+(skel_\w+)\s*\(", txt, re.M))
    return names


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(skel.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return skel.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    assert L.skel_status_string(0) == b"ok"
    assert L.skel_status_string(5).startswith(b"grid")
    assert L.skel_version() >= 100


def test_invalid_arguments_rejected_on_host(L):
    sz = ctypes.c_size_t(0)
    # measurement aids: unknown kind, too few rounds, a 3-CTA cluster, an unaligned column
    ns = ctypes.c_void_p(16)
    assert L.skel_debug_exchange_latency(2, 8, 100, 0, ns, None, ctypes.byref(sz), None, None) == 1
    assert L.skel_debug_exchange_latency(1, 8, 1, 0, ns, None, ctypes.byref(sz), None, None) == 1
    assert L.skel_debug_exchange_latency(1, 3, 100, 0, ns, None, ctypes.byref(sz), None, None) == 1
    assert L.skel_debug_exchange_latency(1, 8, 100, 6, ns, None, ctypes.byref(sz), None, None) == 1
    fl = ctypes.c_int64(0)
    assert L.skel_debug_fma_rate(1, 0, ctypes.byref(fl), ns, None) == 1
    # l = 0
    assert L.skel_sketch(10, 10, 0, ctypes.c_void_p(16), 10, 0, 0, 8, 0, 1, ctypes.c_void_p(16), 10,
                         None, ctypes.byref(sz), None, None) == 1
    # lda < m
    assert L.skel_sketch(10, 10, 0, ctypes.c_void_p(16), 5, 4, 0, 8, 0, 1, ctypes.c_void_p(16), 10,
                         None, ctypes.byref(sz), None, None) == 1
    # FP64 arithmetic on FP32 storage
    assert L.skel_sketch(10, 10, 1, ctypes.c_void_p(16), 10, 4, 0, 8, 0, 1, ctypes.c_void_p(16), 10,
                         None, ctypes.byref(sz), None, None) == 1
    # s > n
    assert L.skel_pivot_lupp(0, ctypes.c_void_p(16), 8, 4, 4, 5, ctypes.c_void_p(16), None, 0, None, 0,
                             None, ctypes.byref(sz), None, None) == 1
    # CPQR with l > 1024
    assert L.skel_pivot_cpqr(0, ctypes.c_void_p(16), 2000, 4000, 4000, 5, ctypes.c_void_p(16), None,
                             0, None, ctypes.byref(sz), None, None) == 1
    # sparse sign zeta > l
    assert L.skel_sketch(10, 10, 0, ctypes.c_void_p(16), 10, 4, 1, 8, 0, 1, ctypes.c_void_p(16), 10,
                         None, ctypes.byref(sz), None, None) == 1
    # SRTT: l > m is invalid; a row offset and FP8 are not supported
    assert L.skel_sketch(10, 10, 0, ctypes.c_void_p(16), 10, 11, 2, 8, 0, 1, ctypes.c_void_p(16), 10,
                         None, ctypes.byref(sz), None, None) == 1
    assert L.skel_sketch_rows(4, 10, 10, 0, ctypes.c_void_p(16), 10, 4, 2, 8, 0, 1, ctypes.c_void_p(16),
                              10, None, ctypes.byref(sz), None, None) == 7
    assert L.skel_sketch(10, 10, 1, ctypes.c_void_p(16), 12, 4, 2, 8, 4, 1, ctypes.c_void_p(16), 10,
                         None, ctypes.byref(sz), None, None) == 7
    # batch plan: unknown flag bits
    one = (ctypes.c_int64 * 1)(64)
    ptr = (ctypes.c_void_p * 1)(16)
    plan = ctypes.c_void_p()
    assert L.skel_batch_plan_create(1, one, one, ptr, one, 8, 4, ctypes.c_double(1e-6), 1, 4,
                                    ctypes.byref(plan)) == 1
    # row-partitioned sketch: row0 not a multiple of 4, negative
    for row0 in (2, -4):
        assert L.skel_sketch_rows(row0, 10, 10, 0, ctypes.c_void_p(16), 10, 4, 0, 8, 0, 1, ctypes.c_void_p(16),
                                  10, None, ctypes.byref(sz), None, None) == 1


def test_host_sketch_arguments_and_workspace(L):
    """The host-A sketches check their arguments on the host before any device call, and the
    streaming sketch's workspace is two staging panels (columns padded to a multiple of 4 rows)
    plus the per-panel sketch's workspace (none for the FP64 Gaussian sketch)."""
    sz = ctypes.c_size_t(0)
    A, X = ctypes.c_void_p(16), ctypes.c_void_p(16)
    # skel_sketch_host: negative panel, lda < m, an unknown storage type
    assert L.skel_sketch_host(10, 10, 0, A, 10, 4, 0, 8, 0, 1, X, 10, -1, None, ctypes.byref(sz), None, None) == 1
    assert L.skel_sketch_host(10, 10, 0, A, 9, 4, 0, 8, 0, 1, X, 10, 0, None, ctypes.byref(sz), None, None) == 1
    assert L.skel_sketch_host(10, 10, 7, A, 10, 4, 0, 8, 0, 1, X, 10, 0, None, ctypes.byref(sz), None, None) == 1
    # m = 10, n = 10 in panels of 4 columns: three panels, two staging buffers of 12 x 4 doubles
    assert L.skel_sketch_host(10, 10, 0, A, 10, 4, 0, 8, 0, 1, X, 10, 4, None, ctypes.byref(sz), None, None) == 0
    assert sz.value == 2 * 512
    # one panel: one staging buffer
    assert L.skel_sketch_host(10, 10, 0, A, 10, 4, 0, 8, 0, 1, X, 10, 0, None, ctypes.byref(sz), None, None) == 0
    assert sz.value == 1024
    # skel_sketch_host_two_sided: a panel not a multiple of 4, negative; FP64 arithmetic on FP32
    # storage; m = 0; FP8
    Y = ctypes.c_void_p(16)
    for panel in (6, -4):
        assert L.skel_sketch_host_two_sided(10, 10, 1, A, 10, 4, 2, 1, 2, X, 10, Y, 10, panel, None,
                                            ctypes.byref(sz), None, None) == 1
    assert L.skel_sketch_host_two_sided(10, 10, 1, A, 10, 4, 0, 1, 2, X, 10, Y, 10, 0, None,
                                        ctypes.byref(sz), None, None) == 1
    assert L.skel_sketch_host_two_sided(0, 10, 1, A, 10, 4, 2, 1, 2, X, 10, Y, 10, 0, None,
                                        ctypes.byref(sz), None, None) == 1
    assert L.skel_sketch_host_two_sided(10, 10, 1, A, 10, 4, 4, 1, 2, X, 10, Y, 10, 0, None,
                                        ctypes.byref(sz), None, None) == 7


def test_workspace_query_gaussian_needs_none(L):
    sz = ctypes.c_size_t(123)
    assert L.skel_sketch(100, 50, 0, ctypes.c_void_p(16), 100, 8, 0, 8, 0, 1, ctypes.c_void_p(16), 50,
                         None, ctypes.byref(sz), None, None) == 0
    assert sz.value == 0


def test_oracle_not_imported_by_product():
    """The product package never references the oracle."""
    pkg = os.path.join(ROOT, "paper_2104_05877_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert "oracle" not in open(os.path.join(dp, f)).read(), f


def test_binding_refuses_host_tensors():
    """The binding never hands a host address to the library (the kernels would dereference
    it on the device): a CPU tensor is refused before any call."""
    import torch
    import paper_2104_05877_gb300 as skel
    with pytest.raises(ValueError):
        skel._ptr(torch.zeros(4))
    assert skel._ptr(None) is None
