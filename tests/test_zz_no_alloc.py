"""GPU: skel_pivot_lupp_static, the LUPP entry point for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Its results must equal those of
skel_pivot_lupp, which takes a caller-allocated workspace, on two calls in a row (the array
keeps the previous call's contents, so the second call checks that the entry point clears
what must start at zero).  This file sorts last so that a run stopping at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _static_fn(skel):
    fn = skel.lib().skel_pivot_lupp_static
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int32, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                   vp, vp, ctypes.c_int64, vp, ctypes.c_int64, vp, vp]
    fn.restype = ctypes.c_int
    return fn


def _run_static(skel, fn, X, s):
    l, n = X.shape
    Js = torch.full((s,), -7, dtype=torch.int32, device=X.device)
    Lf = torch.full((s, s), float("nan"), dtype=X.dtype, device=X.device)
    Rf = torch.full((s, n), float("nan"), dtype=X.dtype, device=X.device)
    st = skel.new_status(X.device)
    dt = 0 if X.dtype == torch.float64 else 1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(dt, ctypes.c_void_p(X.data_ptr()), l, n, n, s, ctypes.c_void_p(Js.data_ptr()),
            ctypes.c_void_p(Lf.data_ptr()), s, ctypes.c_void_p(Rf.data_ptr()), n,
            ctypes.c_void_p(st.data_ptr()), stream)
    assert rc == 0, rc
    skel.check_status(st, "skel_pivot_lupp_static")
    return Js, Lf, Rf


# (FP64, 992, 992, 992) needs 8,373,760 bytes of scratch, just under the 8 MiB array, with the
# column slab in the array rather than in shared memory (32 x 992 FP64 entries per CTA exceed
# the shared-memory budget): the layout where the slab follows the grid's exchange buffers.
@pytest.mark.parametrize("dtype,l,n,s", [(torch.float32, 300, 4096, 256), (torch.float64, 60, 800, 50),
                                         (torch.float32, 8, 8, 8), (torch.float64, 992, 992, 992)])
def test_static_scratch_matches_workspace_entry_point(skel, dev, dtype, l, n, s):
    fn = _static_fn(skel)
    gen = torch.Generator(device="cpu").manual_seed(l * n + s)
    for call in range(2):
        X = torch.randn(l, n, generator=gen, dtype=torch.float64).to(dev, dtype)
        Js_ref, L_ref, R_ref, st = skel.pivot_lupp(X, s)
        skel.check_status(st)
        Js, Lf, Rf = _run_static(skel, fn, X, s)
        torch.cuda.synchronize()
        assert torch.equal(Js.cpu(), Js_ref.cpu()), f"call {call}"
        assert torch.equal(Rf.cpu(), R_ref.cpu()), f"call {call}"
        assert torch.equal(Lf.cpu(), L_ref.cpu()), f"call {call}"


@pytest.mark.parametrize("l,n,s", [(512, 8192, 512), (996, 996, 996)])
def test_static_scratch_rejects_oversized_problem(skel, dev, l, n, s):
    """FP64 with s = 512 over 8192 columns needs a ~33 MB slab, and l = s = n = 996 the first
    square size past the 8 MiB array (992 fits, above): the call returns SKEL_ERR_WORKSPACE,
    launches nothing and leaves no error behind."""
    fn = _static_fn(skel)
    X = torch.ones(l, n, dtype=torch.float64, device=dev)
    Js = torch.full((s,), -7, dtype=torch.int32, device=dev)
    st = skel.new_status(dev)
    torch.cuda.synchronize()
    n0 = skel.launch_count()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(0, ctypes.c_void_p(X.data_ptr()), l, n, n, s, ctypes.c_void_p(Js.data_ptr()),
            None, 0, None, 0, ctypes.c_void_p(st.data_ptr()), stream)
    assert rc == 2
    torch.cuda.synchronize()
    assert skel.launch_count() == n0
    skel.check_status(st, "rejected call")
    assert bool((Js.cpu() == -7).all())
