"""Python binding of libskel (include/skel.h): randomized-pivoting skeletonization on GB300.

Thin argument marshalling over the C ABI: torch tensors supply device memory and the current
CUDA stream; every step of the computation runs in libskel's CUDA kernels.  There is no CPU
path: without the built library (``python -m paper_2104_05877_gb300.build``) or without a
CUDA device every call raises.

Layouts (as in the C header): tall matrices (A, C, Q) are column-major (``t.stride(0) == 1``);
wide matrices (the sketch X, pivot factors, Z) are row-major.  Indices are 0-based int32.
"""

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libskel.so")

F64, F32 = 0, 1
PREC = {"f64": 0, "f32": 1, "tf32": 2, "bf16": 3, "fp8": 4}
KIND = {"gaussian": 0, "sparse_sign": 1, "srtt": 2}
STATUS = {0: "ok", 1: "invalid argument", 2: "workspace", 3: "non-finite", 4: "rank deficient",
          5: "timeout", 6: "cuda error", 7: "unsupported"}

_lib = None


class SkelError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        super().__init__(f"{where}: skel status {self.code} ({STATUS.get(self.code, '?')})")


def lib():
    """Load libskel.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libskel.so not built at {LIB_PATH}; run python -m paper_2104_05877_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    i64, i32, u64, u32, vp, szp = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t))
    sig = {
        "skel_sketch": [i64, i64, i32, vp, i64, i32, i32, i32, i32, u64, vp, i64, vp, szp, vp, vp],
        "skel_sketch_rows": [i64, i64, i64, i32, vp, i64, i32, i32, i32, i32, u64, vp, i64, vp, szp, vp, vp],
        "skel_sketch_host": [i64, i64, i32, vp, i64, i32, i32, i32, i32, u64, vp, i64, i64, vp, szp, vp, vp],
        "skel_sketch_host_two_sided": [i64, i64, i32, vp, i64, i32, i32, u64, u64, vp, i64, vp, i64, i64, vp, szp, vp,
                                       vp],
        "skel_sketch_csc": [i64, i64, i64, vp, vp, vp, i32, i32, i32, u64, vp, i64, vp, szp, vp, vp],
        "skel_pivot_lupp": [i32, vp, i64, i64, i64, i32, vp, vp, i64, vp, i64, vp, szp, vp, vp],
        "skel_pivot_cpqr": [i32, vp, i64, i64, i64, i32, vp, vp, i64, vp, szp, vp, vp],
        "skel_id": [i64, i64, i32, vp, i64, i32, vp, vp, i64, vp, vp, szp, vp, vp],
        "skel_id_refine": [i64, i64, i32, vp, i64, i32, vp, vp, i64, vp, vp, szp, vp, vp],
        "skel_cur": [i64, i64, i32, vp, i64, i32, vp, vp, ctypes.c_int, vp, i64, vp, vp, szp, vp, vp],
        "skel_cur_refine": [i64, i64, i32, vp, i64, i32, vp, vp, ctypes.c_int, vp, i64, vp, vp, szp, vp, vp],
        "skel_pivot_rows": [i64, i64, i32, vp, i64, i32, vp, vp, vp, szp, vp, vp],
        "skel_error": [i64, i64, i32, vp, i64, i32, vp, vp, i64, vp, vp, i64, i32, vp, i64, vp, vp,
                       szp, vp, vp],
        "skel_id_sketch": [i32, vp, i64, i64, i64, i32, vp, vp, i64, vp, szp, vp, vp],
        "skel_cur_sketch": [i64, i64, i32, vp, i64, i32, vp, vp, vp, i64, vp, szp, vp, vp],
        "skel_id_cur": [i64, i64, i32, vp, i64, i32, vp, vp, vp, i64, vp, i64, vp, vp, vp, szp, vp, vp],
        "skel_pivot_skeleton": [i32, vp, i64, i64, i64, i32, vp, i64, i64, vp, vp, vp, i64, vp, i64, vp, szp, vp,
                                vp],
        "skel_sketch_power": [i64, i64, i32, vp, i64, i32, i32, i32, u64, vp, i64, vp, szp, vp, vp],
        "skel_sketch_cols": [i64, i64, i32, vp, i64, i32, i32, u64, vp, i64, vp, szp, vp, vp],
        "skel_debug_gaussian": [i32, i64, u64, ctypes.c_int, vp, vp],
        "skel_debug_philox": [vp, i64, u32, u32, vp, vp],
        "skel_debug_curand_philox": [u64, i64, ctypes.c_int, vp, vp],
        "skel_debug_grid_timeout": [ctypes.c_int, u64, vp, szp, vp, vp],
        "skel_debug_fma_rate": [ctypes.c_int, i64, ctypes.POINTER(i64), vp, vp],
        "skel_debug_exchange_latency": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, szp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.skel_status_string.argtypes = [ctypes.c_int]
    L.skel_status_string.restype = ctypes.c_char_p
    L.skel_version.restype = ctypes.c_int
    L.skel_launch_count.restype = ctypes.c_uint64
    L.skel_debug_kernel_timing.argtypes = [ctypes.c_int]
    L.skel_debug_kernel_timing.restype = ctypes.c_int
    L.skel_debug_kernel_time.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64)]
    L.skel_debug_kernel_time.restype = ctypes.c_int
    L.skel_batch_plan_create.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(vp),
                                         ctypes.POINTER(i64), i32, i32, ctypes.c_double, u64, i32,
                                         ctypes.POINTER(vp)]
    L.skel_batch_plan_create.restype = ctypes.c_int
    L.skel_batch_plan_create_points.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(i64), i32,
                                                ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_double, i32, i32,
                                                ctypes.c_double, ctypes.c_uint64, i32, ctypes.POINTER(vp)]
    L.skel_batch_plan_create_points.restype = ctypes.c_int
    L.skel_batch_copy_sketch.argtypes = [vp, i32, vp, vp]
    L.skel_batch_copy_sketch.restype = ctypes.c_int
    L.skel_batch_plan_info.argtypes = [vp, ctypes.POINTER(i32)]
    L.skel_batch_plan_info.restype = ctypes.c_int
    L.skel_batch_z_offsets.argtypes = [vp, ctypes.POINTER(i64)]
    L.skel_batch_z_offsets.restype = ctypes.c_int
    L.skel_batch_run.argtypes = [vp, vp, vp, vp, vp, vp]
    L.skel_batch_run.restype = ctypes.c_int
    L.skel_batch_plan_destroy.argtypes = [vp]
    L.skel_batch_plan_destroy.restype = None
    _lib = L
    return L


# ------------------------------------------------------------------------------------------
def _ptr(t):
    """Device address of a CUDA tensor (None for None).  Host tensors are refused here: the
    kernels dereference every pointer they get on the device."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libskel takes CUDA tensors; got a tensor on " + str(t.device))
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dt(t):
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _colmajor(A):
    """(tensor, ld) with A column-major; copies only when A is not already column-major."""
    if A.dim() != 2:
        raise ValueError("expected a matrix")
    if A.stride(0) == 1 and (A.stride(1) >= max(1, A.shape[0]) or A.shape[1] <= 1):
        return A, max(A.stride(1), A.shape[0], 1)
    At = A.t().contiguous().t()
    return At, max(At.shape[0], 1)


def _pad16(A):
    """A copy of a column-major A whose columns start on 16-byte boundaries (the tensor-core
    paths stream A with TMA)."""
    m, n = A.shape
    ld4 = (m + 3) // 4 * 4
    Ap = torch.empty(n, ld4, dtype=A.dtype, device=A.device).t()
    Ap[:m].copy_(A)
    return Ap[:m], ld4


def _rowmajor(X):
    if X.dim() != 2:
        raise ValueError("expected a matrix")
    if X.stride(1) == 1 and (X.stride(0) >= max(1, X.shape[1]) or X.shape[0] <= 1):
        return X, max(X.stride(0), X.shape[1], 1)
    Xc = X.contiguous()
    return Xc, max(Xc.shape[1], 1)


def new_status(device=None):
    return torch.zeros(2, dtype=torch.int32, device=device or "cuda")


def check_status(dev_status, where=""):
    """Synchronize and raise SkelError if a kernel recorded an error."""
    code, step = (int(x) for x in dev_status.cpu())
    if code != 0:
        raise SkelError(code, f"{where} (step {step})")


def _call(name, build_args, device):
    """Two-phase call: workspace query, allocate, run.  build_args(ws_ptr, ws_size_ptr)."""
    fn = getattr(lib(), name)
    sz = ctypes.c_size_t(0)
    rc = fn(*build_args(None, ctypes.byref(sz)))
    if rc != 0:
        raise SkelError(rc, name)
    ws = torch.empty(max(int(sz.value), 1), dtype=torch.uint8, device=device)
    rc = fn(*build_args(_ptr(ws), ctypes.byref(sz)))
    if rc != 0:
        raise SkelError(rc, name)
    return ws


# ------------------------------------------------------------------------------------------
def sketch(A, l, kind="gaussian", prec="f32", seed=0, zeta=8, X=None, status=None, row0=0):
    """X = Gamma A (l x n, row-major): FP64 for prec='f64', FP32 otherwise.  With row0 > 0, A
    is the block of rows row0 .. row0+m-1 of a larger matrix and X its partial sketch (Gamma's
    columns row0 ..); the partial sketches of a row partition sum to the whole sketch."""
    A, lda = _colmajor(A)
    m, n = A.shape
    if prec in ("tf32", "bf16", "fp8") and (lda % 4 or A.data_ptr() % 16):
        A, lda = _pad16(A)
    xdt = torch.float64 if prec == "f64" else torch.float32
    if X is None:
        X = torch.empty(l, n, dtype=xdt, device=A.device)
    X, ldx = _rowmajor(X)
    st = status if status is not None else new_status(A.device)
    _call("skel_sketch_rows", lambda w, sz: [row0, m, n, _dt(A), _ptr(A), lda, l, KIND[kind], zeta, PREC[prec],
                                             seed, _ptr(X), ldx, w, sz, _ptr(st), _stream()], A.device)
    return X, st


def sketch_host(A, l, kind="gaussian", prec="f32", seed=0, zeta=8, X=None, status=None, panel=0, device=None):
    """X = Gamma A for a host (CPU) A: the library copies A's column panels to the device (two
    staging buffers in the workspace) while it sketches the panel before; X lands on `device`.
    A pinned A (``pin_memory()``) lets the copies run asynchronously; it must then stay alive and
    unchanged until the current stream has passed this call (synchronize, or an event)."""
    A, lda = _host_colmajor(A)
    m, n = A.shape
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    xdt = torch.float64 if prec == "f64" else torch.float32
    if X is None:
        X = torch.empty(l, n, dtype=xdt, device=dev)
    X, ldx = _rowmajor(X)
    st = status if status is not None else new_status(dev)
    host = ctypes.c_void_p(A.data_ptr())
    _call("skel_sketch_host", lambda w, sz: [m, n, _dt(A), host, lda, l, KIND[kind], zeta, PREC[prec], seed,
                                            _ptr(X), ldx, panel, w, sz, _ptr(st), _stream()], dev)
    return X, st


def _host_colmajor(A):
    if A.is_cuda:
        raise ValueError("expected a host tensor; the device forms take a CUDA tensor")
    if A.dim() != 2:
        raise ValueError("expected a matrix")
    if not (A.stride(0) == 1 and (A.stride(1) >= max(1, A.shape[0]) or A.shape[1] <= 1)):
        A = A.t().contiguous().t()
    return A, max(A.stride(1), A.shape[0], 1)


def sketch_host_two_sided(A, l, prec="f32", seed=0, seed_omega=None, status=None, panel=0, device=None):
    """X = Gamma A (l x n) and Yt = Omega A^T (l x m) from one pass over a host A, streamed in
    column panels: the two sketches of Algorithm 3.  A must stay alive and unchanged until the
    current stream has passed this call."""
    A, lda = _host_colmajor(A)
    m, n = A.shape
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    xdt = torch.float64 if prec == "f64" else torch.float32
    X = torch.empty(l, n, dtype=xdt, device=dev)
    Yt = torch.empty(l, m, dtype=xdt, device=dev)
    st = status if status is not None else new_status(dev)
    so = seed + 1 if seed_omega is None else seed_omega
    host = ctypes.c_void_p(A.data_ptr())
    _call("skel_sketch_host_two_sided", lambda w, sz: [m, n, _dt(A), host, lda, l, PREC[prec], seed, so, _ptr(X), n,
                                                       _ptr(Yt), m, panel, w, sz, _ptr(st), _stream()], dev)
    return X, Yt, st


def skeletonize_streaming_host(A, k, p=10, seed=0, seed_omega=None, prec="f32", status=None, panel=0):
    """Algorithm 3 on a host A in one pass: both sketches from the same streamed panels, then J_s
    by LUPP on X and I_s by LUPP on Y^T."""
    X, Yt, st = sketch_host_two_sided(A, k + p, prec=prec, seed=seed, seed_omega=seed_omega, status=status,
                                      panel=panel)
    Js, _, _, _ = pivot_lupp(X, k, factors=False, status=st)
    Is, _, _, _ = pivot_lupp(Yt, k, factors=False, status=st)
    return Js, Is, st


def sketch_power(A, l, q=1, prec="tf32", seed=0, status=None):
    """X = Omega (A^T A)^q (l x n row-major), Omega l x n Gaussian: the power-iterated row space
    approximator (q = 1: Rand-LUPP-1piter)."""
    A, lda = _colmajor(A)
    m, n = A.shape
    if prec in ("tf32", "f32") and (lda % 4 or A.data_ptr() % 16):
        ld4 = (m + 3) // 4 * 4
        Ap = torch.empty(n, ld4, dtype=A.dtype, device=A.device).t()
        Ap[:m].copy_(A)
        A, lda = Ap[:m], ld4
    X = torch.empty(l, n, dtype=torch.float64 if prec == "f64" else torch.float32, device=A.device)
    st = status if status is not None else new_status(A.device)
    _call("skel_sketch_power", lambda w, sz: [m, n, _dt(A), _ptr(A), lda, l, q, PREC[prec], seed, _ptr(X), n, w,
                                              sz, _ptr(st), _stream()], A.device)
    return X, st


def sketch_cols(A, l, prec="f32", seed=1, status=None):
    """Yt = Omega A^T (l x m row-major): the transposed column sketch Y = A Omega^T of the
    streaming skeleton selection (Algorithm 3); LUPP on Yt gives the row skeletons."""
    A, lda = _colmajor(A)
    m, n = A.shape
    if prec in ("tf32", "bf16") and (lda % 4 or A.data_ptr() % 16):
        A, lda = _pad16(A)
    Yt = torch.empty(l, m, dtype=torch.float64 if prec == "f64" else torch.float32, device=A.device)
    st = status if status is not None else new_status(A.device)
    _call("skel_sketch_cols", lambda w, sz: [m, n, _dt(A), _ptr(A), lda, l, PREC[prec], seed, _ptr(Yt), m, w, sz,
                                             _ptr(st), _stream()], A.device)
    return Yt, st


def skeletonize_streaming(A, k, p=10, seed=0, seed_omega=None, prec="f32", status=None):
    """Algorithm 3: row sketch X = Gamma A and column sketch Y = A Omega^T, J_s from LUPP on X
    and I_s from LUPP on Y^T (no skeleton C is gathered for the row pivots)."""
    A, _ = _colmajor(A)
    st = status if status is not None else new_status(A.device)
    l = k + p
    X, _ = sketch(A, l, prec=prec, seed=seed, status=st)
    Yt, _ = sketch_cols(A, l, prec=prec, seed=seed + 1 if seed_omega is None else seed_omega, status=st)
    Js, _, _, _ = pivot_lupp(X, k, factors=False, status=st)
    Is, _, _, _ = pivot_lupp(Yt, k, factors=False, status=st)
    return Js, Is, st


def sketch_csc(col_ptr, row_idx, val, m, n, l, kind="sparse_sign", seed=0, zeta=8, status=None, X=None):
    """X = Gamma A (l x n FP32, row-major) for a CSC A: col_ptr int64 (n+1), row_idx int32,
    val float32 on the device."""
    if X is None:
        X = torch.empty(l, n, dtype=torch.float32, device=val.device)
    if X.shape != (l, n) or X.dtype != torch.float32 or X.stride() != (n, 1):
        raise ValueError("X must be a contiguous l x n float32 tensor")
    st = status if status is not None else new_status(val.device)
    nnz = val.numel()
    _call("skel_sketch_csc", lambda w, sz: [m, n, nnz, _ptr(col_ptr), _ptr(row_idx), _ptr(val), l,
                                            KIND[kind], zeta, seed, _ptr(X), n, w, sz, _ptr(st),
                                            _stream()], val.device)
    return X, st


def pivot_lupp(X, s, factors=True, status=None):
    """Column-wise LUPP on X (l x n row-major): Js (s,), and optionally L (s x s), R (s x n)."""
    X, ldx = _rowmajor(X)
    l, n = X.shape
    Js = torch.empty(s, dtype=torch.int32, device=X.device)
    Lf = torch.empty(s, s, dtype=X.dtype, device=X.device) if factors else None
    Rf = torch.empty(s, n, dtype=X.dtype, device=X.device) if factors else None
    st = status if status is not None else new_status(X.device)
    _call("skel_pivot_lupp", lambda w, sz: [_dt(X), _ptr(X), l, n, ldx, s, _ptr(Js), _ptr(Lf), s,
                                            _ptr(Rf), n, w, sz, _ptr(st), _stream()], X.device)
    return Js, Lf, Rf, st


def pivot_skeleton(X, A, s, factors=True, status=None):
    """Js (LUPP on the sketch X) and Is (LUPP on C^T, C = A(:, Js)) in one call, the row LUPP
    pipelined behind the column LUPP; returns (Js, Is, L, R, status), L and R as pivot_lupp."""
    X, ldx = _rowmajor(X)
    A, lda = _colmajor(A)
    l, n = X.shape
    m = A.shape[0]
    if A.dtype != X.dtype:
        raise ValueError("X and A must have the same dtype")
    Js = torch.empty(s, dtype=torch.int32, device=X.device)
    Is = torch.empty(s, dtype=torch.int32, device=X.device)
    L = torch.empty(s, s, dtype=X.dtype, device=X.device) if factors else None
    R = torch.empty(s, n, dtype=X.dtype, device=X.device) if factors else None
    st = status if status is not None else new_status(X.device)
    _call("skel_pivot_skeleton", lambda w, sz: [_dt(X), _ptr(X), l, n, ldx, s, _ptr(A), m, lda, _ptr(Js), _ptr(Is),
                                                _ptr(L), s if factors else 0, _ptr(R), n if factors else 0, w, sz,
                                                _ptr(st), _stream()], X.device)
    return Js, Is, L, R, st


def pivot_lupp_rows(C, s, status=None):
    """Row-wise LUPP on a tall C (m x s', column-major): the row skeletons Is."""
    C, ldc = _colmajor(C)
    m, sc = C.shape
    Is = torch.empty(s, dtype=torch.int32, device=C.device)
    st = status if status is not None else new_status(C.device)
    _call("skel_pivot_lupp", lambda w, sz: [_dt(C), _ptr(C), sc, m, ldc, s, _ptr(Is), None, 0, None,
                                            0, w, sz, _ptr(st), _stream()], C.device)
    return Is, st


def pivot_cpqr(X, s, factors=True, status=None):
    X, ldx = _rowmajor(X)
    l, n = X.shape
    Js = torch.empty(s, dtype=torch.int32, device=X.device)
    Rf = torch.empty(s, n, dtype=X.dtype, device=X.device) if factors else None
    st = status if status is not None else new_status(X.device)
    _call("skel_pivot_cpqr", lambda w, sz: [_dt(X), _ptr(X), l, n, ldx, s, _ptr(Js), _ptr(Rf), n, w,
                                            sz, _ptr(st), _stream()], X.device)
    return Js, Rf, st


def column_id(A, Js, status=None):
    """Z (s x n, FP64, row-major) with A ~ A(:, Js) Z, and [||A||_F^2, ||Q_C^T A||_F^2]."""
    A, lda = _colmajor(A)
    m, n = A.shape
    s = Js.numel()
    Z = torch.empty(s, n, dtype=torch.float64, device=A.device)
    sq = torch.empty(2, dtype=torch.float64, device=A.device)
    st = status if status is not None else new_status(A.device)
    _call("skel_id", lambda w, sz: [m, n, _dt(A), _ptr(A), lda, s, _ptr(Js), _ptr(Z), n, _ptr(sq), w,
                                    sz, _ptr(st), _stream()], A.device)
    return Z, sq, st


def column_id_refined(A, Js, status=None):
    """column_id for an FP32 A followed by one FP64 refinement step (corrected seminormal
    equations with exact FP32 products): returns (Z, [||A||^2, ||Q_C^T A||^2], status)."""
    A, lda = _colmajor(A)
    m, n = A.shape
    s = Js.numel()
    Z = torch.empty(s, n, dtype=torch.float64, device=A.device)
    sq = torch.empty(2, dtype=torch.float64, device=A.device)
    st = status if status is not None else new_status(A.device)
    _call("skel_id_refine", lambda w, sz: [m, n, _dt(A), _ptr(A), lda, s, _ptr(Js), _ptr(Z), n, _ptr(sq), w,
                                           sz, _ptr(st), _stream()], A.device)
    return Z, sq, st


def column_id_sketch(X, Js, status=None):
    """Z = X(:, Js)^+ X (s x n FP64): the column ID from the sketch alone (no pass over A), the
    least-squares solution over all l rows of the sketch X (l x n row-major)."""
    X, ldx = _rowmajor(X)
    l, n = X.shape
    s = Js.numel()
    Z = torch.empty(s, n, dtype=torch.float64, device=X.device)
    st = status if status is not None else new_status(X.device)
    _call("skel_id_sketch", lambda w, sz: [_dt(X), _ptr(X), l, n, ldx, s, _ptr(Js), _ptr(Z), n, w, sz, _ptr(st),
                                           _stream()], X.device)
    return Z, st


def id_cur(A, Js, Is, status=None):
    """Column ID and stable CUR in one call (one QR of C and one W = Q_C^T A for both):
    returns (Z, U, sq_id, sq_cur, status) with the meanings of column_id and cur."""
    A, lda = _colmajor(A)
    m, n = A.shape
    s = Js.numel()
    Z = torch.empty(s, n, dtype=torch.float64, device=A.device)
    U = torch.empty(s, s, dtype=torch.float64, device=A.device)
    sq_id = torch.empty(2, dtype=torch.float64, device=A.device)
    sq_cur = torch.empty(2, dtype=torch.float64, device=A.device)
    st = status if status is not None else new_status(A.device)
    _call("skel_id_cur", lambda w, sz: [m, n, _dt(A), _ptr(A), lda, s, _ptr(Js), _ptr(Is), _ptr(Z), n, _ptr(U), s,
                                        _ptr(sq_id), _ptr(sq_cur), w, sz, _ptr(st), _stream()], A.device)
    return Z, U, sq_id, sq_cur, st


def cur_sketch(A, Js, Is, status=None):
    """U = A(Is, Js)^{-1} (s x s FP64): the CUR A ~ C U R without a second pass over A."""
    A, lda = _colmajor(A)
    m, n = A.shape
    s = Js.numel()
    U = torch.empty(s, s, dtype=torch.float64, device=A.device)
    st = status if status is not None else new_status(A.device)
    _call("skel_cur_sketch", lambda w, sz: [m, n, _dt(A), _ptr(A), lda, s, _ptr(Js), _ptr(Is), _ptr(U), s, w, sz,
                                            _ptr(st), _stream()], A.device)
    return U, st


def pivot_rows(A, Js, status=None):
    """Row skeletons Is by row-wise LUPP on C = A(:, Js) (Algorithm 2, row pivoting)."""
    A, lda = _colmajor(A)
    m, n = A.shape
    s = Js.numel()
    Is = torch.empty(s, dtype=torch.int32, device=A.device)
    st = status if status is not None else new_status(A.device)
    _call("skel_pivot_rows", lambda w, sz: [m, n, _dt(A), _ptr(A), lda, s, _ptr(Js), _ptr(Is), w, sz,
                                            _ptr(st), _stream()], A.device)
    return Is, st


def cur(A, Js, Is=None, status=None, refine=False):
    """U (s x s FP64) with A ~ A(:, Js) U A(Is, :) (Remark 3) and [||A||_F^2, ||Q_C^T A Q_R||_F^2].
    Is is computed by row-wise LUPP on C when not given.  refine=True (FP32 A): one FP64
    refinement step of U (skel_cur_refine).  Returns (Is, U, sq_norms, status)."""
    A, lda = _colmajor(A)
    m, n = A.shape
    s = Js.numel()
    given = Is is not None
    if not given:
        Is = torch.empty(s, dtype=torch.int32, device=A.device)
    U = torch.empty(s, s, dtype=torch.float64, device=A.device)
    sq = torch.empty(2, dtype=torch.float64, device=A.device)
    st = status if status is not None else new_status(A.device)
    _call("skel_cur_refine" if refine else "skel_cur",
          lambda w, sz: [m, n, _dt(A), _ptr(A), lda, s, _ptr(Js), _ptr(Is), int(given), _ptr(U), s, _ptr(sq), w, sz,
                         _ptr(st), _stream()], A.device)
    return Is, U, sq, st


def launch_count():
    """Kernels launched by libskel in this process so far."""
    return int(lib().skel_launch_count())


def kernel_timing(enable):
    """Start (True) or stop (False) per-kernel CUDA-event timing of the hot kernels; either
    discards earlier records."""
    rc = lib().skel_debug_kernel_timing(1 if enable else 0)
    if rc != 0:
        raise SkelError(rc, "skel_debug_kernel_timing")


def kernel_time(name):
    """(total ms, launches) of the recorded launches of one kernel ("sketch_tc", "gemm_tc",
    "lupp_panel", "lupp_trail", "qr_panel", "gemm_simt", "trsm")."""
    ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
    rc = lib().skel_debug_kernel_time(name.encode(), ctypes.byref(ms), ctypes.byref(n))
    if rc != 0:
        raise SkelError(rc, "skel_debug_kernel_time")
    return ms.value, n.value


def error(A, Js=None, Z=None, Is=None, U=None, Rf=None, status=None):
    """Device double[4] = [||A||_F, ||A - CZ||_F, ||A - CUR||_F, eta] (NaN where not asked)."""
    A, lda = _colmajor(A)
    m, n = A.shape
    s = 0 if Js is None else Js.numel()
    out = torch.empty(4, dtype=torch.float64, device=A.device)
    st = status if status is not None else new_status(A.device)
    if Rf is not None:
        Rf, ldrf = _rowmajor(Rf)
        rdt = _dt(Rf)
    else:
        ldrf, rdt = 0, F64
    ldz = 0 if Z is None else _rowmajor(Z)[1]
    _call("skel_error", lambda w, sz: [m, n, _dt(A), _ptr(A), lda, s, _ptr(Js), _ptr(Z), ldz, _ptr(Is),
                                       _ptr(U), s, rdt, _ptr(Rf), ldrf, _ptr(out), w, sz, _ptr(st),
                                       _stream()], A.device)
    return out, st


def debug_gaussian(l, m, seed, fp64=False, device="cuda"):
    G = torch.empty(l, m, dtype=torch.float64 if fp64 else torch.float32, device=device)
    rc = lib().skel_debug_gaussian(l, m, seed, int(fp64), _ptr(G), _stream())
    if rc != 0:
        raise SkelError(rc, "skel_debug_gaussian")
    return G


def debug_philox(counters, k0, k1):
    """counters: int64/uint32-valued tensor (N, 4) on the device -> (N, 4) int64 words."""
    c = counters.to(torch.int64).to(torch.int32)   # two's complement bit patterns
    out = torch.empty_like(c)
    rc = lib().skel_debug_philox(_ptr(c), c.shape[0], k0, k1, _ptr(out), _stream())
    if rc != 0:
        raise SkelError(rc, "skel_debug_philox")
    return out.to(torch.int64) & 0xFFFFFFFF


def debug_curand_philox(seed, nseq, per_seq, device="cuda"):
    out = torch.empty(nseq * per_seq * 4, dtype=torch.int32, device=device)
    rc = lib().skel_debug_curand_philox(seed, nseq, per_seq, _ptr(out), _stream())
    if rc != 0:
        raise SkelError(rc, "skel_debug_curand_philox")
    return (out.to(torch.int64) & 0xFFFFFFFF).reshape(nseq, per_seq, 4)


def debug_grid_timeout(grid, wait_ns, device="cuda"):
    """Runs a grid-wide wait that cannot complete; returns the device status tensor."""
    st = new_status(device)
    _call("skel_debug_grid_timeout", lambda w, sz: [grid, wait_ns, w, sz, _ptr(st), _stream()], device)
    return st


def debug_fma_rate(fp64=True, iters=1 << 14, device="cuda"):
    """TFLOP/s of the FP64 (or FP32) FMA pipes, timed with CUDA events on the current stream."""
    sink = torch.empty(8 * torch.cuda.get_device_properties(device).multi_processor_count,
                       dtype=torch.float64 if fp64 else torch.float32, device=device)
    flops = ctypes.c_int64(0)
    fn = lambda: lib().skel_debug_fma_rate(int(fp64), iters, ctypes.byref(flops), _ptr(sink), _stream())
    rc = fn()                                   # warm-up
    if rc != 0:
        raise SkelError(rc, "skel_debug_fma_rate")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rc = fn()
    e1.record()
    torch.cuda.synchronize()
    if rc != 0:
        raise SkelError(rc, "skel_debug_fma_rate")
    return flops.value / (e0.elapsed_time(e1) * 1e-3) / 1e12


def debug_exchange_latency(kind, ctas, steps=2000, col_words=0, device="cuda"):
    """ns per round of the grid barrier (kind 0) or the cluster candidate exchange (kind 1)."""
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=device)
    st = new_status(device)
    _call("skel_debug_exchange_latency", lambda w, sz: [kind, ctas, steps, col_words, _ptr(out), w, sz, _ptr(st),
                                                        _stream()], device)
    check_status(st, "skel_debug_exchange_latency")
    return float(out.cpu()[0])


def skeletonize(A, k, p=10, seed=0, prec="f32", pivot="lupp", kind="gaussian", zeta=8,
                want_cur=True, want_error=True):
    """Algorithm 2 end to end on the device: sketch -> pivots on X -> column ID (-> rows by
    LUPP on C, CUR) (-> errors and eta).  Returns a dict of device tensors."""
    st = new_status(A.device)
    l = k + p
    X, _ = sketch(A, l, kind=kind, prec=prec, seed=seed, zeta=zeta, status=st)
    Is = None
    if pivot == "lupp" and want_cur and X.dtype == A.dtype:
        Js, Is, _, Rf, _ = pivot_skeleton(X, A, k, status=st)     # row LUPP pipelined behind
    elif pivot == "lupp":
        Js, _, Rf, _ = pivot_lupp(X, k, status=st)
    else:
        Js, Rf, _ = pivot_cpqr(X, k, status=st)
    if want_cur:
        if Is is None:
            Is, _ = pivot_rows(A, Js, status=st)
        Z, U, sq, sq_cur, _ = id_cur(A, Js, Is, status=st)      # one QR of C for both
        out = dict(X=X, Js=Js, Rf=Rf, Z=Z, sq_norms=sq, status=st, Is=Is, U=U, sq_norms_cur=sq_cur)
    else:
        Z, sq, _ = column_id(A, Js, status=st)
        out = dict(X=X, Js=Js, Rf=Rf, Z=Z, sq_norms=sq, status=st)
    if want_error:
        e, _ = error(A, Js, Z, out.get("Is"), out.get("U"), Rf, status=st)
        out["errors"] = e
    return out


class BatchPlan:
    """Batched skeletonization of independent FP32 blocks (skel_batch_*): per block the sketch
    with l = kmax + p rows, LUPP stopped at the tolerance-driven rank, and the column ID
    coefficients Z_b = X_b(:, J)^+ X_b (least squares over all l rows of the sketch).  `blocks`: CUDA float32 tensors (m_b x n_b,
    column-major views, kept alive by the plan)."""

    def __init__(self, blocks, kmax, p=16, tol=1e-6, seed=0, graph=False, autotune=False):
        self.blocks = []
        self.l = kmax + p
        if blocks is None:                     # from_points fills the plan in
            return
        for B in blocks:
            if B.dtype != torch.float32 or not B.is_cuda:
                raise ValueError("batch blocks must be float32 CUDA tensors")
            B, ldb = _colmajor(B)
            if ldb % 4 or B.data_ptr() % 16:       # TMA: 16-byte aligned columns
                ld4 = (B.shape[0] + 3) // 4 * 4
                Bp = torch.empty(B.shape[1], ld4, dtype=B.dtype, device=B.device).t()
                Bp[:B.shape[0]].copy_(B)
                B, ldb = Bp[:B.shape[0]], ld4
            self.blocks.append((B, ldb))
        nb = len(self.blocks)
        arr = lambda T, v: (T * nb)(*v)
        m = arr(ctypes.c_int64, [B.shape[0] for B, _ in self.blocks])
        n = arr(ctypes.c_int64, [B.shape[1] for B, _ in self.blocks])
        a = arr(ctypes.c_void_p, [B.data_ptr() for B, _ in self.blocks])
        ld = arr(ctypes.c_int64, [ldb for _, ldb in self.blocks])
        self.kmax, self.nb, self.device = kmax, nb, self.blocks[0][0].device
        self._plan = ctypes.c_void_p()
        flags = (1 if graph else 0) | (2 if autotune else 0)
        rc = lib().skel_batch_plan_create(nb, m, n, a, ld, kmax, p, float(tol), seed, flags, ctypes.byref(self._plan))
        if rc != 0:
            raise SkelError(rc, "skel_batch_plan_create")
        self.ncols = [B.shape[1] for B, _ in self.blocks]
        self._finish(graph)

    @classmethod
    def from_points(cls, xs, ys, h, kmax, p=16, tol=1e-6, seed=0, graph=False, autotune=False):
        """The batch for Gaussian-kernel blocks A_b(i, j) = exp(-||x_i - y_j||^2 / h^2) given by
        point sets (skel_batch_plan_create_points): xs[b] (m_b x dim) and ys[b] (n_b x dim),
        float32 CUDA tensors, dim <= 3, kept alive by the plan and read at every run.  A_b is
        evaluated inside the sketch kernel and never stored."""
        self = cls(None, kmax, p)
        pts = []
        for x, y in zip(xs, ys):
            if x.dtype != torch.float32 or y.dtype != torch.float32 or not (x.is_cuda and y.is_cuda):
                raise ValueError("points must be float32 CUDA tensors")
            if x.dim() != 2 or y.dim() != 2 or x.shape[1] != y.shape[1]:
                raise ValueError("points: (m_b, dim) and (n_b, dim) tensors")
            pts.append((x.contiguous(), y.contiguous()))
        self.points = pts
        nb = len(pts)
        dim = pts[0][0].shape[1]
        arr = lambda T, v: (T * nb)(*v)
        m = arr(ctypes.c_int64, [x.shape[0] for x, _ in pts])
        n = arr(ctypes.c_int64, [y.shape[0] for _, y in pts])
        xp = arr(ctypes.c_void_p, [x.data_ptr() for x, _ in pts])
        yp = arr(ctypes.c_void_p, [y.data_ptr() for _, y in pts])
        self.kmax, self.nb, self.device = kmax, nb, pts[0][0].device
        self._plan = ctypes.c_void_p()
        flags = (1 if graph else 0) | (2 if autotune else 0)
        rc = lib().skel_batch_plan_create_points(nb, m, n, dim, xp, yp, float(h), kmax, p, float(tol), seed, flags,
                                                 ctypes.byref(self._plan))
        if rc != 0:
            raise SkelError(rc, "skel_batch_plan_create_points")
        self.ncols = [y.shape[0] for _, y in pts]
        self._finish(graph)
        return self

    def _finish(self, graph):
        nb = self.nb
        off = (ctypes.c_int64 * (nb + 1))()
        lib().skel_batch_z_offsets(self._plan, off)
        self.z_offsets = list(off)
        info = (ctypes.c_int32 * 4)()
        lib().skel_batch_plan_info(self._plan, info)
        self.info = {"sketch_stages": info[0], "concurrent_classes": bool(info[1]), "flags": info[2],
                     "sketch_items": info[3]}
        self._graph = graph
        self._out = None

    def run(self, status=None):
        """Returns (Js (nb x kmax int32), ranks (nb,), Z_all (float64), status) on the device.
        With graph=True the same output tensors are reused (the captured graph is bound to
        them) and overwritten by the next run."""
        if self._graph and self._out is not None and status is None:
            Js, ranks, Z, st = self._out
        else:
            Js = torch.empty(self.nb, self.kmax, dtype=torch.int32, device=self.device)
            ranks = torch.empty(self.nb, dtype=torch.int32, device=self.device)
            Z = torch.zeros(max(self.z_offsets[-1], 1), dtype=torch.float64, device=self.device)
            st = status if status is not None else new_status(self.device)
            if self._graph and status is None:
                self._out = (Js, ranks, Z, st)
        rc = lib().skel_batch_run(self._plan, _ptr(Js), _ptr(ranks), _ptr(Z), _ptr(st), _stream())
        if rc != 0:
            raise SkelError(rc, "skel_batch_run")
        return Js, ranks, Z, st

    def sketch_block(self, b):
        """X_b ((kmax + p) x n_b float32, a copy) as the last run left it."""
        X = torch.empty(self.l, self.ncols[b], dtype=torch.float32, device=self.device)
        rc = lib().skel_batch_copy_sketch(self._plan, b, _ptr(X), _stream())
        if rc != 0:
            raise SkelError(rc, "skel_batch_copy_sketch")
        return X

    def z_block(self, Z, b, rank=None):
        """Z_b (rank x n_b) as a view of Z_all."""
        n_b = self.ncols[b]
        zb = Z[self.z_offsets[b]:self.z_offsets[b + 1]].view(self.kmax, n_b)
        return zb if rank is None else zb[:rank]

    def __del__(self):
        if getattr(self, "_plan", None) and self._plan.value and _lib is not None:
            _lib.skel_batch_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()
