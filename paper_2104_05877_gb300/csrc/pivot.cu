// Greedy column pivoting on the sketch X (l x n, row-major) -- Sec. 2.5.
//
//   LUPP (Sec. 2.5.2, Algorithm 2, column pivoting): step t picks j_t = argmax |S(t, j)| over the
//   unselected columns, R(t,:) = S(t,:)/S(t,j_t), S(t+1:,:) -= S(t+1:,j_t) R(t,:).
//   CPQR (Sec. 2.5.1): step t picks the largest remaining column norm (downdated, with a
//   recompute guard), then applies a Householder reflector to the remaining columns.
//
// Design: one persistent cooperative grid.  CTA b owns a contiguous slab of columns and
// keeps rows 0..s-1 (LUPP) or 0..l-1 (CPQR) of its slab resident in shared memory (global
// workspace when the slab does not fit).  Each step costs one grid-wide barrier: every CTA
// publishes its best local candidate and that candidate's column, then arrives; the argmax
// is a single packed 64-bit atomicMax per CTA for FP32 data, or a fixed-order scan of the G
// published candidates for FP64 data.  The winner's column is frozen once selected, so its
// published copy stays valid.  LUPP looks one step ahead: after the pivot of step t arrives,
// a CTA first updates row t+1 (and its own next candidate column), publishes its candidate
// for step t+1, and only then applies the rest of the Schur update while the barrier
// completes.  The LUPP updates follow the textbook order with msub / rdiv (common.cuh): in
// FP64 separately rounded multiply and subtract and a correctly rounded division, so FP64
// runs reproduce a plain FP64 restatement bit for bit; in FP32 a fused multiply-subtract and
// a multiply by the pivot's reciprocal, as in every other FP32 LUPP kernel.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace skel {

namespace {

constexpr int kThreads = 256;
constexpr size_t kSmemBudget = 200 * 1024;
constexpr int kHeader = 16;   // slot header: int64 index, then the candidate value

template <typename T>
struct PivParams {
  const T* X;
  int64_t l, n, ldx;
  int s;
  int32_t* Js;
  T* L; int64_t ldl;
  T* R; int64_t ldr;
  T* gblock;          // global slab storage when not in shared memory
  int nloc;           // columns per CTA
  int rows;           // resident rows (s for LUPP, l for CPQR)
  int in_smem;
  GridComm gc;
  int32_t* dev_status;
};

__device__ __forceinline__ unsigned char* carve(unsigned char*& p, size_t bytes) {
  unsigned char* r = p;
  p += (bytes + 15) & ~size_t(15);
  return r;
}

template <typename T>
__device__ void fail_tail(const PivParams<T>& p, int t, int code) {
  if (blockIdx.x == 0) {
    for (int r = t + threadIdx.x; r < p.s; r += blockDim.x) p.Js[r] = -1;
    if (threadIdx.x == 0) record_error(p.dev_status, code, t);
  }
  if (threadIdx.x == 0) atomicExch(p.gc.abort, 1);
}

// Publish this CTA's candidate (index, value, column rows r0..r1-1) for `step`.
template <typename T>
__device__ __forceinline__ void publish(const GridComm& gc, int step, int64_t idx, T val, T key,
                                        const T* W, int64_t ldw, int jb, int r0, int r1) {
  char* sl = gc.slot(step, blockIdx.x);
  T* col = reinterpret_cast<T*>(sl + kHeader);
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) col[r] = W[(int64_t)r * ldw + jb];
  if (threadIdx.x == 0) {
    *reinterpret_cast<long long*>(sl) = idx;
    *reinterpret_cast<T*>(sl + 8) = val;
    if constexpr (sizeof(T) == 4) atomicMax(gc.keys + step, pack_key((float)key, idx));
  }
}

// Winner of `step` (call after comm_wait): its global index, or -1 if nobody published.
template <typename T>
__device__ int64_t winner(const GridComm& gc, int step, bool key_is_mag) {
  if constexpr (sizeof(T) == 4) {
    __shared__ long long s_w;
    if (threadIdx.x == 0) {
      const unsigned long long k = __ldcg(gc.keys + step);
      s_w = k == 0ull ? -1 : key_index(k);
    }
    __syncthreads();
    const long long w = s_w;
    __syncthreads();
    return w;
  } else {
    T key = T(-1);
    int64_t idx = INT64_MAX;
    for (int q = threadIdx.x; q < gc.G; q += blockDim.x) {
      const char* sl = gc.slot(step, q);
      const long long ci = __ldcg(reinterpret_cast<const long long*>(sl));
      if (ci >= 0) {
        const T v = __ldcg(reinterpret_cast<const T*>(sl + 8));
        const T kq = key_is_mag ? pivot_key(v) : (isfinite(v) ? v : T(INFINITY));
        if (better(kq, (int64_t)ci, key, idx)) { key = kq; idx = ci; }
      }
    }
    const KeyIdx<T> r = block_argmax<T>(key, idx);
    return r.idx == INT64_MAX ? -1 : r.idx;
  }
}

// Local argmax of |W(row, jj)| over unselected local columns.
template <typename T>
__device__ __forceinline__ KeyIdx<T> local_best(const T* W, int64_t ldw, int row, int nl, int64_t c0,
                                                const unsigned char* sel) {
  T key = T(-1);
  int64_t idx = INT64_MAX;
  for (int jj = threadIdx.x; jj < nl; jj += blockDim.x) {
    if (sel[jj]) continue;
    const T k = pivot_key(W[(int64_t)row * ldw + jj]);
    if (better(k, c0 + jj, key, idx)) { key = k; idx = c0 + jj; }
  }
  return block_argmax<T>(key, idx);
}

// ------------------------------------------------------------------------------------
// LUPP
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) lupp_kernel(const PivParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const int s = p.s, nloc = p.nloc;
  const int64_t c0 = (int64_t)b * nloc;
  const int nl = (int)(p.n - c0 < 0 ? 0 : (p.n - c0 < nloc ? p.n - c0 : nloc));
  unsigned char* cur = smem;
  T* pivcol = (T*)carve(cur, sizeof(T) * s);
  T* rowt = (T*)carve(cur, sizeof(T) * nloc);
  unsigned char* sel = carve(cur, nloc);
  T* W = p.in_smem ? (T*)carve(cur, sizeof(T) * (size_t)s * nloc) : p.gblock + (int64_t)b * s * nloc;

  for (int r = 0; r < s; ++r)
    for (int jj = tid; jj < nl; jj += bd) W[(int64_t)r * nloc + jj] = p.X[(int64_t)r * p.ldx + c0 + jj];
  for (int jj = tid; jj < nloc; jj += bd) sel[jj] = 0;
  if (b == 0 && p.L)
    for (int r = 0; r < s; ++r)
      for (int c = tid; c < s; c += bd) p.L[(int64_t)r * p.ldl + c] = T(0);
  __syncthreads();

  // step 0 candidate
  {
    const KeyIdx<T> c = local_best<T>(W, nloc, 0, nl, c0, sel);
    if (c.key >= T(0)) {
      const int jb = (int)(c.idx - c0);
      publish<T>(p.gc, 0, c.idx, W[jb], c.key, W, nloc, jb, 0, s);
    } else if (tid == 0) {
      *reinterpret_cast<long long*>(p.gc.slot(0, b)) = -1;
    }
    comm_arrive(p.gc, 0);
  }

  for (int t = 0; t < s; ++t) {
    if (!comm_wait(p.gc, t, p.dev_status)) return;
    const int64_t w = winner<T>(p.gc, t, true);
    if (w < 0) { fail_tail(p, t, SKEL_ERR_INVALID_ARG); return; }
    const char* wsl = p.gc.slot(t, (int)(w / nloc));
    const T piv = __ldcg(reinterpret_cast<const T*>(wsl + 8));
    if (!isfinite(piv)) { fail_tail(p, t, SKEL_ERR_NONFINITE); return; }
    if (piv == T(0)) { fail_tail(p, t, SKEL_ERR_RANK_DEFICIENT); return; }
    const T pr = rdiv_prep(piv);
    const T* wcol = reinterpret_cast<const T*>(wsl + kHeader);
    for (int r = t + tid; r < s; r += bd) pivcol[r] = __ldcg(wcol + r);
    if (b == 0 && tid == 0) p.Js[t] = (int32_t)w;
    const int jw = (w >= c0 && w < c0 + nl) ? (int)(w - c0) : -1;
    // R(t, :) for the local slab: row t is final at step t
    for (int jj = tid; jj < nl; jj += bd) {
      T rv;
      if (jj == jw) rv = T(1);
      else if (sel[jj]) rv = T(0);
      else rv = rdiv(W[(int64_t)t * nloc + jj], pr);
      rowt[jj] = rv;
      if (p.R) p.R[(int64_t)t * p.ldr + c0 + jj] = rv;
    }
    __syncthreads();
    if (b == 0 && p.L)
      for (int r = t + tid; r < s; r += bd) p.L[(int64_t)r * p.ldl + t] = pivcol[r];
    if (jw >= 0 && tid == 0) sel[jw] = 1;
    __syncthreads();
    if (t + 1 == s) break;

    // lookahead: row t+1, then this CTA's candidate for step t+1, then publish + arrive
    const int r1 = t + 1;
    for (int jj = tid; jj < nl; jj += bd) {
      if (sel[jj]) continue;
      T* x = &W[(int64_t)r1 * nloc + jj];
      *x = msub(*x, pivcol[r1], rowt[jj]);
    }
    __syncthreads();
    const KeyIdx<T> c = local_best<T>(W, nloc, r1, nl, c0, sel);
    int jb = -1;
    if (c.key >= T(0)) {
      jb = (int)(c.idx - c0);
      for (int r = t + 2 + tid; r < s; r += bd) {
        T* x = &W[(int64_t)r * nloc + jb];
        *x = msub(*x, pivcol[r], rowt[jb]);
      }
      __syncthreads();
      publish<T>(p.gc, r1, c.idx, W[(int64_t)r1 * nloc + jb], c.key, W, nloc, jb, r1, s);
    } else if (tid == 0) {
      *reinterpret_cast<long long*>(p.gc.slot(r1, b)) = -1;
    }
    comm_arrive(p.gc, r1);
    // rest of the Schur update (rows t+2..s-1), overlapping the barrier
    for (int jj = tid; jj < nl; jj += bd) {
      if (sel[jj] || jj == jb) continue;     // jb's rows > t+1 were updated before publishing
      const T rv = rowt[jj];
      for (int r = t + 2; r < s; ++r) {
        T* x = &W[(int64_t)r * nloc + jj];
        *x = msub(*x, pivcol[r], rv);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// CPQR
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) cpqr_kernel(const PivParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = bd >> 5;
  const int l = p.rows, s = p.s, nloc = p.nloc;
  const int64_t c0 = (int64_t)b * nloc;
  const int nl = (int)(p.n - c0 < 0 ? 0 : (p.n - c0 < nloc ? p.n - c0 : nloc));
  unsigned char* cur = smem;
  T* v = (T*)carve(cur, sizeof(T) * l);
  T* nu = (T*)carve(cur, sizeof(T) * nloc);
  T* nu0 = (T*)carve(cur, sizeof(T) * nloc);
  unsigned char* sel = carve(cur, nloc);
  T* W = p.in_smem ? (T*)carve(cur, sizeof(T) * (size_t)l * nloc) : p.gblock + (int64_t)b * l * nloc;
  // downdating guard: recompute a norm when it fell below sqrt(u) of its last exact value
  const T guard = sizeof(T) == 8 ? T(1.4901161193847656e-08) : T(2.44140625e-04);

  for (int r = 0; r < l; ++r)
    for (int jj = tid; jj < nl; jj += bd) W[(int64_t)r * nloc + jj] = p.X[(int64_t)r * p.ldx + c0 + jj];
  for (int jj = tid; jj < nloc; jj += bd) sel[jj] = 0;
  __syncthreads();
  for (int jj = warp; jj < nl; jj += nwarps) {
    T a = T(0);
    for (int r = lane; r < l; r += 32) { const T x = W[(int64_t)r * nloc + jj]; a += x * x; }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) { nu[jj] = a; nu0[jj] = a; }
  }
  __syncthreads();

  for (int t = 0; t < s; ++t) {
    T key = T(-1);
    int64_t idx = INT64_MAX;
    for (int jj = tid; jj < nl; jj += bd) {
      if (sel[jj]) continue;
      const T k = isfinite(nu[jj]) ? nu[jj] : T(INFINITY);
      if (better(k, c0 + jj, key, idx)) { key = k; idx = c0 + jj; }
    }
    const KeyIdx<T> mine = block_argmax<T>(key, idx);
    if (mine.key >= T(0)) {
      const int jb = (int)(mine.idx - c0);
      publish<T>(p.gc, t, mine.idx, nu[jb], mine.key, W, nloc, jb, t, l);
    } else if (tid == 0) {
      *reinterpret_cast<long long*>(p.gc.slot(t, b)) = -1;
    }
    comm_arrive(p.gc, t);
    if (!comm_wait(p.gc, t, p.dev_status)) return;

    const int64_t w = winner<T>(p.gc, t, false);
    if (w < 0) { fail_tail(p, t, SKEL_ERR_INVALID_ARG); return; }
    const T* wcol = reinterpret_cast<const T*>(p.gc.slot(t, (int)(w / nloc)) + kHeader);
    T part = T(0);
    for (int r = t + tid; r < l; r += bd) {
      const T x = __ldcg(wcol + r);
      v[r] = x;
      part += x * x;
    }
    const T nrm2 = block_sum<T>(part);
    if (!isfinite(nrm2)) { fail_tail(p, t, SKEL_ERR_NONFINITE); return; }
    if (nrm2 == T(0)) { fail_tail(p, t, SKEL_ERR_RANK_DEFICIENT); return; }
    const T nrm = sqrt(nrm2);
    const T alpha = v[t];
    const T beta = alpha != T(0) ? -copysign(nrm, alpha) : -nrm;
    const T tau = (beta - alpha) / beta;
    const T den = alpha - beta;
    __syncthreads();
    for (int r = t + 1 + tid; r < l; r += bd) v[r] = v[r] / den;
    if (tid == 0) v[t] = T(1);
    if (b == 0 && tid == 0) p.Js[t] = (int32_t)w;
    const int jw = (w >= c0 && w < c0 + nl) ? (int)(w - c0) : -1;
    __syncthreads();
    if (jw >= 0 && tid == 0) {
      sel[jw] = 1;
      if (p.R) p.R[(int64_t)t * p.ldr + c0 + jw] = beta;
    }
    __syncthreads();
    // apply H = I - tau v v^T to rows t.. of every remaining local column (one warp per column)
    for (int jj = warp; jj < nl; jj += nwarps) {
      if (sel[jj]) {
        if (jj != jw && lane == 0 && p.R) p.R[(int64_t)t * p.ldr + c0 + jj] = T(0);
        continue;
      }
      T d = T(0);
      for (int r = t + lane; r < l; r += 32) d += v[r] * W[(int64_t)r * nloc + jj];
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      const T f = tau * d;
      T tail = T(0);
      for (int r = t + lane; r < l; r += 32) {
        T* x = &W[(int64_t)r * nloc + jj];
        *x -= f * v[r];
        if (r > t) tail += (*x) * (*x);
      }
      for (int o = 16; o > 0; o >>= 1) tail += __shfl_xor_sync(0xffffffffu, tail, o);
      if (lane == 0) {
        const T rt = W[(int64_t)t * nloc + jj];
        if (p.R) p.R[(int64_t)t * p.ldr + c0 + jj] = rt;
        T nn = nu[jj] - rt * rt;
        if (!(nn > guard * nu0[jj])) { nn = tail; nu0[jj] = tail; }   // recompute exactly
        nu[jj] = nn;
      }
    }
    __syncthreads();
  }
}

int choose_grid(int64_t n, int min_cols) {
  const int sms = device_sm_count();
  int64_t g = (n + min_cols - 1) / min_cols;
  g = std::min<int64_t>(g, std::min(sms, kThreads));
  return (int)std::max<int64_t>(g, 1);
}

template <typename T>
size_t smem_bytes(int rows, int nloc, int s_or_l, bool slab) {
  auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  size_t b = a16(sizeof(T) * s_or_l) + 2 * a16(sizeof(T) * nloc) + a16(nloc);
  if (slab) b += a16(sizeof(T) * (size_t)rows * nloc);
  return b;
}

struct Plan {
  int G, nloc, in_smem, nsteps;
  size_t smem, slot_bytes, comm_bytes, block_bytes, total;
};

template <typename T>
Plan plan_pivot(int64_t n, int rows, int s_or_l_vec, int slot_rows, int nsteps) {
  Plan pl{};
  pl.G = choose_grid(n, 32);
  pl.nloc = (int)((n + pl.G - 1) / pl.G);
  pl.nsteps = nsteps;
  const size_t with = smem_bytes<T>(rows, pl.nloc, s_or_l_vec, true);
  pl.in_smem = with <= kSmemBudget;
  pl.smem = pl.in_smem ? with : smem_bytes<T>(rows, pl.nloc, s_or_l_vec, false);
  pl.slot_bytes = align_up(kHeader + sizeof(T) * slot_rows, 16);
  pl.comm_bytes = comm_header_bytes(nsteps) + align_up(2 * pl.G * pl.slot_bytes);
  pl.block_bytes = pl.in_smem ? 0 : align_up(sizeof(T) * (size_t)pl.G * rows * pl.nloc);
  pl.total = pl.comm_bytes + pl.block_bytes;
  return pl;
}

template <typename T>
skel_status launch_pivot(bool is_lupp, const Plan& pl, PivParams<T>& p, void* ws,
                         cudaStream_t st) {
  char* base = static_cast<char*>(ws);
  p.gc.counter = reinterpret_cast<unsigned int*>(base);
  p.gc.abort = reinterpret_cast<int32_t*>(base + 4);
  p.gc.keys = reinterpret_cast<unsigned long long*>(base + 256);
  p.gc.payload = base + comm_header_bytes(pl.nsteps);
  p.gc.slot_bytes = (int64_t)pl.slot_bytes;
  p.gc.G = pl.G;
  p.gc.wait_ns = kDefaultWaitNs;
  p.gblock = pl.in_smem ? nullptr : reinterpret_cast<T*>(base + pl.comm_bytes);
  p.nloc = pl.nloc;
  p.in_smem = pl.in_smem;
  if (cudaMemsetAsync(base, 0, comm_header_bytes(pl.nsteps), st) != cudaSuccess) return SKEL_ERR_CUDA;
  const void* fn = is_lupp ? (const void*)lupp_kernel<T> : (const void*)cpqr_kernel<T>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) != cudaSuccess)
    return SKEL_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.G);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = is_lupp ? cudaLaunchKernelEx(&cfg, lupp_kernel<T>, p)
                          : cudaLaunchKernelEx(&cfg, cpqr_kernel<T>, p);
  note_launches(1);
  return e == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

}  // namespace

size_t lupp_workspace(skel_dtype dt, int64_t n, int32_t s, int* grid_out) {
  const Plan pl = dt == SKEL_F64 ? plan_pivot<double>(n, s, s, s, s) : plan_pivot<float>(n, s, s, s, s);
  if (grid_out) *grid_out = pl.G;
  return pl.total;
}

skel_status run_lupp(skel_dtype dt, const void* X, int64_t n, int64_t ldx, int32_t s, int32_t* Js,
                     void* L, int64_t ldl, void* R, int64_t ldr, void* ws, size_t ws_bytes,
                     int32_t* dev_status, cudaStream_t st) {
  if (dt == SKEL_F64) {
    const Plan pl = plan_pivot<double>(n, s, s, s, s);
    if (ws_bytes < pl.total) return SKEL_ERR_WORKSPACE;
    PivParams<double> p{};
    p.X = (const double*)X; p.l = s; p.n = n; p.ldx = ldx; p.s = s; p.Js = Js;
    p.L = (double*)L; p.ldl = ldl; p.R = (double*)R; p.ldr = ldr; p.rows = s; p.dev_status = dev_status;
    return launch_pivot<double>(true, pl, p, ws, st);
  }
  const Plan pl = plan_pivot<float>(n, s, s, s, s);
  if (ws_bytes < pl.total) return SKEL_ERR_WORKSPACE;
  PivParams<float> p{};
  p.X = (const float*)X; p.l = s; p.n = n; p.ldx = ldx; p.s = s; p.Js = Js;
  p.L = (float*)L; p.ldl = ldl; p.R = (float*)R; p.ldr = ldr; p.rows = s; p.dev_status = dev_status;
  return launch_pivot<float>(true, pl, p, ws, st);
}

size_t cpqr_workspace(skel_dtype dt, int64_t l, int64_t n, int32_t s, int* grid_out) {
  const Plan pl = dt == SKEL_F64 ? plan_pivot<double>(n, (int)l, (int)l, (int)l, s)
                                 : plan_pivot<float>(n, (int)l, (int)l, (int)l, s);
  if (grid_out) *grid_out = pl.G;
  return pl.total;
}

skel_status run_cpqr(skel_dtype dt, const void* X, int64_t l, int64_t n, int64_t ldx, int32_t s,
                     int32_t* Js, void* R, int64_t ldr, void* ws, size_t ws_bytes,
                     int32_t* dev_status, cudaStream_t st) {
  if (dt == SKEL_F64) {
    const Plan pl = plan_pivot<double>(n, (int)l, (int)l, (int)l, s);
    if (ws_bytes < pl.total) return SKEL_ERR_WORKSPACE;
    PivParams<double> p{};
    p.X = (const double*)X; p.l = l; p.n = n; p.ldx = ldx; p.s = s; p.Js = Js;
    p.R = (double*)R; p.ldr = ldr; p.rows = (int)l; p.dev_status = dev_status;
    return launch_pivot<double>(false, pl, p, ws, st);
  }
  const Plan pl = plan_pivot<float>(n, (int)l, (int)l, (int)l, s);
  if (ws_bytes < pl.total) return SKEL_ERR_WORKSPACE;
  PivParams<float> p{};
  p.X = (const float*)X; p.l = l; p.n = n; p.ldx = ldx; p.s = s; p.Js = Js;
  p.R = (float*)R; p.ldr = ldr; p.rows = (int)l; p.dev_status = dev_status;
  return launch_pivot<float>(false, pl, p, ws, st);
}

}  // namespace skel
