// Panel-blocked column-wise LUPP on X (Sec. 2.5.2, Algorithm 2 line 3) for n small enough
// that a panel of b rows of X fits in the shared memory of one thread-block cluster.
//
// The s pivot steps are grouped into panels of b consecutive rows.  For each panel:
//   * PANEL (one cluster of CL CTAs; each CTA holds b rows x n/CL columns of the current
//     Schur complement in shared memory): b greedy steps.  Each step is a cluster-wide argmax
//     (every CTA reads the CL candidates through distributed shared memory), a read of the
//     winner's column from its owner's shared memory, R(t, :) = S(t, :)/S(t, j_t) and the rank-1
//     update of the panel rows.  Only hardware cluster barriers are involved.
//   * TRAIL (whole grid): for every trailing row r, the multipliers of the b steps,
//     M(r, q) = S^{(q)}(r, j_q), by forward substitution with the unit upper triangular
//     R(panel, J_panel), then the b rank-1 updates S(r, :) -= M(r, q) R(q, :) applied in the
//     same order as one-step-at-a-time elimination.
// Every update is a separately rounded multiply then subtract in the textbook order, so the
// factors equal those of unblocked LUPP bit for bit (FP64 runs reproduce a plain FP64
// restatement exactly).  Kernel boundaries order the phases; the working copy of X(0:s, :)
// lives in the workspace.
#include <algorithm>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace skel {

namespace {

constexpr int kPanelThreads = 512;
constexpr size_t kPanelSmemOptin = 227 * 1024;   // opt-in shared memory per block on sm_103a

template <typename T>
struct PanelParams {
  T* Xg;               // s x n working copy (row-major, ld = n)
  int64_t n;
  int s, t0, b;        // panel rows t0 .. t0+b-1
  int ncl;             // columns per CTA of the cluster
  unsigned char* sel;  // n flags: column already selected
  int32_t* Js;
  T* R; int64_t ldr;   // s x n (always present: user output or workspace)
  T* L; int64_t ldl;   // optional s x s
  int32_t* dev_status;
  int32_t* fail;       // device word: set when a panel stopped early (zero / non-finite pivot)
  T* M;                // (s - t0 - b) x b multipliers of the trailing rows (row-major)
};

// One published candidate: magnitude key, global column index, and the candidate's column
// rows 0..b-1 (only rows q.. are meaningful at step q).
constexpr int kMaxPanel = 64;
template <typename T>
struct Cand {
  T key;
  long long idx;
  T col[kMaxPanel];
};

template <typename T>
__global__ void __launch_bounds__(kPanelThreads) lupp_panel_kernel(const PanelParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31;
  const int b = p.b, ncl = p.ncl;
  const int64_t c0 = (int64_t)crank * ncl;
  const int nl = (int)(p.n - c0 < 0 ? 0 : (p.n - c0 < ncl ? p.n - c0 : ncl));

  // inbox[parity][sender]: every CTA pushes its candidate into every peer's inbox before the
  // cluster barrier, so after the barrier all reads are local.  A slot is rewritten two
  // steps later, after every reader has passed the intervening barrier.
  __shared__ Cand<T> inbox[2][16];
  __shared__ long long s_w;
  __shared__ int s_owner;
  __shared__ T wkey[2][32];
  __shared__ int64_t widx[2][32];
  __shared__ int s_J[kMaxPanel];           // pivots of this panel, written out at the end
  __shared__ T s_L[kMaxPanel][kMaxPanel];  // L(t0+r, t0+q) = pivot column q, row r >= q
  T* P = reinterpret_cast<T*>(smem);                       // [b][ncl]
  T* rowq = P + ((size_t)b * ncl > (size_t)b * b + b ? (size_t)b * ncl : (size_t)b * b + b);   // [ncl]
  T* pivc = rowq + ncl;                                    // [b]
  unsigned char* sl = reinterpret_cast<unsigned char*>(pivc + b);   // [ncl]

  if (*(volatile int32_t*)p.fail) return;   // an earlier panel stopped (uniform over the cluster)
  for (int q = 0; q < b; ++q)
    for (int jj = tid; jj < nl; jj += bd) P[(int64_t)q * ncl + jj] = p.Xg[(int64_t)(p.t0 + q) * p.n + c0 + jj];
  for (int jj = tid; jj < nl; jj += bd) sl[jj] = p.sel[c0 + jj];
  cluster.sync();     // every peer has started before anyone writes into its shared memory

  bool stopped = false;
  int done = 0;                       // completed steps of this panel
  for (int q = 0; q < b; ++q) {
    const int t = p.t0 + q;
    const int par = q & 1;
    // local candidate
    T key = T(-1);
    int64_t idx = INT64_MAX;
    for (int jj = tid; jj < nl; jj += bd) {
      if (sl[jj]) continue;
      const T k = pivot_key(P[(int64_t)q * ncl + jj]);
      if (better(k, c0 + jj, key, idx)) { key = k; idx = c0 + jj; }
    }
    // CTA argmax with one barrier: warp winners go to wbest[par], then every warp reduces them
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T k2 = __shfl_xor_sync(0xffffffffu, key, o);
      const int64_t i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (better(k2, i2, key, idx)) { key = k2; idx = i2; }
    }
    if (lane == 0) { wkey[par][tid >> 5] = key; widx[par][tid >> 5] = idx; }
    __syncthreads();
    KeyIdx<T> mine;
    {
      const int nw = bd >> 5;
      T k = lane < nw ? wkey[par][lane] : T(-1);
      int64_t i = lane < nw ? widx[par][lane] : INT64_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(k2, i2, k, i)) { k = k2; i = i2; }
      }
      mine.key = k;
      mine.idx = i;
    }
    const bool have = mine.idx != INT64_MAX;
    const int jb = have ? (int)(mine.idx - c0) : 0;
    // push: thread tid serves peer (tid % CL), column rows f = q + tid / CL, step bd / CL
    {
      const int dest = tid % CL;
      Cand<T>* slot = &cluster.map_shared_rank(&inbox[0][0], dest)[par * 16 + crank];
      if (tid < CL) {
        slot->key = have ? mine.key : T(-1);
        slot->idx = have ? (long long)mine.idx : (long long)INT64_MAX;
      }
      if (have)
        for (int f = q + tid / CL; f < b; f += bd / CL) slot->col[f] = P[(int64_t)f * ncl + jb];
    }
    cluster.sync();
    if (tid < 32) {
      T k = T(-1);
      int64_t i = INT64_MAX;
      int who = lane;
      if (lane < CL) { k = inbox[par][lane].key; i = inbox[par][lane].idx; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
        const int w2 = __shfl_xor_sync(0xffffffffu, who, o);
        if (better(k2, i2, k, i)) { k = k2; i = i2; who = w2; }
      }
      if (lane == 0) { s_w = i; s_owner = who; }
    }
    __syncthreads();
    const int64_t w = s_w;
    const int owner = s_owner;
    if (w != INT64_MAX)
      for (int r = q + tid; r < b; r += bd) pivc[r] = inbox[par][owner].col[r];
    __syncthreads();
    const T piv = w != INT64_MAX ? pivc[q] : T(0);
    const int code = w == INT64_MAX ? SKEL_ERR_INVALID_ARG
                   : !isfinite(piv) ? SKEL_ERR_NONFINITE
                   : piv == T(0) ? SKEL_ERR_RANK_DEFICIENT : 0;
    if (code != 0) {                       // uniform over the cluster
      if (crank == 0) {
        for (int r = t + tid; r < p.s; r += bd) p.Js[r] = -1;
        if (tid == 0) { record_error(p.dev_status, code, t); atomicExch(p.fail, 1); }
      }
      stopped = true;
      break;
    }
    if (tid == 0) s_J[q] = (int)w;
    if (crank == 0 && p.L)
      for (int r = q + tid; r < b; r += bd) s_L[r][q] = pivc[r];
    const int mine_w = owner == crank ? (int)(w - c0) : -1;
    // R(t, :) replaces row q of P (row q is final at step q); the update of rows q+1.. uses it
    for (int jj = tid; jj < nl; jj += bd) {
      T* pq = &P[(int64_t)q * ncl + jj];
      T rv;
      if (jj == mine_w) rv = T(1);
      else if (sl[jj]) rv = T(0);
      else rv = ddiv(*pq, piv);
      *pq = rv;
      if (jj != mine_w && !sl[jj]) {
        int r = q + 1;
        for (; r + 4 <= b; r += 4) {       // loads of four rows first, then their updates
          const T l0 = pivc[r], l1 = pivc[r + 1], l2 = pivc[r + 2], l3 = pivc[r + 3];
          T* x = &P[(int64_t)r * ncl + jj];
          T x0 = x[0], x1 = x[ncl], x2 = x[2 * ncl], x3 = x[3 * ncl];
          x0 = dsub(x0, dmul(l0, rv));
          x1 = dsub(x1, dmul(l1, rv));
          x2 = dsub(x2, dmul(l2, rv));
          x3 = dsub(x3, dmul(l3, rv));
          x[0] = x0; x[ncl] = x1; x[2 * ncl] = x2; x[3 * ncl] = x3;
        }
        for (; r < b; ++r) {
          T* x = &P[(int64_t)r * ncl + jj];
          *x = dsub(*x, dmul(pivc[r], rv));
        }
      }
    }
    __syncthreads();
    if (mine_w >= 0 && tid == 0) sl[mine_w] = 1;
    done = q + 1;
    __syncthreads();
  }
  // write out what the completed steps produced: R rows, selected flags, pivots, L
  for (int q = 0; q < done; ++q)
    for (int jj = tid; jj < nl; jj += bd) p.R[(int64_t)(p.t0 + q) * p.ldr + c0 + jj] = P[(int64_t)q * ncl + jj];
  for (int jj = tid; jj < nl; jj += bd) p.sel[c0 + jj] = sl[jj];
  if (crank == 0) {
    for (int q = tid; q < done; q += bd) p.Js[p.t0 + q] = s_J[q];
    if (p.L)
      for (int e = tid; e < b * done; e += bd) {
        const int r = e / done, q = e % done;
        if (r >= q) p.L[(int64_t)(p.t0 + r) * p.ldl + p.t0 + q] = s_L[r][q];
      }
  }
  // Multipliers of the trailing rows, M(r, q) = S^{(q)}(r, j_q): one warp per row, lane i
  // owns q = i and q = i + 32; after M(r, qq) is final it is broadcast and every later q
  // subtracts M(r, qq) R(t0+qq, j_q) -- the same operations in the same order as
  // step-by-step elimination.  R(panel, J_panel) is staged in shared memory (reusing P).
  __threadfence();
  cluster.sync();
  if (!stopped && p.s - p.t0 - b > 0) {
    T* RJ = P;                                             // [b][b], b <= 64
    int* J = reinterpret_cast<int*>(RJ + (size_t)b * b);
    for (int q = tid; q < b; q += bd) J[q] = s_J[q];
    __syncthreads();
    for (int qq = 0; qq < b; ++qq)
      for (int q = tid; q < b; q += bd) RJ[qq * b + q] = __ldcg(p.R + (int64_t)(p.t0 + qq) * p.ldr + J[q]);
    __syncthreads();
    const int rows = p.s - p.t0 - b;
    const int warp = tid >> 5, nwarps = bd >> 5;
    for (int ri = crank * nwarps + warp; ri < rows; ri += CL * nwarps) {
      const int64_t r = p.t0 + b + ri;
      const int q0 = lane, q1 = lane + 32;
      T a0 = q0 < b ? p.Xg[r * p.n + J[q0]] : T(0);
      T a1 = q1 < b ? p.Xg[r * p.n + J[q1]] : T(0);
      for (int qq = 0; qq < b; ++qq) {
        const T mq = __shfl_sync(0xffffffffu, qq < 32 ? a0 : a1, qq & 31);   // final M(r, qq)
        if (q0 > qq && q0 < b) a0 = dsub(a0, dmul(mq, RJ[qq * b + q0]));
        if (q1 > qq && q1 < b) a1 = dsub(a1, dmul(mq, RJ[qq * b + q1]));
      }
      T* Mr = p.M + (int64_t)ri * b;
      if (q0 < b) Mr[q0] = a0;
      if (q1 < b) Mr[q1] = a1;
      if (p.L) {
        if (q0 < b) p.L[r * p.ldl + p.t0 + q0] = a0;
        if (q1 < b) p.L[r * p.ldl + p.t0 + q1] = a1;
      }
    }
  }
  cluster.sync();     // no CTA leaves while others may still read its shared memory
}

// Trailing update: rows t0+b .. s-1 of Xg, a block of RB rows x CW columns per CTA, with the
// panel rows R(t0.., j0..j0+CW) staged in shared memory.
constexpr int RB = 16;
template <typename T> constexpr int trail_cw() { return sizeof(T) == 8 ? 256 : 512; }

template <typename T>
size_t trail_smem(int b) {
  return sizeof(T) * ((size_t)RB * b + (size_t)b * trail_cw<T>());
}

template <typename T>
__global__ void __launch_bounds__(256) lupp_trail_kernel(const PanelParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int CW = trail_cw<T>();
  const int b = p.b, tid = threadIdx.x;
  const int r0 = blockIdx.y * RB;                         // index among the trailing rows
  const int rows = p.s - p.t0 - b;
  const int nrows = rows - r0 < RB ? rows - r0 : RB;
  if (nrows <= 0) return;
  if (*(volatile int32_t*)p.fail) return;
  T* M = reinterpret_cast<T*>(smem);                      // [RB][b]
  T* Rt = M + (size_t)RB * b;                             // [b][CW]: R(t0+q, j0+c)
  const int64_t j0 = (int64_t)blockIdx.x * CW;
  const int nc = (int)std::min<int64_t>(CW, p.n - j0);
  for (int q = 0; q < b; ++q)
    for (int c = tid; c < nc; c += blockDim.x) Rt[q * CW + c] = p.R[(int64_t)(p.t0 + q) * p.ldr + j0 + c];
  for (int e = tid; e < nrows * b; e += blockDim.x) M[e] = p.M[(int64_t)r0 * b + e];
  __syncthreads();
  for (int c = tid; c < nc; c += blockDim.x) {
    const int64_t j = j0 + c;
    if (p.sel[j]) continue;
    // four independent elimination chains per thread (rows ri..ri+3), each in step order
    for (int ri = 0; ri < nrows; ri += 4) {
      const int nr4 = nrows - ri < 4 ? nrows - ri : 4;
      T v[4];
      T* x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = &p.Xg[(int64_t)(p.t0 + b + r0 + ri + (u < nr4 ? u : 0)) * p.n + j];
        v[u] = *x[u];
      }
      for (int q = 0; q < b; ++q) {
        const T rq = Rt[q * CW + c];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = dsub(v[u], dmul(M[(ri + (u < nr4 ? u : 0)) * b + q], rq));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < nr4) *x[u] = v[u];
    }
  }
}

template <typename T>
__global__ void lupp_panel_init_kernel(const T* X, int64_t ldx, int s, int64_t n, T* Xg,
                                       unsigned char* sel, int32_t* fail, T* L, int64_t ldl) {
  for (int r = blockIdx.y; r < s; r += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      Xg[(int64_t)r * n + j] = X[(int64_t)r * ldx + j];
      if (r == 0) sel[j] = 0;
    }
  if (L)
    for (int r = blockIdx.y; r < s; r += gridDim.y)
      for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < s; c += gridDim.x * blockDim.x)
        L[(int64_t)r * ldl + c] = T(0);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *fail = 0;
}

struct PanelPlan {
  int CL = 0, b = 0, ncl = 0;
  size_t smem = 0, ws = 0;
};

template <typename T>
size_t panel_smem(int b, int ncl) {
  // P (b x ncl) is reused after the steps for R(panel, J_panel) (b x b) and J (b ints)
  const size_t pbuf = std::max((size_t)b * ncl, (size_t)b * b + (size_t)b);
  return sizeof(T) * (pbuf + ncl + b) + ncl + 64;
}

// Largest cluster the device accepts for the panel kernel (16 non-portable, else 8), and the
// panel height b for it.  b == 0 means "use the grid-barrier kernel".
template <typename T>
PanelPlan plan_panel(int64_t n, int s) {
  PanelPlan pl;
  static int max_cluster = -1;
  static size_t kPanelSmem = 0;       // dynamic budget = opt-in maximum - static shared memory
  if (max_cluster < 0) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, lupp_panel_kernel<T>) != cudaSuccess) {
      cudaGetLastError();
      return pl;
    }
    kPanelSmem = kPanelSmemOptin - fa.sharedSizeBytes - 1024;
    max_cluster = 8;
    if (cudaFuncSetAttribute(lupp_panel_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(lupp_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmem) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(kPanelThreads);
      cfg.dynamicSmemBytes = kPanelSmem;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 16;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, lupp_panel_kernel<T>, &cfg) == cudaSuccess && nclusters > 0)
        max_cluster = 16;
    }
    cudaGetLastError();
  }
  for (int CL : {max_cluster, 8}) {
    const int ncl = (int)((n + CL - 1) / CL);
    int b = std::min(kMaxPanel, s);
    while (b >= 8 && panel_smem<T>(b, ncl) > kPanelSmem) b -= 8;
    if (b >= std::min(8, s) && panel_smem<T>(b, ncl) <= kPanelSmem) {
      pl.CL = CL;
      pl.b = b;
      pl.ncl = ncl;
      pl.smem = panel_smem<T>(b, ncl);
      break;
    }
  }
  return pl;
}

template <typename T>
size_t panel_ws(int64_t n, int s, bool need_r) {
  return align_up(sizeof(T) * (size_t)s * n) + align_up(n) + 256 + align_up(sizeof(T) * (size_t)s * 64) +
         (need_r ? align_up(sizeof(T) * (size_t)s * n) : 0);
}

template <typename T>
skel_status run_panel_t(const PanelPlan& pl, const T* X, int64_t n, int64_t ldx, int s, int32_t* Js,
                        T* L, int64_t ldl, T* R, int64_t ldr, void* ws, int32_t* dev_status,
                        cudaStream_t st) {
  char* base = static_cast<char*>(ws);
  PanelParams<T> p{};
  p.Xg = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)s * n);
  p.sel = reinterpret_cast<unsigned char*>(base);
  base += align_up(n);
  p.fail = reinterpret_cast<int32_t*>(base);
  base += 256;
  p.M = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)s * 64);
  if (R == nullptr) {
    R = reinterpret_cast<T*>(base);
    ldr = n;
  }
  p.n = n; p.s = s; p.ncl = pl.ncl; p.Js = Js; p.R = R; p.ldr = ldr; p.L = L; p.ldl = ldl;
  p.dev_status = dev_status;
  lupp_panel_init_kernel<T><<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min(s, 64)), 256, 0, st>>>(
      X, ldx, s, n, p.Xg, p.sel, p.fail, L, ldl);
  note_launches(1);
  if (cudaFuncSetAttribute(lupp_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) != cudaSuccess)
    return SKEL_ERR_CUDA;
  if (pl.CL > 8 &&
      cudaFuncSetAttribute(lupp_panel_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return SKEL_ERR_CUDA;
  for (int t0 = 0; t0 < s; t0 += pl.b) {
    p.t0 = t0;
    p.b = std::min(pl.b, s - t0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.CL);
    cfg.blockDim = dim3(kPanelThreads);
    cfg.dynamicSmemBytes = panel_smem<T>(p.b, pl.ncl);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pl.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, lupp_panel_kernel<T>, p) != cudaSuccess) return SKEL_ERR_CUDA;
    note_launches(1);
    const int rows = s - t0 - p.b;
    if (rows > 0) {
      constexpr int CW = trail_cw<T>();
      dim3 grid((unsigned)((n + CW - 1) / CW), (unsigned)((rows + RB - 1) / RB));
      const size_t tsm = trail_smem<T>(p.b);
      if (tsm > 48 * 1024 &&
          cudaFuncSetAttribute(lupp_trail_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm) != cudaSuccess)
        return SKEL_ERR_CUDA;
      lupp_trail_kernel<T><<<grid, 256, tsm, st>>>(p);
      note_launches(1);
    }
  }
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

}  // namespace

static bool panel_usable(skel_dtype dt, int64_t n, int32_t s) {
  return (dt == SKEL_F64 ? plan_panel<double>(n, s).b : plan_panel<float>(n, s).b) > 0;
}

static size_t panel_workspace(skel_dtype dt, int64_t n, int32_t s) {
  return dt == SKEL_F64 ? panel_ws<double>(n, s, true) : panel_ws<float>(n, s, true);
}

size_t lupp_auto_workspace(skel_dtype dt, int64_t n, int32_t s) {
  return panel_usable(dt, n, s) ? panel_workspace(dt, n, s) : lupp_workspace(dt, n, s, nullptr);
}

skel_status run_lupp_auto(skel_dtype dt, const void* X, int64_t n, int64_t ldx, int32_t s,
                          int32_t* Js, void* L, int64_t ldl, void* R, int64_t ldr, void* ws,
                          size_t ws_bytes, int32_t* dev_status, cudaStream_t st) {
  if (!panel_usable(dt, n, s))
    return run_lupp(dt, X, n, ldx, s, Js, L, ldl, R, ldr, ws, ws_bytes, dev_status, st);
  if (ws_bytes < panel_workspace(dt, n, s)) return SKEL_ERR_WORKSPACE;
  if (dt == SKEL_F64) {
    const PanelPlan pl = plan_panel<double>(n, s);
    if (pl.b == 0) return SKEL_ERR_UNSUPPORTED;
    return run_panel_t<double>(pl, (const double*)X, n, ldx, s, Js, (double*)L, ldl, (double*)R, ldr, ws,
                               dev_status, st);
  }
  const PanelPlan pl = plan_panel<float>(n, s);
  if (pl.b == 0) return SKEL_ERR_UNSUPPORTED;
  return run_panel_t<float>(pl, (const float*)X, n, ldx, s, Js, (float*)L, ldl, (float*)R, ldr, ws,
                            dev_status, st);
}

}  // namespace skel
