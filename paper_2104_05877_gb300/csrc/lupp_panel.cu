// Panel-blocked column-wise LUPP on X (Sec. 2.5.2, Algorithm 2, column pivoting) for n small enough
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
// Every update is msub(x, m, r) in the textbook order (common.cuh: separately rounded
// multiply then subtract in FP64, one fused multiply-subtract in FP32), and R's rows come from
// rdiv, so the factors equal those of unblocked LUPP in the same arithmetic bit for bit (FP64
// runs reproduce a plain FP64 restatement exactly).  Kernel boundaries order the phases; the working copy of X(0:s, :)
// lives in the workspace.
#include <algorithm>
#include <mutex>

#include <cooperative_groups.h>

#include "cluster.cuh"
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
  T* M;                // trailing-row multipliers M(r, q) at M[(r - trow0) * ldm + q]
  int64_t ldm;         // row stride of M (b when the panel kernel writes it)
  int64_t trow0;       // first trailing row the trailing update covers (t0 + b by default)
  int trows;           // trailing rows it covers (s - t0 - b by default)
  int epi_rows;        // rows t0+b .. whose multipliers the panel kernel's epilogue forms
  unsigned char sel_tag;    // sel value of columns this panel selects: panel index + 1
};

// Per-step exchange.  Every CTA sends every CTA of the cluster (itself included) its step-q
// candidate: a header {key, column index} and the candidate's column, rows q0 .. b-1 of the
// sending step's sub-block [q0, q1), in 16-byte groups.  The stores are st.async into the
// receiver's inbox buffer q % 3, each completing its byte count on the receiver's mbarrier of
// that buffer, so a sender never waits for its stores and a receiver waits only for its own
// barrier phase.  A sender without candidates still sends the full byte count (key -1, index
// INT_MAX).
constexpr int kMaxPanel = 64;
constexpr int kInbox = 3;
constexpr int kPanelKB = 8;    // sub-block of steps whose updates of the rows below are deferred
template <typename T>
struct __align__(16) CandCol {
  T col[kMaxPanel];
};
template <typename T>
struct __align__(16) CandHdr {
  T key;
  int idx;
};

template <typename T>
__host__ __device__ constexpr uint32_t hdr_bytes() { return sizeof(T) + 4; }
// bytes one sender delivers to one receiver when its sub-block starts at row q0s (a multiple
// of 4) in a b-row panel
template <typename T>
__host__ __device__ constexpr uint32_t push_bytes(int q0s, int b) {
  return hdr_bytes<T>() + (uint32_t)((b + 3) / 4 - q0s / 4) * 4u * (uint32_t)sizeof(T);
}
// sub-block start of the step that sends the candidates of step qn
__host__ __device__ constexpr int send_q0(int qn) { return qn == 0 ? 0 : (qn - 1) / kPanelKB * kPanelKB; }

// Pivot order: larger magnitude key, ties to the lower column index.
template <typename T>
__device__ __forceinline__ bool cand_better(T ka, int ia, T kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}

// Warp argmax in the pivot order with warp reductions: keys are >= 0 (magnitudes, +inf for
// non-finite entries) or -1 (no candidate), so their bit patterns order like the values.
__device__ __forceinline__ void warp_argmax(float& k, int& i) {
  const unsigned kbits = k >= 0.f ? __float_as_uint(k) : 0u;
  const unsigned m = __reduce_max_sync(0xffffffffu, kbits);
  const unsigned im = __reduce_min_sync(0xffffffffu, kbits == m ? (unsigned)i : 0x7fffffffu);
  i = (int)im;
  k = im == 0x7fffffffu ? -1.f : __uint_as_float(m);
}
__device__ __forceinline__ void warp_argmax(double& k, int& i) {
  const unsigned long long bits = k >= 0.0 ? (unsigned long long)__double_as_longlong(k) : 0ull;
  const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
  const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
  const unsigned im = __reduce_min_sync(0xffffffffu, hi == mh && lo == ml ? (unsigned)i : 0x7fffffffu);
  i = (int)im;
  k = im == 0x7fffffffu ? -1.0 : __longlong_as_double((long long)(((unsigned long long)mh << 32) | ml));
}

template <typename T> __device__ __forceinline__ uint32_t bits32(T v) { return __float_as_uint((float)v); }
template <typename T> __device__ __forceinline__ uint64_t bits64(T v) { return (uint64_t)__double_as_longlong((double)v); }

// Warp 0 sends this CTA's candidate (key k, index i, local column jb) for step qn = q+1 to
// every CTA of the cluster; step q lies in the sub-block [q0, q1).  Rows qn+1 .. q1-1 of
// column jb take step q's update here (multipliers lcol, R(q, jb) in row q of P) and are
// written back, so the owner thread skips the column; rows from q1 on are sent as they are
// (updated through step q0-1) and the receivers apply the sub-block's steps themselves.  When
// qn = q1 starts the next sub-block, the sub-block's deferred update of the column's rows
// q1+1 .. b-1 (resolved multipliers LkT) is applied here after the send, again in place of the
// owner.  Lane l covers rows 4(l%16) .. 4(l%16)+3 for the receivers of parity l/16.  For the
// first candidate (qn = 0) lcol is null.
template <typename T>
__device__ __forceinline__ void push_candidate(uint32_t col_base, uint32_t hdr_base, uint32_t bar_local,
                                               int crank, int CL, T* P, int ldp, int b, int qn, int q0,
                                               int q1, T k, int i, int jb, const T* lcol,
                                               const T (*LkT)[kPanelKB]) {
  const int lane = threadIdx.x & 31;
  const bool have = i != INT_MAX;
  const int f0 = 4 * (lane & 15);
  const bool active = f0 < b && f0 >= q0;          // groups q0/4 .. ceil(b/4)-1
  T v[4] = {T(0), T(0), T(0), T(0)};
  if (have && active) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (f0 + u < b) v[u] = P[(f0 + u) * ldp + jb];
    if (lcol) {
      const T rq = P[(qn - 1) * ldp + jb];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (f0 + u > qn && f0 + u < q1) v[u] = msub(v[u], lcol[f0 + u], rq);
    }
  }
  __syncwarp();                          // every lane has read column jb before it is rewritten
  if (have && active && lcol && lane < 16)
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (f0 + u > qn && f0 + u < q1) P[(f0 + u) * ldp + jb] = v[u];
  const uint32_t col_off = (uint32_t)(crank * sizeof(CandCol<T>) + f0 * sizeof(T));
  if (active)
    for (int d = lane >> 4; d < CL; d += 2) {
      const uint32_t dst = map_cluster_u32(col_base + col_off, d);
      const uint32_t bar = map_cluster_u32(bar_local, d);
      if constexpr (sizeof(T) == 4) {
        st_async_v4_b32(dst, bits32(v[0]), bits32(v[1]), bits32(v[2]), bits32(v[3]), bar);
      } else {
        st_async_v2_b64(dst, bits64(v[0]), bits64(v[1]), bar);
        st_async_v2_b64(dst + 16, bits64(v[2]), bits64(v[3]), bar);
      }
    }
  if (lane < CL) {
    const uint32_t dst = map_cluster_u32(hdr_base + (uint32_t)(crank * sizeof(CandHdr<T>)), lane);
    const uint32_t bar = map_cluster_u32(bar_local, lane);
    if constexpr (sizeof(T) == 4) st_async_b32(dst, bits32(k), bar);
    else st_async_b64(dst, bits64(k), bar);
    st_async_b32(dst + sizeof(T), (uint32_t)i, bar);
  }
  if (have && lcol && qn == q1 && q1 < b)
    for (int f = q1 + 1 + lane; f < b; f += 32) {
      T x = P[f * ldp + jb];
#pragma unroll
      for (int kk = 0; kk < kPanelKB; ++kk) x = msub(x, LkT[f][kk], P[(q0 + kk) * ldp + jb]);
      P[f * ldp + jb] = x;
    }
}

// Step q of the panel (one-step lookahead; no cluster barrier).  Steps are grouped in
// sub-blocks [q0, q1) of kPanelKB.  Rows inside the current sub-block are updated at every
// step; rows below it once per sub-block with all of its steps (each entry read once, updated
// kPanelKB times in step order, written once), which divides the shared memory traffic of the
// rank-1 updates by kPanelKB.  The multipliers of those deferred rows arrive as the pivot
// columns were stored (updated through step q0-1) and are completed once per sub-block:
//   L(f, k) = raw(f, k) - sum_{q0 <= k' < k} L(f, k') R(k', j_k),  k' in order,
// which is the tail of the textbook sequence for S^(k)(f, j_k).
//   wait    the mbarrier phase of inbox q % 3 (bounded), then a CTA barrier
//   select  every warp reduces the CL headers (same result everywhere); the winner's column
//           holds the multipliers of step q (at a sub-block's first step its rows still lack
//           the previous sub-block and are completed first)
//   row q   R(t, :) = P(q, :) / pivot over row q of P, the update of row q+1 (all steps of
//           the sub-block when row q+1 starts the next one), and this thread's step-(q+1)
//           candidates over row q+1, in one pass over its columns
//   push    CTA argmax (one CTA barrier); warp 0 sends the winner with its column
//   rest    the update of rows q+2 .. q1-1, or at the end of a sub-block the deferred update
//           of rows q1+1 .. b-1 (skipping the sent column), overlaps the exchange
// Inbox q % 3 is rewritten for step q+3 only after its sender has received step q+2 from
// this CTA, which this CTA sends after every warp is done with step q's multipliers.  The
// byte count of step q+3 is armed right after step q's phase completes.
template <typename T>
__global__ void __launch_bounds__(kPanelThreads, 1) lupp_panel_kernel(const PanelParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
  const int b = p.b, ncl = p.ncl;
  const int ldp = ncl + 1;            // odd row stride: a column read across rows is conflict-free
  const int c0 = crank * ncl;
  const int nl = (int)(p.n - c0 < 0 ? 0 : (p.n - c0 < ncl ? p.n - c0 : ncl));

  __shared__ CandCol<T> icol[kInbox][16];    // icol[step % 3][sender]
  __shared__ CandHdr<T> ihdr[kInbox][16];
  __shared__ __align__(8) uint64_t ibar[kInbox];
  __shared__ T wkey[2][32];
  __shared__ int widx[2][32];
  __shared__ int s_J[kMaxPanel];           // pivots of this panel, written out at the end
  __shared__ int s_timeout;
  __shared__ T Lk[2][kPanelKB][kMaxPanel];                 // deferred-row multipliers, step-major
  __shared__ __align__(16) T LkT[2][kMaxPanel][kPanelKB];  // completed ones, row-major
  __shared__ T Rsub[kPanelKB][kPanelKB];                   // Rsub[k][k'] = R(q0+k', j_{q0+k})
  __shared__ T lfix[kMaxPanel];                            // completed pivot column
  T* P = reinterpret_cast<T*>(smem);                        // [b][ldp]
  T* RJ = P + (size_t)b * ldp;                              // [b][b]: R(t0+qq, j_q)
  unsigned char* sl = reinterpret_cast<unsigned char*>(RJ + (size_t)b * b);   // [ncl]

  if (*(volatile int32_t*)p.fail) return;   // an earlier panel stopped (uniform over the cluster)
  if (tid == 0) {
    for (int k = 0; k < kInbox; ++k) mbar_init(smem_u32(&ibar[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_timeout = 0;
  }
  for (int q0 = 0; q0 < b; q0 += 8)         // eight independent loads in flight per thread
    for (int jj = tid; jj < nl; jj += bd) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (q0 + u < b) v[u] = p.Xg[(int64_t)(p.t0 + q0 + u) * p.n + c0 + jj];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (q0 + u < b) P[(q0 + u) * ldp + jj] = v[u];
    }
  for (int jj = tid; jj < nl; jj += bd) sl[jj] = p.sel[c0 + jj];
  const uint32_t col0 = smem_u32(&icol[0][0]), hdr0 = smem_u32(&ihdr[0][0]), bar0 = smem_u32(&ibar[0]);
  auto col_base = [&](int k) { return col0 + (uint32_t)(k * sizeof(icol[0])); };
  auto hdr_base = [&](int k) { return hdr0 + (uint32_t)(k * sizeof(ihdr[0])); };
  auto bar_base = [&](int k) { return bar0 + (uint32_t)(k * sizeof(uint64_t)); };
  __syncthreads();

  // CTA argmax of the per-thread candidates (key, idx) for step qn: one __syncthreads, after
  // which every warp holds the result.
  auto cta_argmax = [&](int qn, T& key, int& idx) {
    warp_argmax(key, idx);
    if (lane == 0) { wkey[qn & 1][warp] = key; widx[qn & 1][warp] = idx; }
    __syncthreads();
    key = lane < nw ? wkey[qn & 1][lane] : T(-1);
    idx = lane < nw ? widx[qn & 1][lane] : INT_MAX;
    warp_argmax(key, idx);
  };

  {
    T key = T(-1);
    int idx = INT_MAX;
    for (int jj = tid; jj < nl; jj += bd) {
      if (sl[jj]) continue;
      const T k = pivot_key(P[jj]);
      if (cand_better(k, c0 + jj, key, idx)) { key = k; idx = c0 + jj; }
    }
    cta_argmax(0, key, idx);
    if (tid == 0)
      for (int k = 0; k < kInbox && k < b; ++k)
        mbar_expect_tx(bar_base(k), (uint32_t)CL * push_bytes<T>(send_q0(k), b));
    cluster.sync();     // barriers initialised and armed everywhere before the first send
    if (warp == 0)
      push_candidate<T>(col_base(0), hdr_base(0), bar_base(0), crank, CL, P, ldp, b, 0, 0, 0, key, idx,
                        idx - c0, nullptr, LkT[0]);
  }

  bool stopped = false;
  int done = 0;                       // completed steps of this panel
  for (int q = 0; q < b; ++q) {
    const int t = p.t0 + q;
    const int buf = q % kInbox;
    if (!mbar_wait(bar_base(buf), (uint32_t)((q / kInbox) & 1), 2000000000ull))
      if (atomicExch(&s_timeout, 1) == 0) {
        record_error(p.dev_status, SKEL_ERR_TIMEOUT, t);
        atomicExch(p.fail, 1);            // later panels and trailing updates skip their work
      }
    __syncthreads();
    if (s_timeout) {                       // uniform in the CTA; the peers time out in turn
      stopped = true;
      break;
    }
    if (tid == bd - 1 && q + kInbox < b)
      mbar_expect_tx(bar_base(buf), (uint32_t)CL * push_bytes<T>(send_q0(q + kInbox), b));
    const int q0 = q - q % kPanelKB;
    const int q1 = q0 + kPanelKB < b ? q0 + kPanelKB : b;
    const int sb = (q / kPanelKB) & 1;
    int w, owner;
    {
      const int i0 = lane < CL ? ihdr[buf][lane].idx : INT_MAX;
      T k = lane < CL ? ihdr[buf][lane].key : T(-1);
      int i = i0;
      warp_argmax(k, i);
      w = i;
      owner = __ffs(__ballot_sync(0xffffffffu, i0 == w && w != INT_MAX)) - 1;
      owner = owner < 0 ? 0 : owner;
    }
    const T* lc = icol[buf][owner].col;          // pivot column as sent
    const T piv = w != INT_MAX ? lc[q] : T(0);
    const T pr = rdiv_prep(piv);
    const int code = w == INT_MAX ? SKEL_ERR_INVALID_ARG
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
    const T* lcol = lc;                          // multipliers of step q, rows q+1 ..
    if (q == q0 && q > 0) {                // rows below q still lack the previous sub-block
      const int p0 = q0 - kPanelKB;
      for (int f = q + 1 + tid; f < b; f += bd) {
        T x = lc[f];
#pragma unroll
        for (int kk = 0; kk < kPanelKB; ++kk) x = msub(x, Lk[sb ^ 1][kk][f], lc[p0 + kk]);
        lfix[f] = x;
      }
      __syncthreads();
      lcol = lfix;
    }
    if (tid == 0) s_J[q] = w;
    if (tid >= q1 && tid < b) Lk[sb][q - q0][tid] = lcol[tid];        // deferred rows, incomplete
    if (tid < q - q0) Rsub[q - q0][tid] = lc[q0 + tid];               // R(q0+tid, j_q)
    if (crank == 0 && p.L)
      for (int r = q + tid; r < q1; r += bd) p.L[(int64_t)(p.t0 + r) * p.ldl + t] = r == q ? piv : lcol[r];
    const bool more = q + 1 < b;
    const bool blk_end = more && q + 1 == q1;    // row q+1 starts the next sub-block
    if (blk_end) {                         // complete the deferred rows' multipliers, in order
      if (tid >= q1 && tid < b) {
        T xs[kPanelKB];
#pragma unroll
        for (int kk = 0; kk < kPanelKB; ++kk) {
          T x = Lk[sb][kk][tid];
#pragma unroll
          for (int k2 = 0; k2 < kk; ++k2)
            x = msub(x, xs[k2], kk == kPanelKB - 1 ? lc[q0 + k2] : Rsub[kk][k2]);
          xs[kk] = x;
        }
#pragma unroll
        for (int kk = 0; kk < kPanelKB; ++kk) {
          Lk[sb][kk][tid] = xs[kk];
          LkT[sb][tid][kk] = xs[kk];
        }
        if (crank == 0 && p.L)
#pragma unroll
          for (int kk = 0; kk < kPanelKB; ++kk) p.L[(int64_t)(p.t0 + tid) * p.ldl + p.t0 + q0 + kk] = xs[kk];
      }
      __syncthreads();
    }
    const int mine_w = owner == crank ? w - c0 : -1;
    const T lnext = more && !blk_end ? lcol[q + 1] : T(0);
    T key = T(-1);
    int idx = INT_MAX;
    // R(t, :) replaces row q of P (row q is final at step q) and goes to global memory; row q+1
    // is updated and scanned
    T* Rg = p.R + (int64_t)t * p.ldr + c0;
    for (int jj = tid; jj < nl; jj += bd) {
      T* pq = &P[q * ldp + jj];
      T rv;
      if (jj == mine_w) {
        rv = T(1);
        sl[jj] = p.sel_tag;
      } else if (sl[jj]) {
        rv = T(0);
      } else {
        rv = rdiv(*pq, pr);
        if (more) {
          T x = pq[ldp];
          if (!blk_end) {
            x = msub(x, lnext, rv);
          } else {                         // all steps of the sub-block for row q1
            const T* Lq1 = LkT[sb][q1];
#pragma unroll
            for (int kk = 0; kk < kPanelKB - 1; ++kk) x = msub(x, Lq1[kk], P[(q0 + kk) * ldp + jj]);
            x = msub(x, Lq1[kPanelKB - 1], rv);
          }
          pq[ldp] = x;
          const T kx = pivot_key(x);
          if (cand_better(kx, c0 + jj, key, idx)) { key = kx; idx = c0 + jj; }
        }
      }
      *pq = rv;
      Rg[jj] = rv;
    }
    int jb = -1;                          // the sent column: warp 0 updates it
    if (more) {
      cta_argmax(q + 1, key, idx);
      if (idx != INT_MAX) jb = idx - c0;
      if (warp == 0) {
        const int nb = (q + 1) % kInbox;
        push_candidate<T>(col_base(nb), hdr_base(nb), bar_base(nb), crank, CL, P, ldp, b, q + 1, q0, q1, key,
                          idx, jb, lcol, LkT[sb]);
      }
    }
    if (more && !blk_end) {                // rows q+2 .. q1-1: step q
      for (int jj = tid; jj < nl; jj += bd) {
        if (sl[jj] || jj == jb) continue;
        const T rv = P[q * ldp + jj];
        for (int r = q + 2; r < q1; ++r) {
          T* x = &P[r * ldp + jj];
          *x = msub(*x, lcol[r], rv);
        }
      }
    } else if (blk_end) {                  // rows q1+1 .. b-1: steps q0 .. q (a full sub-block)
      for (int jj = tid; jj < nl; jj += bd) {
        if (sl[jj] || jj == jb) continue;
        T rk[kPanelKB];
#pragma unroll
        for (int kk = 0; kk < kPanelKB; ++kk) rk[kk] = P[(q0 + kk) * ldp + jj];
        for (int r = q1 + 1; r < b; ++r) {
          T* x = &P[r * ldp + jj];
          T xv = *x;
#pragma unroll
          for (int kk = 0; kk < kPanelKB; ++kk) xv = msub(xv, LkT[sb][r][kk], rk[kk]);
          *x = xv;
        }
      }
    }
    done = q + 1;
  }
  __syncthreads();
  // write out the selected flags and pivots (the R rows went out at their steps)
  for (int jj = tid; jj < nl; jj += bd) p.sel[c0 + jj] = sl[jj];
  if (crank == 0)
    for (int q = tid; q < done; q += bd) p.Js[p.t0 + q] = s_J[q];
  // Multipliers of the trailing rows, M(r, q) = S^{(q)}(r, j_q): one warp per row, lane i
  // owns q = i and q = i + 32; after M(r, qq) is final it is broadcast and every later q
  // subtracts M(r, qq) R(t0+qq, j_q) -- the same operations in the same order as
  // step-by-step elimination.  R(panel, J_panel) is read from the owners' shared memory.
  cluster.sync();     // every CTA's R rows are final in its shared memory
  const bool trail = !stopped && done == b && p.epi_rows > 0;
  if (trail) {                         // eight distributed-shared-memory loads in flight per thread
    for (int e0 = tid; e0 < b * b; e0 += 8 * bd) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * bd;
        if (e < b * b) {
          const int qq = e / b, q = e % b;
          const int j = s_J[q];
          const int o = j / ncl;
          v[u] = cluster.map_shared_rank(P, o)[qq * ldp + (j - o * ncl)];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e0 + u * bd < b * b) RJ[e0 + u * bd] = v[u];
    }
  }
  cluster.sync();     // no CTA leaves or reuses its shared memory while others read it
  if (trail) {
    const int rows = p.epi_rows;
    for (int ri = crank * nw + warp; ri < rows; ri += CL * nw) {
      const int64_t r = p.t0 + b + ri;
      const int q0 = lane, q1 = lane + 32;
      T a0 = q0 < b ? p.Xg[r * p.n + s_J[q0]] : T(0);
      T a1 = q1 < b ? p.Xg[r * p.n + s_J[q1]] : T(0);
      for (int qq = 0; qq < b; ++qq) {
        const T mq = __shfl_sync(0xffffffffu, qq < 32 ? a0 : a1, qq & 31);   // final M(r, qq)
        if (q0 > qq && q0 < b) a0 = msub(a0, mq, RJ[qq * b + q0]);
        if (q1 > qq && q1 < b) a1 = msub(a1, mq, RJ[qq * b + q1]);
      }
      T* Mr = p.M + (int64_t)ri * p.ldm;
      if (q0 < b) Mr[q0] = a0;
      if (q1 < b) Mr[q1] = a1;
      if (p.L) {
        if (q0 < b) p.L[r * p.ldl + p.t0 + q0] = a0;
        if (q1 < b) p.L[r * p.ldl + p.t0 + q1] = a1;
      }
    }
  }
}

// Trailing update: rows t0+b .. s-1 of Xg.  A CTA covers kTrailRows rows x kTrailThreads
// columns; each thread owns one column and keeps its kTrailRows entries in registers, so the
// elimination chains of the rows are independent.  R(t0+q, j) is read from L2 once per q and
// applied to every row; the multipliers sit transposed in shared memory (a broadcast row per
// q).  Each entry sees the same operations in the same order as step-by-step elimination.
constexpr int kTrailRows = 16;
constexpr int kTrailThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kTrailThreads) lupp_trail_kernel(const PanelParams<T> p) {
  __shared__ __align__(16) T Mt[kMaxPanel][kTrailRows];   // Mt[q][u] = M(r0 + u, q)
  const int b = p.b;
  const int r0 = blockIdx.y * kTrailRows;                // index among the trailing rows
  const int rows = p.trows;
  const int nrows = rows - r0 < kTrailRows ? rows - r0 : kTrailRows;
  if (nrows <= 0) return;
  if (*(volatile int32_t*)p.fail) return;
  for (int e = threadIdx.x; e < b * kTrailRows; e += blockDim.x) {
    const int q = e / kTrailRows, u = e % kTrailRows;
    Mt[q][u] = u < nrows ? p.M[(int64_t)(r0 + u) * p.ldm + q] : T(0);
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.n) return;
  // columns selected by this or an earlier panel are updated too, as in the tiled kernel: their
  // trailing entries are never read again
  T* x = p.Xg + (p.trow0 + r0) * p.n + j;
  T v[kTrailRows];
#pragma unroll
  for (int u = 0; u < kTrailRows; ++u) v[u] = u < nrows ? x[(int64_t)u * p.n] : T(0);
  const T* Rj = p.R + (int64_t)p.t0 * p.ldr + j;
  for (int q0 = 0; q0 < b; q0 += 8) {          // R entries of 8 steps loaded together
    T rq[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) rq[e] = q0 + e < b ? Rj[(int64_t)(q0 + e) * p.ldr] : T(0);
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (q0 + e < b)
#pragma unroll
        for (int u = 0; u < kTrailRows; ++u) v[u] = msub(v[u], Mt[q0 + e][u], rq[e]);
  }
#pragma unroll
  for (int u = 0; u < kTrailRows; ++u)
    if (u < nrows) x[(int64_t)u * p.n] = v[u];
}

// The same trailing update as a register-blocked rank-b update: a CTA takes 64 trailing rows
// x 128 columns, stages M's rows (transposed, [q][row]) and R's panel rows ([q][column]) in
// shared memory, and each thread keeps an 8 x 4 block of Xg in registers: per step q two
// 16-byte loads of multipliers (a warp broadcast) and one of R feed 32 multiply-subtract pairs
// (about two instructions per entry and step, against three).  Every entry still sees
// x = msub(x, M(r, q), R(t0 + q, j)) for q = 0 .. b-1 in order, so the results equal the
// column kernel's bit for bit.  Columns selected by this or
// an earlier panel are updated too: from this panel on their R entries are 0 (earlier pivots)
// or belong to this panel's pivot columns, and those trailing entries are never read again.
constexpr int TT_R = 64, TT_C = 128, TT_THREADS = 256;

template <typename T>
size_t trail_tile_smem() { return sizeof(T) * (size_t)kMaxPanel * (TT_R + TT_C); }

template <typename T>
__device__ __forceinline__ void load4(const T* p, int64_t c, int64_t n, bool vec, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    if (vec && c + 3 < n) {
      const float4 q = *reinterpret_cast<const float4*>(p);
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      return;
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) v[u] = c + u < n ? p[u] : T(0);
}

template <typename T>
__device__ __forceinline__ void store4(T* p, int64_t c, int64_t n, bool vec, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    if (vec && c + 3 < n) {
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
      return;
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (c + u < n) p[u] = v[u];
}

template <typename T>
__global__ void __launch_bounds__(TT_THREADS) lupp_trail_tile_kernel(const PanelParams<T> p) {
  extern __shared__ __align__(16) unsigned char tsm[];
  T* Ms = reinterpret_cast<T*>(tsm);                   // [b][TT_R]: Ms[q][rr] = M(r0 + rr, q)
  T* Rs = Ms + (size_t)kMaxPanel * TT_R;               // [b][TT_C]: Rs[q][cc] = R(t0 + q, c0 + cc)
  const int b = p.b;
  const int r0 = blockIdx.y * TT_R;
  const int64_t c0 = (int64_t)blockIdx.x * TT_C;
  const int rows = p.trows;
  if (r0 >= rows) return;
  if (*(volatile int32_t*)p.fail) return;
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;    // rows ty*8 .. +7, columns tx*4 .. +3
  // the block of Xg is loaded first: its loads are in flight while M and R are staged
  const bool vec = (p.n & 3) == 0;
  const int64_t c = c0 + tx * 4;
  T v[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + ty * 8 + i;
    if (r < rows && c < p.n) load4<T>(p.Xg + (p.trow0 + r) * p.n + c, c, p.n, vec, v[i]);
    else {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[i][u] = T(0);
    }
  }
  for (int e = tid; e < b * TT_R; e += TT_THREADS) {
    const int rr = e / b, q = e % b;
    Ms[q * TT_R + rr] = r0 + rr < rows ? p.M[(int64_t)(r0 + rr) * p.ldm + q] : T(0);
  }
  for (int e = tid; e < b * TT_C; e += TT_THREADS) {
    const int q = e / TT_C, cc = e % TT_C;
    Rs[q * TT_C + cc] = c0 + cc < p.n ? p.R[(int64_t)(p.t0 + q) * p.ldr + c0 + cc] : T(0);
  }
  __syncthreads();
  for (int q = 0; q < b; ++q) {
    T m[8], rv[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) m[i] = Ms[q * TT_R + ty * 8 + i];
#pragma unroll
    for (int u = 0; u < 4; ++u) rv[u] = Rs[q * TT_C + tx * 4 + u];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int u = 0; u < 4; ++u) v[i][u] = msub(v[i][u], m[i], rv[u]);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + ty * 8 + i;
    if (r < rows && c < p.n) store4<T>(p.Xg + (p.trow0 + r) * p.n + c, c, p.n, vec, v[i]);
  }
}

// The trailing update of one panel (rows trow0 .. trow0+rows-1 of Xg): the tiled kernel.
template <typename T>
cudaError_t launch_trail(const PanelParams<T>& p, int rows, cudaStream_t st) {
  const int64_t gx = (p.n + TT_C - 1) / TT_C, gy = (rows + TT_R - 1) / TT_R;
  if (gx > (int64_t)INT32_MAX || gy > 65535) {       // beyond the tiled grid: the column kernel
    dim3 grid((unsigned)((p.n + kTrailThreads - 1) / kTrailThreads), (unsigned)((rows + kTrailRows - 1) / kTrailRows));
    KernelTimer kt("lupp_trail", st);
    lupp_trail_kernel<T><<<grid, kTrailThreads, 0, st>>>(p);
    note_launches(1);
    return cudaGetLastError();
  }
  const cudaError_t e = cudaFuncSetAttribute(lupp_trail_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)trail_tile_smem<T>());
  if (e != cudaSuccess) return e;
  KernelTimer kt("lupp_trail", st);
  lupp_trail_tile_kernel<T><<<dim3((unsigned)gx, (unsigned)gy), TT_THREADS, trail_tile_smem<T>(), st>>>(p);
  note_launches(1);
  return cudaGetLastError();
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

// ---------------------------------------------------------------------------------------
// Row chain of the pipelined skeleton pivoting (row LUPP on C^T, C = A(:, Js), run panel by
// panel behind the column LUPP that produces Js).  The row panel [t0, t0+b) is factored as
// soon as its rows exist; the trailing updates that the earlier row panels would have
// applied to these rows are applied then, entry by entry in the same order (panel by panel,
// step by step), and the multipliers are formed by the same forward substitutions as the
// panel kernel's epilogue, so the pivots equal those of the unpipelined factorisation bit
// for bit.
// ---------------------------------------------------------------------------------------

// Rows t0 .. t0+b-1 of the working copy: row r is column Js[r] of A.  A missing pivot (the
// column chain stopped) sets the row chain's fail word instead.
template <typename T>
__global__ void lupp_gather_panel_kernel(const T* A, int64_t lda, int64_t m, int64_t ncols, const int32_t* Js,
                                         int t0, int b, T* Xg, int32_t* fail) {
  for (int r = blockIdx.y; r < b; r += gridDim.y) {
    const int32_t j = Js[t0 + r];
    if (j < 0 || (int64_t)j >= ncols) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(fail, 1);
      continue;
    }
    const T* a = A + (int64_t)j * lda;
    T* x = Xg + (int64_t)(t0 + r) * m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
      x[i] = a[i];
  }
}

// Multipliers M(r, t), t < t0, of the rows r = t0 .. t0+b-1 (earlier panels of height B):
// for each earlier panel q, the entries X(r, J_q) after the updates of the panels before q,
// then forward substitution with R(panel q, J_q).  One warp per row; lane i holds the steps
// i and i + 32 of panel q.  M(r, t) goes to Lw[r * ldw + t].
template <typename T>
__global__ void lupp_defer_m_kernel(const PanelParams<T> p, int B, T* Lw, int64_t ldw) {
  const int lane = threadIdx.x & 31;
  const int ri = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (ri >= p.b) return;
  if (*(volatile int32_t*)p.fail) return;
  const int64_t r = p.t0 + ri;
  T* Mr = Lw + r * ldw;
  const T* xr = p.Xg + r * p.n;
  for (int tq = 0; tq < p.t0; tq += B) {
    const int q0 = lane, q1 = lane + 32;
    const bool h0 = q0 < B, h1 = q1 < B;
    const int j0 = h0 ? p.Js[tq + q0] : 0, j1 = h1 ? p.Js[tq + q1] : 0;
    T a0 = h0 ? xr[j0] : T(0);
    T a1 = h1 ? xr[j1] : T(0);
    for (int t = 0; t < tq; t += 8) {      // the updates of the panels before q, in order
      T r0[8], r1[8], mt[8];               // (B need not be a multiple of 8: steps >= tq are skipped)
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool ok = t + u < tq;
        const int64_t row = (int64_t)(t + u) * p.ldr;
        mt[u] = ok ? Mr[t + u] : T(0);
        r0[u] = ok && h0 ? p.R[row + j0] : T(0);
        r1[u] = ok && h1 ? p.R[row + j1] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (t + u < tq) {
          a0 = msub(a0, mt[u], r0[u]);
          a1 = msub(a1, mt[u], r1[u]);
        }
    }
    for (int c0 = 0; c0 < B; c0 += 8) {    // forward substitution with R(panel q, J_q)
      T r0[8], r1[8];                       // this lane's R entries of 8 steps, loaded together
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int qq = c0 + u;
        const int64_t row = (int64_t)(tq + qq) * p.ldr;
        r0[u] = qq < B && q0 > qq && h0 ? p.R[row + j0] : T(0);
        r1[u] = qq < B && q1 > qq && h1 ? p.R[row + j1] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int qq = c0 + u;
        if (qq < B) {                       // uniform over the warp
          const T mq = __shfl_sync(0xffffffffu, qq < 32 ? a0 : a1, qq & 31);
          if (q0 > qq && h0) a0 = msub(a0, mq, r0[u]);
          if (q1 > qq && h1) a1 = msub(a1, mq, r1[u]);
        }
      }
    }
    if (h0) Mr[tq + q0] = a0;
    if (h1) Mr[tq + q1] = a1;
    __syncwarp();
  }
}

// The earlier panels' trailing updates of rows t0 .. t0+b-1: panel q (steps tq .. tq+B-1)
// subtracts M(r, tq+qq) R(tq+qq, j) for qq in order, skipping the columns selected by panel q
// or earlier (sel tag <= q + 1), exactly as the trailing update after panel q would have.
template <typename T>
__global__ void __launch_bounds__(kTrailThreads) lupp_defer_trail_kernel(const PanelParams<T> p, int B,
                                                                         const T* Lw, int64_t ldw) {
  __shared__ __align__(16) T Mt[kMaxPanel][kTrailRows];
  const int r0 = blockIdx.y * kTrailRows;
  const int nrows = p.b - r0 < kTrailRows ? p.b - r0 : kTrailRows;
  if (nrows <= 0) return;
  if (*(volatile int32_t*)p.fail) return;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = j < p.n;
  const int sj = live ? p.sel[j] : 0;
  const int npan = p.t0 / B;
  const int napply = sj == 0 ? npan : (sj - 1 < npan ? sj - 1 : npan);   // panels q < sel tag - 1
  T* x = p.Xg + (int64_t)(p.t0 + r0) * p.n + j;
  T v[kTrailRows];
#pragma unroll
  for (int u = 0; u < kTrailRows; ++u) v[u] = live && u < nrows ? x[(int64_t)u * p.n] : T(0);
  for (int q = 0; q < npan; ++q) {
    __syncthreads();
    for (int e = threadIdx.x; e < B * kTrailRows; e += blockDim.x) {
      const int qq = e / kTrailRows, u = e % kTrailRows;
      Mt[qq][u] = u < nrows ? Lw[(int64_t)(p.t0 + r0 + u) * ldw + (int64_t)q * B + qq] : T(0);
    }
    __syncthreads();
    if (!live || q >= napply) continue;
    const T* Rj = p.R + (int64_t)q * B * p.ldr + j;
    for (int q0 = 0; q0 < B; q0 += 8) {        // R entries of 8 steps loaded together
      T rq[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) rq[e] = q0 + e < B ? Rj[(int64_t)(q0 + e) * p.ldr] : T(0);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (q0 + e < B)
#pragma unroll
          for (int u = 0; u < kTrailRows; ++u) v[u] = msub(v[u], Mt[q0 + e][u], rq[e]);
    }
  }
  if (live)
#pragma unroll
    for (int u = 0; u < kTrailRows; ++u)
      if (u < nrows) x[(int64_t)u * p.n] = v[u];
}

template <typename T>
__global__ void lupp_row_init_kernel(int64_t n, int s, unsigned char* sel, int32_t* fail, int32_t* Is) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    sel[j] = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s; t += gridDim.x * blockDim.x) Is[t] = -1;
  if (blockIdx.x == 0 && threadIdx.x == 0) *fail = 0;
}

// ---------------------------------------------------------------------------------------
// Grid-wide panels, for matrices too wide for a cluster panel (e.g. the row LUPP on a tall
// C^T with 262144 columns): a persistent grid of G CTAs (all co-resident, cooperative launch),
// CTA g holding columns [g nloc, (g+1) nloc) of the panel's b rows in shared memory.  Per step
// every CTA publishes its best candidate (index, value, and its column below the step) to a
// slot in global memory, arrives at the grid barrier and, after it, all CTAs take the same
// winner (the largest magnitude, ties to the lower index: an atomicMax on a packed key for
// FP32, a scan of the slots for FP64); R(t, :) is written and rows q+1 .. b-1 updated, row q+1
// first so that the next candidate is published before the rest of the update.  The trailing
// rows then get their multipliers (lupp_gmult_kernel: forward substitution with the panel's
// R(panel, J_panel), warp per row) and the tiled trailing update; every entry sees the textbook
// operations in the textbook order, as in the cluster path.
struct GPanelParams {
  int64_t n;
  int s, t0, b, nloc;
  unsigned char* sel;     // n flags (global): columns selected by earlier panels
  unsigned char tag;      // flag value of this panel's pivot columns
  int32_t* Js;
  int32_t* fail;
  int32_t* dev_status;
  GridComm gc;
};

template <typename T>
size_t gpanel_smem(int b, int nloc) {
  auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  return a16(sizeof(T) * (size_t)b * nloc) + a16(sizeof(T) * kMaxPanel) + a16(sizeof(T) * (size_t)nloc) + a16(nloc);
}

template <typename T>
__device__ __forceinline__ KeyIdx<T> gp_best(const T* W, int nloc, int row, int nl, int64_t c0,
                                             const unsigned char* sl) {
  T key = T(-1);
  int64_t idx = INT64_MAX;
  for (int jj = threadIdx.x; jj < nl; jj += blockDim.x) {
    if (sl[jj]) continue;
    const T k = pivot_key(W[(int64_t)row * nloc + jj]);
    if (better(k, c0 + jj, key, idx)) { key = k; idx = c0 + jj; }
  }
  return block_argmax<T>(key, idx);
}

// Slot layout: int64 index (-1: no candidate), T value, then the column rows 0 .. b-1.
template <typename T>
__device__ __forceinline__ void gp_publish(const GridComm& gc, int q, const KeyIdx<T>& c, const T* W, int nloc,
                                           int64_t c0, int b) {
  char* sl = gc.slot(q, blockIdx.x);
  T* col = reinterpret_cast<T*>(sl + 16);
  const bool have = c.idx != INT64_MAX && c.key >= T(0);
  const int jb = have ? (int)(c.idx - c0) : 0;
  if (have)
    for (int r = q + threadIdx.x; r < b; r += blockDim.x) col[r] = W[(int64_t)r * nloc + jb];
  if (threadIdx.x == 0) {
    *reinterpret_cast<long long*>(sl) = have ? (long long)c.idx : -1ll;
    *reinterpret_cast<T*>(sl + 8) = have ? W[(int64_t)q * nloc + jb] : T(0);
    if constexpr (sizeof(T) == 4)
      if (have) atomicMax(gc.keys + q, pack_key((float)c.key, c.idx));
  }
}

template <typename T>
__device__ __forceinline__ int64_t gp_winner(const GridComm& gc, int q) {
  if constexpr (sizeof(T) == 4) {
    __shared__ long long s_w;
    if (threadIdx.x == 0) {
      const unsigned long long k = __ldcg(gc.keys + q);
      s_w = k == 0ull ? -1 : key_index(k);
    }
    __syncthreads();
    const long long w = s_w;
    __syncthreads();
    return w;
  } else {
    T key = T(-1);
    int64_t idx = INT64_MAX;
    for (int g = threadIdx.x; g < gc.G; g += blockDim.x) {
      const char* sl = gc.slot(q, g);
      const long long ci = __ldcg(reinterpret_cast<const long long*>(sl));
      if (ci >= 0) {
        const T kq = pivot_key(__ldcg(reinterpret_cast<const T*>(sl + 8)));
        if (better(kq, (int64_t)ci, key, idx)) { key = kq; idx = ci; }
      }
    }
    const KeyIdx<T> r = block_argmax<T>(key, idx);
    return r.idx == INT64_MAX ? -1 : r.idx;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) lupp_gpanel_kernel(const GPanelParams p, T* Xg, T* R, int64_t ldr, T* L,
                                                          int64_t ldl) {
  extern __shared__ __align__(16) unsigned char gsm[];
  if (*(volatile const int32_t*)p.fail) return;        // an earlier panel stopped: uniform over the grid
  const int b = p.b, nloc = p.nloc, tid = threadIdx.x, bd = blockDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * nloc;
  const int nl = (int)(p.n - c0 < 0 ? 0 : (p.n - c0 < nloc ? p.n - c0 : nloc));
  auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  T* W = reinterpret_cast<T*>(gsm);
  T* pivcol = reinterpret_cast<T*>(gsm + a16(sizeof(T) * (size_t)b * nloc));
  T* rowt = pivcol + kMaxPanel;
  unsigned char* sl = reinterpret_cast<unsigned char*>(rowt) + a16(sizeof(T) * (size_t)nloc);
  for (int q = 0; q < b; ++q)
    for (int jj = tid; jj < nl; jj += bd) W[(int64_t)q * nloc + jj] = Xg[(int64_t)(p.t0 + q) * p.n + c0 + jj];
  for (int jj = tid; jj < nloc; jj += bd) sl[jj] = jj < nl ? p.sel[c0 + jj] : (unsigned char)1;
  __syncthreads();
  auto stop = [&](int t, int code) {
    if (blockIdx.x == 0 && tid == 0) {
      record_error(p.dev_status, code, t);
      atomicExch(p.fail, 1);
    }
    if (blockIdx.x == 0)
      for (int r = t + tid; r < p.s; r += bd) p.Js[r] = -1;
    if (tid == 0) atomicExch(p.gc.abort, 1);
  };
  gp_publish<T>(p.gc, 0, gp_best<T>(W, nloc, 0, nl, c0, sl), W, nloc, c0, b);
  comm_arrive(p.gc, 0);
  for (int q = 0; q < b; ++q) {
    const int t = p.t0 + q;
    if (!comm_wait(p.gc, q, p.dev_status)) {
      if (blockIdx.x == 0 && tid == 0) atomicExch(p.fail, 1);
      return;
    }
    const int64_t w = gp_winner<T>(p.gc, q);
    if (w < 0) { stop(t, SKEL_ERR_RANK_DEFICIENT); return; }
    const char* wsl = p.gc.slot(q, (int)(w / nloc));
    const T piv = __ldcg(reinterpret_cast<const T*>(wsl + 8));
    if (!isfinite(piv)) { stop(t, SKEL_ERR_NONFINITE); return; }
    if (piv == T(0)) { stop(t, SKEL_ERR_RANK_DEFICIENT); return; }
    const T pr = rdiv_prep(piv);
    const T* wcol = reinterpret_cast<const T*>(wsl + 16);
    for (int r = q + tid; r < b; r += bd) pivcol[r] = __ldcg(wcol + r);
    if (blockIdx.x == 0 && tid == 0) p.Js[t] = (int32_t)w;
    const int jw = (w >= c0 && w < c0 + nl) ? (int)(w - c0) : -1;
    for (int jj = tid; jj < nl; jj += bd) {          // R(t, :): row q is final at step q
      T rv;
      if (jj == jw) rv = T(1);
      else if (sl[jj]) rv = T(0);
      else rv = rdiv(W[(int64_t)q * nloc + jj], pr);
      rowt[jj] = rv;
      R[(int64_t)t * ldr + c0 + jj] = rv;
    }
    __syncthreads();
    if (blockIdx.x == 0 && L)
      for (int r = q + tid; r < b; r += bd) L[(int64_t)(p.t0 + r) * ldl + t] = pivcol[r];
    if (jw >= 0 && tid == 0) sl[jw] = p.tag;
    __syncthreads();
    if (q + 1 == b) break;
    const int r1 = q + 1;                            // row q+1 first, then the next candidate
    for (int jj = tid; jj < nl; jj += bd) {
      if (sl[jj]) continue;
      T* x = &W[(int64_t)r1 * nloc + jj];
      *x = msub(*x, pivcol[r1], rowt[jj]);
    }
    __syncthreads();
    const KeyIdx<T> c = gp_best<T>(W, nloc, r1, nl, c0, sl);
    int jb = -1;
    if (c.idx != INT64_MAX && c.key >= T(0)) {
      jb = (int)(c.idx - c0);
      for (int r = q + 2 + tid; r < b; r += bd) {
        T* x = &W[(int64_t)r * nloc + jb];
        *x = msub(*x, pivcol[r], rowt[jb]);
      }
      __syncthreads();
    }
    gp_publish<T>(p.gc, r1, c, W, nloc, c0, b);
    comm_arrive(p.gc, r1);
    for (int jj = tid; jj < nl; jj += bd) {          // rows q+2 .. b-1, overlapping the barrier
      if (sl[jj] || jj == jb) continue;
      const T rv = rowt[jj];
      for (int r = q + 2; r < b; ++r) {
        T* x = &W[(int64_t)r * nloc + jj];
        *x = msub(*x, pivcol[r], rv);
      }
    }
    __syncthreads();
  }
  for (int jj = tid; jj < nl; jj += bd) p.sel[c0 + jj] = sl[jj];
}

// Multipliers of the rows r = r0 .. r1-1 (below a finished panel) for the panel's steps, one
// warp per row: M(r, q) = S^(q)(r, j_q) = X(r, j_q) - sum_{q' < q} M(r, q') R(t0 + q', j_q),
// the subtractions in q' order (lane i owns q = i and i + 32; M(r, q') is broadcast when
// final).  M(r, q) goes to M[(r - r0) * ldm + q] and, when L is given, to L(r, t0 + q).
template <typename T>
__global__ void __launch_bounds__(256) lupp_gmult_kernel(const T* Xg, int64_t n, int64_t r0, int64_t r1, int t0, int b,
                                                         const T* R, int64_t ldr, const int32_t* Js, T* M,
                                                         int64_t ldm, T* L, int64_t ldl, const int32_t* fail) {
  __shared__ T RJ[kMaxPanel][kMaxPanel + 1];           // RJ[qq][q] = R(t0 + qq, j_q)
  __shared__ int jq[kMaxPanel];
  if (*(volatile const int32_t*)fail) return;
  for (int q = threadIdx.x; q < b; q += blockDim.x) jq[q] = Js[t0 + q];
  __syncthreads();
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int qq = e / b, q = e % b;
    RJ[qq][q] = R[(int64_t)(t0 + qq) * ldr + jq[q]];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t r = r0 + (int64_t)blockIdx.x * nw + warp; r < r1; r += (int64_t)gridDim.x * nw) {
    const int qa = lane, qb = lane + 32;
    T xa = qa < b ? Xg[r * n + jq[qa]] : T(0);
    T xb = qb < b ? Xg[r * n + jq[qb]] : T(0);
    for (int qq = 0; qq < b; ++qq) {
      const T m = __shfl_sync(0xffffffffu, qq < 32 ? xa : xb, qq & 31);
      if (lane == 0) {
        M[(r - r0) * ldm + qq] = m;
        if (L) L[r * ldl + t0 + qq] = m;
      }
      if (qa > qq && qa < b) xa = msub(xa, m, RJ[qq][qa]);
      if (qb > qq && qb < b) xb = msub(xb, m, RJ[qq][qb]);
    }
  }
}

struct PanelPlan {
  int CL = 0, b = 0, ncl = 0;
  size_t smem = 0, ws = 0;
};

template <typename T>
size_t panel_smem(int b, int ncl) {
  // P (b x (ncl+1)), R(panel, J_panel) (b x b), selected flags (ncl bytes)
  return sizeof(T) * ((size_t)b * (ncl + 1) + (size_t)b * b) + ncl + 64;
}

// Largest cluster the device accepts for the panel kernel (16 non-portable, else 8), and the
// panel height b for it.  b == 0 means "use the grid-barrier kernel".
template <typename T>
PanelPlan plan_panel(int64_t n, int s) {
  PanelPlan pl;
  if (n >= (int64_t)1 << 30) return pl;   // column indices are 32-bit inside the panel kernel
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
         align_up(sizeof(T) * (size_t)kMaxPanel * kMaxPanel) + (need_r ? align_up(sizeof(T) * (size_t)s * n) : 0);
}

// Streams of the look-ahead schedule (one set per context and device, context_cache.h; used
// under its mutex while a call enqueues): `hi` (highest priority) carries the panels and the
// updates of the next panel's rows, `lo` (lowest priority) the bulk trailing updates.
struct LookaheadSet {
  cudaStream_t hi = nullptr, lo = nullptr;
  cudaEvent_t fork = nullptr, join_hi = nullptr, join_lo = nullptr, panel_done = nullptr, bulk_done = nullptr;
};

std::mutex& lookahead_mutex() {
  static std::mutex mu;
  return mu;
}

LookaheadSet* lookahead_set() {
  static ContextCache<LookaheadSet> sets;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  return sets.get(current_context_id(), dev, [](LookaheadSet& a) {
    int least = 0, greatest = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
              cudaStreamCreateWithPriority(&a.hi, cudaStreamNonBlocking, greatest) == cudaSuccess &&
              cudaStreamCreateWithPriority(&a.lo, cudaStreamNonBlocking, least) == cudaSuccess;
    for (cudaEvent_t* e : {&a.fork, &a.join_hi, &a.join_lo, &a.panel_done, &a.bulk_done})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
  });
}

// Joins both look-ahead streams back into the caller's stream on every return path.
struct LookaheadJoin {
  cudaStream_t st;
  LookaheadSet* la;
  ~LookaheadJoin() {
    if (cudaEventRecord(la->join_hi, la->hi) == cudaSuccess) cudaStreamWaitEvent(st, la->join_hi, 0);
    if (cudaEventRecord(la->join_lo, la->lo) == cudaSuccess) cudaStreamWaitEvent(st, la->join_lo, 0);
  }
};

template <typename T>
cudaError_t launch_panel(const PanelParams<T>& p, const PanelPlan& pl, cudaStream_t st);

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
  T* Mnext = reinterpret_cast<T*>(base);             // multipliers of the next panel's rows
  base += align_up(sizeof(T) * (size_t)kMaxPanel * kMaxPanel);
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
  // Look-ahead schedule.  Panel k (rows [t_k, t_k + b)) needs its rows updated by every
  // earlier panel.  After panel k: on `hi`, the multipliers and the update of panel k+1's rows
  // only (then panel k+1 starts); on `lo`, concurrently with panel k+1, the multipliers and
  // the update of rows t_{k+2} .. s-1 (the bulk).  Panel k+1's look-ahead waits for the bulk
  // of panel k, which holds panel k's update of panel k+2's rows.  Every entry still receives
  // the panels' updates in panel order and, within a panel, step by step with separately
  // rounded multiply and subtract, so the factors equal the sequential schedule's bit for bit.
  std::lock_guard<std::mutex> lock(lookahead_mutex());
  LookaheadSet* la = lookahead_set();
  if (la == nullptr) return SKEL_ERR_CUDA;
  if (cudaEventRecord(la->fork, st) != cudaSuccess || cudaStreamWaitEvent(la->hi, la->fork, 0) != cudaSuccess ||
      cudaStreamWaitEvent(la->lo, la->fork, 0) != cudaSuccess)
    return SKEL_ERR_CUDA;
  LookaheadJoin joiner{st, la};
  auto rows_update = [&](const PanelParams<T>& pp, int64_t r0, int64_t r1, T* Mb, cudaStream_t cs) -> cudaError_t {
    {
      KernelTimer kt("lupp_mult", cs);
      lupp_gmult_kernel<T><<<(unsigned)std::min<int64_t>((r1 - r0 + 7) / 8, 1024), 256, 0, cs>>>(
          pp.Xg, pp.n, r0, r1, pp.t0, pp.b, pp.R, pp.ldr, pp.Js, Mb, pp.b, pp.L, pp.ldl, pp.fail);
    }
    note_launches(1);
    PanelParams<T> q = pp;
    q.M = Mb;
    q.ldm = pp.b;
    q.trow0 = r0;
    q.trows = (int)(r1 - r0);
    return launch_trail<T>(q, q.trows, cs);
  };
  for (int t0 = 0, k = 0; t0 < s; t0 += pl.b, ++k) {
    p.t0 = t0;
    p.b = std::min(pl.b, s - t0);
    p.sel_tag = (unsigned char)(1 + k % 255);   // never 0: 0 marks an unselected column
    p.ldm = p.b;
    p.trow0 = t0 + p.b;
    p.trows = 0;
    p.epi_rows = 0;
    if (launch_panel<T>(p, pl, la->hi) != cudaSuccess) return SKEL_ERR_CUDA;
    const int t1 = t0 + p.b;
    if (t1 >= s) break;
    const int t2 = t1 + std::min(pl.b, s - t1);
    if (t2 < s) {                          // the bulk of panel k
      if (cudaEventRecord(la->panel_done, la->hi) != cudaSuccess ||
          cudaStreamWaitEvent(la->lo, la->panel_done, 0) != cudaSuccess)
        return SKEL_ERR_CUDA;
      if (rows_update(p, t2, s, p.M, la->lo) != cudaSuccess) return SKEL_ERR_CUDA;
    }
    // panel k+1's rows: they hold panel k-1's update once the bulk of panel k-1 is done
    if (k > 0 && cudaStreamWaitEvent(la->hi, la->bulk_done, 0) != cudaSuccess) return SKEL_ERR_CUDA;
    if (rows_update(p, t1, t2, Mnext, la->hi) != cudaSuccess) return SKEL_ERR_CUDA;
    if (t2 < s && cudaEventRecord(la->bulk_done, la->lo) != cudaSuccess) return SKEL_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}


template <typename T>
cudaError_t launch_panel(const PanelParams<T>& p, const PanelPlan& pl, cudaStream_t st) {
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
  cudaError_t e;
  {
    KernelTimer kt("lupp_panel", st);
    e = cudaLaunchKernelEx(&cfg, lupp_panel_kernel<T>, p);
  }
  note_launches(1);
  return e;
}

// Column LUPP on X (Js, optional L, R) and row LUPP on C^T (Is), the row chain on an
// auxiliary stream: row panel [t0, t0+b) starts when the column panel holding step t0+b-1
// has finished (an event) and the previous row panel is done (stream order).  wsc: the
// column chain's panel workspace; wsr: the row chain's (working copy of C^T, sel, fail, R);
// Lw: s x s multipliers of the row chain.
template <typename T>
skel_status run_skeleton_t(const PanelPlan& pc, const PanelPlan& pr, const T* X, int64_t n, int64_t ldx, int s,
                           const T* A, int64_t m, int64_t lda, int32_t* Js, int32_t* Is, T* L, int64_t ldl, T* R,
                           int64_t ldr, void* wsc, void* wsr, T* Lw, int32_t* dev_status, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(aux_mutex());
  AuxSet* aux = aux_set();
  if (aux == nullptr) return SKEL_ERR_CUDA;
  // column chain parameters (as run_panel_t)
  char* base = static_cast<char*>(wsc);
  PanelParams<T> c{};
  c.Xg = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)s * n);
  c.sel = reinterpret_cast<unsigned char*>(base);
  base += align_up(n);
  c.fail = reinterpret_cast<int32_t*>(base);
  base += 256;
  c.M = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)s * 64);
  if (R == nullptr) {
    R = reinterpret_cast<T*>(base);
    ldr = n;
  }
  c.n = n; c.s = s; c.ncl = pc.ncl; c.Js = Js; c.R = R; c.ldr = ldr; c.L = L; c.ldl = ldl;
  c.dev_status = dev_status;
  // row chain parameters
  base = static_cast<char*>(wsr);
  PanelParams<T> r{};
  r.Xg = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)s * m);
  r.sel = reinterpret_cast<unsigned char*>(base);
  base += align_up(m);
  r.fail = reinterpret_cast<int32_t*>(base);
  base += 256;
  r.R = reinterpret_cast<T*>(base);
  r.ldr = m;
  r.n = m; r.ncl = pr.ncl; r.Js = Is; r.L = nullptr; r.ldl = 0; r.M = nullptr;
  r.dev_status = dev_status;

  const size_t smem = std::max(pc.smem, pr.smem);
  if (cudaFuncSetAttribute(lupp_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SKEL_ERR_CUDA;
  if (std::max(pc.CL, pr.CL) > 8 &&
      cudaFuncSetAttribute(lupp_panel_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return SKEL_ERR_CUDA;

  lupp_panel_init_kernel<T><<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min(s, 64)), 256, 0, st>>>(
      X, ldx, s, n, c.Xg, c.sel, c.fail, L, ldl);
  lupp_row_init_kernel<T><<<(unsigned)std::min<int64_t>((m + 255) / 256, 64), 256, 0, st>>>(m, s, r.sel, r.fail, Is);
  note_launches(2);
  if (cudaEventRecord(aux->fork, st) != cudaSuccess) return SKEL_ERR_CUDA;
  // column chain on the caller's stream
  int k = 0;
  for (int t0 = 0; t0 < s; t0 += pc.b, ++k) {
    c.t0 = t0;
    c.b = std::min(pc.b, s - t0);
    c.sel_tag = (unsigned char)(1 + k % 255);   // never 0: 0 marks an unselected column
    c.ldm = c.b;
    c.trow0 = t0 + c.b;
    c.trows = s - t0 - c.b;
    c.epi_rows = c.trows;
    if (launch_panel<T>(c, pc, st) != cudaSuccess) return SKEL_ERR_CUDA;
    if (cudaEventRecord(aux->col[k], st) != cudaSuccess) return SKEL_ERR_CUDA;
    if (c.trows > 0 && launch_trail<T>(c, c.trows, st) != cudaSuccess) return SKEL_ERR_CUDA;
  }
  // row chain on the auxiliary stream
  if (cudaStreamWaitEvent(aux->st, aux->fork, 0) != cudaSuccess) return SKEL_ERR_CUDA;
  AuxJoin joiner{st, aux};              // joins on every return path below
  k = 0;
  for (int t0 = 0; t0 < s; t0 += pr.b, ++k) {
    r.t0 = t0;
    r.b = std::min(pr.b, s - t0);
    r.s = t0 + r.b;                       // no rows below: the epilogue forms no multipliers
    r.epi_rows = 0;
    r.sel_tag = (unsigned char)(1 + k % 255);   // never 0: 0 marks an unselected column
    if (cudaStreamWaitEvent(aux->st, aux->col[(t0 + r.b - 1) / pc.b], 0) != cudaSuccess) return SKEL_ERR_CUDA;
    lupp_gather_panel_kernel<T><<<dim3((unsigned)std::min<int64_t>((m + 255) / 256, 32), (unsigned)r.b), 256, 0, aux->st>>>(
        A, lda, m, n, Js, t0, r.b, r.Xg, r.fail);
    note_launches(1);
    if (t0 > 0) {
      lupp_defer_m_kernel<T><<<(unsigned)((r.b + 7) / 8), 256, 0, aux->st>>>(r, pr.b, Lw, s);
      dim3 grid((unsigned)((m + kTrailThreads - 1) / kTrailThreads), (unsigned)((r.b + kTrailRows - 1) / kTrailRows));
      {
        KernelTimer kt("lupp_trail", aux->st);
        lupp_defer_trail_kernel<T><<<grid, kTrailThreads, 0, aux->st>>>(r, pr.b, Lw, s);
      }
      note_launches(2);
    }
    if (launch_panel<T>(r, pr, aux->st) != cudaSuccess) return SKEL_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

}  // namespace

size_t skeleton_pivot_workspace(skel_dtype dt, int64_t n, int64_t m, int32_t s) {
  const size_t es = dt == SKEL_F64 ? 8 : 4;
  const size_t col = dt == SKEL_F64 ? panel_ws<double>(n, s, true) : panel_ws<float>(n, s, true);
  const size_t row = align_up(es * (size_t)s * m) + align_up(m) + 256 + align_up(es * (size_t)s * m);
  return col + row + align_up(es * (size_t)s * s);
}

std::mutex& aux_mutex() {
  static std::mutex mu;
  return mu;
}

AuxSet* aux_set() {
  static ContextCache<AuxSet> sets;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  return sets.get(current_context_id(), dev, [](AuxSet& a) {
    bool ok = cudaStreamCreateWithFlags(&a.st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < kAuxEvents; ++k)
      ok = cudaEventCreateWithFlags(&a.col[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
  });
}

bool skeleton_pivot_pipelined(skel_dtype dt, int64_t n, int64_t m, int32_t s) {
  if (dt == SKEL_F64) {
    const PanelPlan pc = plan_panel<double>(n, s), pr = plan_panel<double>(m, s);
    return pc.b > 0 && pr.b > 0 && (s + std::min(pc.b, pr.b) - 1) / std::min(pc.b, pr.b) <= kAuxEvents;
  }
  const PanelPlan pc = plan_panel<float>(n, s), pr = plan_panel<float>(m, s);
  return pc.b > 0 && pr.b > 0 && (s + std::min(pc.b, pr.b) - 1) / std::min(pc.b, pr.b) <= kAuxEvents;
}

skel_status run_skeleton_pivot(skel_dtype dt, const void* X, int64_t n, int64_t ldx, int32_t s, const void* A,
                               int64_t m, int64_t lda, int32_t* Js, int32_t* Is, void* L, int64_t ldl, void* R,
                               int64_t ldr, void* ws, size_t ws_bytes, int32_t* dev_status, cudaStream_t st) {
  if (!skeleton_pivot_pipelined(dt, n, m, s)) return SKEL_ERR_UNSUPPORTED;
  if (ws_bytes < skeleton_pivot_workspace(dt, n, m, s)) return SKEL_ERR_WORKSPACE;
  const size_t es = dt == SKEL_F64 ? 8 : 4;
  char* wsc = static_cast<char*>(ws);
  char* wsr = wsc + (dt == SKEL_F64 ? panel_ws<double>(n, s, true) : panel_ws<float>(n, s, true));
  char* lw = wsr + align_up(es * (size_t)s * m) + align_up(m) + 256 + align_up(es * (size_t)s * m);
  if (dt == SKEL_F64)
    return run_skeleton_t<double>(plan_panel<double>(n, s), plan_panel<double>(m, s), (const double*)X, n, ldx, s,
                                  (const double*)A, m, lda, Js, Is, (double*)L, ldl, (double*)R, ldr, wsc, wsr,
                                  (double*)lw, dev_status, st);
  return run_skeleton_t<float>(plan_panel<float>(n, s), plan_panel<float>(m, s), (const float*)X, n, ldx, s,
                               (const float*)A, m, lda, Js, Is, (float*)L, ldl, (float*)R, ldr, wsc, wsr, (float*)lw,
                               dev_status, st);
}

struct GPanelPlan {
  int G = 0, nloc = 0, b = 0;
  size_t smem = 0, slot_bytes = 0, comm = 0;
};

// Grid panels: every SM holds n/G columns of a panel of b rows (b as large as 200 KB of shared
// memory allows, at most 64); 0 when not even one row fits or the grid cannot be co-resident.
template <typename T>
GPanelPlan plan_gpanel(int64_t n, int s) {
  GPanelPlan pl;
  if (n >= (int64_t)1 << 31) return pl;
  const int sms = device_sm_count();
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (n + 31) / 32));
  const int nloc = (int)((n + G - 1) / G);
  int b = std::min(kMaxPanel, s);
  while (b > 1 && gpanel_smem<T>(b, nloc) > 200 * 1024) --b;
  if (gpanel_smem<T>(b, nloc) > 200 * 1024) return pl;
  const size_t smem = gpanel_smem<T>(b, nloc);
  if (cudaFuncSetAttribute(lupp_gpanel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return pl;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lupp_gpanel_kernel<T>, 256, smem) != cudaSuccess ||
      per_sm * sms < G) {
    cudaGetLastError();
    return pl;
  }
  pl.G = G;
  pl.nloc = nloc;
  pl.b = b;
  pl.smem = smem;
  pl.slot_bytes = align_up(16 + sizeof(T) * (size_t)kMaxPanel, 16);
  pl.comm = comm_header_bytes(kMaxPanel) + align_up(2 * (size_t)G * pl.slot_bytes);
  return pl;
}

template <typename T>
size_t gpanel_ws(int64_t n, int s, const GPanelPlan& pl) {
  return panel_ws<T>(n, s, true) + pl.comm;
}

template <typename T>
skel_status run_gpanel_t(const GPanelPlan& pl, const T* X, int64_t n, int64_t ldx, int s, int32_t* Js, T* L,
                         int64_t ldl, T* R, int64_t ldr, void* ws, int32_t* dev_status, cudaStream_t st) {
  char* base = static_cast<char*>(ws);
  T* Xg = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)s * n);
  unsigned char* sel = reinterpret_cast<unsigned char*>(base);
  base += align_up(n);
  int32_t* fail = reinterpret_cast<int32_t*>(base);
  base += 256;
  T* M = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)s * 64);
  T* Rw = reinterpret_cast<T*>(base);
  base += align_up(sizeof(T) * (size_t)s * n);
  if (R == nullptr) {
    R = Rw;
    ldr = n;
  }
  char* comm = base;
  lupp_panel_init_kernel<T><<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min(s, 64)), 256, 0, st>>>(
      X, ldx, s, n, Xg, sel, fail, L, ldl);
  note_launches(1);
  if (cudaFuncSetAttribute(lupp_gpanel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) != cudaSuccess)
    return SKEL_ERR_CUDA;
  int k = 0;
  for (int t0 = 0; t0 < s; t0 += pl.b, ++k) {
    const int bb = std::min(pl.b, s - t0);
    if (cudaMemsetAsync(comm, 0, comm_header_bytes(kMaxPanel), st) != cudaSuccess) return SKEL_ERR_CUDA;
    GPanelParams gp{};
    gp.n = n; gp.s = s; gp.t0 = t0; gp.b = bb; gp.nloc = pl.nloc;
    gp.sel = sel;
    gp.tag = (unsigned char)std::min(k + 1, 255);
    gp.Js = Js; gp.fail = fail; gp.dev_status = dev_status;
    gp.gc.counter = reinterpret_cast<unsigned int*>(comm);
    gp.gc.abort = reinterpret_cast<int32_t*>(comm + 4);
    gp.gc.keys = reinterpret_cast<unsigned long long*>(comm + 256);
    gp.gc.payload = comm + comm_header_bytes(kMaxPanel);
    gp.gc.slot_bytes = (int64_t)pl.slot_bytes;
    gp.gc.G = pl.G;
    gp.gc.wait_ns = kDefaultWaitNs;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.G);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    {
      KernelTimer kt("lupp_panel", st);
      if (cudaLaunchKernelEx(&cfg, lupp_gpanel_kernel<T>, gp, Xg, R, ldr, L, ldl) != cudaSuccess) return SKEL_ERR_CUDA;
    }
    note_launches(1);
    const int trows = s - t0 - bb;
    if (trows <= 0) continue;
    {
      KernelTimer kt("lupp_mult", st);
      lupp_gmult_kernel<T><<<(unsigned)std::min<int64_t>((trows + 7) / 8, 1024), 256, 0, st>>>(
          Xg, n, t0 + bb, s, t0, bb, R, ldr, Js, M, bb, L, ldl, fail);
    }
    note_launches(1);
    PanelParams<T> tp{};
    tp.Xg = Xg; tp.n = n; tp.s = s; tp.t0 = t0; tp.b = bb; tp.R = R; tp.ldr = ldr; tp.fail = fail;
    tp.M = M; tp.ldm = bb; tp.trow0 = t0 + bb; tp.trows = trows; tp.sel = sel;
    if (launch_trail<T>(tp, trows, st) != cudaSuccess) return SKEL_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ERR_CUDA;
}

static bool gpanel_usable(skel_dtype dt, int64_t n, int32_t s) {
  return (dt == SKEL_F64 ? plan_gpanel<double>(n, s).b : plan_gpanel<float>(n, s).b) > 0;
}

static size_t gpanel_workspace(skel_dtype dt, int64_t n, int32_t s) {
  return dt == SKEL_F64 ? gpanel_ws<double>(n, s, plan_gpanel<double>(n, s))
                        : gpanel_ws<float>(n, s, plan_gpanel<float>(n, s));
}

static bool panel_usable(skel_dtype dt, int64_t n, int32_t s) {
  return (dt == SKEL_F64 ? plan_panel<double>(n, s).b : plan_panel<float>(n, s).b) > 0;
}

static size_t panel_workspace(skel_dtype dt, int64_t n, int32_t s) {
  return dt == SKEL_F64 ? panel_ws<double>(n, s, true) : panel_ws<float>(n, s, true);
}

size_t lupp_auto_workspace(skel_dtype dt, int64_t n, int32_t s) {
  if (panel_usable(dt, n, s)) return panel_workspace(dt, n, s);
  if (gpanel_usable(dt, n, s)) return gpanel_workspace(dt, n, s);
  return lupp_workspace(dt, n, s, nullptr);
}

skel_status run_lupp_auto(skel_dtype dt, const void* X, int64_t n, int64_t ldx, int32_t s,
                          int32_t* Js, void* L, int64_t ldl, void* R, int64_t ldr, void* ws,
                          size_t ws_bytes, int32_t* dev_status, cudaStream_t st) {
  if (!panel_usable(dt, n, s)) {
    if (gpanel_usable(dt, n, s)) {           // wider than a cluster panel: grid-wide panels
      if (ws_bytes < gpanel_workspace(dt, n, s)) return SKEL_ERR_WORKSPACE;
      if (dt == SKEL_F64)
        return run_gpanel_t<double>(plan_gpanel<double>(n, s), (const double*)X, n, ldx, s, Js, (double*)L, ldl,
                                    (double*)R, ldr, ws, dev_status, st);
      return run_gpanel_t<float>(plan_gpanel<float>(n, s), (const float*)X, n, ldx, s, Js, (float*)L, ldl, (float*)R,
                                 ldr, ws, dev_status, st);
    }
    return run_lupp(dt, X, n, ldx, s, Js, L, ldl, R, ldr, ws, ws_bytes, dev_status, st);
  }
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
