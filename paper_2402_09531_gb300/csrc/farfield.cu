// Far-field phases of the DW-FMM matvec (Sec. 5.2, Eq. (5.4) with the
// two-scale relation of the nested cluster bases).
//
// With mu_c = P_c^T x (Legendre moments), m_c = V^{-T} mu_c (charges at the
// nodes a_c(xi_alpha)), l_c = sum_{s in far(c)} S_{c,s} m_s (potentials at
// the nodes) and lambda_c = V^{-1} l_c + T_c lambda_parent (Legendre
// coefficients of the local expansion), the far-field part of y is
// P_leaf lambda_leaf.  With T_c = V^{-1} B_c, B_c[alpha][alpha'] =
// p_hat_alpha'(a_parent^{-1}(a_c(xi_alpha))):
//   P2M:  mu_leaf[b]   = sum_{i in leaf} p_hat_b(a_leaf^{-1} x_i) x_i
//   M2M:  mu_p[b]      = sum_{c child} sum_a p_hat_b(a_p^{-1} y^c_a) m_c[a]
//   L2L:  l_c[a]      += sum_b lambda_p[b] p_hat_b(a_p^{-1} y^c_a)
//   L2P:  y_i          = sum_b lambda_leaf[b] p_hat_b(a_leaf^{-1} x_i)
// P2M and M2M are one kernel (Legendre moments of a box from point charges,
// then V^{-T}); L2L, V^{-1} and (on the leaf level) L2P are one kernel.
#include <algorithm>

#include "dwfmm_internal.cuh"
#include "sum_f32.cuh"

namespace dw {

namespace {

constexpr int kFarThreads = 128;
constexpr int kChunk = 32;

// p_hat_j(t) = sqrt(2j+1) P_j(2t-1), j = 0..qk.
template <typename T>
__device__ __forceinline__ void legendre_row(T t, int qk, T* tab) {
  const T u = T(2) * t - T(1);
  T pm = T(1), pc = u;
  tab[0] = T(1);
  if (qk >= 1) tab[1] = u * sqrt(T(3));
  for (int j = 1; j < qk; ++j) {
    const T pn = (T(2 * j + 1) * u * pc - T(j) * pm) / T(j + 1);
    tab[j + 1] = pn * sqrt(T(2 * j + 3));
    pm = pc;
    pc = pn;
  }
}

template <typename T>
__device__ __forceinline__ T basis_value(const T* tab, const int16_t* fac, int nnz) {
  T v = T(1);
  for (int z = 0; z < nnz; ++z) {
    const int o = fac[z];
    if (o < 0) break;
    v *= tab[o];
  }
  return v;
}

// Legendre table of one point: for every dimension k the values at
// t_k = (y_k - lo_k) * iext_k.
template <typename T>
__device__ __forceinline__ void point_table(const ExpDev& e, const T* y, int64_t ystride,
                                            const T* lo, const T* iext, T* tab) {
  for (int k = 0; k < e.d; ++k) {
    const T t = (y[k * ystride] - lo[k]) * iext[k];
    legendre_row<T>(t, e.qk[k], tab + e.loff[k]);
  }
}

// Moments of cluster g = first + blockIdx.x, then m = V^{-T} mu.
//  leaf mode:     sources = the leaf's sites, charges = right-hand sides.
//  children mode: sources = nodes of both children, charges = their m.
template <typename T>
__device__ __forceinline__ void moments_body(const ExpDev& e, int g, int leaf_mode, int L, const int32_t* count,
                                             const T* pts, int m_pad, const T* xb, const T* ynode,
                                             const T* lo_all, const T* iext_all, const T* vinv, int Rc, T* mom) {
  extern __shared__ unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);          // [kChunk][lsum]
  T* qs = tab + kChunk * e.lsum;                   // [kChunk][kRC]
  T* mu = qs + kChunk * kRC;                       // [n_pad][kRC]
  const int n = e.n, np = e.n_pad, d = e.d;
  const T* lo = lo_all + static_cast<int64_t>(g) * d;
  const T* iext = iext_all + static_cast<int64_t>(g) * d;
  int S;
  if (leaf_mode) S = count[g];
  else S = 2 * n;

  for (int ab = 0; ab < n; ab += kFarThreads) {
    const int a = ab + threadIdx.x;
    T acc[kRC];
#pragma unroll
    for (int r = 0; r < kRC; ++r) acc[r] = T(0);
    for (int cb = 0; cb < S; cb += kChunk) {
      const int cn = min(kChunk, S - cb);
      if (threadIdx.x < cn) {
        const int p = cb + threadIdx.x;
        const T* y;
        int64_t ys;
        if (leaf_mode) {
          y = pts + static_cast<int64_t>(g - (L - 1)) * d * m_pad + p;
          ys = m_pad;
        } else {
          const int ch = 2 * g + 1 + (p >= n);
          const int pa = p % n;
          y = ynode + static_cast<int64_t>(ch) * d * np + pa;
          ys = np;
        }
        point_table<T>(e, y, ys, lo, iext, tab + threadIdx.x * e.lsum);
      }
      for (int idx = threadIdx.x; idx < cn * kRC; idx += kFarThreads) {
        const int pl = idx / kRC, r = idx % kRC;
        const int p = cb + pl;
        T v = T(0);
        if (r < Rc) {
          if (leaf_mode) v = xb[(static_cast<int64_t>(g - (L - 1)) * kRC + r) * m_pad + p];
          else {
            const int ch = 2 * g + 1 + (p >= n);
            v = mom[(static_cast<int64_t>(ch) * kRC + r) * np + (p % n)];
          }
        }
        qs[idx] = v;
      }
      __syncthreads();
      if (a < n) {
        const int16_t* fac = e.fac + a * e.nnz_max;
        for (int pl = 0; pl < cn; ++pl) {
          const T b = basis_value<T>(tab + pl * e.lsum, fac, e.nnz_max);
#pragma unroll
          for (int r = 0; r < kRC; ++r) acc[r] += b * qs[pl * kRC + r];
        }
      }
      __syncthreads();
    }
    if (a < np) {
#pragma unroll
      for (int r = 0; r < kRC; ++r) mu[a * kRC + r] = (a < n) ? acc[r] : T(0);
    }
  }
  __syncthreads();
  // m = V^{-T} mu
  for (int a = threadIdx.x; a < np; a += kFarThreads) {
    T out[kRC];
#pragma unroll
    for (int r = 0; r < kRC; ++r) out[r] = T(0);
    for (int b = 0; b < n; ++b) {
      const T v = vinv[b * np + a];
#pragma unroll
      for (int r = 0; r < kRC; ++r) out[r] += v * mu[b * kRC + r];
    }
    for (int r = 0; r < kRC; ++r) mom[(static_cast<int64_t>(g) * kRC + r) * np + a] = r < Rc ? out[r] : T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(kFarThreads)
k_moments(ExpDev e, int first, int leaf_mode, int L, const int32_t* count, const T* pts, int m_pad,
          const T* xb, const T* ynode, const T* lo_all, const T* iext_all, const T* vinv, int Rc,
          T* mom) {
  moments_body<T>(e, first + blockIdx.x, leaf_mode, L, count, pts, m_pad, xb, ynode, lo_all, iext_all, vinv,
                  Rc, mom);
}

// Downward pass on cluster g = first + blockIdx.x (level `level`):
//   l_g += B_g lambda_parent  (if level > jmin), lambda_g = V^{-1} l_g,
//   and on the leaf level y_far = P_leaf lambda_leaf.
template <typename T>
__device__ __forceinline__ void downward_body(const ExpDev& e, int g, int level, int jmin, int J, int L,
                                              const int32_t* count, const T* pts, int m_pad, const T* ynode,
                                              const T* lo_all, const T* iext_all, const T* loc, T* lco,
                                              const T* vinv, int Rc, T* yfar) {
  extern __shared__ unsigned char smem_raw[];
  T* lamp = reinterpret_cast<T*>(smem_raw);        // [n_pad][kRC]
  T* lsm = lamp + e.n_pad * kRC;                  // [n_pad][kRC]
  T* tab = lsm + e.n_pad * kRC;                   // [kFarThreads][lsum]
  const int n = e.n, np = e.n_pad, d = e.d;
  for (int idx = threadIdx.x; idx < np * kRC; idx += kFarThreads) {
    const int a = idx / kRC, r = idx % kRC;
    lsm[idx] = (r < Rc && a < n) ? loc[(static_cast<int64_t>(g) * kRC + r) * np + a] : T(0);
  }
  if (level > jmin) {
    const int p = (g - 1) / 2;
    for (int idx = threadIdx.x; idx < np * kRC; idx += kFarThreads) {
      const int a = idx / kRC, r = idx % kRC;
      lamp[idx] = (r < Rc && a < n) ? lco[(static_cast<int64_t>(p) * kRC + r) * np + a] : T(0);
    }
    __syncthreads();
    const T* lo = lo_all + static_cast<int64_t>(p) * d;
    const T* iext = iext_all + static_cast<int64_t>(p) * d;
    T* mytab = tab + threadIdx.x * e.lsum;
    for (int ab = 0; ab < n; ab += kFarThreads) {
      const int a = ab + threadIdx.x;
      if (a < n) {
        point_table<T>(e, ynode + static_cast<int64_t>(g) * d * np + a, np, lo, iext, mytab);
        T acc[kRC];
#pragma unroll
        for (int r = 0; r < kRC; ++r) acc[r] = T(0);
        for (int b = 0; b < n; ++b) {
          const T v = basis_value<T>(mytab, e.fac + b * e.nnz_max, e.nnz_max);
#pragma unroll
          for (int r = 0; r < kRC; ++r) acc[r] += v * lamp[b * kRC + r];
        }
#pragma unroll
        for (int r = 0; r < kRC; ++r) lsm[a * kRC + r] += acc[r];
      }
    }
  }
  __syncthreads();
  // lambda_g = V^{-1} l_g  (into lamp)
  for (int a = threadIdx.x; a < np; a += kFarThreads) {
    T out[kRC];
#pragma unroll
    for (int r = 0; r < kRC; ++r) out[r] = T(0);
    for (int b = 0; b < n; ++b) {
      const T v = vinv[a * np + b];
#pragma unroll
      for (int r = 0; r < kRC; ++r) out[r] += v * lsm[b * kRC + r];
    }
#pragma unroll
    for (int r = 0; r < kRC; ++r) {
      lamp[a * kRC + r] = out[r];
      if (level < J) lco[(static_cast<int64_t>(g) * kRC + r) * np + a] = out[r];
    }
  }
  if (level < J) return;
  __syncthreads();
  // L2P on the leaf's sites
  const int leaf = g - (L - 1);
  const int cnt = count[g];
  const T* lo = lo_all + static_cast<int64_t>(g) * d;
  const T* iext = iext_all + static_cast<int64_t>(g) * d;
  T* mytab = tab + threadIdx.x * e.lsum;
  for (int ib = 0; ib < m_pad; ib += kFarThreads) {
    const int i = ib + threadIdx.x;
    if (i >= m_pad) break;
    T acc[kRC];
#pragma unroll
    for (int r = 0; r < kRC; ++r) acc[r] = T(0);
    if (i < cnt) {
      point_table<T>(e, pts + static_cast<int64_t>(leaf) * d * m_pad + i, m_pad, lo, iext, mytab);
      for (int b = 0; b < n; ++b) {
        const T v = basis_value<T>(mytab, e.fac + b * e.nnz_max, e.nnz_max);
#pragma unroll
        for (int r = 0; r < kRC; ++r) acc[r] += v * lamp[b * kRC + r];
      }
    }
    for (int r = 0; r < Rc; ++r) yfar[(static_cast<int64_t>(leaf) * kRC + r) * m_pad + i] = acc[r];
  }
}

template <typename T>
__global__ void __launch_bounds__(kFarThreads)
k_downward(ExpDev e, int first, int level, int jmin, int J, int L, const int32_t* count,
           const T* pts, int m_pad, const T* ynode, const T* lo_all, const T* iext_all,
           const T* loc, T* lco, const T* vinv, int Rc, T* yfar) {
  downward_body<T>(e, first + blockIdx.x, level, jmin, J, L, count, pts, m_pad, ynode, lo_all, iext_all, loc,
                   lco, vinv, Rc, yfar);
}

// ---- many problems in one launch (batches) --------------------------------
// Work item = (problem, cluster); every problem's arrays come from its entry
// of the problem table.

__device__ __forceinline__ int level_of(int g) { return 31 - __clz(g + 1); }

__global__ void __launch_bounds__(kFarThreads)
k_moments_batched(const ProbF32* probs, const int2* work) {
  const int2 w = work[blockIdx.x];
  const ProbF32& p = probs[w.x];
  moments_body<float>(p.e, w.y, level_of(w.y) == p.J, p.L, p.count, p.pts, p.m_pad, p.xb, p.ynode, p.lo, p.iext,
                      p.vinv, p.R, p.mom);
}

__global__ void __launch_bounds__(kFarThreads)
k_downward_batched(const ProbF32* probs, const int2* work) {
  const int2 w = work[blockIdx.x];
  const ProbF32& p = probs[w.x];
  downward_body<float>(p.e, w.y, level_of(w.y), p.jmin, p.J, p.L, p.count, p.pts, p.m_pad, p.ynode, p.lo, p.iext,
                       p.loc, p.lco, p.vinv, p.R, p.yfar);
}

// Problem of a global leaf (binary search in the leaf offsets).
__device__ __forceinline__ int problem_of(const int* leaf_off, int P, int gl) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (leaf_off[mid] <= gl) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Element t of the gathered right-hand sides xb[leaf][r][ld] (t < Ltot * 16 * ld).
__device__ __forceinline__ void gather_elem(const ProbF32* probs, const int* leaf_off, int P, int ld, float* xb,
                                            int64_t t) {
  const int i = static_cast<int>(t % ld);
  const int64_t lr = t / ld;
  const int r = static_cast<int>(lr % kRC);
  const int gl = static_cast<int>(lr / kRC);
  const int pi = problem_of(leaf_off, P, gl);
  const ProbF32& p = probs[pi];
  const int c = p.L - 1 + (gl - leaf_off[pi]);
  float v = 0.0f;
  if (r < p.R && i < p.count[c]) v = static_cast<float>(p.x[static_cast<int64_t>(r) * p.ldx + p.perm[p.begin[c] + i]]);
  xb[t] = v;
}

__global__ void k_gather_batched(const ProbF32* probs, const int* leaf_off, int P, int Ltot, int ld, float* xb) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= static_cast<int64_t>(Ltot) * kRC * ld) return;
  gather_elem(probs, leaf_off, P, ld, xb, t);
}

// Element t of y = near + far, written to the caller's order (t < Ltot * 16 * ld).
__device__ __forceinline__ void scatter_elem(const ProbF32* probs, const int* leaf_off, int P, int ld,
                                             const float* ynear, const float* yfar, int64_t t) {
  const int i = static_cast<int>(t % ld);
  const int64_t lr = t / ld;
  const int r = static_cast<int>(lr % kRC);
  const int gl = static_cast<int>(lr / kRC);
  const int pi = problem_of(leaf_off, P, gl);
  const ProbF32& p = probs[pi];
  const int c = p.L - 1 + (gl - leaf_off[pi]);
  if (r >= p.R || i >= p.count[c]) return;
  double v = static_cast<double>(ynear[t]);
  if (p.jmin <= p.J) v += static_cast<double>(yfar[t]);
  p.y[static_cast<int64_t>(r) * p.ldy + p.perm[p.begin[c] + i]] = v;
}

__global__ void k_scatter_batched(const ProbF32* probs, const int* leaf_off, int P, int Ltot, int ld,
                                  const float* ynear, const float* yfar) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= static_cast<int64_t>(Ltot) * kRC * ld) return;
  scatter_elem(probs, leaf_off, P, ld, ynear, yfar, t);
}

// ---------------------------------------------------------------------------
// Persistent batch matvec: the whole fused matvec of a batch as one
// cooperative launch (every CTA resident at once).  Phases, each ended by a
// grid-wide barrier (one arrival counter per phase, bounded wait):
//   gather | interleave of the near-field charges, P2M of the leaves |
//   M2M, one phase per height | interleave of the moments | the couplings
//   (M2L, work queue) | L2L and L2P, one phase per level | the rest of the
//   near field | scatter.
// The near field (P2P) needs only the gathered charges, so from the second
// barrier on a CTA that has done its share of a far-field phase takes
// near-field target groups from a work queue while it waits for the others:
// the short phases of the coarse levels no longer leave SMs idle, and all
// right-hand-side classes share one queue (no tail per class).  Near-field
// and coupling target groups run on groups of gs threads (several per CTA:
// the tuned width), each group with its own stages and stage barriers,
// taking items on its own until its queue is empty or its barrier completes;
// the summation order inside a target group is that of k_sum_f32, so the
// result equals the launch-per-phase matvec bit for bit.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// A barrier waits at most this long with nothing to do (every CTA is
// resident, so the others only have their share of one phase left).
constexpr uint64_t kPersistWaitNs = 4000000000ull;

template <int D, int KER>
__device__ __forceinline__ bool persist_sum_item(const PersistSeg* segs, int nseg, int idx, const sk::Grp& G,
                                                 unsigned char* sm, uint64_t* full, int& tiles) {
  int s = 0;
  while (s + 1 < nseg && idx >= segs[s].count) {
    idx -= segs[s].count;
    ++s;
  }
  const PersistSeg& sg = segs[s];
  const int g = sg.a.first + idx;
  switch (sg.rc) {
    case 1: return sk::sum_block<D, 1, KER>(sg.a, g, G, sm, full, tiles);
    case 4: return sk::sum_block<D, 4, KER>(sg.a, g, G, sm, full, tiles);
    case 8: return sk::sum_block<D, 8, KER>(sg.a, g, G, sm, full, tiles);
    default: return sk::sum_block<D, 16, KER>(sg.a, g, G, sm, full, tiles);
  }
}

// Shared state of a persistent CTA: stage barriers and completed-stage counts
// of up to four groups, the item each group took, a broadcast word.
struct PShared {
  uint64_t full[kPersistThreads / 32][2];
  int tiles[kPersistThreads / 32];
  int item[kPersistThreads / 32];
  int flag;
};

// Summation items from a queue (head `head`, `total` items): every group of
// gs threads takes target groups one at a time and sums them, on its own,
// until the queue is empty or, if `stop` is given, the barrier counter *stop
// has reached gridDim.x (checked by the group's first thread between items).
// 0: the queue is empty; 1: stopped by the barrier; -1: a copy wait gave up
// (error flag set).
template <int D, int KER>
__device__ __noinline__ int persist_drain(const PersistSeg* segs, int nseg, int total, unsigned* head, int gs,
                                          int gbytes, unsigned char* smem, PShared& sh, const unsigned* stop) {
  const int gid = static_cast<int>(threadIdx.x) / gs;
  const sk::Grp G{static_cast<int>(threadIdx.x) % gs, gs, 1 + gid};
  unsigned char* gsm = smem + static_cast<size_t>(gid) * gbytes;
  int tiles = sh.tiles[gid];
  bool ok = true, empty = false;
  for (;;) {
    if (G.tid == 0) {
      int it = -1;   // -1: the barrier is complete
      if (!stop || ld_acquire_gpu(stop) < gridDim.x) it = static_cast<int>(atomicAdd(head, 1u));
      sh.item[gid] = it;
    }
    sk::grp_sync(G);
    const int it = sh.item[gid];
    sk::grp_sync(G);   // read by every thread before the next item overwrites it
    if (it < 0) break;
    if (it >= total) {
      empty = true;
      break;
    }
    if (!persist_sum_item<D, KER>(segs, nseg, it, G, gsm, sh.full[gid], tiles)) {
      ok = false;
      break;
    }
  }
  if (G.tid == 0) sh.tiles[gid] = tiles;
  const int bad = __syncthreads_or(!ok);
  const int emp = __syncthreads_or(empty);
  return bad ? -1 : (emp ? 0 : 1);
}

// Arrive at barrier `ph` and wait until every CTA has; meanwhile, if `near`,
// the CTA's groups take near-field items from their queue until the barrier
// completes or the queue is empty.  False when the wait gave up (error flag
// 4) or a copy wait did.
template <int D, int KER>
__device__ __noinline__ bool persist_barrier(const PersistArgs& pa, int ph, bool near, bool& near_left, unsigned char* smem,
                                PShared& sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(pa.sync + ph, 1u);
  }
  uint64_t t0 = threadIdx.x == 0 ? global_ns() : 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const bool all = ld_acquire_gpu(pa.sync + ph) >= gridDim.x;
      sh.flag = all ? 1 : (global_ns() - t0 > kPersistWaitNs ? 2 : 0);
    }
    __syncthreads();
    const int f = sh.flag;
    __syncthreads();
    if (f == 1) break;
    if (f == 2) {
      if (threadIdx.x == 0) atomicExch(pa.err, 4);
      return false;
    }
    if (near && near_left) {
      const int r = persist_drain<D, KER>(pa.near, pa.nnear, pa.near_total, pa.sync + kPersistSync - 2,
                                          pa.gs_near, pa.near_group_bytes, smem, sh, pa.sync + ph);
      if (r < 0) return false;
      if (r == 0) near_left = false;
      if (threadIdx.x == 0) t0 = global_ns();
      continue;
    }
    if (threadIdx.x == 0) __nanosleep(256);
  }
  // the other CTAs' writes are now visible; order them before this CTA's
  // bulk copies (async proxy) as well
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  return true;
}

__device__ __forceinline__ void persist_up_items(const PersistArgs& pa, int h) {
  for (int i = static_cast<int>(blockIdx.x); i < pa.up_cnt[h]; i += static_cast<int>(gridDim.x)) {
    const int2 w = pa.work[pa.up_off[h] + i];
    const ProbF32& p = pa.probs[w.x];
    moments_body<float>(p.e, w.y, level_of(w.y) == p.J, p.L, p.count, p.pts, p.m_pad, p.xb, p.ynode, p.lo, p.iext,
                        p.vinv, p.R, p.mom);
    __syncthreads();
  }
}

__device__ __forceinline__ void persist_down_items(const PersistArgs& pa, int j) {
  for (int i = static_cast<int>(blockIdx.x); i < pa.down_cnt[j]; i += static_cast<int>(gridDim.x)) {
    const int2 w = pa.work[pa.down_off[j] + i];
    const ProbF32& p = pa.probs[w.x];
    downward_body<float>(p.e, w.y, level_of(w.y), p.jmin, p.J, p.L, p.count, p.pts, p.m_pad, p.ynode, p.lo, p.iext,
                         p.loc, p.lco, p.vinv, p.R, p.yfar);
    __syncthreads();
  }
}

__device__ __forceinline__ void persist_interleave(const PersistSeg* segs, int nseg, int64_t t0, int64_t stride) {
  for (int s = 0; s < nseg; ++s) {
    const PersistSeg& sg = segs[s];
    const int ld = sg.a.ld;
    const int64_t n = static_cast<int64_t>(sg.count) * ld * sg.rc;
    const float* src = sg.ilv_src + static_cast<int64_t>(sg.a.first) * kRC * ld;
    float* dst = const_cast<float*>(sg.a.q) + static_cast<int64_t>(sg.a.first) * sg.rc * ld;
    for (int64_t t = t0; t < n; t += stride) sk::interleave_elem(src, ld, sg.rc, dst, t);
  }
}

template <int D, int KER>
__global__ void __launch_bounds__(kPersistThreads, 3) k_batch_persistent(const __grid_constant__ PersistArgs pa) {
  extern __shared__ __align__(128) unsigned char psm[];
  __shared__ PShared sh;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kPersistThreads / 32; ++k) {
      sk::mbar_init(&sh.full[k][0], 1);
      sk::mbar_init(&sh.full[k][1], 1);
      sh.tiles[k] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int ph = 0;
  bool near_left = pa.near_total > 0;
  // gather
  const int64_t nel = static_cast<int64_t>(pa.Ltot) * kRC * pa.ld;
  if (pa.io)
    for (int64_t t = t0; t < nel; t += stride) gather_elem(pa.probs, pa.leaf_off, pa.P, pa.ld, pa.xb, t);
  if (!persist_barrier<D, KER>(pa, ph++, false, near_left, psm, sh)) return;
  // near-field charges; P2M of the leaves
  persist_interleave(pa.near, pa.nnear, t0, stride);
  if (pa.nup > 0) persist_up_items(pa, 0);
  if (!persist_barrier<D, KER>(pa, ph++, false, near_left, psm, sh)) return;
  // M2M by height
  for (int h = 1; h < pa.nup; ++h) {
    persist_up_items(pa, h);
    if (!persist_barrier<D, KER>(pa, ph++, true, near_left, psm, sh)) return;
  }
  // M2L
  if (pa.m2l_total > 0) {
    persist_interleave(pa.m2l, pa.nm2l, t0, stride);
    if (!persist_barrier<D, KER>(pa, ph++, true, near_left, psm, sh)) return;
    if (persist_drain<D, KER>(pa.m2l, pa.nm2l, pa.m2l_total, pa.sync + kPersistSync - 1, pa.gs_m2l,
                              pa.m2l_group_bytes, psm, sh, nullptr) < 0)
      return;
    if (!persist_barrier<D, KER>(pa, ph++, true, near_left, psm, sh)) return;
  }
  // L2L / L2P by level
  for (int j = 0; j < pa.ndown; ++j) {
    persist_down_items(pa, j);
    if (!persist_barrier<D, KER>(pa, ph++, true, near_left, psm, sh)) return;
  }
  // the rest of the near field
  if (near_left && persist_drain<D, KER>(pa.near, pa.nnear, pa.near_total, pa.sync + kPersistSync - 2, pa.gs_near,
                                          pa.near_group_bytes, psm, sh, nullptr) < 0)
    return;
  if (!persist_barrier<D, KER>(pa, ph++, false, near_left, psm, sh)) return;
  if (pa.io)
    for (int64_t t = t0; t < nel; t += stride)
      scatter_elem(pa.probs, pa.leaf_off, pa.P, pa.ld, pa.ynear, pa.yfar, t);
}

// x (caller order, column-major) -> xb[leaf][r][m_pad] for r in [r0, r0+Rc).
template <typename T>
__global__ void k_gather(const double* x, int64_t ldx, int r0, int Rc, const int32_t* perm,
                         const int32_t* begin, const int32_t* count, int L, int m_pad, T* xb) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(L) * kRC * m_pad;
  if (t >= total) return;
  const int i = static_cast<int>(t % m_pad);
  const int64_t lr = t / m_pad;
  const int r = static_cast<int>(lr % kRC);
  const int leaf = static_cast<int>(lr / kRC);
  const int c = L - 1 + leaf;
  T v = T(0);
  if (r < Rc && i < count[c]) v = static_cast<T>(x[static_cast<int64_t>(r0 + r) * ldx + perm[begin[c] + i]]);
  xb[t] = v;
}

template <typename T>
__global__ void k_scatter(double* y, int64_t ldy, int r0, int Rc, const int32_t* perm,
                          const int32_t* begin, const int32_t* count, int L, int m_pad,
                          const T* ynear, const T* yfar, int has_far) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(L) * kRC * m_pad;
  if (t >= total) return;
  const int i = static_cast<int>(t % m_pad);
  const int64_t lr = t / m_pad;
  const int r = static_cast<int>(lr % kRC);
  const int leaf = static_cast<int>(lr / kRC);
  const int c = L - 1 + leaf;
  if (r >= Rc || i >= count[c]) return;
  double v = static_cast<double>(ynear[t]);
  if (has_far) v += static_cast<double>(yfar[t]);
  y[static_cast<int64_t>(r0 + r) * ldy + perm[begin[c] + i]] = v;
}

template <typename T>
struct Bufs {
  T *xb, *ynear, *yfar, *mom, *loc, *lco;
  const T *pts, *ynode, *lo, *iext, *vinv;
};

template <typename T>
Bufs<T> bufs(Plan& P);

template <>
Bufs<double> bufs<double>(Plan& P) {
  return Bufs<double>{P.xb64.p,   P.ynear64.p, P.yfar64.p,  P.mom64.p,  P.loc64.p, P.lco64.p,
                      P.d_pts64.p, P.d_ynode64.p, P.d_lo.p, P.d_iext.p, P.d_vinv.p};
}
template <>
Bufs<float> bufs<float>(Plan& P) {
  return Bufs<float>{P.xb32.p,   P.ynear32.p, P.yfar32.p,  P.mom32.p,   P.loc32.p,  P.lco32.p,
                     P.d_pts32.p, P.d_ynode32.p, P.d_lo32.p, P.d_iext32.p, P.d_vinv32.p};
}

template <typename T>
void farfield_impl(Plan& P, int Rc) {
  cudaStream_t s = P.stream;
  Bufs<T> B = bufs<T>(P);
  const ExpDev e = P.exp_dev();
  const int J = P.J, L = P.L;
  const int64_t ny = static_cast<int64_t>(L) * kRC * P.m_pad;
  if (P.jmin > J) {  // no admissible block: the far field is empty
    DW_CUDA(cudaMemsetAsync(B.yfar, 0, ny * sizeof(T), s));
    P.far_engine = sizeof(T) == 8 ? 0 : 1;
    return;
  }
  if (sizeof(T) == 4 && farfield_tc_eligible(P)) {
    P.far_engine = 2;
    farfield_tc(P, Rc);
    return;
  }
  P.far_engine = sizeof(T) == 8 ? 0 : 1;
  const size_t sm_mom = (static_cast<size_t>(kChunk) * e.lsum + kChunk * kRC + static_cast<size_t>(e.n_pad) * kRC) * sizeof(T);
  const size_t sm_down = (2 * static_cast<size_t>(e.n_pad) * kRC + static_cast<size_t>(kFarThreads) * e.lsum) * sizeof(T);
  timer_begin(P, 1, s);
  int launches = 0;
  for (int j = J; j >= P.jmin; --j) {
    const int first = (1 << j) - 1;
    k_moments<T><<<1 << j, kFarThreads, sm_mom, s>>>(e, first, j == J, L, P.d_count.p, B.pts, P.m_pad,
                                                     B.xb, B.ynode, B.lo, B.iext, B.vinv, Rc, B.mom);
    ++launches;
  }
  timer_end(P, 1, s, launches);
  timer_begin(P, 2, s);
  launch_m2l(P, Rc, sizeof(T) == 8);
  timer_end(P, 2, s, 1);
  timer_begin(P, 3, s);
  launches = 0;
  for (int j = P.jmin; j <= J; ++j) {
    const int first = (1 << j) - 1;
    k_downward<T><<<1 << j, kFarThreads, sm_down, s>>>(e, first, j, P.jmin, J, L, P.d_count.p, B.pts,
                                                       P.m_pad, B.ynode, B.lo, B.iext, B.loc, B.lco,
                                                       B.vinv, Rc, B.yfar);
    ++launches;
  }
  timer_end(P, 3, s, launches);
  DW_CUDA(cudaGetLastError());
}

}  // namespace

void farfield_set_smem_limits(Plan& P) {
  // Raise the dynamic shared-memory limit once per plan (large index sets).
  const int big = 200 * 1024;
  DW_CUDA(cudaFuncSetAttribute(k_moments<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DW_CUDA(cudaFuncSetAttribute(k_moments<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DW_CUDA(cudaFuncSetAttribute(k_downward<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DW_CUDA(cudaFuncSetAttribute(k_downward<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  (void)P;
}

size_t farfield_smem_need(const Plan& P, bool fp64) {
  const size_t es = fp64 ? 8 : 4;
  const size_t a = (static_cast<size_t>(kChunk) * P.lsum + kChunk * kRC + static_cast<size_t>(P.n_pad) * kRC) * es;
  const size_t b = (2 * static_cast<size_t>(P.n_pad) * kRC + static_cast<size_t>(kFarThreads) * P.lsum) * es;
  return std::max(a, b);
}

void launch_gather(Plan& P, const double* x, int64_t ldx, int r0, int Rc, bool fp64) {
  const int64_t total = static_cast<int64_t>(P.L) * kRC * P.m_pad;
  if (fp64)
    k_gather<double><<<ceil_div(total, 256), 256, 0, P.stream>>>(x, ldx, r0, Rc, P.d_perm.p, P.d_begin.p,
                                                                 P.d_count.p, P.L, P.m_pad, P.xb64.p);
  else
    k_gather<float><<<ceil_div(total, 256), 256, 0, P.stream>>>(x, ldx, r0, Rc, P.d_perm.p, P.d_begin.p,
                                                                P.d_count.p, P.L, P.m_pad, P.xb32.p);
  DW_CUDA(cudaGetLastError());
}

void launch_scatter(Plan& P, double* y, int64_t ldy, int r0, int Rc, bool fp64) {
  const int64_t total = static_cast<int64_t>(P.L) * kRC * P.m_pad;
  const int has_far = P.jmin <= P.J;
  if (fp64)
    k_scatter<double><<<ceil_div(total, 256), 256, 0, P.stream>>>(y, ldy, r0, Rc, P.d_perm.p, P.d_begin.p,
                                                                  P.d_count.p, P.L, P.m_pad, P.ynear64.p,
                                                                  P.yfar64.p, has_far);
  else
    k_scatter<float><<<ceil_div(total, 256), 256, 0, P.stream>>>(y, ldy, r0, Rc, P.d_perm.p, P.d_begin.p,
                                                                 P.d_count.p, P.L, P.m_pad, P.ynear32.p,
                                                                 P.yfar32.p, has_far);
  DW_CUDA(cudaGetLastError());
}

void batch_far_attrs() {
  const int big = 200 * 1024;
  DW_CUDA(cudaFuncSetAttribute(k_moments_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DW_CUDA(cudaFuncSetAttribute(k_downward_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
}

size_t batch_far_smem(int lsum, int n_pad) {
  const size_t a = (static_cast<size_t>(kChunk) * lsum + kChunk * kRC + static_cast<size_t>(n_pad) * kRC) * 4;
  const size_t b = (2 * static_cast<size_t>(n_pad) * kRC + static_cast<size_t>(kFarThreads) * lsum) * 4;
  return std::max(a, b);
}

void launch_moments_batched(const ProbF32* probs, const int2* work, int items, size_t smem, cudaStream_t s) {
  if (items > 0) k_moments_batched<<<items, kFarThreads, smem, s>>>(probs, work);
}

void launch_downward_batched(const ProbF32* probs, const int2* work, int items, size_t smem, cudaStream_t s) {
  if (items > 0) k_downward_batched<<<items, kFarThreads, smem, s>>>(probs, work);
}

void launch_gather_batched(const ProbF32* probs, const int* leaf_off, int P, int Ltot, int ld, float* xb,
                           cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(Ltot) * kRC * ld;
  k_gather_batched<<<ceil_div(total, 256), 256, 0, s>>>(probs, leaf_off, P, Ltot, ld, xb);
}

void launch_scatter_batched(const ProbF32* probs, const int* leaf_off, int P, int Ltot, int ld, const float* ynear,
                            const float* yfar, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(Ltot) * kRC * ld;
  k_scatter_batched<<<ceil_div(total, 256), 256, 0, s>>>(probs, leaf_off, P, Ltot, ld, ynear, yfar);
}

size_t persist_group_bytes(int D, int RC, int ld, int threads) { return sk::group_stage_bytes(D, RC, ld, threads); }

namespace {

template <int D>
const void* persist_fn_d(int kernel) {
  switch (kernel) {
    case DWFMM_K_EXP: return reinterpret_cast<const void*>(k_batch_persistent<D, DWFMM_K_EXP>);
    case DWFMM_K_MATERN32: return reinterpret_cast<const void*>(k_batch_persistent<D, DWFMM_K_MATERN32>);
    default: return reinterpret_cast<const void*>(k_batch_persistent<D, DWFMM_K_GAUSS>);
  }
}

const void* persist_fn(int D, int kernel) {
  switch (D) {
    case 4: return persist_fn_d<4>(kernel);
    case 8: return persist_fn_d<8>(kernel);
    case 10: return persist_fn_d<10>(kernel);
    case 12: return persist_fn_d<12>(kernel);
    case 16: return persist_fn_d<16>(kernel);
    default: return persist_fn_d<20>(kernel);
  }
}

template <int D>
cudaError_t persist_launch_d(int kernel, const cudaLaunchConfig_t& cfg, const PersistArgs& pa) {
  switch (kernel) {
    case DWFMM_K_EXP: return cudaLaunchKernelEx(&cfg, k_batch_persistent<D, DWFMM_K_EXP>, pa);
    case DWFMM_K_MATERN32: return cudaLaunchKernelEx(&cfg, k_batch_persistent<D, DWFMM_K_MATERN32>, pa);
    default: return cudaLaunchKernelEx(&cfg, k_batch_persistent<D, DWFMM_K_GAUSS>, pa);
  }
}

}  // namespace

int persist_blocks_per_sm(int D, int kernel, size_t smem) {
  const void* f = persist_fn(D, kernel);
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kPersistThreads, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_batch_persistent(int D, int kernel, const PersistArgs& pa, int grid, size_t smem,
                                    cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  switch (D) {
    case 4: return persist_launch_d<4>(kernel, cfg, pa);
    case 8: return persist_launch_d<8>(kernel, cfg, pa);
    case 10: return persist_launch_d<10>(kernel, cfg, pa);
    case 12: return persist_launch_d<12>(kernel, cfg, pa);
    case 16: return persist_launch_d<16>(kernel, cfg, pa);
    default: return persist_launch_d<20>(kernel, cfg, pa);
  }
}

void launch_farfield(Plan& P, int Rc, bool fp64) {
  if (fp64) farfield_impl<double>(P, Rc);
  else farfield_impl<float>(P, Rc);
}

}  // namespace dw
