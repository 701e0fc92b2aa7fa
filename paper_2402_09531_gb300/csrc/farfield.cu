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

__global__ void k_gather_batched(const ProbF32* probs, const int* leaf_off, int P, int Ltot, int ld, float* xb) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= static_cast<int64_t>(Ltot) * kRC * ld) return;
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

__global__ void k_scatter_batched(const ProbF32* probs, const int* leaf_off, int P, int Ltot, int ld,
                                  const float* ynear, const float* yfar) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= static_cast<int64_t>(Ltot) * kRC * ld) return;
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

void launch_farfield(Plan& P, int Rc, bool fp64) {
  if (fp64) farfield_impl<double>(P, Rc);
  else farfield_impl<float>(P, Rc);
}

}  // namespace dw
