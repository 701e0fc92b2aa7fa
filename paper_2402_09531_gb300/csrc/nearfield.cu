// Kernel summation y_i = sum_j phi(||x_i - x_j|| / sigma) q_j over lists of
// (target group, source group) blocks.  Two instances:
//   P2P: targets = a leaf's sites, sources = the sites of its near leaves
//        (the nearfield N of Sec. 5.2), charges = right-hand sides;
//   M2L: targets = the nodes a_c(xi_alpha) of cluster c, sources = the nodes
//        of every s with (c, s) in the farfield F, charges = m_s; this is
//        l_c = sum_s S_{c,s} m_s with the coupling matrices of Sec. 5.2.
// One CTA per target group, one thread per target, sources staged through
// shared memory in chunks.  This generic kernel serves float64 (parity) and
// the fallback float32 shapes; the tuned float32 P2P lives in p2p_f32.cu.
//
// The float64 P2P has a symmetric form as well: phi is symmetric and so is
// the near relation, so each unordered pair of near leaves (T, S) is
// evaluated once and contributes to both y_T (with x_S) and y_S (with x_T).
// One CTA per entry (T, S >= T) of the upper near list writes a forward
// partial (sums over S for the targets of T) and, off the diagonal, a
// transposed partial (sums over T for the sources of S: warp butterflies,
// then the four warps in order); a second kernel adds each leaf's partials
// in list order, so the result is deterministic.
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <vector>

#include "dwfmm_internal.cuh"

namespace dw {

int sm_count() {
  static std::atomic<int> n[64];   // per device; 0 = not looked up yet
  int dev = 0;
  DW_CUDA(cudaGetDevice(&dev));
  int v = dev < 64 ? n[dev].load() : 0;
  if (v == 0) {
    DW_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 64) n[dev].store(v);
  }
  return v;
}

namespace {

constexpr int kThreads = 128;
constexpr int kSrcChunk = 128;

template <typename T, int KER>
__device__ __forceinline__ T phi_r2(T r2, T inv_sigma) {
  if (KER == DWFMM_K_GAUSS) return exp(T(-0.5) * r2 * inv_sigma * inv_sigma);
  const T s = sqrt(r2) * inv_sigma;
  if (KER == DWFMM_K_EXP) return exp(-s);
  const T t = T(1.7320508075688772) * s;
  return (T(1) + t) * exp(-t);
}

struct Side {
  int64_t gstride;   // elements between groups
  int ld;            // elements between coordinate rows (or rhs rows)
  const int32_t* count;
  int count_off;
  int count_const;   // used when count == nullptr
};

// DM: compile-time bound on d (coordinates beyond d are zero, so the extra
// terms of the squared distance are exactly 0); RC: right-hand sides held in
// registers (rows beyond Rc are zero charges).
// splits > 1: CTA blockIdx.x handles part (blockIdx.x % splits) of group
// blockIdx.x / splits's list and writes its partial sums to out + part *
// split_stride (the caller adds the parts in a fixed order).
template <typename T, int KER, int DM, int RC>
__global__ void __launch_bounds__(kThreads)
k_ksum(int first_group, const int32_t* rowptr, const int32_t* col, int d, T inv_sigma,
       const T* tcoord, Side ts, const T* scoord, Side ss, const T* sq, int64_t sq_gstride,
       int sq_ld, T* out, int64_t o_gstride, int o_ld, int Rc, int splits, int64_t split_stride) {
  __shared__ T sc[DM * kSrcChunk];
  __shared__ T sqs[RC * kSrcChunk];
  const int g = first_group + static_cast<int>(blockIdx.x) / splits;
  const int part = static_cast<int>(blockIdx.x) % splits;
  const int r0 = rowptr[g], len = rowptr[g + 1] - r0;
  const int rb = r0 + static_cast<int>((static_cast<int64_t>(len) * part) / splits);
  const int re = r0 + static_cast<int>((static_cast<int64_t>(len) * (part + 1)) / splits);
  out += part * split_stride;
  const int tcnt = ts.count ? ts.count[ts.count_off + g] : ts.count_const;
  for (int tb = 0; tb < ts.ld; tb += kThreads) {
    const int i = tb + threadIdx.x;
    T xt[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k)
      xt[k] = (k < d && i < tcnt) ? tcoord[g * ts.gstride + static_cast<int64_t>(k) * ts.ld + i] : T(0);
    T acc[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) acc[r] = T(0);
    for (int e = rb; e < re; ++e) {
      const int s = col[e];
      const int scnt = ss.count ? ss.count[ss.count_off + s] : ss.count_const;
      for (int cb = 0; cb < scnt; cb += kSrcChunk) {
        const int cn = min(kSrcChunk, scnt - cb);
        __syncthreads();
        for (int idx = threadIdx.x; idx < DM * kSrcChunk; idx += kThreads) {
          const int k = idx / kSrcChunk, j = idx % kSrcChunk;
          sc[idx] = (j < cn && k < d) ? scoord[s * ss.gstride + static_cast<int64_t>(k) * ss.ld + cb + j] : T(0);
        }
        for (int idx = threadIdx.x; idx < RC * kSrcChunk; idx += kThreads) {
          const int r = idx / kSrcChunk, j = idx % kSrcChunk;
          sqs[idx] = (j < cn && r < Rc) ? sq[s * sq_gstride + static_cast<int64_t>(r) * sq_ld + cb + j] : T(0);
        }
        __syncthreads();
        for (int j = 0; j < cn; ++j) {
          T r2 = T(0);
#pragma unroll
          for (int k = 0; k < DM; ++k) {
            const T df = xt[k] - sc[k * kSrcChunk + j];
            r2 += df * df;
          }
          const T ph = phi_r2<T, KER>(r2, inv_sigma);
#pragma unroll
          for (int r = 0; r < RC; ++r) acc[r] += ph * sqs[r * kSrcChunk + j];
        }
      }
    }
    if (i < o_ld) {
#pragma unroll
      for (int r = 0; r < RC; ++r)
        if (r < Rc) out[g * o_gstride + static_cast<int64_t>(r) * o_ld + i] = acc[r];
    }
  }
}

template <typename T, int KER, int DM>
void launch_ksum_rc(int ngroups, int first_group, const int32_t* rowptr, const int32_t* col, int d,
                    T inv_sigma, const T* tcoord, Side ts, const T* scoord, Side ss, const T* sq,
                    int64_t sq_gstride, int sq_ld, T* out, int64_t o_gstride, int o_ld, int Rc,
                    cudaStream_t s, int splits, int64_t split_stride) {
#define DW_KS(RCV)                                                                                      \
  k_ksum<T, KER, DM, RCV><<<ngroups * splits, kThreads, 0, s>>>(first_group, rowptr, col, d, inv_sigma,   \
                                                                tcoord, ts, scoord, ss, sq, sq_gstride,   \
                                                                sq_ld, out, o_gstride, o_ld, Rc, splits,  \
                                                                split_stride)
  if (Rc <= 1) DW_KS(1);
  else if (Rc <= 4) DW_KS(4);
  else DW_KS(16);
#undef DW_KS
}

template <typename T, int KER>
void launch_ksum(int ngroups, int first_group, const int32_t* rowptr, const int32_t* col, int d,
                 T inv_sigma, const T* tcoord, Side ts, const T* scoord, Side ss, const T* sq,
                 int64_t sq_gstride, int sq_ld, T* out, int64_t o_gstride, int o_ld, int Rc,
                 cudaStream_t s, int splits, int64_t split_stride) {
  if (ngroups <= 0) return;
#define DW_KD(DMV)                                                                                 \
  launch_ksum_rc<T, KER, DMV>(ngroups, first_group, rowptr, col, d, inv_sigma, tcoord, ts, scoord, \
                              ss, sq, sq_gstride, sq_ld, out, o_gstride, o_ld, Rc, s, splits, split_stride)
  if (d <= 4) DW_KD(4);
  else if (d <= 8) DW_KD(8);
  else if (d <= 12) DW_KD(12);
  else if (d <= 16) DW_KD(16);
  else if (d <= 20) DW_KD(20);
  else DW_KD(kMaxDim);
#undef DW_KD
}

template <typename T>
void dispatch_ksum(int kernel, int ngroups, int first_group, const int32_t* rowptr, const int32_t* col,
                   int d, T inv_sigma, const T* tcoord, Side ts, const T* scoord, Side ss, const T* sq,
                   int64_t sq_gstride, int sq_ld, T* out, int64_t o_gstride, int o_ld, int Rc,
                   cudaStream_t s, int splits = 1, int64_t split_stride = 0) {
  switch (kernel) {
    case DWFMM_K_EXP:
      launch_ksum<T, DWFMM_K_EXP>(ngroups, first_group, rowptr, col, d, inv_sigma, tcoord, ts, scoord, ss,
                                  sq, sq_gstride, sq_ld, out, o_gstride, o_ld, Rc, s, splits, split_stride);
      break;
    case DWFMM_K_MATERN32:
      launch_ksum<T, DWFMM_K_MATERN32>(ngroups, first_group, rowptr, col, d, inv_sigma, tcoord, ts, scoord,
                                       ss, sq, sq_gstride, sq_ld, out, o_gstride, o_ld, Rc, s, splits, split_stride);
      break;
    default:
      launch_ksum<T, DWFMM_K_GAUSS>(ngroups, first_group, rowptr, col, d, inv_sigma, tcoord, ts, scoord, ss,
                                    sq, sq_gstride, sq_ld, out, o_gstride, o_ld, Rc, s, splits, split_stride);
  }
}

template <typename T>
void m2l_impl(Plan& P, int Rc, const T* ynode, const T* mom, T* loc) {
  // Targets: every cluster on levels >= jmin (clusters above have empty rows).
  const int first = (1 << P.jmin) - 1;
  const int ngroups = P.C - first;
  const int64_t gs = static_cast<int64_t>(P.d) * P.n_pad;
  Side side{gs, P.n_pad, nullptr, 0, P.n};
  dispatch_ksum<T>(P.kernel, ngroups, first, P.d_far_rowptr.p, P.d_far_col.p, P.d, T(1.0 / P.sigma), ynode,
                   side, ynode, side, mom, static_cast<int64_t>(kRC) * P.n_pad, P.n_pad, loc,
                   static_cast<int64_t>(kRC) * P.n_pad, P.n_pad, Rc, P.stream);
}

// out[g][r][i] = sum over parts of part[p][g][r][i] in part order (r < Rc).
__global__ void k_sum_parts(const double* part, int splits, int64_t stride, int64_t n, int64_t o_gstride,
                            int o_ld, int Rc, double* out) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int r = static_cast<int>((t % o_gstride) / o_ld);
  if (r >= Rc) return;
  double acc = 0.0;
  for (int p = 0; p < splits; ++p) acc += part[p * stride + t];
  out[t] = acc;
}


template <typename T>
void p2p_impl(Plan& P, int Rc, const T* pts, const T* xb, T* ynear, cudaStream_t s) {
  const int64_t gs = static_cast<int64_t>(P.d) * P.m_pad;
  Side side{gs, P.m_pad, P.d_count.p, P.L - 1, 0};
  const int64_t o_gstride = static_cast<int64_t>(kRC) * P.m_pad;
  // Small float64 problems: one CTA per leaf would leave most SMs idle (and
  // GB300's float64 unit is narrow), so each leaf's near list is split over
  // several CTAs whose partial sums are added in a fixed order.
  int splits = 1;
  if (std::is_same<T, double>::value) {
    const int want = 2 * sm_count();
    if (P.L < want) splits = std::min(16, (want + P.L - 1) / P.L);
  }
  if (splits == 1) {
    dispatch_ksum<T>(P.kernel, P.L, 0, P.d_near_rowptr.p, P.d_near_col.p, P.d, T(1.0 / P.sigma), pts, side,
                     pts, side, xb, o_gstride, P.m_pad, ynear, o_gstride, P.m_pad, Rc, s);
    return;
  }
  const int64_t stride = static_cast<int64_t>(P.L) * o_gstride;
  P.near_parts64.alloc(static_cast<size_t>(splits) * stride);
  T* part = reinterpret_cast<T*>(P.near_parts64.p);
  dispatch_ksum<T>(P.kernel, P.L, 0, P.d_near_rowptr.p, P.d_near_col.p, P.d, T(1.0 / P.sigma), pts, side, pts,
                   side, xb, o_gstride, P.m_pad, part, o_gstride, P.m_pad, Rc, s, splits, stride);
  k_sum_parts<<<ceil_div(stride, 256), 256, 0, s>>>(reinterpret_cast<const double*>(part), splits, stride, stride,
                                                     o_gstride, P.m_pad, Rc, reinterpret_cast<double*>(ynear));
}

// ---- symmetric float64 near field -------------------------------------

constexpr int kSymMaxRc = 4;

// Per row T of the near list: entries with S >= T (upper) and S < T (lower).
// One warp per leaf t: the counts of its upper (s >= t) and lower entries.
__global__ void k_sym_count(const int32_t* rowptr, const int32_t* col, int L, int* nup, int* nlo) {
  const int t = static_cast<int>((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= L) return;
  int u = 0, l = 0;
  for (int e = rowptr[t] + lane; e < rowptr[t + 1]; e += 32) (col[e] >= t ? u : l) += 1;
  for (int o = 16; o > 0; o >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, o);
    l += __shfl_xor_sync(0xffffffffu, l, o);
  }
  if (lane == 0) {
    nup[t] = u;
    nlo[t] = l;
  }
}

// One warp per leaf t: its upper and lower entries in list order (a ballot
// per 32 entries keeps the order, so every upper row stays sorted by source).
__global__ void k_sym_fill(const int32_t* rowptr, const int32_t* col, int L, const int32_t* uprow,
                           const int32_t* lorow, int32_t* up_t, int32_t* up_s, int32_t* lo_src) {
  const int t = static_cast<int>((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= L) return;
  const unsigned below = (1u << lane) - 1u;
  int u = uprow[t], l = lorow[t];
  const int end = rowptr[t + 1];
  for (int e0 = rowptr[t]; e0 < end; e0 += 32) {
    const int e = e0 + lane;
    const int s = e < end ? col[e] : -1;
    const bool isup = e < end && s >= t, islo = e < end && s < t;
    const unsigned mu = __ballot_sync(0xffffffffu, isup), ml = __ballot_sync(0xffffffffu, islo);
    if (isup) {
      up_t[u + __popc(mu & below)] = t;
      up_s[u + __popc(mu & below)] = s;
    }
    if (islo) lo_src[l + __popc(ml & below)] = s;
    u += __popc(mu);
    l += __popc(ml);
  }
}

// Slot of the lower entry (X, T < X): the position of (T, X) in the upper
// list (each upper row is sorted by source, so a binary search finds it); a
// missing one means the near relation is not symmetric.  One warp per leaf
// X, its lanes over X's lower entries.
__global__ void k_sym_slots(const int32_t* lorow, const int32_t* lo_src, const int32_t* uprow, const int32_t* up_s,
                            int L, int32_t* lo_slot, int* bad) {
  const int x = static_cast<int>((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (x >= L) return;
  for (int k = lorow[x] + lane; k < lorow[x + 1]; k += 32) {
    const int t = lo_src[k];
    int a = uprow[t], b = uprow[t + 1];   // first entry with up_s >= x in [a, b)
    while (a < b) {
      const int m = (a + b) >> 1;
      if (up_s[m] < x) a = m + 1;
      else b = m;
    }
    const int slot = (a < uprow[t + 1] && up_s[a] == x) ? a : -1;
    if (slot < 0) atomicExch(bad, 1);
    lo_slot[k] = slot < 0 ? 0 : slot;
  }
}

// One CTA per upper entry e = (T, S): forward sums pf[e][r][i] over the
// sources of S for target i of T; for S != T also pt[e][r][j] = sum over
// the targets of T of phi * x_T for source j of S.  Leaves hold <= 128
// points (one target per thread).
template <int KER, int DM, int RC>
__global__ void __launch_bounds__(kThreads)
k_near_sym(const int32_t* up_t, const int32_t* up_s, int d, double inv_sigma, const double* pts, int64_t gstride,
           int ld, const int32_t* count, int count_off, const double* xb, int64_t q_gstride, int Rc, double* pf,
           double* pt) {
  __shared__ double sc[DM * kSrcChunk];
  __shared__ double sqs[RC * kSrcChunk];
  __shared__ double zw[4 * RC * kSrcChunk];
  const int64_t e = blockIdx.x;
  const int T = up_t[e], S = up_s[e];
  const int tcnt = count[count_off + T], scnt = count[count_off + S];
  const int i = threadIdx.x, warp = i >> 5, lane = i & 31;
  double xt[DM], qt[RC], acc[RC];
#pragma unroll
  for (int k = 0; k < DM; ++k) xt[k] = (k < d && i < tcnt) ? pts[T * gstride + static_cast<int64_t>(k) * ld + i] : 0.0;
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    qt[r] = (r < Rc && i < tcnt) ? xb[T * q_gstride + static_cast<int64_t>(r) * ld + i] : 0.0;
    acc[r] = 0.0;
  }
  const bool transposed = S != T;
  for (int cb = 0; cb < scnt; cb += kSrcChunk) {
    const int cn = min(kSrcChunk, scnt - cb);
    __syncthreads();
    for (int idx = i; idx < DM * kSrcChunk; idx += kThreads) {
      const int k = idx / kSrcChunk, j = idx % kSrcChunk;
      sc[idx] = (j < cn && k < d) ? pts[S * gstride + static_cast<int64_t>(k) * ld + cb + j] : 0.0;
    }
    for (int idx = i; idx < RC * kSrcChunk; idx += kThreads) {
      const int r = idx / kSrcChunk, j = idx % kSrcChunk;
      sqs[idx] = (j < cn && r < Rc) ? xb[S * q_gstride + static_cast<int64_t>(r) * ld + cb + j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < cn; ++j) {
      double r2 = 0.0;
#pragma unroll
      for (int k = 0; k < DM; ++k) {
        const double df = xt[k] - sc[k * kSrcChunk + j];
        r2 += df * df;
      }
      const double ph = phi_r2<double, KER>(r2, inv_sigma);
#pragma unroll
      for (int r = 0; r < RC; ++r) acc[r] += ph * sqs[r * kSrcChunk + j];
      if (transposed) {
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          double v = ph * qt[r];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          if (lane == 0) zw[(warp * RC + r) * kSrcChunk + j] = v;
        }
      }
    }
    if (transposed) {
      __syncthreads();
      if (i < cn) {
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          if (r >= Rc) break;
          const double v = ((zw[(0 * RC + r) * kSrcChunk + i] + zw[(1 * RC + r) * kSrcChunk + i]) +
                            zw[(2 * RC + r) * kSrcChunk + i]) +
                           zw[(3 * RC + r) * kSrcChunk + i];
          pt[(e * Rc + r) * ld + cb + i] = v;
        }
      }
    }
  }
  if (transposed) {   // sources of the padding: zero, so the sum over partials may run to ld
    for (int j = scnt + i; j < ld; j += kThreads)
      for (int r = 0; r < Rc; ++r) pt[(e * Rc + r) * ld + j] = 0.0;
  }
  if (i < ld) {
#pragma unroll
    for (int r = 0; r < RC; ++r)
      if (r < Rc) pf[(e * Rc + r) * ld + i] = acc[r];
  }
}

// y[X][r][i] = sum of X's forward partials, then of the transposed partials
// of its lower entries, each in list order.
__global__ void k_sym_reduce(const int32_t* uprow, const int32_t* lorow, const int32_t* lo_slot, int L, int ld,
                             int Rc, const double* pf, const double* pt, double* y, int64_t o_gstride) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= static_cast<int64_t>(L) * Rc * ld) return;
  const int i = static_cast<int>(t % ld);
  const int r = static_cast<int>((t / ld) % Rc);
  const int x = static_cast<int>(t / (static_cast<int64_t>(ld) * Rc));
  double acc = 0.0;
  for (int e = uprow[x]; e < uprow[x + 1]; ++e) acc += pf[(static_cast<int64_t>(e) * Rc + r) * ld + i];
  for (int k = lorow[x]; k < lorow[x + 1]; ++k) acc += pt[(static_cast<int64_t>(lo_slot[k]) * Rc + r) * ld + i];
  y[x * o_gstride + static_cast<int64_t>(r) * ld + i] = acc;
}

template <int KER, int DM>
void launch_near_sym_rc(Plan& P, int Rc, cudaStream_t s) {
  const int64_t gs = static_cast<int64_t>(P.d) * P.m_pad;
  const int64_t qg = static_cast<int64_t>(kRC) * P.m_pad;
#define DW_SYM(RCV)                                                                                                k_near_sym<KER, DM, RCV><<<static_cast<unsigned>(P.sym_nup), kThreads, 0, s>>>(                                      P.sym_t.p, P.sym_s.p, P.d, 1.0 / P.sigma, P.d_pts64.p, gs, P.m_pad, P.d_count.p, P.L - 1, P.xb64.p, qg, Rc,       P.sym_pf.p, P.sym_pt.p)
  if (Rc <= 1) DW_SYM(1);
  else DW_SYM(kSymMaxRc);
#undef DW_SYM
}

template <int KER>
void launch_near_sym_k(Plan& P, int Rc, cudaStream_t s) {
  if (P.d <= 4) launch_near_sym_rc<KER, 4>(P, Rc, s);
  else if (P.d <= 8) launch_near_sym_rc<KER, 8>(P, Rc, s);
  else if (P.d <= 12) launch_near_sym_rc<KER, 12>(P, Rc, s);
  else if (P.d <= 16) launch_near_sym_rc<KER, 16>(P, Rc, s);
  else launch_near_sym_rc<KER, 20>(P, Rc, s);
}

// Partial sums of the symmetric form: 2 x upper entries x RHS x leaf doubles;
// above this the list kernel runs instead.
constexpr size_t kSymMaxBytes = size_t(8) << 30;

bool near_sym(Plan& P, int Rc, cudaStream_t s) {
  if (!P.sym_ok || Rc > kSymMaxRc || P.m_pad > kThreads || P.d > 20 || P.sym_nup <= 0) return false;
  const size_t per = static_cast<size_t>(P.sym_nup) * Rc * P.m_pad;
  if (2 * per * sizeof(double) > kSymMaxBytes) return false;
  P.sym_pf.alloc(per);
  P.sym_pt.alloc(per);
  switch (P.kernel) {
    case DWFMM_K_EXP: launch_near_sym_k<DWFMM_K_EXP>(P, Rc, s); break;
    case DWFMM_K_MATERN32: launch_near_sym_k<DWFMM_K_MATERN32>(P, Rc, s); break;
    default: launch_near_sym_k<DWFMM_K_GAUSS>(P, Rc, s);
  }
  const int64_t n = static_cast<int64_t>(P.L) * Rc * P.m_pad;
  k_sym_reduce<<<ceil_div(n, 256), 256, 0, s>>>(P.sym_uprow.p, P.sym_lorow.p, P.sym_loslot.p, P.L, P.m_pad, Rc,
                                                 P.sym_pf.p, P.sym_pt.p, P.ynear64.p,
                                                 static_cast<int64_t>(kRC) * P.m_pad);
  return true;
}

}  // namespace

uint64_t device_bit() {
  int dev = 0;
  DW_CUDA(cudaGetDevice(&dev));
  return dev < 64 ? (uint64_t(1) << dev) : 0;
}

// Upper / lower near lists of the symmetric float64 near field (tree build).
void build_sym_lists(Plan& P) {
  P.sym_ok = false;
  P.sym_nup = 0;
  const int L = P.L;
  if (P.N == 0 || L <= 0 || P.nnear <= 0) return;
  cudaStream_t s = P.stream;
  DBuf<int> cu, cl, bad;
  cu.alloc(L);
  cl.alloc(L);
  bad.alloc(1);
  DW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  const int warps_grid = ceil_div(static_cast<int64_t>(L) * 32, 128);   // one warp per leaf
  k_sym_count<<<warps_grid, 128, 0, s>>>(P.d_near_rowptr.p, P.d_near_col.p, L, cu.p, cl.p);
  std::vector<int> hu(L), hl(L);
  DW_CUDA(cudaMemcpyAsync(hu.data(), cu.p, sizeof(int) * L, cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaMemcpyAsync(hl.data(), cl.p, sizeof(int) * L, cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> up(L + 1, 0), lo(L + 1, 0);
  for (int t = 0; t < L; ++t) {
    up[t + 1] = up[t] + hu[t];
    lo[t + 1] = lo[t] + hl[t];
  }
  const int64_t nup = up[L], nlo = lo[L];
  // a symmetric relation with every leaf near itself has nup = nlo + L
  if (nup != nlo + L) return;
  P.sym_uprow.alloc(L + 1);
  P.sym_lorow.alloc(L + 1);
  P.sym_t.alloc(static_cast<size_t>(nup));
  P.sym_s.alloc(static_cast<size_t>(nup));
  P.sym_loslot.alloc(static_cast<size_t>(std::max<int64_t>(nlo, 1)));
  DBuf<int32_t> lo_src;
  lo_src.alloc(static_cast<size_t>(std::max<int64_t>(nlo, 1)));
  DW_CUDA(cudaMemcpyAsync(P.sym_uprow.p, up.data(), sizeof(int32_t) * (L + 1), cudaMemcpyHostToDevice, s));
  DW_CUDA(cudaMemcpyAsync(P.sym_lorow.p, lo.data(), sizeof(int32_t) * (L + 1), cudaMemcpyHostToDevice, s));
  k_sym_fill<<<warps_grid, 128, 0, s>>>(P.d_near_rowptr.p, P.d_near_col.p, L, P.sym_uprow.p, P.sym_lorow.p,
                                        P.sym_t.p, P.sym_s.p, lo_src.p);
  k_sym_slots<<<warps_grid, 128, 0, s>>>(P.sym_lorow.p, lo_src.p, P.sym_uprow.p, P.sym_s.p, L, P.sym_loslot.p,
                                         bad.p);
  int hbad = 0;
  DW_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  DW_CUDA(cudaGetLastError());
  if (hbad) return;
  P.sym_nup = nup;
  P.sym_ok = true;
  sym_tc_order(P, hu);
}

// Upper entries (t, s > t) of the far list (Eq. (5.1): admissible pairs of
// one level, both orderings listed) for the symmetric tensor-core M2L: rows
// by target cluster, sorted by source like the list; target clusters ordered
// by decreasing upper-row length, the ones with entries first.  The relation
// must be symmetric (checked through the slots of the lower entries) and
// holds no diagonal entry.
void build_far_sym_lists(Plan& P) {
  P.fsym_ok = false;
  P.fsym_rows = 0;
  const int C = P.C;
  if (P.N == 0 || C <= 0 || P.nfar <= 0) return;
  cudaStream_t s = P.stream;
  DBuf<int> cu, cl, bad;
  cu.alloc(C);
  cl.alloc(C);
  bad.alloc(1);
  DW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  const int warps_grid = ceil_div(static_cast<int64_t>(C) * 32, 128);   // one warp per cluster
  k_sym_count<<<warps_grid, 128, 0, s>>>(P.d_far_rowptr.p, P.d_far_col.p, C, cu.p, cl.p);
  std::vector<int> hu(C), hl(C);
  DW_CUDA(cudaMemcpyAsync(hu.data(), cu.p, sizeof(int) * C, cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaMemcpyAsync(hl.data(), cl.p, sizeof(int) * C, cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> up(C + 1, 0), lo(C + 1, 0);
  for (int t = 0; t < C; ++t) {
    up[t + 1] = up[t] + hu[t];
    lo[t + 1] = lo[t] + hl[t];
  }
  const int64_t nup = up[C], nlo = lo[C];
  if (nup != nlo || nup <= 0) return;   // a symmetric relation without diagonal entries
  P.fsym_uprow.alloc(C + 1);
  P.fsym_s.alloc(static_cast<size_t>(nup));
  DBuf<int32_t> lorow, up_t, lo_src, lo_slot;
  lorow.alloc(C + 1);
  up_t.alloc(static_cast<size_t>(nup));
  lo_src.alloc(static_cast<size_t>(nlo));
  lo_slot.alloc(static_cast<size_t>(nlo));
  DW_CUDA(cudaMemcpyAsync(P.fsym_uprow.p, up.data(), sizeof(int32_t) * (C + 1), cudaMemcpyHostToDevice, s));
  DW_CUDA(cudaMemcpyAsync(lorow.p, lo.data(), sizeof(int32_t) * (C + 1), cudaMemcpyHostToDevice, s));
  k_sym_fill<<<warps_grid, 128, 0, s>>>(P.d_far_rowptr.p, P.d_far_col.p, C, P.fsym_uprow.p, lorow.p, up_t.p,
                                        P.fsym_s.p, lo_src.p);
  k_sym_slots<<<warps_grid, 128, 0, s>>>(lorow.p, lo_src.p, P.fsym_uprow.p, P.fsym_s.p, C, lo_slot.p, bad.p);
  int hbad = 0;
  DW_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  DW_CUDA(cudaGetLastError());
  if (hbad) return;
  std::vector<int32_t> ord(C);
  for (int i = 0; i < C; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return hu[x] > hu[y]; });
  int rows = 0;
  while (rows < C && hu[ord[rows]] > 0) ++rows;
  P.fsym_order.alloc(C);
  DW_CUDA(cudaMemcpyAsync(P.fsym_order.p, ord.data(), sizeof(int32_t) * C, cudaMemcpyHostToDevice, s));
  DW_CUDA(cudaStreamSynchronize(s));
  P.fsym_rows = rows;
  P.fsym_ok = true;
}

// Every target block against every source leaf in float64 (exact evaluation).
void eval_f64(Plan& P, const double* tgt64, int G, const int32_t* rowptr, const int32_t* col, int Rc, double* out,
              cudaStream_t s) {
  const int64_t gs = static_cast<int64_t>(P.d) * P.m_pad;
  Side ts{gs, P.m_pad, nullptr, 0, P.m_pad};
  Side ss{gs, P.m_pad, P.d_count.p, P.L - 1, 0};
  dispatch_ksum<double>(P.kernel, G, 0, rowptr, col, P.d, 1.0 / P.sigma, tgt64, ts, P.d_pts64.p, ss, P.xb64.p,
                        static_cast<int64_t>(kRC) * P.m_pad, P.m_pad, out, static_cast<int64_t>(kRC) * P.m_pad,
                        P.m_pad, Rc, s);
}

void launch_m2l(Plan& P, int Rc, bool fp64) {
  if (P.jmin > P.J) return;
  if (fp64) {
    P.m2l_engine = 0;
    m2l_impl<double>(P, Rc, P.d_ynode64.p, P.mom64.p, P.loc64.p);
  } else if (!m2l_f32_tuned(P, Rc)) {
    P.m2l_engine = 1;
    m2l_impl<float>(P, Rc, P.d_ynode32.p, P.mom32.p, P.loc32.p);
  }
  DW_CUDA(cudaGetLastError());
}

void launch_nearfield(Plan& P, int Rc, bool fp64, cudaStream_t s) {
  if (fp64) {
    P.near_engine = 1;
    if (!near_sym(P, Rc, s)) {
      P.near_engine = 0;
      p2p_impl<double>(P, Rc, P.d_pts64.p, P.xb64.p, P.ynear64.p, s);
    }
  } else if (!p2p_f32_tuned(P, Rc, s)) {
    P.near_engine = 2;
    p2p_impl<float>(P, Rc, P.d_pts32.p, P.xb32.p, P.ynear32.p, s);
  }
  DW_CUDA(cudaGetLastError());
}

}  // namespace dw
