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
#include <algorithm>
#include <type_traits>

#include "dwfmm_internal.cuh"

namespace dw {

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

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    DW_CUDA(cudaGetDevice(&dev));
    DW_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
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

}  // namespace

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
  if (fp64) m2l_impl<double>(P, Rc, P.d_ynode64.p, P.mom64.p, P.loc64.p);
  else if (!m2l_f32_tuned(P, Rc)) m2l_impl<float>(P, Rc, P.d_ynode32.p, P.mom32.p, P.loc32.p);
  DW_CUDA(cudaGetLastError());
}

void launch_nearfield(Plan& P, int Rc, bool fp64, cudaStream_t s) {
  if (fp64) p2p_impl<double>(P, Rc, P.d_pts64.p, P.xb64.p, P.ynear64.p, s);
  else if (!p2p_f32_tuned(P, Rc, s)) p2p_impl<float>(P, Rc, P.d_pts32.p, P.xb32.p, P.ynear32.p, s);
  DW_CUDA(cudaGetLastError());
}

}  // namespace dw
