// Tuned float32 kernel summation for sm_103a: the P2P near field and the M2L
// couplings of the DW-FMM (Sec. 5.2), y_i = sum_j phi(|x_i - x_j| / sigma) q_j.
//
// Design (one CTA per target group: a leaf, or a cluster's node set):
//  - Source blocks (scaled coordinates plus a norm row, then R charge rows)
//    are contiguous and 32-byte aligned in HBM, so each block is two 1-D TMA
//    bulk copies (cp.async.bulk, mbarrier completion) into a double-buffered
//    shared-memory stage; thread 0 issues, every thread waits with a bounded
//    try_wait loop that raises an error flag instead of hanging.
//  - Each thread owns TT targets; sources are read as float4 broadcasts from
//    shared memory, 4 sources per step.
//  - The kernel constants are folded into the coordinates when the source
//    blocks are built:
//      Gaussian:  x' = x sqrt(log2 e / (2 sigma^2)),  phi = ex2(2 x'.s' - |x'|^2 - |s'|^2)
//      exp:       x' = x log2 e / sigma,               phi = ex2(-|x' - s'|)
//      Matern:    x' = x sqrt3 / sigma,                phi = (1 + r') ex2(-r' log2 e)
//    so the Gaussian costs D FMAs, one add and one MUFU.EX2 per pair.
//  - Arithmetic is packed: fma/add/sub.f32x2 (two lanes per instruction) for
//    distances and accumulation; charges are interleaved per source.
//  - Per source block the contributions are summed in float32 partials, then
//    folded into per-target running sums with Kahan compensation (kept in
//    shared memory).
#include <atomic>
#include <cstdint>
#include <string>

#include "dwfmm_internal.cuh"
#include "sum_f32.cuh"

namespace dw {

namespace {

using namespace sk;

// One CTA per target group g = a.first + blockIdx.x (the whole CTA is the group).
template <int D, int RC, int KER>
__global__ void __launch_bounds__(kThreadsMax, 3) k_sum_f32(SumArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[2];
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int tile_base = 0;
  const Grp G{static_cast<int>(threadIdx.x), static_cast<int>(blockDim.x), 0};
  (void)sum_block<D, RC, KER>(a, a.first + static_cast<int>(blockIdx.x), G, smem, full, tile_base);
}

// Row layout [g][16][ld] -> interleaved [g][ld][RC] (first RC rows).
__global__ void k_interleave(const float* src, int64_t groups, int ld, int RC, float* dst) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= groups * ld * RC) return;
  interleave_elem(src, ld, RC, dst, t);
}

// Scaled source blocks [g][D+1][ld] from float64 coordinates [g][d][ld].
__global__ void k_scaled_blocks(const double* src, int64_t groups, int d, int D, int ld, int kernel,
                                double sigma, float* dst) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= groups * ld) return;
  const int64_t g = t / ld;
  const int i = static_cast<int>(t % ld);
  double scale;
  if (kernel == DWFMM_K_GAUSS) scale = sqrt(1.4426950408889634 / (2.0 * sigma * sigma));
  else if (kernel == DWFMM_K_EXP) scale = 1.4426950408889634 / sigma;
  else scale = 1.7320508075688772 / sigma;
  double n2 = 0.0;
  for (int k = 0; k < D; ++k) {
    const double v = k < d ? src[(g * d + k) * ld + i] * scale : 0.0;
    const float f = static_cast<float>(v);
    dst[(g * (D + 1) + k) * ld + i] = f;
    n2 += static_cast<double>(f) * static_cast<double>(f);
  }
  dst[(g * (D + 1) + D) * ld + i] = static_cast<float>(n2);
}

template <int D, int RC>
void launch_kernel_type(int kernel, SumArgs a, int groups, int threads, size_t smem, cudaStream_t s) {
  switch (kernel) {
    case DWFMM_K_EXP:
      k_sum_f32<D, RC, DWFMM_K_EXP><<<groups, threads, smem, s>>>(a);
      break;
    case DWFMM_K_MATERN32:
      k_sum_f32<D, RC, DWFMM_K_MATERN32><<<groups, threads, smem, s>>>(a);
      break;
    default:
      k_sum_f32<D, RC, DWFMM_K_GAUSS><<<groups, threads, smem, s>>>(a);
  }
}

template <int D>
void launch_rc(int kernel, int RC, SumArgs a, int groups, int threads, size_t smem, cudaStream_t s) {
  if (RC <= 1) launch_kernel_type<D, 1>(kernel, a, groups, threads, smem, s);
  else if (RC <= 4) launch_kernel_type<D, 4>(kernel, a, groups, threads, smem, s);
  else if (RC <= 8) launch_kernel_type<D, 8>(kernel, a, groups, threads, smem, s);
  else launch_kernel_type<D, 16>(kernel, a, groups, threads, smem, s);
}

template <int D>
void set_attrs() {
  const int big = 200 * 1024;
#define DW_ATTR(RC)                                                                                           \
  cudaFuncSetAttribute(k_sum_f32<D, RC, DWFMM_K_EXP>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);      \
  cudaFuncSetAttribute(k_sum_f32<D, RC, DWFMM_K_MATERN32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); \
  cudaFuncSetAttribute(k_sum_f32<D, RC, DWFMM_K_GAUSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  DW_ATTR(1)
  DW_ATTR(4)
  DW_ATTR(8)
  DW_ATTR(16)
#undef DW_ATTR
}

int padded_dim(int d) {
  if (d <= 4) return 4;
  if (d <= 8) return 8;
  if (d <= 10) return 10;
  if (d <= 12) return 12;
  if (d <= 16) return 16;
  if (d <= 20) return 20;
  return -1;
}

int padded_rc(int Rc) { return Rc <= 1 ? 1 : Rc <= 4 ? 4 : Rc <= 8 ? 8 : 16; }

void dispatch(int D, int kernel, int RC, SumArgs a, int groups, int threads, size_t smem, cudaStream_t s) {
  switch (D) {
    case 4: launch_rc<4>(kernel, RC, a, groups, threads, smem, s); break;
    case 8: launch_rc<8>(kernel, RC, a, groups, threads, smem, s); break;
    case 10: launch_rc<10>(kernel, RC, a, groups, threads, smem, s); break;
    case 12: launch_rc<12>(kernel, RC, a, groups, threads, smem, s); break;
    case 16: launch_rc<16>(kernel, RC, a, groups, threads, smem, s); break;
    default: launch_rc<20>(kernel, RC, a, groups, threads, smem, s); break;
  }
}

// Devices whose kernel attributes are set.  Atomic: host threads may make
// their first call on a device at the same time (both then set the same
// attributes, which is harmless).
std::atomic<uint64_t> g_attrs_dev{0};

void ensure_attrs() {
  const uint64_t bit = device_bit();
  if (g_attrs_dev.load() & bit) return;
  set_attrs<4>();
  set_attrs<8>();
  set_attrs<10>();
  set_attrs<12>();
  set_attrs<16>();
  set_attrs<20>();
  DW_CUDA(cudaGetLastError());
  g_attrs_dev.fetch_or(bit);
}

// Scaled blocks for the current tree: leaf sites and cluster nodes.
void ensure_scaled(Plan& P, int D) {
  if (P.dpad == D && P.d_ptsk.p && P.d_ynodek.p) return;
  const int64_t nl = static_cast<int64_t>(P.L) * (D + 1) * P.m_pad;
  const int64_t nc = static_cast<int64_t>(P.C) * (D + 1) * P.n_pad;
  P.d_ptsk.alloc(nl);
  P.d_ynodek.alloc(nc);
  k_scaled_blocks<<<ceil_div(static_cast<int64_t>(P.L) * P.m_pad, 256), 256, 0, P.stream>>>(
      P.d_pts64.p, P.L, P.d, D, P.m_pad, P.kernel, P.sigma, P.d_ptsk.p);
  k_scaled_blocks<<<ceil_div(static_cast<int64_t>(P.C) * P.n_pad, 256), 256, 0, P.stream>>>(
      P.d_ynode64.p, P.C, P.d, D, P.n_pad, P.kernel, P.sigma, P.d_ynodek.p);
  DW_CUDA(cudaGetLastError());
  P.dpad = D;
}

size_t stage_bytes(int D, int RC, int ld) {
  const size_t comp = static_cast<size_t>(kTT) * (RC >= 2 ? RC / 2 : 1) * kThreadsMax * sizeof(unsigned long long);
  return 2 * static_cast<size_t>((D + 1) * ld + RC * ld) * sizeof(float) + comp;
}

}  // namespace

int sum_padded_dim(int d) { return padded_dim(d); }
int sum_padded_rc(int r) { return padded_rc(r); }
size_t sum_stage_bytes(int D, int RC, int ld) { return stage_bytes(D, RC, ld); }
void ensure_sum_attrs() { ensure_attrs(); }

void launch_sum_f32(int D, int kernel, int RC, const SumArgs& a, int groups, int threads, size_t smem,
                    cudaStream_t s) {
  if (groups > 0) dispatch(D, kernel, RC, a, groups, threads, smem, s);
}

void launch_interleave(const float* src, int64_t groups, int ld, int RC, float* dst, cudaStream_t s) {
  const int64_t nq = groups * ld * RC;
  if (nq > 0) k_interleave<<<ceil_div(nq, 256), 256, 0, s>>>(src, groups, ld, RC, dst);
}

void launch_scaled_blocks(const double* src, int64_t groups, int d, int D, int ld, int kernel, double sigma,
                          float* dst, cudaStream_t s) {
  if (groups > 0)
    k_scaled_blocks<<<ceil_div(groups * ld, 256), 256, 0, s>>>(src, groups, d, D, ld, kernel, sigma, dst);
}

bool p2p_f32_tuned(Plan& P, int Rc, cudaStream_t s) {
  const int D = padded_dim(P.d);
  if (D < 0) return false;
  const int RC = padded_rc(Rc);
  const size_t smem = stage_bytes(D, RC, P.m_pad);
  if (smem > 200 * 1024) return false;
  ensure_attrs();
  ensure_scaled(P, D);
  // the tree build made the scaled blocks on P.stream; the side stream waits
  if (s != P.stream) {
    DW_CUDA(cudaEventRecord(P.ev_scaled, P.stream));
    DW_CUDA(cudaStreamWaitEvent(s, P.ev_scaled, 0));
  }
  P.xq32.alloc(static_cast<size_t>(P.L) * P.m_pad * kRC);
  const int64_t nq = static_cast<int64_t>(P.L) * P.m_pad * RC;
  k_interleave<<<ceil_div(nq, 256), 256, 0, s>>>(P.xb32.p, P.L, P.m_pad, RC, P.xq32.p);
  // MIXED plans with 9..16 right-hand sides: contraction on the tensor cores,
  // each unordered near pair once where the symmetric kernel applies
  P.near_engine = 4;
  if (P.prec == DWFMM_P_MIXED && RC == 16 && near_sym_tc(P, D, Rc, s)) return true;
  P.near_engine = 3;
  if (P.prec == DWFMM_P_MIXED && RC == 16 &&
      sum_tc(D, P.kernel, P.d_ptsk.p, static_cast<int64_t>(D + 1) * P.m_pad, P.d_ptsk.p,
             static_cast<int64_t>(D + 1) * P.m_pad, P.xq32.p, P.L, P.bq32, P.ynear32.p,
             static_cast<int64_t>(kRC) * P.m_pad, P.d_near_rowptr.p, P.d_near_col.p, P.d_count.p, P.L - 1, 0, 0,
             P.L, P.m_pad, Rc, P.gauss_fact, P.d_err.p, s))
    return true;
  P.near_engine = 2;
  SumArgs a{};
  a.tgt = P.d_ptsk.p;
  a.tgt_gstride = static_cast<int64_t>(D + 1) * P.m_pad;
  a.src = P.d_ptsk.p;
  a.src_gstride = a.tgt_gstride;
  a.q = P.xq32.p;
  a.q_gstride = static_cast<int64_t>(RC) * P.m_pad;
  a.out = P.ynear32.p;
  a.out_gstride = static_cast<int64_t>(kRC) * P.m_pad;
  a.rowptr = P.d_near_rowptr.p;
  a.col = P.d_near_col.p;
  a.count = P.d_count.p;
  a.count_off = P.L - 1;
  a.count_const = 0;
  a.first = 0;
  a.ld = P.m_pad;
  a.Rc = Rc;
  a.err = P.d_err.p;
  const int threads = std::min(kThreadsMax, round_up(ceil_div(P.m_pad, kTT), 32));
  dispatch(D, P.kernel, RC, a, P.L, threads, smem, s);
  DW_CUDA(cudaGetLastError());
  return true;
}

// Every target block against every source leaf in float32 (exact evaluation);
// falls back to the generic kernel when d > 20.
void eval_f32(Plan& P, const double* tgt64, int G, const int32_t* rowptr, const int32_t* col, int Rc, float* out,
              DBuf<float>& scratch, cudaStream_t s) {
  const int D = padded_dim(P.d);
  if (D < 0) fail(DWFMM_ERR_INVALID_ARG, "evaluation in float32 needs d <= 20");
  const int RC = padded_rc(Rc);
  ensure_attrs();
  ensure_scaled(P, D);
  scratch.alloc(static_cast<size_t>(G) * (D + 1) * P.m_pad);
  k_scaled_blocks<<<ceil_div(static_cast<int64_t>(G) * P.m_pad, 256), 256, 0, s>>>(tgt64, G, P.d, D, P.m_pad, P.kernel,
                                                                                  P.sigma, scratch.p);
  P.xq32.alloc(static_cast<size_t>(P.L) * P.m_pad * kRC);
  const int64_t nq = static_cast<int64_t>(P.L) * P.m_pad * RC;
  k_interleave<<<ceil_div(nq, 256), 256, 0, s>>>(P.xb32.p, P.L, P.m_pad, RC, P.xq32.p);
  SumArgs a{};
  a.tgt = scratch.p;
  a.tgt_gstride = static_cast<int64_t>(D + 1) * P.m_pad;
  a.src = P.d_ptsk.p;
  a.src_gstride = a.tgt_gstride;
  a.q = P.xq32.p;
  a.q_gstride = static_cast<int64_t>(RC) * P.m_pad;
  a.out = out;
  a.out_gstride = static_cast<int64_t>(kRC) * P.m_pad;
  a.rowptr = rowptr;
  a.col = col;
  a.count = P.d_count.p;
  a.count_off = P.L - 1;
  a.count_const = 0;
  a.first = 0;
  a.ld = P.m_pad;
  a.Rc = Rc;
  a.err = P.d_err.p;
  const int threads = std::min(kThreadsMax, round_up(ceil_div(P.m_pad, kTT), 32));
  dispatch(D, P.kernel, RC, a, G, threads, stage_bytes(D, RC, P.m_pad), s);
  DW_CUDA(cudaGetLastError());
}

namespace {

// The ordered-pair tensor-core M2L (every far block, both orderings):
// interleaved moments, then the kernel-summation engine on node sets.
bool m2l_ordered_tc(Plan& P, int D, int Rc) {
  const int first = (1 << P.jmin) - 1;
  P.momq32.alloc(static_cast<size_t>(P.C) * P.n_pad * kRC);
  const int64_t nq = static_cast<int64_t>(P.C) * P.n_pad * 16;
  k_interleave<<<ceil_div(nq, 256), 256, 0, P.stream>>>(P.mom32.p, P.C, P.n_pad, 16, P.momq32.p);
  // own charge-block scratch: the near field runs concurrently on the side stream
  return sum_tc(D, P.kernel, P.d_ynodek.p, static_cast<int64_t>(D + 1) * P.n_pad, P.d_ynodek.p,
                static_cast<int64_t>(D + 1) * P.n_pad, P.momq32.p, P.C, P.bqm32, P.loc32.p,
                static_cast<int64_t>(kRC) * P.n_pad, P.d_far_rowptr.p, P.d_far_col.p, nullptr, 0, P.n, first,
                P.C - first, P.n_pad, Rc, P.gauss_fact, P.d_err.p, P.stream);
}

}  // namespace

// MIXED plans with 9..16 right-hand sides have two tensor-core M2L engines
// (every ordered far pair, TF32 hi/lo; each unordered pair once, FP16 hi/lo
// with fixed-point transposed sums).  Unless the caller chose one, the
// first such matvec of a tree times both on the plan's moments buffer (set
// to zero; values do not change the time) before the near field starts,
// and the faster is kept for the tree.  Not while the stream is being
// captured or the phase timers run (the ordered engine then).
void m2l_autotune(Plan& P, int Rc) {
  if (P.prec != DWFMM_P_MIXED || Rc < 9 || Rc > 16 || P.m2l_pref >= 0 || P.m2l_tuned >= 0) return;
  if (P.jmin > P.J || P.tm.on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DW_CUDA(cudaStreamIsCapturing(P.stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return;
  const int D = padded_dim(P.d);
  if (D < 0 || stage_bytes(D, 16, P.n_pad) > 200 * 1024) return;
  ensure_attrs();
  ensure_scaled(P, D);
  DW_CUDA(cudaMemsetAsync(P.mom32.p, 0, static_cast<size_t>(P.C) * kRC * P.n_pad * sizeof(float), P.stream));
  cudaEvent_t e0, e1, e2;
  DW_CUDA(cudaEventCreate(&e0));
  DW_CUDA(cudaEventCreate(&e1));
  DW_CUDA(cudaEventCreate(&e2));
  DW_CUDA(cudaEventRecord(e0, P.stream));
  const bool sym = m2l_sym_tc(P, D, Rc, P.stream);
  DW_CUDA(cudaEventRecord(e1, P.stream));
  const bool ord = m2l_ordered_tc(P, D, Rc);
  DW_CUDA(cudaEventRecord(e2, P.stream));
  DW_CUDA(cudaEventSynchronize(e2));
  float ms_sym = 0.f, ms_ord = 0.f;
  DW_CUDA(cudaEventElapsedTime(&ms_sym, e0, e1));
  DW_CUDA(cudaEventElapsedTime(&ms_ord, e1, e2));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  P.m2l_tune_ms[0] = sym ? ms_sym : -1.0;
  P.m2l_tune_ms[1] = ord ? ms_ord : -1.0;
  P.m2l_tuned = (sym && (!ord || ms_sym < ms_ord)) ? 3 : 2;
}

bool m2l_f32_tuned(Plan& P, int Rc) {
  const int D = padded_dim(P.d);
  if (D < 0) return false;
  const int RC = padded_rc(Rc);
  const size_t smem = stage_bytes(D, RC, P.n_pad);
  if (smem > 200 * 1024) return false;
  ensure_attrs();
  ensure_scaled(P, D);
  if (P.prec == DWFMM_P_MIXED && RC == 16) {
    const int want = P.m2l_pref >= 0 ? P.m2l_pref : (P.m2l_tuned >= 0 ? P.m2l_tuned : 2);
    if (want == 3 && m2l_sym_tc(P, D, Rc, P.stream)) {
      P.m2l_engine = 3;
      return true;
    }
    if (m2l_ordered_tc(P, D, Rc)) {
      P.m2l_engine = 2;
      return true;
    }
  }
  const int first = (1 << P.jmin) - 1;
  P.momq32.alloc(static_cast<size_t>(P.C) * P.n_pad * kRC);
  const int64_t nq = static_cast<int64_t>(P.C) * P.n_pad * RC;
  k_interleave<<<ceil_div(nq, 256), 256, 0, P.stream>>>(P.mom32.p, P.C, P.n_pad, RC, P.momq32.p);
  P.m2l_engine = 1;
  SumArgs a{};
  a.tgt = P.d_ynodek.p;
  a.tgt_gstride = static_cast<int64_t>(D + 1) * P.n_pad;
  a.src = P.d_ynodek.p;
  a.src_gstride = a.tgt_gstride;
  a.q = P.momq32.p;
  a.q_gstride = static_cast<int64_t>(RC) * P.n_pad;
  a.out = P.loc32.p;
  a.out_gstride = static_cast<int64_t>(kRC) * P.n_pad;
  a.rowptr = P.d_far_rowptr.p;
  a.col = P.d_far_col.p;
  a.count = nullptr;
  a.count_off = 0;
  a.count_const = P.n;
  a.first = first;
  a.ld = P.n_pad;
  a.Rc = Rc;
  a.err = P.d_err.p;
  const int threads = std::min(kThreadsMax, round_up(ceil_div(P.n_pad, kTT), 32));
  dispatch(D, P.kernel, RC, a, P.C - first, threads, smem, P.stream);
  DW_CUDA(cudaGetLastError());
  return true;
}


// ---------------------------------------------------------------------------
// Allocation-free direct sum (dwfmm_direct_sum_noalloc).
//
// Some callers cannot call cudaMalloc: host applications whose framework
// owns the device memory pool (a caching allocator that has reserved nearly
// all of it, so a fresh cudaMalloc fails or fragments the pool), and
// latency-sensitive loops that cannot afford the device synchronisation
// that cudaMalloc/cudaFree imply.  For them this entry point computes the
// exact y = K x over all N sites (no tree) with the same tuned kernel as the
// near field, and keeps every intermediate in one file-scope device array.
//
// The array is shared by every call on a device and holds the last call's
// data; each call rewrites all of it that it reads.  Calls whose work
// overlaps on the GPU (different streams, no ordering) race on it.
// ---------------------------------------------------------------------------

namespace {

constexpr int kNaBlock = 256;                       // sites per block
constexpr int kNaMaxN = 8192;                       // largest N
constexpr int kNaMaxD = 16;                         // largest d (padded dimension <= 16)
constexpr int kNaGroups = kNaMaxN / kNaBlock;       // 32
constexpr size_t kNaCoord = static_cast<size_t>(kNaGroups) * (kNaMaxD + 1) * kNaBlock;
constexpr size_t kNaCharge = static_cast<size_t>(kNaGroups) * kRC * kNaBlock;
constexpr size_t kNaInts = 1 + kNaGroups + 1 + kNaGroups + static_cast<size_t>(kNaGroups) * kNaGroups;
constexpr size_t kNaFloats = kNaCoord + 2 * kNaCharge + kNaInts;

static __device__ __align__(256) float g_noalloc_scratch[kNaFloats];

// Scratch layout (floats): coords [G][D+1][256] | charges [G][16][256] |
// out [G][16][256] | ints: err, counts[G], rowptr[G+1], col[G*G].
struct NaLayout {
  float* coord;
  float* charge;
  float* out;
  int* err;
  int* count;
  int* rowptr;
  int* col;
};

NaLayout na_layout(float* base) {
  NaLayout l;
  l.coord = base;
  l.charge = base + kNaCoord;
  l.out = l.charge + kNaCharge;
  int* ints = reinterpret_cast<int*>(l.out + kNaCharge);
  l.err = ints;
  l.count = ints + 1;
  l.rowptr = l.count + kNaGroups;
  l.col = l.rowptr + kNaGroups + 1;
  return l;
}

// Fills every scratch entry the sum reads: scaled coordinates and norm row,
// charges (zero past N and past nrhs), counts, a complete block list, and
// clears the error flag.
__global__ void k_na_prepare(const double* pts, int64_t n, int d, int64_t ldp, int D, int kernel,
                             double sigma, const double* x, int R, int RC, int64_t ldx, NaLayout l, int G) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t == 0) *l.err = 0;
  if (t < G) {
    const int64_t rem = n - t * kNaBlock;
    l.count[t] = static_cast<int>(rem < kNaBlock ? rem : kNaBlock);
    l.rowptr[t] = static_cast<int>(t) * G;
    if (t == G - 1) l.rowptr[G] = G * G;
  }
  if (t < static_cast<int64_t>(G) * G) l.col[t] = static_cast<int>(t % G);
  if (t >= static_cast<int64_t>(G) * kNaBlock) return;
  const int g = static_cast<int>(t / kNaBlock), i = static_cast<int>(t % kNaBlock);
  const int64_t src = t < n ? t : static_cast<int64_t>(g) * kNaBlock;   // padding repeats the block's first site
  double scale;
  if (kernel == DWFMM_K_GAUSS) scale = sqrt(1.4426950408889634 / (2.0 * sigma * sigma));
  else if (kernel == DWFMM_K_EXP) scale = 1.4426950408889634 / sigma;
  else scale = 1.7320508075688772 / sigma;
  double n2 = 0.0;
  for (int k = 0; k < D; ++k) {
    const float f = k < d ? static_cast<float>(pts[src * ldp + k] * scale) : 0.0f;
    l.coord[(static_cast<int64_t>(g) * (D + 1) + k) * kNaBlock + i] = f;
    n2 += static_cast<double>(f) * static_cast<double>(f);
  }
  l.coord[(static_cast<int64_t>(g) * (D + 1) + D) * kNaBlock + i] = static_cast<float>(n2);
  for (int r = 0; r < RC; ++r)   // interleaved per site: [g][256][RC]
    l.charge[(static_cast<int64_t>(g) * kNaBlock + i) * RC + r] =
        (t < n && r < R) ? static_cast<float>(x[r * ldx + t]) : 0.0f;
}

// y[:, r] from the per-block sums; NaN if a bounded wait gave up.
__global__ void k_na_finish(NaLayout l, int64_t n, int R, double* y, int64_t ldy) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * R) return;
  const int r = static_cast<int>(t / n);
  const int64_t i = t % n;
  const int g = static_cast<int>(i / kNaBlock), j = static_cast<int>(i % kNaBlock);
  const double v = static_cast<double>(l.out[(static_cast<int64_t>(g) * kRC + r) * kNaBlock + j]);
  y[r * ldy + i] = (*l.err) ? __longlong_as_double(0x7ff8000000000000ll) : v;
}

// Device address of the scratch array.  Outside stream capture it is looked
// up on every call (cudaGetSymbolAddress allocates nothing), so a context
// that was reset still gets the right address; the last address seen per
// device serves calls made during capture, where the first call on a device
// must not load the module or set kernel attributes.
constexpr int kNaMaxDevices = 64;
std::atomic<float*> g_na_ptr[kNaMaxDevices];

float* na_scratch_for_current_device(cudaStream_t s) {
  int dev = 0;
  DW_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) fail(DWFMM_ERR_INVALID_ARG, "device index out of range");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  DW_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) {
    float* p = g_na_ptr[dev].load();
    if (!p)
      fail(DWFMM_ERR_STATE,
           "direct_sum_noalloc: the first call on a device sets it up and must come before any stream capture");
    return p;
  }
  ensure_attrs();
  void* p = nullptr;
  DW_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  g_na_ptr[dev].store(static_cast<float*>(p));
  return static_cast<float*>(p);
}

// Buffers the kernels read or write directly: device (or managed) memory of
// the current device.  A host pointer would fault on the GPU.
void na_check_device_buffer(const void* p, int dev, const char* name) {
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) (void)cudaGetLastError();
  const bool ok = e == cudaSuccess &&
                  ((a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged);
  if (!ok)
    fail(DWFMM_ERR_INVALID_ARG, std::string("direct_sum_noalloc: ") + name +
                                    " must be device memory of the current device");
}

}  // namespace

dwfmm_status direct_sum_noalloc(int kernel, double sigma, const double* pts, int64_t n, int d, int64_t ldp,
                                const double* x, double* y, int R, int64_t ldx, int64_t ldy,
                                cudaStream_t s) {
  if (kernel < 0 || kernel > 2 || !(sigma > 0.0) || n < 0 || n > kNaMaxN || d < 1 || d > kNaMaxD ||
      R < 1 || R > kRC)
    fail(DWFMM_ERR_INVALID_ARG, "direct_sum_noalloc: needs N <= 8192, 1 <= d <= 16, 1 <= nrhs <= 16");
  if (n == 0) return DWFMM_OK;
  if (!pts || !x || !y || ldp < d || ldx < n || ldy < n)
    fail(DWFMM_ERR_INVALID_ARG, "direct_sum_noalloc: NULL buffer or leading dimension too small");
  int dev = 0;
  DW_CUDA(cudaGetDevice(&dev));
  na_check_device_buffer(pts, dev, "pts");
  na_check_device_buffer(x, dev, "x");
  na_check_device_buffer(y, dev, "y");
  const int D = padded_dim(d);
  const int RC = padded_rc(R);
  const int G = static_cast<int>((n + kNaBlock - 1) / kNaBlock);
  const NaLayout l = na_layout(na_scratch_for_current_device(s));
  k_na_prepare<<<ceil_div(static_cast<int64_t>(G) * kNaBlock + G * G, 256), 256, 0, s>>>(
      pts, n, d, ldp, D, kernel, sigma, x, R, RC, ldx, l, G);
  SumArgs a{};
  a.tgt = l.coord;
  a.tgt_gstride = static_cast<int64_t>(D + 1) * kNaBlock;
  a.src = l.coord;
  a.src_gstride = a.tgt_gstride;
  a.q = l.charge;
  a.q_gstride = static_cast<int64_t>(RC) * kNaBlock;
  a.out = l.out;
  a.out_gstride = static_cast<int64_t>(kRC) * kNaBlock;
  a.rowptr = l.rowptr;
  a.col = l.col;
  a.count = l.count;
  a.count_off = 0;
  a.count_const = 0;
  a.first = 0;
  a.ld = kNaBlock;
  a.Rc = R;
  a.err = l.err;
  dispatch(D, kernel, RC, a, G, kThreadsMax, stage_bytes(D, RC, kNaBlock), s);
  k_na_finish<<<ceil_div(n * R, 256), 256, 0, s>>>(l, n, R, y, ldy);
  DW_CUDA(cudaGetLastError());
  return DWFMM_OK;
}

}  // namespace dw
