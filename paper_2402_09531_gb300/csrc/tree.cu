// Cluster tree (Sec. 5.1) and far/near interaction lists (Sec. 5.2, Eq. (5.1))
// built level by level on the GPU.
//
// Tree: every cluster on level j < J is split along the longest edge of its
// tight bounding box (ties: lowest k); the first child receives the
// ceil(n/2) sites that are smallest by (x_k, position), both children keep
// the parent's order.  Per level this is a segmented median selection by
// MSB-first radix select on order-preserving 64-bit keys, then a stable
// partition by two exclusive scans.  Bounding boxes are segmented min/max
// reductions with warp shuffles and one atomic per run of a segment.
//
// Lists: candidate block pairs are kept in CSR order by target cluster; a
// candidate is far if admissible, else its four child pairs become the next
// level's candidates (the rows of the children are built directly in sorted
// order), or, on the leaf level, a near pair.
//
// This file is compiled with -fmad=false so that the admissibility sums are
// plain float64 products and adds in k order.
#include <algorithm>
#include <cmath>
#include <utility>

#include "dwfmm_internal.cuh"

namespace dw {

namespace {

constexpr unsigned long long kSign = 0x8000000000000000ull;

__device__ __forceinline__ unsigned long long dkey(double x) {
  x = x + 0.0;  // -0.0 -> +0.0
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  return (u & kSign) ? ~u : (u | kSign);
}

__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  const unsigned long long u = (k & kSign) ? (k & ~kSign) : ~k;
  return __longlong_as_double(static_cast<long long>(u));
}

// ---- scans (exclusive, int32) ----------------------------------------------

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int s = lane < nw ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  const int before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void k_scan_tiles(const int* in, int* out, int64_t n, int* tile_sums) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  int total;
  int run = block_exclusive_scan(s, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_tile_sums(int* sums, int ntiles, int* grand_total) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b = 0; b < ntiles; b += blockDim.x) {
    const int i = b + threadIdx.x;
    const int v = i < ntiles ? sums[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, &total);
    if (i < ntiles) sums[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0 && grand_total) *grand_total = carry;
}

__global__ void k_scan_add(int* out, int64_t n, const int* tile_sums) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_sums[i / kScanTile];
}

// out[i] = sum_{j<i} in[j] for i < n, and out[n] = total (out has n+1 slots).
void scan_exclusive(const int* in, int* out, int64_t n, DBuf<int>& tmp, cudaStream_t s) {
  const int ntiles = std::max(1, ceil_div(n, kScanTile));
  tmp.alloc(ntiles + 1);
  if (n > 0) k_scan_tiles<<<ntiles, kScanThreads, 0, s>>>(in, out, n, tmp.p);
  else DW_CUDA(cudaMemsetAsync(tmp.p, 0, sizeof(int), s));
  k_scan_tile_sums<<<1, 1024, 0, s>>>(tmp.p, n > 0 ? ntiles : 1, out + n);
  if (n > 0) k_scan_add<<<ceil_div(n, 256), 256, 0, s>>>(out, n, tmp.p);
}

// ---- point loading ----------------------------------------------------------

__global__ void k_load_points(const double* pts, int64_t n, int64_t ld, int d, double* soa,
                              int32_t* perm, int* bad) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < d; ++k) {
    const double v = pts[i * ld + k];
    if (!isfinite(v)) *bad = 1;
    soa[k * n + i] = v;
  }
  perm[i] = static_cast<int32_t>(i);
}

// Segment (cluster, local to the level) of every tree position.
__global__ void k_segment_ids(const int32_t* lvl_begin, int nseg, int64_t n, int32_t* seg) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {  // last segment with begin <= i
    const int mid = (lo + hi + 1) >> 1;
    if (lvl_begin[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  seg[i] = lo;
}

// ---- segmented bounding boxes ----------------------------------------------

__global__ void k_box_init(unsigned long long* kmin, unsigned long long* kmax, int cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  kmin[i] = ~0ull;
  kmax[i] = 0ull;
}

// Warp-level segmented min/max over 32 consecutive positions; the last lane of
// each run of equal segment ids does one atomic per dimension.
__global__ void k_box_reduce(const double* soa, int64_t n, int d, const int32_t* seg,
                             unsigned long long* kmin, unsigned long long* kmax) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = i < n;
  const int sg = valid ? seg[i] : -1;
  const int sg_next = __shfl_down_sync(0xffffffffu, sg, 1);
  const bool tail = valid && (lane == 31 || sg_next != sg);
  for (int k = 0; k < d; ++k) {
    unsigned long long mn = valid ? dkey(soa[k * n + i]) : ~0ull;
    unsigned long long mx = valid ? mn : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long a = __shfl_up_sync(0xffffffffu, mn, o);
      const unsigned long long b = __shfl_up_sync(0xffffffffu, mx, o);
      const int s2 = __shfl_up_sync(0xffffffffu, sg, o);
      if (lane >= o && s2 == sg) {
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
      }
    }
    if (tail) {
      atomicMin(&kmin[static_cast<int64_t>(sg) * d + k], mn);
      atomicMax(&kmax[static_cast<int64_t>(sg) * d + k], mx);
    }
  }
}

// Decode the keys into lo/hi of clusters first..first+nseg-1 and choose the
// split dimension: argmax_k (hi_k - lo_k), first maximum.
__global__ void k_box_finish(const unsigned long long* kmin, const unsigned long long* kmax,
                             int nseg, int d, int first, double* lo, double* hi, int32_t* kstar) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  double best = -1.0;
  int bk = 0;
  for (int k = 0; k < d; ++k) {
    const double a = dkey_inv(kmin[static_cast<int64_t>(s) * d + k]);
    const double b = dkey_inv(kmax[static_cast<int64_t>(s) * d + k]);
    lo[static_cast<int64_t>(first + s) * d + k] = a;
    hi[static_cast<int64_t>(first + s) * d + k] = b;
    const double e = b - a;
    if (e > best) {
      best = e;
      bk = k;
    }
  }
  if (kstar) kstar[s] = bk;
}

// ---- median selection ---------------------------------------------------------

__global__ void k_make_keys(const double* soa, int64_t n, const int32_t* seg, const int32_t* kstar,
                            unsigned long long* key) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = dkey(soa[static_cast<int64_t>(kstar[seg[i]]) * n + i]);
}

struct SelState {
  unsigned long long prefix;
  unsigned long long mask;
  int rank;   // rank (0-based) still sought among keys matching prefix
  int pad;
};

__global__ void k_sel_init(SelState* st, const int32_t* lvl_count, int nseg) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const int c = lvl_count[s];
  st[s] = SelState{0ull, 0ull, (c + 1) / 2 - 1, 0};
}

constexpr int kHistThreads = 256;
constexpr int kHistItems = 16;

// Histogram of the digit at `shift` of the keys that match their segment's
// prefix.  A block whose positions all lie in one segment aggregates in
// shared memory first.
__global__ void k_sel_hist(const unsigned long long* key, const int32_t* seg, int64_t n,
                           const SelState* st, int shift, unsigned int* hist) {
  __shared__ unsigned int sh[256];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kHistThreads * kHistItems;
  const int64_t last = std::min<int64_t>(base + kHistThreads * kHistItems, n) - 1;
  const bool one = seg[base] == seg[last];
  if (one) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) sh[b] = 0;
    __syncthreads();
  }
  for (int it = 0; it < kHistItems; ++it) {
    const int64_t i = base + static_cast<int64_t>(it) * kHistThreads + threadIdx.x;
    if (i > last) break;
    const int sg = seg[i];
    const unsigned long long k = key[i];
    const SelState s = st[sg];
    if ((k & s.mask) != s.prefix || s.rank < 0) continue;
    const int digit = static_cast<int>((k >> shift) & 0xFFull);
    if (one) atomicAdd(&sh[digit], 1u);
    else atomicAdd(&hist[static_cast<int64_t>(sg) * 256 + digit], 1u);
  }
  if (one) {
    __syncthreads();
    const int sg = seg[base];
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
      if (sh[b]) atomicAdd(&hist[static_cast<int64_t>(sg) * 256 + b], sh[b]);
  }
}

__global__ void k_sel_pick(SelState* st, unsigned int* hist, int nseg, int shift) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  SelState t = st[s];
  unsigned int* h = hist + static_cast<int64_t>(s) * 256;
  if (t.rank >= 0) {
    unsigned int cum = 0;
    int b = 0;
    for (; b < 256; ++b) {
      if (cum + h[b] > static_cast<unsigned int>(t.rank)) break;
      cum += h[b];
    }
    if (b == 256) b = 255;  // unreachable for consistent counts
    t.prefix |= static_cast<unsigned long long>(b) << shift;
    t.mask |= 0xFFull << shift;
    t.rank -= static_cast<int>(cum);
    st[s] = t;
  }
  for (int b = 0; b < 256; ++b) h[b] = 0;
}

// eq[i] = key equals the segment's median key.
__global__ void k_flag_equal(const unsigned long long* key, const int32_t* seg, int64_t n,
                             const SelState* st, int* eq) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  eq[i] = key[i] == st[seg[i]].prefix;
}

// left[i]: below the median, or equal to it with rank among equals <= rank.
__global__ void k_flag_left(const unsigned long long* key, const int32_t* seg, int64_t n,
                            const SelState* st, const int* eqscan, const int32_t* lvl_begin,
                            int* left) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sg = seg[i];
  const SelState s = st[sg];
  const unsigned long long k = key[i];
  int l = k < s.prefix;
  if (k == s.prefix) l = (eqscan[i] - eqscan[lvl_begin[sg]]) <= s.rank;
  left[i] = l;
}

__global__ void k_partition(const double* soa_in, const int32_t* perm_in, int64_t n, int d,
                            const int32_t* seg, const int* left, const int* lscan,
                            const int32_t* lvl_begin, const int32_t* lvl_count, double* soa_out,
                            int32_t* perm_out, int* bad) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sg = seg[i];
  const int b = lvl_begin[sg];
  const int n1 = (lvl_count[sg] + 1) / 2;
  const int lr = lscan[i] - lscan[b];
  const int64_t pos = left[i] ? b + lr : b + n1 + (static_cast<int>(i) - b - lr);
  if (pos < b || pos >= b + lvl_count[sg]) {  // inconsistent selection: record, do not write
    *bad = 2;
    return;
  }
  perm_out[pos] = perm_in[i];
  for (int k = 0; k < d; ++k) soa_out[k * n + pos] = soa_in[k * n + i];
}

// ---- lists ------------------------------------------------------------------

__device__ __forceinline__ bool admissible(const double* lo, const double* hi, int d, int t, int s,
                                           double eta2) {
  double D2 = 0.0, da = 0.0, db = 0.0;
  for (int k = 0; k < d; ++k) {
    const double lt = lo[static_cast<int64_t>(t) * d + k], ht = hi[static_cast<int64_t>(t) * d + k];
    const double ls = lo[static_cast<int64_t>(s) * d + k], hs = hi[static_cast<int64_t>(s) * d + k];
    const double g = fmax(0.0, fmax(ls - ht, lt - hs));
    D2 = D2 + g * g;
    const double ea = ht - lt, eb = hs - ls;
    da = da + ea * ea;
    db = db + eb * eb;
  }
  return D2 > 0.0 && D2 >= eta2 * fmax(da, db);
}

__global__ void k_adm(const int32_t* ct, const int32_t* cs, int64_t nc, const double* lo,
                      const double* hi, int d, double eta2, int* adm) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  adm[c] = admissible(lo, hi, d, ct[c], cs[c], eta2) ? 1 : 0;
}

__global__ void k_compact_pairs(const int32_t* ct, const int32_t* cs, int64_t nc, const int* adm,
                                const int* admscan, int want_adm, int32_t* out) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  if (adm[c] != want_adm) return;
  const int64_t pos = want_adm ? admscan[c] : c - admscan[c];
  out[2 * pos] = ct[c];
  out[2 * pos + 1] = cs[c];
}

// Rows of the next level: child t' of t gets 2 * (non-admissible count of t's row).
__global__ void k_child_rows(const int* rowptr, const int* admscan, int nrows, int* child_cnt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int b = rowptr[r], e = rowptr[r + 1];
  const int non = (e - b) - (admscan[e] - admscan[b]);
  child_cnt[2 * r] = 2 * non;
  child_cnt[2 * r + 1] = 2 * non;
}

__global__ void k_expand(const int32_t* ct, const int32_t* cs, int64_t nc, const int* adm,
                         const int* admscan, const int* rowptr, int first, const int* next_rowptr,
                         int next_first, int32_t* nt, int32_t* ns) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nc || adm[c]) return;
  const int t = ct[c], s = cs[c];
  const int row = t - first;
  const int rb = rowptr[row];
  const int rank = static_cast<int>((c - admscan[c]) - (rb - admscan[rb]));
  for (int a = 0; a < 2; ++a) {
    const int tc = 2 * t + 1 + a;
    const int base = next_rowptr[tc - next_first] + 2 * rank;
    for (int b = 0; b < 2; ++b) {
      nt[base + b] = tc;
      ns[base + b] = 2 * s + 1 + b;
    }
  }
}

// Pairs per row; the pairs are sorted by row, so the lanes of a warp that
// share a row add their count with one atomic.
__global__ void k_count_rows(const int32_t* pairs, int64_t np, int offset, int* cnt) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const unsigned act = __ballot_sync(0xffffffffu, i < np);
  if (i >= np) return;
  const int row = pairs[2 * i] - offset;
  const unsigned same = __match_any_sync(act, row);
  if ((threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&cnt[row], __popc(same));
}

__global__ void k_pair_cols(const int32_t* pairs, int64_t np, int offset, int32_t* col) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= np) return;
  col[i] = pairs[2 * i + 1] - offset;
}

// ---- per-cluster data -----------------------------------------------------------

// Affine maps a_c(t) = lo + t * ext; a degenerate edge is widened to
// 1e-12 * max(1, longest edge).
__global__ void k_extents(const double* lo, const double* hi, int C, int d, double* ext,
                          double* iext, float* lo32, float* iext32) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double mx = 0.0;
  for (int k = 0; k < d; ++k) mx = fmax(mx, hi[static_cast<int64_t>(c) * d + k] - lo[static_cast<int64_t>(c) * d + k]);
  const double guard = 1e-12 * fmax(1.0, mx);
  for (int k = 0; k < d; ++k) {
    const int64_t o = static_cast<int64_t>(c) * d + k;
    const double e = fmax(hi[o] - lo[o], guard);
    ext[o] = e;
    iext[o] = 1.0 / e;
    lo32[o] = static_cast<float>(lo[o]);
    iext32[o] = static_cast<float>(1.0 / e);
  }
}

// ynode[c][k][alpha] = lo_c + xi_alpha * ext_c (padding slots repeat alpha = 0).
__global__ void k_nodes(const double* lo, const double* ext, const double* xi, int C, int d, int n,
                        int n_pad, double* y64, float* y32) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(C) * d * n_pad;
  if (t >= total) return;
  const int a = static_cast<int>(t % n_pad);
  const int64_t ck = t / n_pad;
  const int k = static_cast<int>(ck % d);
  const int64_t c = ck / d;
  const int aa = a < n ? a : 0;
  const double v = lo[c * d + k] + xi[static_cast<int64_t>(aa) * d + k] * ext[c * d + k];
  y64[t] = v;
  y32[t] = static_cast<float>(v);
}

// Leaf-blocked sites pts[leaf][k][m_pad]; padding slots copy the leaf's first site.
__global__ void k_leaf_block(const double* soa, int64_t n, int d, const int32_t* begin,
                             const int32_t* count, int L, int m_pad, double* p64, float* p32) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(L) * d * m_pad;
  if (t >= total) return;
  const int i = static_cast<int>(t % m_pad);
  const int64_t lk = t / m_pad;
  const int k = static_cast<int>(lk % d);
  const int leaf = static_cast<int>(lk / d);
  const int c = L - 1 + leaf;
  const int ii = i < count[c] ? i : 0;
  const double v = soa[static_cast<int64_t>(k) * n + begin[c] + ii];
  p64[t] = v;
  p32[t] = static_cast<float>(v);
}

}  // namespace

// ---------------------------------------------------------------------------

static void cluster_layout(int64_t N, int J, std::vector<int32_t>& begin, std::vector<int32_t>& count) {
  const int C = (1 << (J + 1)) - 1;
  begin.assign(C, 0);
  count.assign(C, 0);
  begin[0] = 0;
  count[0] = static_cast<int32_t>(N);
  for (int c = 0; c < (1 << J) - 1; ++c) {
    const int n1 = (count[c] + 1) / 2;
    begin[2 * c + 1] = begin[c];
    count[2 * c + 1] = n1;
    begin[2 * c + 2] = begin[c] + n1;
    count[2 * c + 2] = count[c] - n1;
  }
}

void build_tree(Plan& P, const double* pts_dev, int64_t N, int64_t ld) {
  cudaStream_t s = P.stream;
  P.free_tree();
  const int d = P.d;
  int J = 0;
  while ((N + (int64_t(1) << J) - 1) / (int64_t(1) << J) > P.leaf) ++J;
  P.N = N;
  P.J = J;
  P.L = 1 << J;
  P.C = (1 << (J + 1)) - 1;
  cluster_layout(N, J, P.h_begin, P.h_count);
  P.d_begin.alloc(P.C);
  P.d_count.alloc(P.C);
  DW_CUDA(cudaMemcpyAsync(P.d_begin.p, P.h_begin.data(), P.C * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  DW_CUDA(cudaMemcpyAsync(P.d_count.p, P.h_count.data(), P.C * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  P.d_lo.alloc(static_cast<size_t>(P.C) * d);
  P.d_hi.alloc(static_cast<size_t>(P.C) * d);
  P.d_perm.alloc(std::max<int64_t>(N, 1));
  if (N == 0) {
    DW_CUDA(cudaMemsetAsync(P.d_lo.p, 0, sizeof(double) * d, s));
    DW_CUDA(cudaMemsetAsync(P.d_hi.p, 0, sizeof(double) * d, s));
    return;
  }
  DBuf<double> soa0, soa1;
  DBuf<int32_t> perm1, seg, kstar;
  DBuf<unsigned long long> key, kmin, kmax;
  DBuf<int> bad, eq, eqscan, left, lscan, tmp;
  DBuf<SelState> st;
  DBuf<unsigned int> hist;
  soa0.alloc(static_cast<size_t>(N) * d);
  soa1.alloc(static_cast<size_t>(N) * d);
  perm1.alloc(N);
  seg.alloc(N);
  key.alloc(N);
  eq.alloc(N);
  left.alloc(N);
  eqscan.alloc(N + 1);
  lscan.alloc(N + 1);
  bad.alloc(1);
  const int maxseg = P.L;
  kstar.alloc(maxseg);
  kmin.alloc(static_cast<size_t>(maxseg) * d);
  kmax.alloc(static_cast<size_t>(maxseg) * d);
  st.alloc(maxseg);
  hist.alloc(static_cast<size_t>(maxseg) * 256);
  DW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  DW_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(unsigned int) * maxseg * 256, s));
  const int nb = ceil_div(N, 256);
  k_load_points<<<nb, 256, 0, s>>>(pts_dev, N, ld, d, soa0.p, P.d_perm.p, bad.p);
  int h_bad = 0;
  DW_CUDA(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  if (h_bad) fail(DWFMM_ERR_INVALID_ARG, "sites contain NaN or Inf");

  double* cur = soa0.p;
  double* nxt = soa1.p;
  int32_t* pcur = P.d_perm.p;
  int32_t* pnxt = perm1.p;
  const int hist_blocks = ceil_div(N, kHistThreads * kHistItems);
  for (int j = 0; j <= J; ++j) {
    const int first = (1 << j) - 1;
    const int nseg = 1 << j;
    const int32_t* lvl_begin = P.d_begin.p + first;
    const int32_t* lvl_count = P.d_count.p + first;
    k_segment_ids<<<nb, 256, 0, s>>>(lvl_begin, nseg, N, seg.p);
    k_box_init<<<ceil_div(nseg * d, 256), 256, 0, s>>>(kmin.p, kmax.p, nseg * d);
    k_box_reduce<<<nb, 256, 0, s>>>(cur, N, d, seg.p, kmin.p, kmax.p);
    k_box_finish<<<ceil_div(nseg, 128), 128, 0, s>>>(kmin.p, kmax.p, nseg, d, first, P.d_lo.p,
                                                     P.d_hi.p, j < J ? kstar.p : nullptr);
    if (j == J) break;
    k_make_keys<<<nb, 256, 0, s>>>(cur, N, seg.p, kstar.p, key.p);
    k_sel_init<<<ceil_div(nseg, 128), 128, 0, s>>>(st.p, lvl_count, nseg);
    for (int shift = 56; shift >= 0; shift -= 8) {
      k_sel_hist<<<hist_blocks, kHistThreads, 0, s>>>(key.p, seg.p, N, st.p, shift, hist.p);
      k_sel_pick<<<ceil_div(nseg, 128), 128, 0, s>>>(st.p, hist.p, nseg, shift);
    }
    k_flag_equal<<<nb, 256, 0, s>>>(key.p, seg.p, N, st.p, eq.p);
    scan_exclusive(eq.p, eqscan.p, N, tmp, s);
    k_flag_left<<<nb, 256, 0, s>>>(key.p, seg.p, N, st.p, eqscan.p, lvl_begin, left.p);
    scan_exclusive(left.p, lscan.p, N, tmp, s);
    k_partition<<<nb, 256, 0, s>>>(cur, pcur, N, d, seg.p, left.p, lscan.p, lvl_begin, lvl_count,
                                   nxt, pnxt, bad.p);
    std::swap(cur, nxt);
    std::swap(pcur, pnxt);
  }
  DW_CUDA(cudaGetLastError());
  if (pcur != P.d_perm.p)
    DW_CUDA(cudaMemcpyAsync(P.d_perm.p, pcur, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  // keep the tree-ordered SoA sites for the leaf blocks
  P.scratch.alloc(static_cast<size_t>(N) * d * sizeof(double));
  DW_CUDA(cudaMemcpyAsync(P.scratch.p, cur, static_cast<size_t>(N) * d * sizeof(double),
                          cudaMemcpyDeviceToDevice, s));
  DW_CUDA(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  if (h_bad) fail(DWFMM_ERR_CUDA, "median selection produced an inconsistent partition");
}

void build_lists(Plan& P) {
  cudaStream_t s = P.stream;
  const int J = P.J, d = P.d;
  P.far_level_count.assign(J + 1, 0);
  P.nfar = P.nnear = 0;
  if (P.N == 0) {
    P.d_far_rowptr.alloc(P.C + 1);
    DW_CUDA(cudaMemsetAsync(P.d_far_rowptr.p, 0, sizeof(int32_t) * (P.C + 1), s));
    P.d_near_rowptr.alloc(P.L + 1);
    DW_CUDA(cudaMemsetAsync(P.d_near_rowptr.p, 0, sizeof(int32_t) * (P.L + 1), s));
    P.jmin = J + 1;
    return;
  }
  const double eta2 = P.eta * P.eta;
  DBuf<int32_t> ct, cs, nt, ns;
  DBuf<int> adm, admscan, rowptr, nrowptr, childcnt, tmp;
  std::vector<DBuf<int32_t>> far_lvl(J + 1);
  int64_t nc = 1;
  ct.alloc(1);
  cs.alloc(1);
  rowptr.alloc(2);
  {
    const int32_t z[2] = {0, 0};
    const int rp[2] = {0, 1};
    DW_CUDA(cudaMemcpyAsync(ct.p, z, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DW_CUDA(cudaMemcpyAsync(cs.p, z, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DW_CUDA(cudaMemcpyAsync(rowptr.p, rp, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    DW_CUDA(cudaStreamSynchronize(s));
  }
  DBuf<int32_t> near_pairs;
  for (int j = 0; j <= J; ++j) {
    const int first = (1 << j) - 1;
    const int nrows = 1 << j;
    adm.alloc(std::max<int64_t>(nc, 1));
    admscan.alloc(nc + 1);
    if (nc > 0) k_adm<<<ceil_div(nc, 256), 256, 0, s>>>(ct.p, cs.p, nc, P.d_lo.p, P.d_hi.p, d, eta2, adm.p);
    scan_exclusive(adm.p, admscan.p, nc, tmp, s);
    int nadm = 0;
    DW_CUDA(cudaMemcpyAsync(&nadm, admscan.p + nc, sizeof(int), cudaMemcpyDeviceToHost, s));
    DW_CUDA(cudaStreamSynchronize(s));
    P.far_level_count[j] = nadm;
    if (nadm > 0) {
      far_lvl[j].alloc(2 * static_cast<size_t>(nadm));
      k_compact_pairs<<<ceil_div(nc, 256), 256, 0, s>>>(ct.p, cs.p, nc, adm.p, admscan.p, 1, far_lvl[j].p);
    }
    const int64_t non = nc - nadm;
    if (j == J) {
      P.nnear = non;
      near_pairs.alloc(std::max<int64_t>(2 * non, 2));
      if (non > 0)
        k_compact_pairs<<<ceil_div(nc, 256), 256, 0, s>>>(ct.p, cs.p, nc, adm.p, admscan.p, 0, near_pairs.p);
      break;
    }
    childcnt.alloc(2 * nrows);
    nrowptr.alloc(2 * nrows + 1);
    k_child_rows<<<ceil_div(nrows, 128), 128, 0, s>>>(rowptr.p, admscan.p, nrows, childcnt.p);
    scan_exclusive(childcnt.p, nrowptr.p, 2 * nrows, tmp, s);
    const int64_t nnext = 4 * non;
    nt.alloc(std::max<int64_t>(nnext, 1));
    ns.alloc(std::max<int64_t>(nnext, 1));
    if (nc > 0)
      k_expand<<<ceil_div(nc, 256), 256, 0, s>>>(ct.p, cs.p, nc, adm.p, admscan.p, rowptr.p, first,
                                                 nrowptr.p, 2 * first + 1, nt.p, ns.p);
    std::swap(ct, nt);
    std::swap(cs, ns);
    std::swap(rowptr, nrowptr);
    nc = nnext;
  }
  DW_CUDA(cudaGetLastError());
  // far pairs of all levels, CSR over all clusters (targets)
  P.nfar = 0;
  for (int j = 0; j <= J; ++j) P.nfar += P.far_level_count[j];
  P.d_far_pairs.alloc(std::max<int64_t>(2 * P.nfar, 2));
  int64_t off = 0;
  P.jmin = J + 1;
  for (int j = 0; j <= J; ++j) {
    if (P.far_level_count[j] == 0) continue;
    P.jmin = std::min(P.jmin, j);
    DW_CUDA(cudaMemcpyAsync(P.d_far_pairs.p + 2 * off, far_lvl[j].p,
                            2 * P.far_level_count[j] * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    off += P.far_level_count[j];
  }
  DBuf<int> cnt;
  cnt.alloc(std::max(P.C, P.L) + 1);
  P.d_far_rowptr.alloc(P.C + 1);
  P.d_far_col.alloc(std::max<int64_t>(P.nfar, 1));
  DW_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (P.C + 1), s));
  if (P.nfar > 0) {
    k_count_rows<<<ceil_div(P.nfar, 256), 256, 0, s>>>(P.d_far_pairs.p, P.nfar, 0, cnt.p);
    k_pair_cols<<<ceil_div(P.nfar, 256), 256, 0, s>>>(P.d_far_pairs.p, P.nfar, 0, P.d_far_col.p);
  }
  scan_exclusive(cnt.p, P.d_far_rowptr.p, P.C, tmp, s);
  // near pairs, CSR over leaves (leaf-local ids)
  P.d_near_pairs = std::move(near_pairs);
  P.d_near_rowptr.alloc(P.L + 1);
  P.d_near_col.alloc(std::max<int64_t>(P.nnear, 1));
  DW_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (P.L + 1), s));
  if (P.nnear > 0) {
    k_count_rows<<<ceil_div(P.nnear, 256), 256, 0, s>>>(P.d_near_pairs.p, P.nnear, P.L - 1, cnt.p);
    k_pair_cols<<<ceil_div(P.nnear, 256), 256, 0, s>>>(P.d_near_pairs.p, P.nnear, P.L - 1, P.d_near_col.p);
  }
  scan_exclusive(cnt.p, P.d_near_rowptr.p, P.L, tmp, s);
  DW_CUDA(cudaGetLastError());
  DW_CUDA(cudaStreamSynchronize(s));
  for (auto& b : far_lvl) b.release();
}

void build_cluster_data(Plan& P) {
  cudaStream_t s = P.stream;
  const int d = P.d, C = P.C;
  P.d_ext.alloc(static_cast<size_t>(C) * d);
  P.d_iext.alloc(static_cast<size_t>(C) * d);
  P.d_lo32.alloc(static_cast<size_t>(C) * d);
  P.d_iext32.alloc(static_cast<size_t>(C) * d);
  k_extents<<<ceil_div(C, 128), 128, 0, s>>>(P.d_lo.p, P.d_hi.p, C, d, P.d_ext.p, P.d_iext.p,
                                             P.d_lo32.p, P.d_iext32.p);
  const int64_t ny = static_cast<int64_t>(C) * d * P.n_pad;
  P.d_ynode64.alloc(ny);
  P.d_ynode32.alloc(ny);
  k_nodes<<<ceil_div(ny, 256), 256, 0, s>>>(P.d_lo.p, P.d_ext.p, P.d_nodes.p, C, d, P.n, P.n_pad,
                                            P.d_ynode64.p, P.d_ynode32.p);
  // one block stride per leaf size (not per tree), so plans with equal leaf
  // sizes share a layout and can be fused into one batch
  int maxleaf = 1;
  for (int l = 0; l < P.L; ++l) maxleaf = std::max(maxleaf, P.h_count[P.L - 1 + l]);
  P.m_pad = round_up(std::max(maxleaf, std::min<int>(P.leaf, static_cast<int>(std::max<int64_t>(P.N, 1)))), 8);
  const int64_t np = static_cast<int64_t>(P.L) * d * P.m_pad;
  P.d_pts64.alloc(std::max<int64_t>(np, 1));
  P.d_pts32.alloc(std::max<int64_t>(np, 1));
  if (P.N > 0)
    k_leaf_block<<<ceil_div(np, 256), 256, 0, s>>>(reinterpret_cast<const double*>(P.scratch.p), P.N, d,
                                                   P.d_begin.p, P.d_count.p, P.L, P.m_pad, P.d_pts64.p,
                                                   P.d_pts32.p);
  DW_CUDA(cudaGetLastError());
  DW_CUDA(cudaStreamSynchronize(s));
  P.scratch.release();
}

}  // namespace dw
