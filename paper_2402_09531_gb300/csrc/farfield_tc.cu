// Far-field expansion phases of the MIXED matvec on the tensor cores
// (Sec. 5.2, Eq. (5.4); the same algebra as the CUDA-core kernels of
// farfield.cu, with mu the Legendre moments, m the charges at the nodes,
// l the potentials at the nodes and lambda the local coefficients):
//   P2M / M2M  mu_c[b]     = sum_s p_hat_b(a_c^{-1} y_s) q_s[r]   (sites or child nodes s)
//              m_c         = V^{-T} mu_c
//   L2L        l_c[a]      = loc_c[a] + sum_b p_hat_b(a_p^{-1} y^c_a) lambda_p[b]
//              lambda_c    = V^{-1} l_c
//   L2P        y_i         = sum_b p_hat_b(a_leaf^{-1} x_i) lambda_leaf[b]
//
// Basis contractions (k_far_basis_tc, one CTA per cluster): the CUDA cores
// evaluate the basis values of a 128-row x 64-column tile (Legendre tables
// per point, products along each multi-index) and split each into FP16
// hi + lo; the 16 right-hand sides are scaled per column by a power of two
// (largest |entry| in [0.5, 1)) and split the same way.  tcgen05.mma
// kind::f16 (M = 128) forms A_hi [B_hi | B_lo] and A_lo [B_hi | B_lo]
// (N = 32 each: all four products, so each term carries the ~2^-23
// precision of its operands' splits) in FP32 TMEM accumulators, the large
// and the small terms in separate columns.  The upward tile is the A
// operand as stored (rows = basis indices); the downward passes read the
// same layout transposed (MN-major: rows = points), so every tile is built
// one basis row at a time.  Every 64-wide chunk starts fresh accumulators (four
// K = 16 steps) and is folded into FP32 registers, so that the tensor
// cores' per-step rounding of the accumulator acts on four steps at most.
// The CUDA cores build chunk c + 1 while the MMAs of chunk c run (two
// operand stages, two accumulator sets).
//
// Transforms (k_far_vgemm): V^{-T} and V^{-1} act on all clusters of a
// level at once, one GEMM whose A operand is the constant 128 x 128 tile
// (FP16 hi + lo of V^{-1} scaled by a power of two, built once per node
// set by k_far_vtiles) and whose columns are the level's (cluster,
// right-hand side) pairs, 64 per MMA (N = 64), split per column like the
// charges.
//
// Per element the pair hi + lo carries ~2^-23 relative down to ~2^-14 of
// the operand's scale (the lo part is stored times 2^11 so that it stays in
// FP16's normal range), about the precision of the float32 CUDA-core path it
// replaces.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "dwfmm_internal.cuh"
#include "tcgen05_util.cuh"

namespace dw {

namespace {

using namespace tc;

constexpr int kFT = 256;                      // threads of both kernels (8 warps)
constexpr int kKC = 64;                       // contraction length of one chunk
constexpr int kAHalf = 128 * kKC * 2;         // 16 KB: hi or lo of an A chunk
constexpr int kAStage = 2 * kAHalf;           // 32 KB
constexpr int kBStage = (kKC / 8) * 512;      // 4 KB: 32 rows (16 hi, 16 lo) x 64
constexpr int kBasisTmem = 128;               // two accumulator sets of 64 columns (at 0 and 64)
constexpr int kNzMax = 20;                    // nonzeros of a multi-index on this path
// Basis tile of a chunk, rows b, 8 FP16 points per 16-byte core row:
//  upward (A = the tile, K-major, M = b, K = 64 points): core (b/8, p/8) at
//    (b/8)*1024 + (p/8)*128;
//  downward (A = its transpose, read MN-major, M = 128 points, K = 64 b):
//    core (b/8, p/8) at (b/8)*2048 + (p/8)*128, so the leading byte offset
//    (along K) is 2048 and the stride byte offset (along M) 128.
// B chunk (right-hand sides, K-major): core (k/8, n/8) at (k/8)*512 + (n/8)*128.
constexpr uint32_t kLboA = 128, kSboA = 1024;
constexpr uint32_t kLboT = 2048, kSboT = 128;
constexpr uint32_t kLboB = 512, kSboB = 128;
// V tile: core (a/8, b/8) at (a/8)*2048 + (b/8)*128; hi then lo.
constexpr int kVHalf = 128 * 128 * 2;         // 32 KB
constexpr int kVTile = 2 * kVHalf;            // 64 KB
constexpr uint32_t kLboV = 128, kSboV = 2048;
// Column tile of the transform: core (k/8, n/8) at (k/8)*1024 + (n/8)*128.
constexpr int kVgCols = 64;
constexpr int kVgBHalf = 128 * kVgCols * 2;   // 16 KB
constexpr uint32_t kLboVB = 1024, kSboVB = 128;
constexpr int kVgTmem = 256;   // hi*hi (k < 64) at 0, one lo factor at 64, hi*hi (k >= 64) at 128, lo*lo at 192

// Instruction descriptor of kind::f16: D F32, A and B F16, both K-major.
__host__ __device__ constexpr uint32_t idesc_h(uint32_t m, uint32_t n) {
  return (1u << 4) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
constexpr uint32_t kId32 = idesc_h(128, 32), kId64 = idesc_h(128, 64);
constexpr uint32_t kId32T = kId32 | (1u << 15);   // A read MN-major

__device__ __forceinline__ void mma_h(uint32_t d_tmem, u64 adesc, u64 bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void st_shared128(uint32_t addr, const uint32_t* v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}

// Two values -> packed FP16 hi and lo: hi = the value rounded to FP16, lo =
// (value - hi) * 2^11 rounded to FP16 (the remainder is exact in FP32; the
// factor 2^11 keeps lo in FP16's normal range for values down to ~2^-14,
// where an unscaled remainder would be subnormal and lose its bits).  The
// pair carries ~2^-23 relative; products with a lo factor are accumulated in
// their own TMEM columns and scaled back by 2^-11 per lo factor.
constexpr float kLoScale = 2048.0f, kLoInv = 1.0f / 2048.0f;
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn((x0 - hf.x) * kLoScale, (x1 - hf.y) * kLoScale);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void split8(const float* v, uint32_t* hi, uint32_t* lo) {
#pragma unroll
  for (int u = 0; u < 4; ++u) split_h2(v[2 * u], v[2 * u + 1], hi[u], lo[u]);
}

// Four 8-column TMEM loads of the warp's lanes, one wait.
__device__ __forceinline__ void tmem_ld8x4(uint32_t ta, uint32_t tb, uint32_t tcc, uint32_t td, uint32_t* r,
                                           uint32_t* q, uint32_t* s, uint32_t* u) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7])
               : "r"(tb));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7])
               : "r"(tcc));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
               : "r"(td));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Coefficients of the three-term recurrence of the Legendre polynomials,
// P_{j+1}(u) = ((2j+1) u P_j(u) - j P_{j-1}(u)) / (j+1), and the
// normalisation sqrt(2j+1) of p_hat_j, for j < kLegMax.
constexpr int kLegMax = 48;
__constant__ float c_leg_a[kLegMax];   // (2j+1)/(j+1)
__constant__ float c_leg_b[kLegMax];   // j/(j+1)
__constant__ float c_leg_s[kLegMax];   // sqrt(2j+1)

// p_hat_j(t) = sqrt(2j+1) P_j(2t-1), j = 0..qk (qk < kLegMax).
__device__ __forceinline__ void legendre_f(float t, int qk, float* tab) {
  const float u = 2.0f * t - 1.0f;
  float pm = 1.0f, pc = u;
  tab[0] = 1.0f;
  if (qk >= 1) tab[1] = u * c_leg_s[1];
  for (int j = 1; j < qk; ++j) {
    const float pn = c_leg_a[j] * u * pc - c_leg_b[j] * pm;
    tab[j + 1] = pn * c_leg_s[j + 1];
    pm = pc;
    pc = pn;
  }
}

// Bounded wait on an mbarrier phase without a suspend-time hint (the waits
// here are short: one chunk's MMAs); false if it gave up.
__device__ __forceinline__ bool wait_spin(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = sptr(bar);
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Power of two s with max * s in [0.5, 1) (1 for an empty column); *inv = 1/s.
__device__ __forceinline__ float pow2_scale(float mx, float* inv) {
  int ex = 0;
  if (mx > 0.0f) (void)frexpf(mx, &ex);
  *inv = ldexpf(1.0f, ex);
  return ldexpf(1.0f, -ex);
}

struct BasisArgs {
  ExpDev e;
  int mode;       // 0: upward (P2M on the leaf level, M2M above), 1: L2L, 2: L2P
  int first;      // first cluster of the level
  int leaves;     // upward: the level is the leaf level
  int L, m_pad, LS, Rc;
  const int32_t* count;   // [C] sites per cluster
  const float* pts;       // [L][d][m_pad]
  const float* ynode;     // [C][d][n_pad]
  const float* lo;        // [C][d]
  const float* iext;      // [C][d]
  const float* xb;        // [L][16][m_pad] charges (upward, leaf level)
  float* mom;             // [C][16][n_pad] children's m (read), the cluster's mu (written)
  const float* loc;       // [C][16][n_pad] M2L potentials (L2L)
  float* lco;             // [C][16][n_pad] parent's lambda (L2L, read), own l (L2L, written), own lambda (L2P)
  float* yfar;            // [L][16][m_pad] (L2P)
  int* err;
};

// One cluster per CTA; see the file comment.
__global__ void __launch_bounds__(kFT, 2) k_far_basis_tc(BasisArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tslot;
  __shared__ float cscl[16], cinv[16];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int n = a.e.n, np = a.e.n_pad, d = a.e.d, LS = a.LS, nz = a.e.nnz_max;
  const int mode = a.mode;
  const int g = a.first + blockIdx.x;
  const int tabN = mode == 0 ? kKC : 128;
  float* tab = reinterpret_cast<float*>(smem + 2 * kAStage + 2 * kBStage);
  int16_t* fac = reinterpret_cast<int16_t*>(tab + tabN * LS);
  // the points' coordinates, copied in by the TMA engine: [d][m_pad] (sites
  // of a leaf), [d][n_pad] (nodes of a cluster) or two such node blocks
  float* crd = reinterpret_cast<float*>(smem + 2 * kAStage + 2 * kBStage +
                                        ((static_cast<size_t>(tabN) * LS * 4 + static_cast<size_t>(n) * nz * 2 + 15) &
                                         ~static_cast<size_t>(15)));
  __shared__ __align__(8) uint64_t cbar;
  __shared__ uint8_t nzc[128];   // nonzero factors of each multi-index
  __shared__ float cred[kFT / 32][16];

  const int box = mode == 1 ? (g - 1) / 2 : g;   // the expansion's box
  const float* blo = a.lo + static_cast<int64_t>(box) * d;
  const float* bie = a.iext + static_cast<int64_t>(box) * d;
  const int leaf = g - (a.L - 1);
  const int cnt = (mode == 1 || (mode == 0 && !a.leaves)) ? 0 : a.count[g];
  const int K = mode == 0 ? (a.leaves ? a.m_pad : 256) : 128;
  const int tiles = mode == 2 ? a.m_pad / 128 : 1;
  const int nchunk = K / kKC;
  const int units = tiles * nchunk;

  // point p of the contraction (mode 0: column k; modes 1, 2: row of the tile)
  auto point_ok = [&](int p) -> bool {
    if (mode == 0) return a.leaves ? p < cnt : (p & 127) < n;
    if (mode == 1) return p < n;
    return p < cnt;
  };
  auto point_ptr = [&](int p, int& stride) -> const float* {
    if (mode == 0 && !a.leaves) {
      stride = np;
      return crd + (p >> 7) * d * np + (p & 127);
    }
    stride = mode == 1 ? np : a.m_pad;
    return crd + p;
  };
  // eight consecutive entries k0..k0+7 of right-hand side r of the B operand
  auto load8 = [&](int r, int k0, float* v) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.0f;
    if (r >= a.Rc) return;
    const float* src = nullptr;
    int valid = 8;
    if (mode == 0 && a.leaves) {
      src = a.xb + (static_cast<int64_t>(leaf) * 16 + r) * a.m_pad + k0;
    } else if (mode == 0) {
      const int a0 = k0 & 127;
      if (a0 < np) src = a.mom + (static_cast<int64_t>(2 * g + 1 + (k0 >> 7)) * 16 + r) * np + a0;
      valid = n - a0;
    } else {
      const int pc = mode == 1 ? (g - 1) / 2 : g;
      if (k0 < np) src = a.lco + (static_cast<int64_t>(pc) * 16 + r) * np + k0;
      valid = n - k0;
    }
    if (!src || valid <= 0) return;
    const float4 x0 = *reinterpret_cast<const float4*>(src);
    const float4 x1 = *reinterpret_cast<const float4*>(src + 4);
    const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = j < valid ? xs[j] : 0.0f;
  };

  if (t == 0) {
    bar_init(&bars[0], 1);
    bar_init(&bars[1], 1);
    bar_init(&cbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // coordinates of the contraction's points
    if (mode == 0 && !a.leaves) {
      const uint32_t bytes = static_cast<uint32_t>(d * np * 4);
      bar_expect_tx(&cbar, 2 * bytes);
      bulk_load(crd, a.ynode + static_cast<int64_t>(2 * g + 1) * d * np, bytes, &cbar);
      bulk_load(crd + d * np, a.ynode + static_cast<int64_t>(2 * g + 2) * d * np, bytes, &cbar);
    } else if (mode == 1) {
      const uint32_t bytes = static_cast<uint32_t>(d * np * 4);
      bar_expect_tx(&cbar, bytes);
      bulk_load(crd, a.ynode + static_cast<int64_t>(g) * d * np, bytes, &cbar);
    } else {
      const uint32_t bytes = static_cast<uint32_t>(d * a.m_pad * 4);
      bar_expect_tx(&cbar, bytes);
      bulk_load(crd, a.pts + static_cast<int64_t>(leaf) * d * a.m_pad, bytes, &cbar);
    }
  }
  if (w == 0) tmem_alloc(&tslot, kBasisTmem);
  for (int i = t; i < n * nz; i += kFT) fac[i] = a.e.fac[i];
  if (t < 128) {
    int c = 0;
    if (t < n)
      while (c < nz && a.e.fac[t * nz + c] >= 0) ++c;
    nzc[t] = static_cast<uint8_t>(c);
  }
  // the B operand, read once into registers: thread (r = t % 16, g8 = t / 16)
  // holds entries g8*8 + 128 i .. + 7 of right-hand side r (i < K / 128),
  // i.e. chunk 2 i + t / 128, core column g8 % 8; the per-column scale is
  // the largest |entry| over the whole contraction
  const int br = t & 15, bg8 = t >> 4;
  float bv[2][8];
  {
    float mx = 0.0f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (i * 128 < K) load8(br, bg8 * 8 + 128 * i, bv[i]);
      else
#pragma unroll
        for (int j = 0; j < 8; ++j) bv[i][j] = 0.0f;
#pragma unroll
      for (int j = 0; j < 8; ++j) mx = fmaxf(mx, fabsf(bv[i][j]));
    }
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
    if (lane < 16) cred[w][lane] = mx;
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (t < 16) {
    float mx = 0.0f;
#pragma unroll
    for (int i = 0; i < kFT / 32; ++i) mx = fmaxf(mx, cred[i][t]);
    cscl[t] = pow2_scale(mx, &cinv[t]);
  }
  const uint32_t tmem = tslot;
  if (!wait_spin(&cbar, 0)) atomicExch(a.err, 3);

  auto fill_tab = [&](int base) {   // one (point, dimension) pair per thread and pass
    const int sh = mode == 0 ? 6 : 7;   // log2(tabN)
    for (int i = t; i < tabN * d; i += kFT) {
      const int pt = i & (tabN - 1), k = i >> sh;
      if (point_ok(base + pt)) {
        int ys;
        const float* y = point_ptr(base + pt, ys);
        legendre_f((y[k * ys] - blo[k]) * bie[k], a.e.qk[k], tab + pt * LS + a.e.loff[k]);
      }
    }
  };

  // operands of unit u (tile u / nchunk, chunk u % nchunk) into stage u & 1
  auto gen = [&](int u) {
    const int tl = u / nchunk, c = u % nchunk, st = u & 1;
    if (mode == 0) fill_tab(c * kKC);
    else if (c == 0) fill_tab(tl * 128);
    __syncthreads();
    const uint32_t abase = sptr(smem + st * kAStage);
    // Basis tile G[b][point] (rows b, FP16 along the points): mode 0 all 128
    // basis rows x the chunk's 64 points (the A operand, K-major); modes 1, 2
    // the chunk's 64 basis rows x the tile's 128 points (the A operand read
    // MN-major: M = points, K = b).  Item q: 8 consecutive rows per quarter
    // warp (one 128-byte core matrix), 8 points per thread.
    const int cshift = mode == 0 ? 3 : 4;   // log2 of the point groups per row
    for (int q = t; q < 1024; q += kFT) {
      const int lo8 = q & 7, pg = (q >> 3) & ((1 << cshift) - 1);
      const int row = ((q >> (3 + cshift)) << 3) | lo8;
      const int b = mode == 0 ? row : c * kKC + row;
      const int p0 = pg * 8;   // first point of the group, index into the table
      const int nzb = b < n ? nzc[b] : 0;
      const float* t0 = tab + p0 * LS;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = 1.0f;
      for (int z = 0; z < nzb; ++z) {
        const int fz = fac[b * nz + z];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] *= t0[j * LS + fz];
      }
      const int pbase = mode == 0 ? c * kKC + p0 : tl * 128 + p0;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (b >= n || !point_ok(pbase + j)) v[j] = 0.0f;
      uint32_t hi[4], lo[4];
      split8(v, hi, lo);
      const uint32_t off = mode == 0 ? static_cast<uint32_t>(row >> 3) * kSboA + pg * kLboA + lo8 * 16
                                     : static_cast<uint32_t>(row >> 3) * kLboT + pg * kSboT + lo8 * 16;
      st_shared128(abase + off, hi);
      st_shared128(abase + kAHalf + off, lo);
    }
    if ((t >> 7) == (c & 1)) {   // the half of the CTA that holds chunk c
      const int kg = bg8 & 7;
      const bool second = (c >> 1) != 0;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = (second ? bv[1][j] : bv[0][j]) * cscl[br];
      uint32_t hi[4], lo[4];
      split8(v, hi, lo);
      const uint32_t bbase = sptr(smem + 2 * kAStage + st * kBStage) + kg * kLboB + (br & 7) * 16;
      st_shared128(bbase + (br >> 3) * kSboB, hi);
      st_shared128(bbase + ((br + 16) >> 3) * kSboB, lo);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  };

  auto issue = [&](int u) {
    if (t != 0) return;
    fence_after();
    const int st = u & 1;
    const uint32_t ab = sptr(smem + st * kAStage), bb = sptr(smem + 2 * kAStage + st * kBStage);
    const uint32_t dc = tmem + st * 64;
#pragma unroll
    for (int kk = 0; kk < kKC / 16; ++kk) {
      u64 ahi, alo;
      if (mode == 0) {
        ahi = smem_desc(ab + kk * 2 * kLboA, kLboA, kSboA);
        alo = smem_desc(ab + kAHalf + kk * 2 * kLboA, kLboA, kSboA);
      } else {
        ahi = smem_desc(ab + kk * 2 * kLboT, kLboT, kSboT);
        alo = smem_desc(ab + kAHalf + kk * 2 * kLboT, kLboT, kSboT);
      }
      const uint32_t id = mode == 0 ? kId32 : kId32T;
      const u64 bd = smem_desc(bb + kk * 2 * kLboB, kLboB, kSboB);
      mma_h(dc, ahi, bd, id, kk > 0 ? 1u : 0u);        // hi*hi (cols 0-15), hi*lo (16-31)
      mma_h(dc + 32, alo, bd, id, kk > 0 ? 1u : 0u);   // lo*hi (32-47), lo*lo (48-63)
    }
    mma_commit(&bars[st]);
  };

  const int wg = w >> 2;   // warps 0-3: right-hand sides 0-7, warps 4-7: 8-15
  const uint32_t lanes = tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16);
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0f;

  gen(0);
  issue(0);
  for (int u = 0; u < units; ++u) {
    if (u + 1 < units) {
      gen(u + 1);
      issue(u + 1);
    }
    const int st = u & 1;
    if (!wait_spin(&bars[st], (u >> 1) & 1)) atomicExch(a.err, 3);
    fence_after();
    uint32_t hh[8], hl[8], lh[8], ll[8];
    const uint32_t cb = lanes + st * 64 + 8 * wg;
    tmem_ld8x4(cb, cb + 16, cb + 32, cb + 48, hh, hl, lh, ll);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float small = (__uint_as_float(hl[j]) + __uint_as_float(lh[j])) + __uint_as_float(ll[j]) * kLoInv;
      acc[j] += __uint_as_float(hh[j]) + small * kLoInv;
    }
    fence_before();
    if (u % nchunk == nchunk - 1) {   // the tile is complete
      const int tl = u / nchunk;
      const int m = 32 * (w & 3) + lane;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = 8 * wg + j;
        const float val = r < a.Rc ? acc[j] * cinv[r] : 0.0f;
        if (mode == 0) {
          if (m < np) a.mom[(static_cast<int64_t>(g) * 16 + r) * np + m] = val;
        } else if (mode == 1) {
          if (m < np) {
            const int64_t o = (static_cast<int64_t>(g) * 16 + r) * np + m;
            a.lco[o] = (r < a.Rc && m < n) ? a.loc[o] + val : 0.0f;
          }
        } else {
          a.yfar[(static_cast<int64_t>(leaf) * 16 + r) * a.m_pad + tl * 128 + m] = val;
        }
        acc[j] = 0.0f;
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (w == 0) tmem_dealloc(tmem, kBasisTmem);
}

struct VgArgs {
  const uint16_t* vt;   // the tile (hi, then lo) in the A-operand layout
  const int* vexp;      // tile entries = V^{-1} entries * 2^-vexp
  const float* in;      // [cols][n_pad], column = cluster * 16 + r, from the level's first cluster
  float* out;           // same layout (may alias `in`: each CTA reads its columns before writing them)
  int n, np, cols, Rc;
  int* err;
};

// out[col] = V_x in[col] for every column of the level; see the file comment.
__global__ void __launch_bounds__(kFT, 2) k_far_vgemm(VgArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tslot;
  __shared__ unsigned cmax[kVgCols];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int n = a.n, np = a.np;
  unsigned char* vt = smem;
  unsigned char* bt = smem + kVTile;
  if (t == 0) {
    bar_init(&bars[0], 1);
    bar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) tmem_alloc(&tslot, kVgTmem);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tslot;
  if (t == 0) {
    bar_expect_tx(&bars[0], kVTile);
    bulk_load(vt, a.vt, kVHalf, &bars[0]);
    bulk_load(vt + kVHalf, a.vt + kVHalf / 2, kVHalf, &bars[0]);
  }
  const float vs = ldexpf(1.0f, *a.vexp);
  const int ntiles = (a.cols + kVgCols - 1) / kVgCols;
  const int nn = t & (kVgCols - 1), part = t >> 6;   // column of the tile, quarter of the contraction
  const int wg = w >> 2;
  const uint32_t lanes = tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16);
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    if (t < kVgCols) cmax[t] = 0u;
    __syncthreads();
    const int col = tile * kVgCols + nn;
    const bool cok = col < a.cols && (col & 15) < a.Rc;
    float v[32];
    float mx = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int b0 = part * 32 + 4 * i;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (cok && b0 < np) x = *reinterpret_cast<const float4*>(a.in + static_cast<int64_t>(col) * np + b0);
      v[4 * i + 0] = b0 + 0 < n ? x.x : 0.0f;
      v[4 * i + 1] = b0 + 1 < n ? x.y : 0.0f;
      v[4 * i + 2] = b0 + 2 < n ? x.z : 0.0f;
      v[4 * i + 3] = b0 + 3 < n ? x.w : 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) mx = fmaxf(mx, fabsf(v[4 * i + j]));
    }
    if (mx > 0.0f) atomicMax(&cmax[nn], __float_as_uint(mx));
    __syncthreads();
    float cinv_unused;
    const float sc = pow2_scale(__uint_as_float(cmax[nn]), &cinv_unused);
#pragma unroll
    for (int i2 = 0; i2 < 4; ++i2) {
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = v[8 * i2 + j] * sc;
      uint32_t hi[4], lo[4];
      split8(x, hi, lo);
      const uint32_t off = static_cast<uint32_t>(part * 4 + i2) * kLboVB + (nn >> 3) * kSboVB + (nn & 7) * 16;
      st_shared128(sptr(bt) + off, hi);
      st_shared128(sptr(bt) + kVgBHalf + off, lo);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      if (it == 0 && !wait_spin(&bars[0], 0)) atomicExch(a.err, 3);
      fence_after();
      const uint32_t va = sptr(vt), ba = sptr(bt);
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const u64 ahi = smem_desc(va + kk * 256, kLboV, kSboV);
        const u64 alo = smem_desc(va + kVHalf + kk * 256, kLboV, kSboV);
        const u64 bhi = smem_desc(ba + kk * 2 * kLboVB, kLboVB, kSboVB);
        const u64 blo = smem_desc(ba + kVgBHalf + kk * 2 * kLboVB, kLboVB, kSboVB);
        mma_h(tmem + (kk < 4 ? 0 : 128), ahi, bhi, kId64, (kk & 3) ? 1u : 0u);   // hi*hi, two halves
        mma_h(tmem + 64, ahi, blo, kId64, kk ? 1u : 0u);                        // one lo factor
        mma_h(tmem + 64, alo, bhi, kId64, 1u);
        mma_h(tmem + 192, alo, blo, kId64, kk ? 1u : 0u);                       // two lo factors
      }
      mma_commit(&bars[1]);
    }
    if (!wait_spin(&bars[1], it & 1)) atomicExch(a.err, 3);
    fence_after();
    const int ar = 32 * (w & 3) + lane;   // row of V_x: node index
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c0 = wg * 32 + h * 16;
      uint32_t d0[16], d1[16], d2[16], d3[16];
      tmem_ld16(lanes + c0, d0);
      tmem_ld16(lanes + 64 + c0, d1);
      tmem_ld16(lanes + 128 + c0, d2);
      tmem_ld16(lanes + 192 + c0, d3);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int cc = c0 + j, col2 = tile * kVgCols + cc;
        if (col2 < a.cols && ar < np) {
          float ci;
          (void)pow2_scale(__uint_as_float(cmax[cc]), &ci);
          const float small = __uint_as_float(d1[j]) + __uint_as_float(d3[j]) * kLoInv;
          const float val = (__uint_as_float(d0[j]) + __uint_as_float(d2[j])) + small * kLoInv;
          a.out[static_cast<int64_t>(col2) * np + ar] = (ar < n && (col2 & 15) < a.Rc) ? val * ci * vs : 0.0f;
        }
      }
    }
    fence_before();
    __syncthreads();
  }
  fence_after();
  if (w == 0) tmem_dealloc(tmem, kVgTmem);
}

// Tiles of V^{-T} (up) and V^{-1} (down), FP16 hi and lo (the remainder
// times 2^11, as in split_h2) of the entries scaled by 2^-vexp (largest
// |entry| in [0.5, 1)), zero outside n x n:
// tiles = [up hi][up lo][down hi][down lo], 16384 halves each.
__global__ void k_far_vtiles(const double* vinv, int n, int np, uint16_t* tiles, int* vexp) {
  __shared__ double red[kFT / 32];
  __shared__ int s_ex;
  const int t = threadIdx.x;
  double mx = 0.0;
  for (int i = t; i < n * n; i += blockDim.x) mx = fmax(mx, fabs(vinv[static_cast<int64_t>(i / n) * np + i % n]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) red[t >> 5] = mx;
  __syncthreads();
  if (t == 0) {
    double m = 0.0;
    for (int i = 0; i < kFT / 32; ++i) m = fmax(m, red[i]);
    int ex = 0;
    if (m > 0.0) (void)frexp(m, &ex);
    s_ex = ex;
    *vexp = ex;
  }
  __syncthreads();
  const double s = ldexp(1.0, -s_ex);
  for (int i = t; i < 128 * 128; i += blockDim.x) {
    const int r = i >> 7, c = i & 127;
    const int off = (r >> 3) * 1024 + (c >> 3) * 64 + (r & 7) * 8 + (c & 7);
    const bool in = r < n && c < n;
    const double up = in ? vinv[static_cast<int64_t>(c) * np + r] * s : 0.0;
    const double dn = in ? vinv[static_cast<int64_t>(r) * np + c] * s : 0.0;
    const __half uh = __double2half(up), dh = __double2half(dn);
    const __half ul = __double2half((up - static_cast<double>(__half2float(uh))) * 2048.0);
    const __half dl = __double2half((dn - static_cast<double>(__half2float(dh))) * 2048.0);
    tiles[off] = __half_as_ushort(uh);
    tiles[16384 + off] = __half_as_ushort(ul);
    tiles[32768 + off] = __half_as_ushort(dh);
    tiles[49152 + off] = __half_as_ushort(dl);
  }
}

std::atomic<uint64_t> g_far_attrs_dev{0};

size_t basis_smem(const Plan& P, int mode) {
  const int LS = P.lsum | 1;
  const size_t tabN = mode == 0 ? kKC : 128;
  const size_t head = (tabN * LS * 4 + static_cast<size_t>(P.n) * P.nnz_max * 2 + 15) & ~static_cast<size_t>(15);
  const size_t crd = static_cast<size_t>(P.d) * std::max(P.m_pad, 2 * P.n_pad) * 4;
  return 2 * static_cast<size_t>(kAStage) + 2 * kBStage + head + crd;
}

constexpr size_t kVgSmem = kVTile + 2 * kVgBHalf;

void ensure_far_attrs() {
  const uint64_t bit = device_bit();
  if (g_far_attrs_dev.load() & bit) return;
  float la[kLegMax], lb[kLegMax], ls[kLegMax];
  for (int j = 0; j < kLegMax; ++j) {
    la[j] = static_cast<float>((2.0 * j + 1.0) / (j + 1.0));
    lb[j] = static_cast<float>(j / (j + 1.0));
    ls[j] = static_cast<float>(std::sqrt(2.0 * j + 1.0));
  }
  DW_CUDA(cudaMemcpyToSymbol(c_leg_a, la, sizeof(la)));
  DW_CUDA(cudaMemcpyToSymbol(c_leg_b, lb, sizeof(lb)));
  DW_CUDA(cudaMemcpyToSymbol(c_leg_s, ls, sizeof(ls)));
  DW_CUDA(cudaFuncSetAttribute(k_far_basis_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  DW_CUDA(cudaFuncSetAttribute(k_far_vgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kVgSmem));
  g_far_attrs_dev.fetch_or(bit);
}

BasisArgs basis_args(Plan& P, int mode, int j, int Rc) {
  BasisArgs a;
  a.e = P.exp_dev();
  a.mode = mode;
  a.first = (1 << j) - 1;
  a.leaves = j == P.J;
  a.L = P.L;
  a.m_pad = P.m_pad;
  a.LS = P.lsum | 1;
  a.Rc = Rc;
  a.count = P.d_count.p;
  a.pts = P.d_pts32.p;
  a.ynode = P.d_ynode32.p;
  a.lo = P.d_lo32.p;
  a.iext = P.d_iext32.p;
  a.xb = P.xb32.p;
  a.mom = P.mom32.p;
  a.loc = P.loc32.p;
  a.lco = P.lco32.p;
  a.yfar = P.yfar32.p;
  a.err = P.d_err.p;
  return a;
}

void launch_vgemm(Plan& P, bool up, const float* in, float* out, int clusters, int Rc, cudaStream_t s) {
  VgArgs v;
  v.vt = P.far_vt.p + (up ? 0 : 32768);
  v.vexp = P.far_vexp.p;
  v.in = in;
  v.out = out;
  v.n = P.n;
  v.np = P.n_pad;
  v.cols = clusters * 16;
  v.Rc = Rc;
  v.err = P.d_err.p;
  const int ntiles = ceil_div(v.cols, kVgCols);
  const int grid = std::min(ntiles, 2 * sm_count());
  k_far_vgemm<<<grid, kFT, kVgSmem, s>>>(v);
}

}  // namespace

bool farfield_tc_eligible(const Plan& P) {
  if (P.prec != DWFMM_P_MIXED || P.n < 1 || P.n_pad > 128 || P.nnz_max > kNzMax || P.nnz_max < 1) return false;
  if (P.m_pad != 128 && P.m_pad != 256) return false;
  for (int k = 0; k < P.d; ++k)
    if (P.qk[k] >= kLegMax) return false;
  if (basis_smem(P, 1) > 200 * 1024) return false;
  return true;
}

void farfield_tc(Plan& P, int Rc) {
  cudaStream_t s = P.stream;
  ensure_far_attrs();
  if (!P.far_vt_ok) {
    P.far_vt.alloc(4 * 16384);
    P.far_vexp.alloc(1);
    k_far_vtiles<<<1, kFT, 0, s>>>(P.d_vinv.p, P.n, P.n_pad, P.far_vt.p, P.far_vexp.p);
    DW_CUDA(cudaGetLastError());
    P.far_vt_ok = true;
  }
  const int J = P.J, np = P.n_pad;
  const size_t sm_up = basis_smem(P, 0), sm_dn = basis_smem(P, 1);
  timer_begin(P, 1, s);
  int launches = 0;
  for (int j = J; j >= P.jmin; --j) {
    k_far_basis_tc<<<1 << j, kFT, sm_up, s>>>(basis_args(P, 0, j, Rc));
    float* m = P.mom32.p + static_cast<int64_t>((1 << j) - 1) * 16 * np;
    launch_vgemm(P, true, m, m, 1 << j, Rc, s);
    launches += 2;
  }
  timer_end(P, 1, s, launches);
  timer_begin(P, 2, s);
  launch_m2l(P, Rc, false);
  timer_end(P, 2, s, 1);
  timer_begin(P, 3, s);
  launches = 0;
  for (int j = P.jmin; j <= J; ++j) {
    const int64_t off = static_cast<int64_t>((1 << j) - 1) * 16 * np;
    if (j > P.jmin) {
      k_far_basis_tc<<<1 << j, kFT, sm_dn, s>>>(basis_args(P, 1, j, Rc));
      launch_vgemm(P, false, P.lco32.p + off, P.lco32.p + off, 1 << j, Rc, s);
      launches += 2;
    } else {
      launch_vgemm(P, false, P.loc32.p + off, P.lco32.p + off, 1 << j, Rc, s);
      launches += 1;
    }
  }
  k_far_basis_tc<<<P.L, kFT, sm_dn, s>>>(basis_args(P, 2, J, Rc));
  timer_end(P, 3, s, launches + 1);
  DW_CUDA(cudaGetLastError());
}

}  // namespace dw
