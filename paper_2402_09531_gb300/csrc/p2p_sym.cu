// Symmetric near field (P2P) on the tensor cores for MIXED plans with 9..16
// right-hand sides: each unordered near pair of leaves (T, S >= T) of the
// near list N (Eq. (5.1); both orderings are in the list, K is symmetric)
// is evaluated once and serves both directions,
//
//   y_T += E q_S    (forward),     y_S += E^T q_T    (transposed, S != T),
//
// with E[t][s] = phi(|x_t - x_s| / sigma).  For the Gaussian the factored
// form E = 2^(-|x'|^2) 2^(2 x'.s') 2^(-|s'|^2) is used (scaled coordinates,
// kernel constant folded in): the CUDA cores evaluate E' = 2^(2 x'.s'), the
// point factors sit on the charges and on the finished sums.
//
// Arithmetic.  E' is split into FP16 hi + lo (hi = E' rounded to FP16,
// lo = (E' - hi) * 2^11 rounded to FP16, so that lo stays in FP16's normal
// range for small E'); the charges q' = q * factor, normalised per
// right-hand side by a power of two so that |q'| <= 1, are split the same
// way.  tcgen05.mma.kind::f16 (FP32 accumulation) forms hi*hi in its own
// columns and hi*lo + lo*hi in others, scaled back by 2^-11 when read.  The
// plan takes this path only where E' stays inside the FP16 range (E' <=
// 2^15: the bound on |x'|^2 of the tree's root box) and E' <= 1 otherwise.
//
// Work.  One CTA per target leaf T (rows ordered by their upper-list length,
// longest first), looping over the upper entries S >= T in 64-source
// chunks.  Sixteen compute warps evaluate E for all targets of T (two per
// thread: t and t + 128) against the chunk and store E_hi / E_lo into a
// shared-memory tile in the no-swizzle core-matrix layout; one core row is
// 8 sources of one target (16 bytes), so the same tile is
//   * the K-major A operand of the forward product (M = 128 targets,
//     K = 16 sources, N = 32: E_hi*[q_hi | q_lo], then N = 16: E_lo*q_hi), and
//   * the MN-major A operand of the transposed product with M = 128 rows =
//     [E_hi of the 64 sources ; E_lo of the 64 sources], K = 16 targets,
//     N = 32 ([q_hi | q_lo] of T): one MMA per K step.
// The tensor core rounds its FP32 accumulator toward zero at every MMA, so
// the large hi*hi terms get their own columns with one update per K step.
//
// Accumulation.  The forward sums of T stay in the CTA: TMEM accumulators per
// (upper entry, 128-target tile), folded into Kahan-compensated running sums
// in shared memory and written once.  The transposed sums of S (64 sources x
// 16 right-hand sides per chunk) are combined from the hi and lo rows and
// added to a 64-bit fixed-point accumulator per site with
// red.global.add.u64: integer addition is associative, so the result does
// not depend on the order in which CTAs finish (repeated matvecs are bit
// identical).  The fixed-point step 2^-sb is chosen from a bound on every
// partial sum (N sites times the largest E'), far below the FP32 rounding.
// A finishing kernel adds both parts and applies the point factors.
//
// Roles: 16 compute warps, one warp whose lane 0 issues the MMAs, one whose
// lane 0 issues the TMA bulk copies; hand-over through mbarriers only; every
// wait is bounded and raises the plan's error flag instead of hanging.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_fp16.h>

#include "dwfmm_internal.cuh"
#include "tcgen05_util.cuh"

namespace dw {

namespace {

using namespace tc;

constexpr int kSymCompWarps = 16;
constexpr int kSymTcThreads = (kSymCompWarps + 3) * 32;  // forward and transposed issuers, TMA warp
constexpr int kSymGThreads = (kSymCompWarps + 4) * 32;   // three MMA-issuing warps, one TMA warp
constexpr int kChunk = 64;          // sources per chunk
constexpr int kStages = 4;          // TMA stages (coordinates + FP16 charges of one chunk)
constexpr int kTmemCols = 256;      // forward 2 entries x 2 tiles x 32, transposed 2 x 32
constexpr int kQChunkBytes = kChunk * 16 * 2 * 2;   // [s/8][4 cores][128 B]: 4 KB

// Instruction descriptor, kind::f16: D F32, A and B F16; a_mn = 1 reads A
// MN-major.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t m, uint32_t n, uint32_t a_mn) {
  return (1u << 4) | (a_mn << 15) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
constexpr uint32_t kIdFwd32 = idesc_f16(128, 32, 0);
constexpr uint32_t kIdFwd16 = idesc_f16(128, 16, 0);
constexpr uint32_t kIdTrn32 = idesc_f16(128, 32, 1);

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, u64 adesc, u64 bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// E tile of one chunk: core (t/8, hl, s/8) at (t/8)*2048 + hl*1024 + (s/8)*128,
// row t%8 at 16 bytes, 8 FP16 sources per row.
constexpr int kTS = 2048, kHL = 1024;
// Descriptor of the transposed (MN-major) A operand: for this layout the
// leading byte offset is the stride between core matrices along K (targets,
// kTS) and the stride byte offset the one along M (sources, 128 bytes).
constexpr uint32_t kSymTrnLbo = kTS, kSymTrnSbo = 128;

template <int KER>
__device__ __forceinline__ float phi_sym(float a) {
  if (KER == DWFMM_K_GAUSS) return ex2f(a);
  const float r = sqrtf_a(a);
  if (KER == DWFMM_K_EXP) return ex2f(-r);
  const float e = ex2f(-1.4426950408889634f * r);
  return fmaf(r, e, e);
}

// Two values -> packed FP16 hi and lo: hi = the value rounded to FP16, lo =
// (value - hi) * 2^11 rounded to FP16 (the remainder is exact in FP32; the
// factor 2^11 keeps lo inside FP16's normal range for values down to
// ~2^-14, where an unscaled remainder would be subnormal and lose its bits).
// The pair carries ~2^-23 relative; every product with one lo factor is
// scaled back by 2^-11 when it is read from TMEM.
constexpr float kLoScale = 2048.0f, kLoInv = 1.0f / 2048.0f;
__device__ __forceinline__ void split_f16x2(float e0, float e1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(e0, e1);
  const float2 hf = __half22float2(h);
  float l0, l1;
  up(sub2(pk(e0, e1), pk(hf.x, hf.y)), l0, l1);
  const __half2 l = __floats2half2_rn(l0 * kLoScale, l1 * kLoScale);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// E' for two targets (A, B) and sources j..j+7 of the stage (row stride 64
// floats); results as FP16 hi / lo rows (4 words each).
template <int D, int KER>
__device__ __forceinline__ void eval8x2(const float* sc, int j, const u64* xa, const u64* xb, uint32_t* ha,
                                        uint32_t* la, uint32_t* hb, uint32_t* lb) {
  u64 pa[4], pb[4];
  if (KER == DWFMM_K_GAUSS) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sc + k * kChunk + j);
      const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sc + k * kChunk + j + 4);
      if (k == 0) {
        pa[0] = mul2(xa[0], v0.x); pa[1] = mul2(xa[0], v0.y); pa[2] = mul2(xa[0], v1.x); pa[3] = mul2(xa[0], v1.y);
        pb[0] = mul2(xb[0], v0.x); pb[1] = mul2(xb[0], v0.y); pb[2] = mul2(xb[0], v1.x); pb[3] = mul2(xb[0], v1.y);
      } else {
        pa[0] = fma2(xa[k], v0.x, pa[0]); pa[1] = fma2(xa[k], v0.y, pa[1]);
        pa[2] = fma2(xa[k], v1.x, pa[2]); pa[3] = fma2(xa[k], v1.y, pa[3]);
        pb[0] = fma2(xb[k], v0.x, pb[0]); pb[1] = fma2(xb[k], v0.y, pb[1]);
        pb[2] = fma2(xb[k], v1.x, pb[2]); pb[3] = fma2(xb[k], v1.y, pb[3]);
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) pa[u] = pb[u] = 0ull;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sc + k * kChunk + j);
      const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sc + k * kChunk + j + 4);
      u64 df;
      df = sub2(xa[k], v0.x); pa[0] = fma2(df, df, pa[0]);
      df = sub2(xa[k], v0.y); pa[1] = fma2(df, df, pa[1]);
      df = sub2(xa[k], v1.x); pa[2] = fma2(df, df, pa[2]);
      df = sub2(xa[k], v1.y); pa[3] = fma2(df, df, pa[3]);
      df = sub2(xb[k], v0.x); pb[0] = fma2(df, df, pb[0]);
      df = sub2(xb[k], v0.y); pb[1] = fma2(df, df, pb[1]);
      df = sub2(xb[k], v1.x); pb[2] = fma2(df, df, pb[2]);
      df = sub2(xb[k], v1.y); pb[3] = fma2(df, df, pb[3]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float f0, f1;
    up(pa[u], f0, f1);
    split_f16x2(phi_sym<KER>(f0), phi_sym<KER>(f1), ha[u], la[u]);
    up(pb[u], f0, f1);
    split_f16x2(phi_sym<KER>(f0), phi_sym<KER>(f1), hb[u], lb[u]);
  }
}

// E' for one target (A) against sources j..j+7 (a) and j+8..j+15 (b) of
// the stage: the one-tile (128-slot) form of eval8x2.
template <int D, int KER>
__device__ __forceinline__ void eval16x1(const float* sc, int j, const u64* xa, uint32_t* ha, uint32_t* la,
                                         uint32_t* hb, uint32_t* lb) {
  u64 pa[4], pb[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) pa[u] = pb[u] = 0ull;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sc + k * kChunk + j);
    const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sc + k * kChunk + j + 4);
    const ulonglong2 w0 = *reinterpret_cast<const ulonglong2*>(sc + k * kChunk + j + 8);
    const ulonglong2 w1 = *reinterpret_cast<const ulonglong2*>(sc + k * kChunk + j + 12);
    if (KER == DWFMM_K_GAUSS) {
      pa[0] = fma2(xa[k], v0.x, pa[0]); pa[1] = fma2(xa[k], v0.y, pa[1]);
      pa[2] = fma2(xa[k], v1.x, pa[2]); pa[3] = fma2(xa[k], v1.y, pa[3]);
      pb[0] = fma2(xa[k], w0.x, pb[0]); pb[1] = fma2(xa[k], w0.y, pb[1]);
      pb[2] = fma2(xa[k], w1.x, pb[2]); pb[3] = fma2(xa[k], w1.y, pb[3]);
    } else {
      u64 df;
      df = sub2(xa[k], v0.x); pa[0] = fma2(df, df, pa[0]);
      df = sub2(xa[k], v0.y); pa[1] = fma2(df, df, pa[1]);
      df = sub2(xa[k], v1.x); pa[2] = fma2(df, df, pa[2]);
      df = sub2(xa[k], v1.y); pa[3] = fma2(df, df, pa[3]);
      df = sub2(xa[k], w0.x); pb[0] = fma2(df, df, pb[0]);
      df = sub2(xa[k], w0.y); pb[1] = fma2(df, df, pb[1]);
      df = sub2(xa[k], w1.x); pb[2] = fma2(df, df, pb[2]);
      df = sub2(xa[k], w1.y); pb[3] = fma2(df, df, pb[3]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float f0, f1;
    up(pa[u], f0, f1);
    split_f16x2(phi_sym<KER>(f0), phi_sym<KER>(f1), ha[u], la[u]);
    up(pb[u], f0, f1);
    split_f16x2(phi_sym<KER>(f0), phi_sym<KER>(f1), hb[u], lb[u]);
  }
}

__device__ __forceinline__ void sts128(uint32_t addr, const uint32_t* v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}

__device__ __forceinline__ void red_add_u64(unsigned long long* p, long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(static_cast<unsigned long long>(v)) : "memory");
}

__device__ __forceinline__ void tmem_ld4x2(uint32_t ta, uint32_t tb, uint32_t* r, uint32_t* q) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(ta));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3])
               : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 columns, load only: the registers are valid after tmem_wait_ld16 on
// the same array (which names them, so no use moves above the wait).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// 32 columns of the warp's TMEM lanes in one load, one wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct SymArgs {
  const float* pts;          // scaled blocks [L][D+1][ld] (coordinates, row D = |x'|^2)
  int64_t gstride;           // (D+1) * ld
  const uint16_t* bq;        // FP16 charge blocks [L][ld/8][4][64] (hi r0-7, hi r8-15, lo r0-7, lo r8-15)
  const int32_t* uprow;      // [L+1] upper entries of each target leaf
  const int32_t* ups;        // [nup] source leaf of each upper entry (ascending, the first is T itself)
  const int32_t* order;      // [L] target leaves, longest upper row first
  float* fwd;                // [L][16][ld] forward sums (normalised units)
  unsigned long long* acc;   // [L][16][ld] fixed-point transposed sums
  float acc_scale;           // 2^sb
  int ld;                    // 128 or 256
  int* err;
};

template <int D, int KER>
__global__ void __launch_bounds__(kSymTcThreads, 1) k_near_sym_tc(SymArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[32];
  __shared__ uint32_t tmem_slot;
  uint64_t* full = bars;                    // [kStages] TMA landed
  uint64_t* sfree = full + kStages;         // [kStages] stage consumed (16 warps + MMA commit)
  uint64_t* efull = sfree + kStages;        // [2] E tile written (16 warps)
  uint64_t* efree = efull + 2;              // [2] E tile read by the MMAs (commit)
  uint64_t* tfull = efree + 2;              // [2] transposed accumulator complete (commit)
  uint64_t* tempty = tfull + 2;             // [2] transposed accumulator drained (16 warps)
  uint64_t* cready = tempty + 2;            // [2] lo rows combined into shared memory (8 warps)
  uint64_t* ffull = cready + 2;             // [2] forward accumulators of an entry complete (commit)
  uint64_t* fempty = ffull + 2;             // [2] forward accumulators folded (16 warps)
  uint64_t* qfull = fempty + 2;             // q_T landed
  uint64_t* fin = qfull + 1;                // [2] every MMA of an issuer done
  static_assert(2 * kStages + 17 <= 32, "barrier array");

  const int ld = a.ld;
  const int NT = ld / 128;                    // 128-target tiles
  const int NC = ld / kChunk;                 // chunks per source leaf
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int T = a.order[blockIdx.x];
  const int e0 = a.uprow[T], ne = a.uprow[T + 1] - e0;

  // shared memory carve-up
  const uint32_t ebytes = static_cast<uint32_t>(NT * 16 * kTS);        // one E tile
  const uint32_t coord_bytes = static_cast<uint32_t>(D * kChunk * 4);
  const uint32_t qoff = (coord_bytes + 1023u) & ~1023u;
  const uint32_t stage_bytes = qoff + kQChunkBytes;
  unsigned char* ebuf = smem;                                       // 2 tiles
  unsigned char* stages = smem + 2 * ebytes;                         // kStages
  unsigned char* qT = stages + kStages * stage_bytes;               // ld * 64 bytes
  float* ksum = reinterpret_cast<float*>(qT + ld * 64);              // [NT][16][128] sums, then compensations
  float* comb = ksum + 2 * NT * 16 * 128;                            // [2][16][64]

  if (t == 0) {
    for (int i = 0; i < kStages; ++i) {
      bar_init(&full[i], 1);
      bar_init(&sfree[i], kSymCompWarps + 1);
    }
    for (int i = 0; i < 2; ++i) {
      bar_init(&efull[i], kSymCompWarps);
      bar_init(&efree[i], 2);   // the forward and the transposed issuer
      bar_init(&tfull[i], 1);
      bar_init(&tempty[i], kSymCompWarps);
      bar_init(&cready[i], kSymCompWarps / 2);
      bar_init(&ffull[i], 1);
      bar_init(&fempty[i], kSymCompWarps);
    }
    bar_init(qfull, 1);
    bar_init(&fin[0], 1);
    bar_init(&fin[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kSymCompWarps + 1) {
    // ---- TMA producer
    if (lane == 0) {
      bool bad = false;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_expect_tx(qfull, static_cast<uint32_t>(ld * 64));
      bulk_load(qT, a.bq + static_cast<int64_t>(T) * ld * 32, static_cast<uint32_t>(ld * 64), qfull);
      int i = 0;
      for (int e = 0; e < ne && !bad; ++e) {
        const int S = a.ups[e0 + e];
        for (int c = 0; c < NC; ++c, ++i) {
          const int st = i % kStages;
          if (i >= kStages && !wait_sleep(&sfree[st], static_cast<uint32_t>(((i - kStages) / kStages) & 1))) {
            bad = true;
            break;
          }
          unsigned char* dst = stages + st * stage_bytes;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar_expect_tx(&full[st], coord_bytes + kQChunkBytes);
          const float* src = a.pts + static_cast<int64_t>(S) * a.gstride + c * kChunk;
#pragma unroll 1
          for (int k = 0; k < D; ++k) bulk_load(dst + k * kChunk * 4, src + static_cast<int64_t>(k) * ld, kChunk * 4,
                                                &full[st]);
          bulk_load(dst + qoff, a.bq + (static_cast<int64_t>(S) * ld + c * kChunk) * 32, kQChunkBytes, &full[st]);
        }
      }
      // copies in flight land before the CTA exits
      (void)wait_sleep(qfull, 0u);
      for (int j = i > kStages ? i - kStages : 0; j < i; ++j)
        (void)wait_sleep(&full[j % kStages], static_cast<uint32_t>((j / kStages) & 1));
      if (bad) atomicExch(a.err, 3);
    }
  } else if (warp == kSymCompWarps + 2) {
    // ---- transposed-product issuer (MMAs issued by two threads proceed
    // concurrently; one thread's issue rate bounded the kernel)
    if (lane == 0) {
      bool bad = !wait_sleep(qfull, 0u);
      const uint32_t ebase = sptr(ebuf), qtb = sptr(qT);
      int i = 0, jt = 0;
      for (int e = 0; e < ne && !bad; ++e) {
        const bool diag = a.ups[e0 + e] == T;
        for (int c = 0; c < NC; ++c, ++i) {
          const int eb = i & 1;
          if (!wait_sleep(&efull[eb], static_cast<uint32_t>((i >> 1) & 1))) {
            bad = true;
            break;
          }
          if (!diag) {
            const int tb = jt & 1;
            if (jt >= 2 && !wait_sleep(&tempty[tb], static_cast<uint32_t>(((jt - 2) >> 1) & 1))) {
              bad = true;
              break;
            }
            fence_after();
            const uint32_t et = ebase + eb * ebytes;
            const uint32_t dcol = tmem + static_cast<uint32_t>(128 + tb * 32);
            for (int j = 0; j < NT * 8; ++j) {
              // A: rows [E_hi of 64 sources ; E_lo of 64 sources], MN-major
              const u64 at = smem_desc(et + j * 2 * kTS, kSymTrnLbo, kSymTrnSbo);
              const u64 bq = smem_desc(qtb + j * 2 * 512, 512, 128);
              mma_f16(dcol, at, bq, kIdTrn32, j > 0 ? 1u : 0u);
            }
            mma_commit(&tfull[tb]);
            ++jt;
          }
          mma_commit(&efree[eb]);
        }
      }
      mma_commit(&fin[1]);
      (void)wait_sleep(&fin[1], 0u);
      if (bad) atomicExch(a.err, 3);
    }
  } else if (warp == kSymCompWarps) {
    // ---- forward-product issuer
    if (lane == 0) {
      bool bad = false;
      const uint32_t ebase = sptr(ebuf), sbase = sptr(stages);
      int i = 0;
      for (int e = 0; e < ne && !bad; ++e) {
        const int fb = e & 1;
        for (int c = 0; c < NC; ++c, ++i) {
          const int st = i % kStages, eb = i & 1;
          if (!wait_sleep(&full[st], static_cast<uint32_t>((i / kStages) & 1)) ||
              !wait_sleep(&efull[eb], static_cast<uint32_t>((i >> 1) & 1)) ||
              (c == 0 && e >= 2 && !wait_sleep(&fempty[fb], static_cast<uint32_t>(((e - 2) >> 1) & 1)))) {
            bad = true;
            break;
          }
          fence_after();
          const uint32_t et = ebase + eb * ebytes;
          const uint32_t qs = sbase + st * stage_bytes + qoff;
          // forward: D[t][r] over the chunk's sources, K = 16 per MMA
          for (int at = 0; at < NT; ++at) {
            const uint32_t dcol = tmem + static_cast<uint32_t>(fb * 64 + at * 32);
            for (int kk = 0; kk < kChunk / 16; ++kk) {
              const uint32_t aoff = et + at * 16 * kTS + kk * 2 * 128;
              const u64 ahi = smem_desc(aoff, 128, kTS);
              const u64 alo = smem_desc(aoff + kHL, 128, kTS);
              const u64 bq = smem_desc(qs + kk * 2 * 512, 512, 128);
              mma_f16(dcol, ahi, bq, kIdFwd32, (c > 0 || kk > 0) ? 1u : 0u);
              mma_f16(dcol + 16, alo, bq, kIdFwd16, 1u);
            }
          }
          mma_commit(&efree[eb]);
          mma_commit(&sfree[st]);
          if (c == NC - 1) mma_commit(&ffull[fb]);
        }
      }
      mma_commit(&fin[0]);
      (void)wait_sleep(&fin[0], 0u);
      if (bad) atomicExch(a.err, 3);
    }
  } else {
    // ---- compute warps
    const int qd = warp & 3, part = warp >> 2;   // TMEM lane quadrant, source quarter of a chunk
    const int ta = qd * 32 + lane;               // targets ta and ta + 128 (tile 1, if NT == 2)
    const float* tp = a.pts + static_cast<int64_t>(T) * a.gstride;
    u64 xa[D], xb[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float va = tp[k * ld + ta];
      float vb = NT == 2 ? tp[k * ld + ta + 128] : va;
      if (KER == DWFMM_K_GAUSS) {
        va *= 2.0f;
        vb *= 2.0f;
      }
      xa[k] = pk(va, va);
      xb[k] = pk(vb, vb);
    }
    // Kahan sums: warp (qd, part) owns tile part / 2, right-hand sides 8 (part % 2) .. + 7
    const int ftile = part >> 1, fr0 = 8 * (part & 1);
    const bool fown = ftile < NT;
    if (fown) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        ksum[(ftile * 16 + fr0 + r) * 128 + ta] = 0.0f;
        ksum[NT * 16 * 128 + (ftile * 16 + fr0 + r) * 128 + ta] = 0.0f;
      }
    }
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(qd * 32) << 16);
    bool bad = false;

    // fold the forward accumulators of entry e into the sums
    auto fold = [&](int e) {
      const int fb = e & 1;
      const bool ok = wait_sleep(&ffull[fb], static_cast<uint32_t>((e >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok)) {
        bad = true;
        return;
      }
      fence_after();
      if (fown) {
        uint32_t dv[8], dl[8];
        const uint32_t col = lane_base + static_cast<uint32_t>(fb * 64 + ftile * 32 + fr0);
        tmem_ld8x2(col, col + 16, dv, dl);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          float* pa = ksum + (ftile * 16 + fr0 + r) * 128 + ta;
          const float acc = pa[0], comp = pa[NT * 16 * 128];
          const float y = (__uint_as_float(dv[r]) + __uint_as_float(dl[r]) * kLoInv) - comp;
          const float s = acc + y;
          pa[NT * 16 * 128] = (s - acc) - y;
          pa[0] = s;
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(&fempty[fb]);
    };
    // drain transposed accumulator jt (chunk c of source leaf S) into the
    // fixed-point sums of S
    auto flush = [&](int jt, int S, int c) {
      const int tb = jt & 1;
      const bool ok = wait_sleep(&tfull[tb], static_cast<uint32_t>((jt >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok)) {
        bad = true;
        return;
      }
      fence_after();
      const int r0 = 4 * part;
      const uint32_t col = lane_base + static_cast<uint32_t>(128 + tb * 32 + r0);
      uint32_t x[4], y[4];
      tmem_ld4x2(col, col + 16, x, y);
      float* cb = comb + tb * (64 * 16);
      if (qd >= 2) {
        // rows 64..127: E_lo of source 32 (qd - 2) + lane
        const int s = (qd - 2) * 32 + lane;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          cb[(r0 + j) * 64 + s] = (__uint_as_float(x[j]) + __uint_as_float(y[j]) * kLoInv) * kLoInv;
        fence_before();
        __syncwarp();
        if (lane == 0) {
          bar_arrive(&cready[tb]);
          bar_arrive(&tempty[tb]);
        }
      } else {
        const int s = qd * 32 + lane;
        const bool okc = wait_sleep(&cready[tb], static_cast<uint32_t>((jt >> 1) & 1));
        if (__any_sync(0xffffffffu, !okc)) {
          bad = true;
          fence_before();
          if (lane == 0) bar_arrive(&tempty[tb]);
          return;
        }
        unsigned long long* dst = a.acc + (static_cast<int64_t>(S) * 16 + r0) * ld + c * kChunk + s;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float v = (__uint_as_float(x[j]) + __uint_as_float(y[j]) * kLoInv) + cb[(r0 + j) * 64 + s];
          red_add_u64(dst + static_cast<int64_t>(j) * ld, __float2ll_rn(v * a.acc_scale));
        }
        fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(&tempty[tb]);
      }
    };

    int i = 0, jt = 0;
    int pend_jt = -1, pend_S = 0, pend_c = 0;
    for (int e = 0; e < ne && !bad; ++e) {
      const int S = a.ups[e0 + e];
      const bool diag = S == T;
      for (int c = 0; c < NC; ++c, ++i) {
        const int st = i % kStages, eb = i & 1;
        const bool ok = wait_sleep(&full[st], static_cast<uint32_t>((i / kStages) & 1)) &&
                        (i < 2 || wait_sleep(&efree[eb], static_cast<uint32_t>(((i - 2) >> 1) & 1)));
        if (__any_sync(0xffffffffu, !ok)) {
          bad = true;
          break;
        }
        const float* sc = reinterpret_cast<const float*>(stages + st * stage_bytes);
        const uint32_t et = sptr(ebuf + eb * ebytes);
        if (NT == 2) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = part * 16 + h * 8;   // source within the chunk
            uint32_t ha[4], la[4], hb[4], lb[4];
            eval8x2<D, KER>(sc, j, xa, xb, ha, la, hb, lb);
            const uint32_t off = static_cast<uint32_t>((ta >> 3) * kTS + (j >> 3) * 128 + (ta & 7) * 16);
            sts128(et + off, ha);
            sts128(et + off + kHL, la);
            sts128(et + off + 16 * kTS, hb);
            sts128(et + off + 16 * kTS + kHL, lb);
          }
        } else {   // one tile: the thread's target against 16 sources
          const int j = part * 16;
          uint32_t ha[4], la[4], hb[4], lb[4];
          eval16x1<D, KER>(sc, j, xa, ha, la, hb, lb);
          const uint32_t off = static_cast<uint32_t>((ta >> 3) * kTS + (j >> 3) * 128 + (ta & 7) * 16);
          sts128(et + off, ha);
          sts128(et + off + kHL, la);
          sts128(et + off + 128, hb);
          sts128(et + off + 128 + kHL, lb);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          bar_arrive(&efull[eb]);
          bar_arrive(&sfree[st]);
        }
        // service: the previous chunk's transposed sums, the previous entry's forward sums
        if (pend_jt >= 0) {
          flush(pend_jt, pend_S, pend_c);
          pend_jt = -1;
          if (bad) break;
        }
        if (c == 0 && e >= 1) {
          fold(e - 1);
          if (bad) break;
        }
        if (!diag) {
          pend_jt = jt;
          pend_S = S;
          pend_c = c;
          ++jt;
        }
      }
    }
    if (!bad && pend_jt >= 0) flush(pend_jt, pend_S, pend_c);
    if (!bad && ne >= 1) fold(ne - 1);
    if (bad && lane == 0) atomicExch(a.err, 3);
    if (fown) {
      float* op = a.fwd + static_cast<int64_t>(T) * 16 * ld + ftile * 128 + ta;
#pragma unroll
      for (int r = 0; r < 8; ++r) op[(fr0 + r) * ld] = ksum[(ftile * 16 + fr0 + r) * 128 + ta];
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// Per right-hand side: the largest |q * factor| (float bits, atomicMax).
// Charges xb[g][r][s] with row stride xld; slots s >= nvalid hold none.
__global__ void k_sym_colmax(const float* xb, int64_t xld, int nvalid, const float* pts, int64_t gstride, int L,
                             int ld, int D, int gauss, int Rc, unsigned* colmax) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = static_cast<int64_t>(L) * ld;
  float m[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) m[r] = 0.0f;
  for (int64_t p = i; p < n; p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t g = p / ld;
    const int s = static_cast<int>(p % ld);
    if (s >= nvalid) continue;
    const float f = gauss ? exp2f(-pts[g * gstride + static_cast<int64_t>(D) * ld + s]) : 1.0f;
    for (int r = 0; r < Rc; ++r) m[r] = fmaxf(m[r], fabsf(xb[(g * 16 + r) * xld + s] * f));
  }
  for (int r = 0; r < Rc; ++r) {
    float v = m[r];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.0f) atomicMax(&colmax[r], __float_as_uint(v));
  }
}

// Power of two that brings the column's largest |q'| into [0.5, 1).
__device__ __forceinline__ float col_scale_exp(unsigned bits, int* e) {
  const float m = __uint_as_float(bits);
  int ex = 0;
  if (m > 0.0f) (void)frexpf(m, &ex);
  *e = ex;
  return ldexpf(1.0f, -ex);
}

// FP16 hi / lo charge blocks: q' = q * factor * 2^-e_r, core (s/8, n/8) at
// (s/8)*512 + (n/8)*128, row n%8 at 16 bytes, source s%8 at 2 bytes; n < 16
// hi, n >= 16 lo.
__global__ void k_sym_make_bq(const float* xb, int64_t xld, int nvalid, const float* pts, int64_t gstride, int L,
                              int ld, int D, int gauss, int Rc, const unsigned* colmax, uint16_t* bq) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(L) * ld * 16) return;
  const int r = static_cast<int>(i % 16);
  const int64_t gs = i / 16;
  const int s = static_cast<int>(gs % ld);
  const int64_t g = gs / ld;
  float v = 0.0f;
  if (r < Rc && s < nvalid) {
    int ex;
    const float sc = col_scale_exp(colmax[r], &ex);
    const float f = gauss ? exp2f(-pts[g * gstride + static_cast<int64_t>(D) * ld + s]) : 1.0f;
    v = xb[(g * 16 + r) * xld + s] * f * sc;
  }
  const __half h = __float2half_rn(v);
  const __half l = __float2half_rn((v - __half2float(h)) * kLoScale);
  uint16_t* blk = bq + g * static_cast<int64_t>(ld) * 32;
  const int64_t base = (s / 8) * 256 + (s % 8);               // in 2-byte units
  blk[base + (r / 8) * 64 + (r % 8) * 8] = __half_as_ushort(h);
  blk[base + (2 + r / 8) * 64 + (r % 8) * 8] = __half_as_ushort(l);
}

// y = (forward + fixed-point transposed) * 2^e_r * factor(t), written to
// y[g * ystride + r * yrow + s] for slots s < nvalid.
__global__ void k_sym_finish(const float* fwd, const unsigned long long* acc, double inv_scale, const float* pts,
                             int64_t gstride, int L, int ld, int D, int gauss, int Rc, const unsigned* colmax,
                             float* ynear, int64_t ystride, int64_t yrow, int nvalid) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(L) * 16 * ld) return;
  const int s = static_cast<int>(i % ld);
  const int r = static_cast<int>((i / ld) % 16);
  const int64_t g = i / (16 * static_cast<int64_t>(ld));
  if (r >= Rc || s >= nvalid) return;
  int ex;
  (void)col_scale_exp(colmax[r], &ex);
  const double tr = static_cast<double>(static_cast<long long>(acc[i])) * inv_scale;
  double v = (static_cast<double>(fwd[i]) + tr) * ldexp(1.0, ex);
  if (gauss) v *= static_cast<double>(exp2f(-pts[g * gstride + static_cast<int64_t>(D) * ld + s]));
  ynear[g * ystride + static_cast<int64_t>(r) * yrow + s] = static_cast<float>(v);
}

// ---------------------------------------------------------------------------
// Gaussian variant with the exponent on the tensor cores.
//
// For the factored Gaussian the exponent is a dot product, G = 2 x'.s'
// (padded dimension <= 16), so it is one more small contraction:
// G = X2 S^T with X2 = 2x' of the 256 targets (A, M = 128 per tile) and S =
// s' of the chunk's 64 sources (B, N = 64), both as FP16 hi + lo, K = 16.
// The two small products (hi*lo, lo*hi) are accumulated first and the large
// one (hi*hi) last, so the accumulator's round-toward-zero step applies
// once at the magnitude of G: ~1 ulp of |G| <= 2 * bound, as the FP32
// multiply-add chain.  The CUDA cores only read G from tensor memory,
// apply ex2, split E' into FP16 hi / lo and store the E tile; the rest
// (forward and transposed products, folds, fixed-point flushes) is the
// kernel above.
//
// Coordinate blocks [L][2 (hi, lo)][ld/8][2][128 B]: core (p/8, k/8) of
// point p, coordinate k (8 FP16 per row); the target tile of T (2x') stays
// resident, the source chunk (x') comes with the stage.
// ---------------------------------------------------------------------------

constexpr int kKD = 16;                                  // padded dimension of the G contraction
constexpr uint32_t kIdG = idesc_f16(128, 64, 0);
constexpr int kXChunkHalf = (kChunk / 8) * (kKD / 8) * 128;   // 2 KB: one of hi / lo of a chunk

// hi / lo FP16 coordinate blocks: xa = 2x' (target role), xb = x' (source role).
// hi = the coordinate rounded to FP16, lo = the exact FP32 remainder rounded
// to FP16: |lo| <= 2^-11 |v| with either sign, so the lo * lo product the G
// contraction leaves out is <= 2^-22 of a term and unbiased.  (Truncating hi
// instead leaves a remainder of up to 2^-10 |v| with the sign of v: the
// dropped lo * lo terms then all shrink |G| and bias E' = 2^G by up to
// 2^-20 |G| relative, a smooth error that does not average out in K x.)
// Remainders of coordinates below 2^-3 are FP16 subnormals: absolute error
// <= 2^-25, far below the accumulator's rounding of G.
__global__ void k_sym_make_x16(const float* pts, int64_t gstride, int L, int ld, int D, uint16_t* xa, uint16_t* xb) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(L) * ld * kKD) return;
  const int k = static_cast<int>(i % kKD);
  const int64_t gp = i / kKD;
  const int p = static_cast<int>(gp % ld);
  const int64_t g = gp / ld;
  const float v = k < D ? pts[g * gstride + static_cast<int64_t>(k) * ld + p] : 0.0f;
  const __half hh = __float2half_rn(v);
  const float r = v - __half2float(hh);                                   // exact
  const __half hl = __float2half_rn(r);
  const __half ah = __float2half_rn(2.0f * __half2float(hh)), al = __float2half_rn(2.0f * r);
  const int64_t blk = g * static_cast<int64_t>(ld) * kKD * 2;            // halfs per leaf
  const int64_t off = (p / 8) * (kKD / 8) * 64 + (k / 8) * 64 + (p % 8) * 8 + (k % 8);
  const int64_t lo = static_cast<int64_t>(ld) * kKD;                      // hi -> lo
  xb[blk + off] = __half_as_ushort(hh);
  xb[blk + lo + off] = __half_as_ushort(hl);
  xa[blk + off] = __half_as_ushort(ah);
  xa[blk + lo + off] = __half_as_ushort(al);
}

struct SymGArgs {
  const uint16_t* xa;        // [L][2][ld/8][2][64] 2x' hi / lo
  const uint16_t* xb;        // x' hi / lo
  const uint16_t* bq;        // FP16 charge blocks [L][ld/8][4][64]
  const int32_t* uprow;
  const int32_t* ups;
  const int32_t* order;
  float* fwd;
  unsigned long long* acc;
  float acc_scale;
  int ld;                    // 256
  int* err;
};

// NT target tiles of 128 (leaves of 256 slots: NT = 2; node sets of 128: NT = 1).
template <int NT>
__global__ void __launch_bounds__(kSymGThreads, 1) k_near_sym_gtc(SymGArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[32];
  __shared__ uint32_t tmem_slot;
  uint64_t* full = bars;                    // [kStages] TMA landed (coordinates + charges of a chunk)
  uint64_t* sfree = full + kStages;         // [kStages] stage read by the MMAs
  uint64_t* efull = sfree + kStages;        // [2] E tile written (16 warps)
  uint64_t* efree = efull + 2;              // [2] E tile read by the MMAs
  uint64_t* tfull = efree + 2;              // [2] transposed accumulator complete
  uint64_t* tempty = tfull + 2;             // [2] transposed accumulator drained (16 warps)
  uint64_t* cready = tempty + 2;            // [2] lo rows combined (8 warps)
  uint64_t* ffull = cready + 2;             // [2] forward accumulators of an entry complete
  uint64_t* fempty = ffull + 2;             // [2] forward accumulators folded (16 warps)
  uint64_t* gfull = fempty + 2;             // [2] G of a chunk complete
  uint64_t* gfree = gfull + 2;              // [2] G read by the compute warps (16 warps)
  uint64_t* qfull = gfree + 2;              // q_T and 2x'_T landed
  uint64_t* fin = qfull + 1;                // [4] all MMAs of an issuer complete (3 used)
  static_assert(2 * kStages + 23 <= 32, "barrier array");

  constexpr int ld = 128 * NT;      // NT 128-target tiles, 2 NT 64-source chunks
  constexpr int NC = 2 * NT;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int T = a.order[blockIdx.x];
  const int e0 = a.uprow[T], ne = a.uprow[T + 1] - e0;
  const int nchunks = ne * NC;

  constexpr uint32_t ebytes = NT * 16 * kTS;                         // 32 KB per tile
  constexpr uint32_t stage_bytes = 2 * kXChunkHalf + kQChunkBytes;  // 8 KB
  unsigned char* ebuf = smem;
  unsigned char* stages = smem + 2 * ebytes;
  constexpr uint32_t xbytes = ld * kKD * 2 * 2;                     // target coordinates, hi and lo
  unsigned char* qT = stages + kStages * stage_bytes;               // ld * 64 bytes
  unsigned char* xT = qT + ld * 64;                                  // ld * 64 bytes
  float* comb = reinterpret_cast<float*>(xT + xbytes);              // [2][16][64]
  // TMEM column bases: G (2 buffers x NT tiles x 64), forward accumulators
  // (2 x NT x 32), transposed accumulators (2 x 32 per K half: one half per
  // target tile)
  constexpr uint32_t kGB = NT * 64, kFB = NT * 32;
  constexpr uint32_t kG = 0, kF = 2 * kGB, kTr = kF + 2 * kFB, kTr1 = kTr + 64;
  constexpr uint32_t kCols = NT == 2 ? 512 : 256;
  static_assert(kTr + 64 * NT <= kCols, "TMEM columns");

  if (t == 0) {
    // barriers the MMAs complete count one commit of each issuer that uses
    // the resource: the stage and G (two G / forward issuers), the E tile
    // (all three), the transposed accumulators (the transposed issuer)
    for (int i = 0; i < kStages; ++i) {
      bar_init(&full[i], 1);
      bar_init(&sfree[i], NT);
    }
    for (int i = 0; i < 2; ++i) {
      bar_init(&efull[i], kSymCompWarps);
      bar_init(&efree[i], NT + 1);
      bar_init(&tfull[i], 1);
      bar_init(&tempty[i], kSymCompWarps);
      bar_init(&cready[i], kSymCompWarps / 2);
      bar_init(&ffull[i], NT);
      bar_init(&fempty[i], kSymCompWarps);
      bar_init(&gfull[i], NT);
      bar_init(&gfree[i], kSymCompWarps);
    }
    bar_init(qfull, 1);
    for (int i = 0; i < 4; ++i) bar_init(&fin[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kSymCompWarps + 1) {
    // ---- TMA producer
    if (lane == 0) {
      bool bad = false;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_expect_tx(qfull, static_cast<uint32_t>(ld * 64 + xbytes));
      bulk_load(qT, a.bq + static_cast<int64_t>(T) * ld * 32, static_cast<uint32_t>(ld * 64), qfull);
      bulk_load(xT, a.xa + static_cast<int64_t>(T) * ld * kKD * 2, xbytes, qfull);
      int i = 0;
      for (int e = 0; e < ne && !bad; ++e) {
        const int S = a.ups[e0 + e];
        const uint16_t* xs = a.xb + static_cast<int64_t>(S) * ld * kKD * 2;
        for (int c = 0; c < NC; ++c, ++i) {
          const int st = i % kStages;
          if (i >= kStages && !wait_sleep(&sfree[st], static_cast<uint32_t>(((i - kStages) / kStages) & 1))) {
            bad = true;
            break;
          }
          unsigned char* dst = stages + st * stage_bytes;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar_expect_tx(&full[st], stage_bytes);
          bulk_load(dst, xs + c * (kXChunkHalf / 2), kXChunkHalf, &full[st]);
          bulk_load(dst + kXChunkHalf, xs + static_cast<int64_t>(ld) * kKD + c * (kXChunkHalf / 2), kXChunkHalf,
                    &full[st]);
          bulk_load(dst + 2 * kXChunkHalf, a.bq + (static_cast<int64_t>(S) * ld + c * kChunk) * 32, kQChunkBytes,
                    &full[st]);
        }
      }
      (void)wait_sleep(qfull, 0u);
      for (int j = i > kStages ? i - kStages : 0; j < i; ++j)
        (void)wait_sleep(&full[j % kStages], static_cast<uint32_t>((j / kStages) & 1));
      if (bad) atomicExch(a.err, 3);
    }
  } else if (warp == kSymCompWarps + 3) {
    // ---- transposed-product issuer (E^T q_T over both target tiles, one K
    // half per TMEM accumulator), beside the two G / forward issuers: MMAs
    // issued by several threads proceed concurrently, and one thread's issue
    // rate bounded the kernel.  Three issuers and one TMA warp leave 96
    // registers per thread (a fourth issuer forced spills and was slower)
    if (lane == 0) {
      bool bad = !wait_sleep(qfull, 0u);
      const u64 dT_a = smem_desc(sptr(ebuf), kSymTrnLbo, kSymTrnSbo);   // E tile 0, transposed A
      const u64 dT_b = smem_desc(sptr(qT), 512, 128);                     // q_T
      int i = 0, jt = 0;
      for (int e = 0; e < ne && !bad; ++e) {
        const bool diag = a.ups[e0 + e] == T;
        for (int c = 0; c < NC; ++c, ++i) {
          const int eb = i & 1;
          if (!wait_sleep(&efull[eb], static_cast<uint32_t>((i >> 1) & 1))) {
            bad = true;
            break;
          }
          if (!diag) {
            const int tb = jt & 1;
            if (jt >= 2 && !wait_sleep(&tempty[tb], static_cast<uint32_t>(((jt - 2) >> 1) & 1))) {
              bad = true;
              break;
            }
            fence_after();
            const u64 ta = dT_a + ((eb * ebytes) >> 4);
#pragma unroll
            for (int h = 0; h < NT; ++h) {
              const uint32_t dcol = tmem + (h == 0 ? kTr : kTr1) + static_cast<uint32_t>(tb * 32);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const int j = 8 * h + jj;
                mma_f16(dcol, ta + ((j * 2 * kTS) >> 4), dT_b + ((j * 2 * 512) >> 4), kIdTrn32, jj > 0 ? 1u : 0u);
              }
            }
            mma_commit(&tfull[tb]);
            ++jt;
          }
          mma_commit(&efree[eb]);
        }
      }
      mma_commit(&fin[2]);
      (void)wait_sleep(&fin[2], 0u);
      if (bad) atomicExch(a.err, 3);
    }
  } else if (warp == kSymCompWarps || warp == kSymCompWarps + 2) {
    // ---- G / forward issuers, one per target tile: G of chunk i + 2 ahead
    // of the forward products of chunk i
    const int at = warp == kSymCompWarps ? 0 : 1;
    if (lane == 0 && at < NT) {
      bool bad = !wait_sleep(qfull, 0u);
      const uint32_t ebase = sptr(ebuf), sbase = sptr(stages), xtb = sptr(xT);
      constexpr uint32_t xlo = ld * kKD * 2;             // hi -> lo in the target block (bytes)
      // G MMAs of chunk i (stage i % kStages) into G buffer i & 1
      // descriptors: the start address is the low field (address / 16), so a
      // byte offset o moves a descriptor by o / 16
      const u64 dG_b = smem_desc(sbase, 128, 256);                  // stage 0 coordinates (hi)
      const u64 dG_a = smem_desc(xtb, 128, 256);                    // target tile 0 (hi)
      const u64 dF_a = smem_desc(ebase, 128, kTS);                  // E tile 0, forward A (hi)
      const u64 dF_b = smem_desc(sbase + 2 * kXChunkHalf, 512, 128);   // stage 0 charges
      auto issue_g = [&](int i) -> bool {
        const int st = i % kStages, gb = i & 1;
        if (!wait_sleep(&full[st], static_cast<uint32_t>((i / kStages) & 1))) return false;
        if (i >= 2 && !wait_sleep(&gfree[gb], static_cast<uint32_t>(((i - 2) >> 1) & 1))) return false;
        fence_after();
        const u64 bhi = dG_b + ((st * stage_bytes) >> 4), blo = bhi + (kXChunkHalf >> 4);
        {
          const u64 ahi = dG_a + ((at * 16 * 256) >> 4), alo = ahi + (xlo >> 4);
          const uint32_t d = tmem + kG + static_cast<uint32_t>(gb * kGB + at * 64);
          mma_f16(d, ahi, blo, kIdG, 0u);                // small terms first,
          mma_f16(d, alo, bhi, kIdG, 1u);
          mma_f16(d, ahi, bhi, kIdG, 1u);                // the large one last
        }
        mma_commit(&gfull[gb]);
        return true;
      };
      // G runs two chunks ahead of the products: G(i + 2) goes into the
      // buffer of G(i) as soon as the compute warps have read G(i), so the
      // products never wait on a G still queued behind other MMAs
      if (nchunks > 0 && !bad) bad = !issue_g(0);
      if (nchunks > 1 && !bad) bad = !issue_g(1);
      int i = 0;
      for (int e = 0; e < ne && !bad; ++e) {
        const int fb = e & 1;
        for (int c = 0; c < NC; ++c, ++i) {
          if (i + 2 < nchunks && !issue_g(i + 2)) {
            bad = true;
            break;
          }
          const int st = i % kStages, eb = i & 1;
          if (!wait_sleep(&efull[eb], static_cast<uint32_t>((i >> 1) & 1)) ||
              (c == 0 && e >= 2 && !wait_sleep(&fempty[fb], static_cast<uint32_t>(((e - 2) >> 1) & 1)))) {
            bad = true;
            break;
          }
          fence_after();
          const u64 fa = dF_a + ((eb * ebytes) >> 4);
          const u64 fb_desc = dF_b + ((st * stage_bytes) >> 4);
          {
            const uint32_t dcol = tmem + kF + static_cast<uint32_t>(fb * kFB + at * 32);
#pragma unroll
            for (int kk = 0; kk < kChunk / 16; ++kk) {
              const u64 ahi = fa + ((at * 16 * kTS + kk * 2 * 128) >> 4);
              const u64 bq = fb_desc + ((kk * 2 * 512) >> 4);
              mma_f16(dcol, ahi, bq, kIdFwd32, (c > 0 || kk > 0) ? 1u : 0u);
              mma_f16(dcol + 16, ahi + (kHL >> 4), bq, kIdFwd16, 1u);
            }
          }
          mma_commit(&efree[eb]);
          mma_commit(&sfree[st]);
          if (c == NC - 1) mma_commit(&ffull[fb]);
        }
      }
      mma_commit(&fin[at]);
      (void)wait_sleep(&fin[at], 0u);
      if (bad) atomicExch(a.err, 3);
    }
  } else {
    // ---- compute warps: (quadrant qd, part p): NT = 2: target tile p / 2,
    // sources 32 (p % 2) .. + 31 of each chunk and right-hand sides 8 (p % 2)
    // .. + 7 of the forward sums; NT = 1: sources 16 p .. + 15, right-hand
    // sides 8 p .. + 7 for p < 2
    const int qd = warp & 3, part = warp >> 2;
    const int at = NT == 2 ? part >> 1 : 0, sh = NT == 2 ? part & 1 : part;
    constexpr int kSrc = NT == 2 ? 32 : 16;   // sources per warp and chunk
    const bool fown = NT == 2 || part < 2;
    const int tl = qd * 32 + lane;                 // target within the tile (TMEM lane)
    const int tt = at * 128 + tl;                  // target within T
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(qd * 32) << 16);
    // Kahan sums in registers: tile `at`, right-hand sides 8 sh .. 8 sh + 7
    float ks[8], kc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) ks[r] = kc[r] = 0.0f;
    bool bad = false;

    auto fold = [&](int e) {
      const int fb = e & 1;
      const bool ok = wait_sleep(&ffull[fb], static_cast<uint32_t>((e >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok)) {
        bad = true;
        return;
      }
      fence_after();
      if (fown) {
        uint32_t dv[8], dl[8];
        const uint32_t col = lane_base + kF + static_cast<uint32_t>(fb * kFB + at * 32 + 8 * sh);
        tmem_ld8x2(col, col + 16, dv, dl);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float y = (__uint_as_float(dv[r]) + __uint_as_float(dl[r]) * kLoInv) - kc[r];
          const float s = ks[r] + y;
          kc[r] = (s - ks[r]) - y;
          ks[r] = s;
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(&fempty[fb]);
    };
    auto flush = [&](int jt, int S, int c) {
      const int tb = jt & 1;
      const bool ok = wait_sleep(&tfull[tb], static_cast<uint32_t>((jt >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok)) {
        bad = true;
        return;
      }
      fence_after();
      const int r0 = 4 * part;
      const uint32_t col = lane_base + kTr + static_cast<uint32_t>(tb * 32 + r0);
      uint32_t x[4], y[4];
      tmem_ld4x2(col, col + 16, x, y);
      if (NT == 2) {
        uint32_t x1[4], y1[4];
        tmem_ld4x2(col + (kTr1 - kTr), col + (kTr1 - kTr) + 16, x1, y1);   // the other K half
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          x[j] = __float_as_uint(__uint_as_float(x[j]) + __uint_as_float(x1[j]));
          y[j] = __float_as_uint(__uint_as_float(y[j]) + __uint_as_float(y1[j]));
        }
      }
      float* cb = comb + tb * (64 * 16);
      if (qd >= 2) {
        const int s = (qd - 2) * 32 + lane;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          cb[(r0 + j) * 64 + s] = (__uint_as_float(x[j]) + __uint_as_float(y[j]) * kLoInv) * kLoInv;
        fence_before();
        __syncwarp();
        if (lane == 0) {
          bar_arrive(&cready[tb]);
          bar_arrive(&tempty[tb]);
        }
      } else {
        const int s = qd * 32 + lane;
        const bool okc = wait_sleep(&cready[tb], static_cast<uint32_t>((jt >> 1) & 1));
        if (__any_sync(0xffffffffu, !okc)) {
          bad = true;
          fence_before();
          if (lane == 0) bar_arrive(&tempty[tb]);
          return;
        }
        unsigned long long* dst = a.acc + (static_cast<int64_t>(S) * 16 + r0) * ld + c * kChunk + s;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float v = (__uint_as_float(x[j]) + __uint_as_float(y[j]) * kLoInv) + cb[(r0 + j) * 64 + s];
          red_add_u64(dst + static_cast<int64_t>(j) * ld, __float2ll_rn(v * a.acc_scale));
        }
        fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(&tempty[tb]);
      }
    };

    int i = 0, jt = 0;
    int pend_jt = -1, pend_S = 0, pend_c = 0;
    for (int e = 0; e < ne && !bad; ++e) {
      const int S = a.ups[e0 + e];
      const bool diag = S == T;
      for (int c = 0; c < NC; ++c, ++i) {
        const int gb = i & 1, eb = i & 1;
        // G[t][32 sources] from tensor memory, then the G buffer is free
        const bool okg = wait_sleep(&gfull[gb], static_cast<uint32_t>((i >> 1) & 1));
        if (__any_sync(0xffffffffu, !okg)) {
          bad = true;
          break;
        }
        fence_after();
        // G in two halves (NT = 2): the second half's load is in flight
        // while the first half is evaluated
        uint32_t g[32];
        const uint32_t gaddr = lane_base + kG + static_cast<uint32_t>(gb * kGB + at * 64 + kSrc * sh);
        tmem_ld16(gaddr, g);
        if (NT == 2) tmem_ld16_async(gaddr + 16, g + 16);
        const bool oke = i < 2 || wait_sleep(&efree[eb], static_cast<uint32_t>(((i - 2) >> 1) & 1));
        const uint32_t et = sptr(ebuf + eb * ebytes) +
                            static_cast<uint32_t>((tt >> 3) * kTS + (tt & 7) * 16 + (kSrc / 8 * sh) * 128);
        if (__all_sync(0xffffffffu, oke)) {
#pragma unroll
          for (int q8 = 0; q8 < 2; ++q8) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              split_f16x2(ex2f(__uint_as_float(g[8 * q8 + 2 * u])), ex2f(__uint_as_float(g[8 * q8 + 2 * u + 1])),
                          hi[u], lo[u]);
            sts128(et + q8 * 128, hi);
            sts128(et + q8 * 128 + kHL, lo);
          }
        }
        if (NT == 2) tmem_wait_ld16(g + 16);
        fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(&gfree[gb]);
        if (__any_sync(0xffffffffu, !oke)) {
          bad = true;
          break;
        }
#pragma unroll
        for (int q8 = 2; q8 < kSrc / 8; ++q8) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            split_f16x2(ex2f(__uint_as_float(g[8 * q8 + 2 * u])), ex2f(__uint_as_float(g[8 * q8 + 2 * u + 1])), hi[u],
                        lo[u]);
          sts128(et + q8 * 128, hi);
          sts128(et + q8 * 128 + kHL, lo);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) bar_arrive(&efull[eb]);
        if (pend_jt >= 0) {
          flush(pend_jt, pend_S, pend_c);
          pend_jt = -1;
          if (bad) break;
        }
        if (c == 0 && e >= 1) {
          fold(e - 1);
          if (bad) break;
        }
        if (!diag) {
          pend_jt = jt;
          pend_S = S;
          pend_c = c;
          ++jt;
        }
      }
    }
    if (!bad && pend_jt >= 0) flush(pend_jt, pend_S, pend_c);
    if (!bad && ne >= 1) fold(ne - 1);
    if (bad && lane == 0) atomicExch(a.err, 3);
    if (fown) {
      float* op = a.fwd + static_cast<int64_t>(T) * 16 * ld + tt;
#pragma unroll
      for (int r = 0; r < 8; ++r) op[(8 * sh + r) * ld] = ks[r];
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

size_t sym_g_smem(int NT) {
  const size_t ld = 128 * static_cast<size_t>(NT);
  return 2 * static_cast<size_t>(NT * 16 * kTS) + kStages * static_cast<size_t>(2 * kXChunkHalf + kQChunkBytes) +
         ld * 64 + ld * kKD * 2 * 2 + 2 * 64 * 16 * 4;
}

size_t sym_smem(int D, int ld) {
  const int NT = ld / 128;
  const size_t ebytes = static_cast<size_t>(NT) * 16 * kTS;
  const size_t coord = static_cast<size_t>(D) * kChunk * 4;
  const size_t stage = ((coord + 1023) & ~size_t(1023)) + kQChunkBytes;
  return 2 * ebytes + kStages * stage + static_cast<size_t>(ld) * 64 + 2 * NT * 16 * 128 * 4 + 2 * 64 * 16 * 4;
}

template <int D>
void sym_launch_d(int kernel, const SymArgs& a, int grid, size_t smem, cudaStream_t s) {
  switch (kernel) {
    case DWFMM_K_EXP: k_near_sym_tc<D, DWFMM_K_EXP><<<grid, kSymTcThreads, smem, s>>>(a); break;
    case DWFMM_K_MATERN32: k_near_sym_tc<D, DWFMM_K_MATERN32><<<grid, kSymTcThreads, smem, s>>>(a); break;
    default: k_near_sym_tc<D, DWFMM_K_GAUSS><<<grid, kSymTcThreads, smem, s>>>(a);
  }
}

template <int D>
void sym_attrs_d(int bytes) {
  cudaFuncSetAttribute(k_near_sym_tc<D, DWFMM_K_EXP>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_near_sym_tc<D, DWFMM_K_MATERN32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_near_sym_tc<D, DWFMM_K_GAUSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

std::atomic<uint64_t> g_sym_attrs_dev{0};
constexpr int kSymSmemMax = 220 * 1024;

// The exponent on the tensor cores: Gaussian in factored form, leaves of 256
// slots, padded dimension <= 16.
bool sym_g_applies(const Plan& P, int D) {
  return P.kernel == DWFMM_K_GAUSS && P.m_pad == 256 && D <= kKD && sym_g_smem(2) <= static_cast<size_t>(kSymSmemMax);
}

}  // namespace

// Rows of the symmetric tensor-core near field: target leaves in order of
// decreasing upper-list length (longest first, so the short rows fill the
// tail of the launch).  Host counts of the upper rows come from the tree
// build.
void sym_tc_order(Plan& P, const std::vector<int>& upper_counts) {
  std::vector<int32_t> ord(P.L);
  for (int i = 0; i < P.L; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return upper_counts[x] > upper_counts[y]; });
  P.sym_order.alloc(P.L);
  DW_CUDA(cudaMemcpyAsync(P.sym_order.p, ord.data(), sizeof(int32_t) * P.L, cudaMemcpyHostToDevice, P.stream));
  DW_CUDA(cudaStreamSynchronize(P.stream));
}

// Whether the symmetric tensor-core near field applies: MIXED with 9..16
// right-hand sides, a symmetric near list, leaves of 128 or 256 slots, a
// padded dimension the kernel is built for, and E' inside the FP16 range.
bool sym_tc_eligible(const Plan& P, int D, int RC) {
  if (P.prec != DWFMM_P_MIXED || RC != 16 || !P.sym_ok || P.sym_nup <= 0 || !P.sym_order.p) return false;
  if (P.m_pad != 128 && P.m_pad != 256) return false;
  if (D != 4 && D != 8 && D != 10 && D != 12 && D != 16 && D != 20) return false;
  if (P.kernel == DWFMM_K_GAUSS && !(P.gauss_fact && 2.0 * P.gauss_bound <= 15.0)) return false;
  return sym_smem(D, P.m_pad) <= static_cast<size_t>(kSymSmemMax);
}

// Fixed-point bits of the transposed sums: every partial sum is at most N
// sites times the largest E' times max |q'| <= 1.
int sym_tc_bits(const Plan& P) {
  const double emax = P.kernel == DWFMM_K_GAUSS ? std::exp2(2.0 * P.gauss_bound) : 1.0;
  const double bound = static_cast<double>(std::max<int64_t>(P.N, 1)) * emax * 2.0;
  return 62 - static_cast<int>(std::ceil(std::log2(bound)));
}

namespace {

void ensure_sym_attrs() {
  const uint64_t dbit = device_bit();
  if (g_sym_attrs_dev.load() & dbit) return;
  sym_attrs_d<4>(kSymSmemMax);
  sym_attrs_d<8>(kSymSmemMax);
  sym_attrs_d<10>(kSymSmemMax);
  sym_attrs_d<12>(kSymSmemMax);
  sym_attrs_d<16>(kSymSmemMax);
  sym_attrs_d<20>(kSymSmemMax);
  cudaFuncSetAttribute(k_near_sym_gtc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSymSmemMax);
  cudaFuncSetAttribute(k_near_sym_gtc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSymSmemMax);
  DW_CUDA(cudaGetLastError());
  g_sym_attrs_dev.fetch_or(dbit);
}

void launch_sym_tc(int D, int kernel, const SymArgs& a, int grid, size_t smem, cudaStream_t s) {
  switch (D) {
    case 4: sym_launch_d<4>(kernel, a, grid, smem, s); break;
    case 8: sym_launch_d<8>(kernel, a, grid, smem, s); break;
    case 10: sym_launch_d<10>(kernel, a, grid, smem, s); break;
    case 12: sym_launch_d<12>(kernel, a, grid, smem, s); break;
    case 16: sym_launch_d<16>(kernel, a, grid, smem, s); break;
    default: sym_launch_d<20>(kernel, a, grid, smem, s); break;
  }
}

// Node coordinates of every cluster in 128-slot blocks: [C][D+1][128] from
// the scaled node blocks [C][D+1][n_pad] (row D = |y'|^2), slots >= n_pad zero.
__global__ void k_m2l_crd(const float* ynodek, int C, int D, int np, float* out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(C) * (D + 1) * 128) return;
  const int a = static_cast<int>(i & 127);
  const int64_t row = i >> 7;
  out[i] = a < np ? ynodek[row * np + a] : 0.0f;
}

}  // namespace

bool near_sym_tc(Plan& P, int D, int Rc, cudaStream_t s) {
  const int RC = 16;
  if (!sym_tc_eligible(P, D, RC)) return false;
  ensure_sym_attrs();
  const int ld = P.m_pad;
  const int64_t nsite = static_cast<int64_t>(P.L) * 16 * ld;
  const int64_t gstride = static_cast<int64_t>(D + 1) * ld;
  const int gauss = P.kernel == DWFMM_K_GAUSS ? 1 : 0;
  P.sym_bq16.alloc(static_cast<size_t>(P.L) * ld * 32);
  P.sym_acc.alloc(static_cast<size_t>(nsite));
  P.sym_fwd.alloc(static_cast<size_t>(nsite));
  P.sym_colmax.alloc(16);
  DW_CUDA(cudaMemsetAsync(P.sym_colmax.p, 0, 16 * sizeof(unsigned), s));
  DW_CUDA(cudaMemsetAsync(P.sym_acc.p, 0, static_cast<size_t>(nsite) * sizeof(unsigned long long), s));
  k_sym_colmax<<<2 * sm_count(), 256, 0, s>>>(P.xb32.p, ld, ld, P.d_ptsk.p, gstride, P.L, ld, D, gauss, Rc,
                                               P.sym_colmax.p);
  k_sym_make_bq<<<ceil_div(static_cast<int64_t>(P.L) * ld * 16, 256), 256, 0, s>>>(
      P.xb32.p, ld, ld, P.d_ptsk.p, gstride, P.L, ld, D, gauss, Rc, P.sym_colmax.p, P.sym_bq16.p);
  const int sb = sym_tc_bits(P);
  if (sym_g_applies(P, D)) {
    P.near_engine = 5;
    if (!P.sym_x16_ok) {
      P.sym_xa16.alloc(static_cast<size_t>(P.L) * ld * kKD * 2);
      P.sym_xb16.alloc(static_cast<size_t>(P.L) * ld * kKD * 2);
      k_sym_make_x16<<<ceil_div(static_cast<int64_t>(P.L) * ld * kKD, 256), 256, 0, s>>>(
          P.d_ptsk.p, gstride, P.L, ld, D, P.sym_xa16.p, P.sym_xb16.p);
      P.sym_x16_ok = true;
    }
    SymGArgs g{};
    g.xa = P.sym_xa16.p;
    g.xb = P.sym_xb16.p;
    g.bq = P.sym_bq16.p;
    g.uprow = P.sym_uprow.p;
    g.ups = P.sym_s.p;
    g.order = P.sym_order.p;
    g.fwd = P.sym_fwd.p;
    g.acc = P.sym_acc.p;
    g.acc_scale = std::ldexp(1.0f, sb);
    g.ld = ld;
    g.err = P.d_err.p;
    k_near_sym_gtc<2><<<P.L, kSymGThreads, sym_g_smem(2), s>>>(g);
    DW_CUDA(cudaGetLastError());
    k_sym_finish<<<ceil_div(nsite, 256), 256, 0, s>>>(P.sym_fwd.p, P.sym_acc.p, std::ldexp(1.0, -sb), P.d_ptsk.p,
                                                       gstride, P.L, ld, D, gauss, Rc, P.sym_colmax.p, P.ynear32.p,
                                                       static_cast<int64_t>(kRC) * ld, ld, ld);
    DW_CUDA(cudaGetLastError());
    return true;
  }
  SymArgs a{};
  a.pts = P.d_ptsk.p;
  a.gstride = gstride;
  a.bq = P.sym_bq16.p;
  a.uprow = P.sym_uprow.p;
  a.ups = P.sym_s.p;
  a.order = P.sym_order.p;
  a.fwd = P.sym_fwd.p;
  a.acc = P.sym_acc.p;
  a.acc_scale = std::ldexp(1.0f, sb);
  a.ld = ld;
  a.err = P.d_err.p;
  launch_sym_tc(D, P.kernel, a, P.L, sym_smem(D, ld), s);
  DW_CUDA(cudaGetLastError());
  k_sym_finish<<<ceil_div(nsite, 256), 256, 0, s>>>(P.sym_fwd.p, P.sym_acc.p, std::ldexp(1.0, -sb), P.d_ptsk.p,
                                                     gstride, P.L, ld, D, gauss, Rc, P.sym_colmax.p, P.ynear32.p,
                                                     static_cast<int64_t>(kRC) * ld, ld, ld);
  DW_CUDA(cudaGetLastError());
  return true;
}

// The couplings (M2L, Eq. (5.4)) of MIXED plans with 9..16 right-hand sides
// on the symmetric engine: the far list holds both orderings of every
// admissible pair of clusters and K is symmetric, so each unordered pair
// (t, s > t) is evaluated once, targets = the nodes of t, sources = the
// nodes of s, charges = the moments m_s; the forward sums go to t, the
// transposed ones (fixed point, order independent) to s.  Node sets are
// padded to 128 slots (zero charges); only the levels with far blocks are
// touched (the moments of coarser clusters are never computed).  Returns
// false where the path does not apply (the ordered-pair engines run
// instead).
bool m2l_sym_tc(Plan& P, int D, int Rc, cudaStream_t s) {
  if (P.prec != DWFMM_P_MIXED || Rc < 9 || Rc > 16 || !P.fsym_ok || P.fsym_rows <= 0) return false;
  if (P.n_pad > 128 || (D != 4 && D != 8 && D != 10 && D != 12 && D != 16 && D != 20)) return false;
  if (P.kernel == DWFMM_K_GAUSS && !(P.gauss_fact && 2.0 * P.gauss_bound <= 15.0)) return false;
  if (sym_smem(D, 128) > static_cast<size_t>(kSymSmemMax) || !P.d_ynodek.p || P.dpad != D) return false;
  ensure_sym_attrs();
  const int C = P.C, ld = 128, np = P.n_pad;
  const int64_t gstride = static_cast<int64_t>(D + 1) * ld;
  const int64_t nslot = static_cast<int64_t>(C) * 16 * ld;
  const int gauss = P.kernel == DWFMM_K_GAUSS ? 1 : 0;
  if (P.m2l_crd_D != D || !P.m2l_crd.p) {
    P.m2l_crd.alloc(static_cast<size_t>(C) * gstride);
    k_m2l_crd<<<ceil_div(static_cast<int64_t>(C) * gstride, 256), 256, 0, s>>>(P.d_ynodek.p, C, D, np,
                                                                             P.m2l_crd.p);
    P.m2l_crd_D = D;
    P.m2l_x16_D = -1;
  }
  P.m2l_bq16.alloc(static_cast<size_t>(C) * ld * 32);
  P.m2l_acc.alloc(static_cast<size_t>(nslot));
  P.m2l_fwd.alloc(static_cast<size_t>(nslot));
  P.m2l_colmax.alloc(16);
  DW_CUDA(cudaMemsetAsync(P.m2l_colmax.p, 0, 16 * sizeof(unsigned), s));
  DW_CUDA(cudaMemsetAsync(P.m2l_acc.p, 0, static_cast<size_t>(nslot) * sizeof(unsigned long long), s));
  // targets without upper entries get no CTA; their forward sums stay zero
  DW_CUDA(cudaMemsetAsync(P.m2l_fwd.p, 0, static_cast<size_t>(nslot) * sizeof(float), s));
  // only the clusters of the levels with far blocks (>= jmin) carry moments
  const int first = (1 << P.jmin) - 1, nc = C - first;
  const float* mom = P.mom32.p + static_cast<int64_t>(first) * 16 * np;
  const float* crd = P.m2l_crd.p + static_cast<int64_t>(first) * gstride;
  k_sym_colmax<<<2 * sm_count(), 256, 0, s>>>(mom, np, P.n, crd, gstride, nc, ld, D, gauss, Rc, P.m2l_colmax.p);
  k_sym_make_bq<<<ceil_div(static_cast<int64_t>(nc) * ld * 16, 256), 256, 0, s>>>(
      mom, np, P.n, crd, gstride, nc, ld, D, gauss, Rc, P.m2l_colmax.p,
      P.m2l_bq16.p + static_cast<int64_t>(first) * ld * 32);
  // fixed-point bits: a partial sum is at most (all nodes) x E'max x max |q'|
  const double emax = gauss ? std::exp2(2.0 * P.gauss_bound) : 1.0;
  const int sb = 62 - static_cast<int>(std::ceil(std::log2(static_cast<double>(C) * ld * emax * 2.0)));
  if (gauss && D <= kKD && sym_g_smem(1) <= static_cast<size_t>(kSymSmemMax)) {
    // the Gaussian's exponent on the tensor cores, one 128-target tile
    if (P.m2l_x16_D != D || !P.m2l_xa16.p) {
      P.m2l_xa16.alloc(static_cast<size_t>(C) * ld * kKD * 2);
      P.m2l_xb16.alloc(static_cast<size_t>(C) * ld * kKD * 2);
      k_sym_make_x16<<<ceil_div(static_cast<int64_t>(C) * ld * kKD, 256), 256, 0, s>>>(
          P.m2l_crd.p, gstride, C, ld, D, P.m2l_xa16.p, P.m2l_xb16.p);
      P.m2l_x16_D = D;
    }
    SymGArgs g{};
    g.xa = P.m2l_xa16.p;
    g.xb = P.m2l_xb16.p;
    g.bq = P.m2l_bq16.p;
    g.uprow = P.fsym_uprow.p;
    g.ups = P.fsym_s.p;
    g.order = P.fsym_order.p;
    g.fwd = P.m2l_fwd.p;
    g.acc = P.m2l_acc.p;
    g.acc_scale = std::ldexp(1.0f, sb);
    g.ld = ld;
    g.err = P.d_err.p;
    k_near_sym_gtc<1><<<P.fsym_rows, kSymGThreads, sym_g_smem(1), s>>>(g);
  } else {
    SymArgs a{};
    a.pts = P.m2l_crd.p;
    a.gstride = gstride;
    a.bq = P.m2l_bq16.p;
    a.uprow = P.fsym_uprow.p;
    a.ups = P.fsym_s.p;
    a.order = P.fsym_order.p;
    a.fwd = P.m2l_fwd.p;
    a.acc = P.m2l_acc.p;
    a.acc_scale = std::ldexp(1.0f, sb);
    a.ld = ld;
    a.err = P.d_err.p;
    launch_sym_tc(D, P.kernel, a, P.fsym_rows, sym_smem(D, ld), s);
  }
  DW_CUDA(cudaGetLastError());
  const int64_t off = static_cast<int64_t>(first) * 16 * ld;
  k_sym_finish<<<ceil_div(static_cast<int64_t>(nc) * 16 * ld, 256), 256, 0, s>>>(
      P.m2l_fwd.p + off, P.m2l_acc.p + off, std::ldexp(1.0, -sb), crd, gstride, nc, ld, D, gauss, Rc,
      P.m2l_colmax.p, P.loc32.p + static_cast<int64_t>(first) * 16 * np, static_cast<int64_t>(kRC) * np, np, np);
  DW_CUDA(cudaGetLastError());
  return true;
}

}  // namespace dw
