// Kernel summation with the contraction on the tensor cores (sm_103a
// tcgen05), used for the near field (P2P) of MIXED plans with 9..16
// right-hand sides:
//
//   y[t][r] = sum_s E[t][s] q[s][r],   E[t][s] = phi(|x_t - x_s| / sigma).
//
// CUDA cores evaluate E (as in k_sum_f32: scaled coordinates, packed
// fma.f32x2 distances, one ex2), split it into TF32 hi + lo and store both
// into tensor memory as the A operand; one thread issues
// tcgen05.mma.kind::tf32 (M=128 targets, K=8 sources) with B = the charges,
// pre-split into TF32 hi + lo in the no-swizzle K-major core-matrix layout
// and staged by TMA bulk copies.  The hi and lo charge blocks are adjacent
// in that layout, so one N=32 product gives E_hi*[q_hi | q_lo] and a second,
// N=16, adds E_lo*q_hi: three terms (~2^-20 relative each) in two MMAs per
// K step.  Each source block accumulates into a 32-column TMEM tile (FP32):
// columns 0..15 hold E_hi*q_hi, columns 16..31 the two small terms.  The
// tensor core rounds its accumulator toward zero at every MMA, a bias that
// grows with the number of updates, so the large terms get one update per
// K step and the small ones the other.  The two halves are read back, added
// and folded into Kahan-compensated running sums kept in shared memory.
//
// One CTA = 128 targets, warp-specialised: twelve compute warps (warps w,
// w+4 and w+8 share the TMEM lanes of quadrant w, each evaluating a third
// of every 48-source chunk, 8 sources per call), one warp whose lane 0
// issues the MMAs and one whose lane 0 issues the TMA loads.  The roles hand
// over through mbarriers only (stage full / coordinates free / charges free,
// A full / A empty, D full / D empty), so the compute warps never wait at a
// CTA-wide barrier inside the loop; every waiting thread sleeps in the
// barrier (mbarrier.try_wait with a suspend-time hint) until the phase
// completes.  TMEM: two A buffers (2 x 96 columns: 48 sources hi + lo) and
// two 32-column accumulators, 256 columns allocated.  72 registers per
// thread, two CTAs per SM.  Every wait is bounded.
#include <atomic>
#include <cstdint>

#include "dwfmm_internal.cuh"
#include "tcgen05_util.cuh"

namespace dw {

namespace {

using namespace tc;

constexpr int kCompWarps = 12;
constexpr int kFoldWarps = 8;                        // parts 0 and 1 of each quadrant fold the sums
constexpr int kTcThreads = (kCompWarps + 2) * 32;   // compute warps, MMA warp, TMA warp
constexpr int kChunkS = 48;                          // sources per A buffer
constexpr int kTmemCols = 256;
constexpr int kRow = 256;                // shared-memory row stride (floats) of the coordinates

template <int KER>
__device__ __forceinline__ float phi_of(float a) {
  if (KER == DWFMM_K_GAUSS) return ex2f(a);
  const float r = sqrtf_a(a);
  if (KER == DWFMM_K_EXP) return ex2f(-r);
  const float e = ex2f(-1.4426950408889634f * r);
  return fmaf(r, e, e);
}

// Instruction descriptors: M = 128 targets; N = 32 (the hi and lo charge
// blocks together) or 16 (hi only).
constexpr uint32_t kIdesc32 = idesc_tf32(128, 32);
constexpr uint32_t kIdesc16 = idesc_tf32(128, 16);

// Charges [g][ld][16] (interleaved per source) -> TF32 hi and lo blocks in
// the K-major core layout: block g = [hi | lo], each 16 x ld, core (nb, kb)
// at kb * 128 + nb * (ld * 32) bytes, row i of a core at i * 16 bytes.
// Gaussian kernel: each charge carries its source's factor 2^(-|s'|^2)
// (norm row D of the scaled source block).
__global__ void k_make_bq(const float* xq, int64_t groups, int ld, const float* src, int64_t src_gstride, int D,
                          int gauss, float* bq) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= groups * ld * 16) return;
  const int r = static_cast<int>(t % 16);
  const int64_t gs = t / 16;
  const int s = static_cast<int>(gs % ld);
  const int64_t g = gs / ld;
  float v = xq[t];
  if (gauss) v *= exp2f(-src[g * src_gstride + static_cast<int64_t>(D) * ld + s]);
  uint32_t hi, lo;
  split_tf32(v, hi, lo);
  const int64_t off = (static_cast<int64_t>(s / 4) * 128 + (r / 8) * static_cast<int64_t>(ld) * 32 + (r % 8) * 16 +
                       (s % 4) * 4) / 4;
  float* blk = bq + g * (2 * 16 * static_cast<int64_t>(ld));
  blk[off] = __uint_as_float(hi);
  blk[16 * static_cast<int64_t>(ld) + off] = __uint_as_float(lo);
}

struct TcArgs {
  const float* tgt;       // [g][D+1][ld] scaled coordinates + norm row
  int64_t tgt_gstride;
  const float* src;
  int64_t src_gstride;
  const float* bq;        // [g][2][16 x ld] TF32 hi | lo charge blocks
  float* out;             // [g][16][ld]
  int64_t out_gstride;
  const int32_t* rowptr;
  const int32_t* col;
  const int32_t* count;
  int count_off;
  int count_const;
  int first;
  int ld;
  int halves;             // CTAs per target group (ld / 128, rounded up)
  int Rc;
  int* err;
};

// 8 pairs (one target, sources j..j+7 of the stage): phi, TF32 split.  The
// Gaussian is evaluated in factored form, E' = 2^(2 x'.s'): the factors
// 2^(-|x'|^2) and 2^(-|s'|^2) sit on the sums and the charges.
template <int D, int KER>
__device__ __forceinline__ void eval8(const float* sc, int j, const u64* xt2, uint32_t* hi, uint32_t* lo) {
  u64 p[4];
  if (KER == DWFMM_K_GAUSS) {
    {
      const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sc + j);
      const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sc + j + 4);
      p[0] = mul2(xt2[0], v0.x);
      p[1] = mul2(xt2[0], v0.y);
      p[2] = mul2(xt2[0], v1.x);
      p[3] = mul2(xt2[0], v1.y);
    }
#pragma unroll
    for (int k = 1; k < D; ++k) {
      const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sc + k * kRow + j);
      const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sc + k * kRow + j + 4);
      p[0] = fma2(xt2[k], v0.x, p[0]);
      p[1] = fma2(xt2[k], v0.y, p[1]);
      p[2] = fma2(xt2[k], v1.x, p[2]);
      p[3] = fma2(xt2[k], v1.y, p[3]);
    }
  } else {
    p[0] = p[1] = p[2] = p[3] = 0ull;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sc + k * kRow + j);
      const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sc + k * kRow + j + 4);
      u64 df = sub2(xt2[k], v0.x);
      p[0] = fma2(df, df, p[0]);
      df = sub2(xt2[k], v0.y);
      p[1] = fma2(df, df, p[1]);
      df = sub2(xt2[k], v1.x);
      p[2] = fma2(df, df, p[2]);
      df = sub2(xt2[k], v1.y);
      p[3] = fma2(df, df, p[3]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float f0, f1;
    up(p[u], f0, f1);
    const float e0 = phi_of<KER>(f0), e1 = phi_of<KER>(f1);
    const uint32_t h0 = __float_as_uint(e0) & 0xFFFFE000u, h1 = __float_as_uint(e1) & 0xFFFFE000u;
    float l0, l1;
    up(sub2(pk(e0, e1), pk(__uint_as_float(h0), __uint_as_float(h1))), l0, l1);
    hi[2 * u] = h0;
    hi[2 * u + 1] = h1;
    lo[2 * u] = __float_as_uint(l0);
    lo[2 * u + 1] = __float_as_uint(l1);
  }
}


template <int D, int KER>
__global__ void __launch_bounds__(kTcThreads, (D <= 12 ? 2 : 1)) k_sum_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // full: TMA landed; cfree: compute warps done with the coordinates;
  // bqfree: MMAs done with the charges; afull / aempty: A buffer written /
  // read; dfull / dempty: accumulator complete / folded; fin: all MMAs done.
  __shared__ __align__(8) uint64_t bars[15];
  __shared__ uint32_t tmem_slot;
  __shared__ int stage_s8[2];   // sources (rounded up to 8) of the block in each stage
  uint64_t* full = bars;
  uint64_t* cfree = bars + 2;
  uint64_t* bqfree = bars + 4;
  uint64_t* afull = bars + 6;
  uint64_t* aempty = bars + 8;
  uint64_t* dfull = bars + 10;
  uint64_t* dempty = bars + 12;
  uint64_t* fin = bars + 14;
  const int ld = a.ld;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int g = a.first + blockIdx.x / a.halves;
  const int half = blockIdx.x % a.halves;
  const int rb = a.rowptr[g];
  const int nb = a.rowptr[g + 1] - rb;
  const uint32_t coord_bytes = static_cast<uint32_t>((D + 1) * ld * 4);
  const uint32_t coord_pad = static_cast<uint32_t>((D + 1) * kRow * 4);   // rows at a fixed stride
  const uint32_t bq_bytes = static_cast<uint32_t>(2 * 16 * ld * 4);
  const uint32_t stage_bytes = coord_pad + bq_bytes;
  unsigned char* stage0 = smem;

  if (t == 0) {
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sptr(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(&cfree[i])), "r"(kCompWarps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sptr(&bqfree[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(&afull[i])), "r"(kCompWarps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sptr(&aempty[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sptr(&dfull[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(&dempty[i])), "r"(kFoldWarps));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sptr(fin)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sptr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == kCompWarps + 1) {
    // ---- TMA producer: block b into stage b & 1 once block b - 2 is done
    if (lane == 0) {
      bool bad = false;
      int issued = 0;
      for (int b = 0; b < nb; ++b) {
        const int st = b & 1;
        if (b >= 2) {
          const uint32_t par = static_cast<uint32_t>(((b - 2) >> 1) & 1);
          if (!wait_sleep(&cfree[st], par) || !wait_sleep(&bqfree[st], par)) {
            bad = true;
            break;
          }
        }
        const int s = a.col[rb + b];
        const int scnt = a.count ? a.count[a.count_off + s] : a.count_const;
        stage_s8[st] = (scnt + 7) & ~7;   // published by the arrive below
        unsigned char* dst = stage0 + st * stage_bytes;
        const uint32_t bar = sptr(&full[st]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(coord_bytes + bq_bytes)
                     : "memory");
        if (ld == kRow) {
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  sptr(dst)),
              "l"(a.src + s * a.src_gstride), "r"(coord_bytes), "r"(bar)
              : "memory");
        } else {
          for (int k = 0; k <= D; ++k)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    sptr(dst + k * kRow * 4)),
                "l"(a.src + s * a.src_gstride + static_cast<int64_t>(k) * ld), "r"(static_cast<uint32_t>(ld * 4)),
                "r"(bar)
                : "memory");
        }
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sptr(dst + coord_pad)),
            "l"(a.bq + s * (2 * 16 * static_cast<int64_t>(ld))), "r"(bq_bytes), "r"(bar)
            : "memory");
        issued = b + 1;
      }
      // the copies in flight land before the CTA exits
      for (int b = issued >= 2 ? issued - 2 : 0; b < issued; ++b)
        (void)wait_sleep(&full[b & 1], static_cast<uint32_t>((b >> 1) & 1));
      if (bad) atomicExch(a.err, 3);
    }
  } else if (warp == kCompWarps) {
    // ---- MMA issuer: two TF32 products per 8-source step of every chunk
    if (lane == 0) {
      bool bad = false;
      int chunk = 0, kb = 0;
      for (int b = 0; b < nb && !bad; ++b) {
        const int st = b & 1;
        if (!wait_sleep(&full[st], static_cast<uint32_t>((b >> 1) & 1))) {
          bad = true;
          break;
        }
        const int s8 = stage_s8[st];
        if (s8 > 0) {
          const int db = kb & 1;
          if (kb >= 2 && !wait_sleep(&dempty[db], static_cast<uint32_t>(((kb - 2) >> 1) & 1))) {
            bad = true;
            break;
          }
          const uint32_t bq_addr = sptr(stage0 + st * stage_bytes + coord_pad);
          const uint32_t d_tmem = tmem + 192 + 32 * db;
          for (int c0 = 0; c0 < s8; c0 += kChunkS) {
            const int ab = chunk & 1;
            if (!wait_sleep(&afull[ab], static_cast<uint32_t>((chunk >> 1) & 1))) {
              bad = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int ns = min(kChunkS, s8 - c0);
            const uint32_t a_tmem = tmem + 96 * ab;
            for (int ks = 0; ks < ns; ks += 8) {
              const uint32_t boff = static_cast<uint32_t>(((c0 + ks) / 4) * 128);
              // rows 0..15 of B = q_hi, rows 16..31 = q_lo (the lo block
              // starts 16 * ld floats = two 8-row groups after the hi block)
              const u64 bq = smem_desc(bq_addr + boff, 128, static_cast<uint32_t>(ld * 32));
              mma_tf32(d_tmem, a_tmem + ks, bq, kIdesc32, (c0 + ks) > 0 ? 1u : 0u);
              // the small term E_lo*q_hi joins E_hi*q_lo in columns 16..31:
              // the tensor core truncates its FP32 accumulator at every
              // MMA, so the large E_hi*q_hi columns take one update per step
              mma_tf32(d_tmem + 16, a_tmem + kChunkS + ks, bq, kIdesc16, 1u);
            }
            mma_commit(&aempty[ab]);
            ++chunk;
          }
          if (bad) break;
          mma_commit(&dfull[db]);
          ++kb;
        }
        mma_commit(&bqfree[st]);
      }
      mma_commit(fin);
      (void)wait_sleep(fin, 0u);
      if (bad) atomicExch(a.err, 3);
    }
  } else {
    // ---- compute warps: E for (quadrant targets) x (half of each chunk)
    const int qd = warp & 3, hf = warp >> 2;   // hf: part 0..2 of each chunk
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(qd * 32) << 16);
    const int ti = half * 128 + qd * 32 + lane;
    const int tsafe = ti < ld ? ti : 0;
    const float* tp = a.tgt + g * a.tgt_gstride + tsafe;
    u64 xt2[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float v = (KER == DWFMM_K_GAUSS) ? 2.0f * tp[k * ld] : tp[k * ld];
      xt2[k] = pk(v, v);
    }
    // target factor of the factored Gaussian
    const float tfac = (KER == DWFMM_K_GAUSS) ? exp2f(-tp[D * ld]) : 1.0f;
    // Kahan sums in shared memory: [16 RHS][128 targets], values then compensations
    float* ksum = reinterpret_cast<float*>(stage0 + 2 * stage_bytes);
    const int trow = qd * 32 + lane;
    if (hf < 2) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        ksum[(8 * hf + r) * 128 + trow] = 0.0f;
        ksum[2048 + (8 * hf + r) * 128 + trow] = 0.0f;
      }
    }
    bool bad = false;
    // fold accumulator k (this warp's 8 right-hand sides) into the sums
    auto fold = [&](int k) {
      if (hf >= 2) return;
      const int db = k & 1;
      const bool ok = wait_sleep(&dfull[db], static_cast<uint32_t>((k >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok)) {
        bad = true;
        return;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t dv[8], dl[8];
      tmem_ld8x2(lane_base + 192 + 32 * db + 8 * hf, lane_base + 192 + 32 * db + 16 + 8 * hf, dv, dl);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        float* pa = ksum + (8 * hf + r) * 128 + trow;
        const float acc = pa[0], comp = pa[2048];
        const float y = (__uint_as_float(dv[r]) + __uint_as_float(dl[r])) - comp;
        const float s = acc + y;
        pa[2048] = (s - acc) - y;
        pa[0] = s;
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) bar_arrive(&dempty[db]);
    };
    int chunk = 0, kb = 0;
    for (int b = 0; b < nb; ++b) {
      const int st = b & 1;
      const bool ok = wait_sleep(&full[st], static_cast<uint32_t>((b >> 1) & 1));
      if (__any_sync(0xffffffffu, !ok)) {
        bad = true;
        break;
      }
      const float* sc = reinterpret_cast<const float*>(stage0 + st * stage_bytes);
      const int s8 = stage_s8[st];
      for (int c0 = 0; c0 < s8; c0 += kChunkS) {
        const int ab = chunk & 1;
        const bool okA = chunk < 2 || wait_sleep(&aempty[ab], static_cast<uint32_t>(((chunk - 2) >> 1) & 1));
        if (__any_sync(0xffffffffu, !okA)) {
          bad = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int j0 = c0 + 16 * hf;
        const int jn = min(16, s8 - j0);
        const uint32_t col = static_cast<uint32_t>(96 * ab + 16 * hf);
        if (jn > 0) {
          uint32_t hi[8], lo[8];
          eval8<D, KER>(sc, j0, xt2, hi, lo);
          tmem_st8(lane_base + col, hi);
          tmem_st8(lane_base + col + kChunkS, lo);
        }
        if (jn > 8) {
          uint32_t hi[8], lo[8];
          eval8<D, KER>(sc, j0 + 8, xt2, hi, lo);
          tmem_st8(lane_base + col + 8, hi);
          tmem_st8(lane_base + col + kChunkS + 8, lo);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) bar_arrive(&afull[ab]);
        ++chunk;
      }
      if (bad) break;
      __syncwarp();
      if (lane == 0) bar_arrive(&cfree[st]);
      if (s8 > 0) {
        if (kb >= 1) {
          fold(kb - 1);
          if (bad) break;
        }
        ++kb;
      }
    }
    if (!bad && kb >= 1) fold(kb - 1);
    if (bad && lane == 0) atomicExch(a.err, 3);
    if (ti < ld && hf < 2) {
      float* op = a.out + g * a.out_gstride + ti;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float v = ksum[(8 * hf + r) * 128 + trow];
        if (8 * hf + r < a.Rc) op[(8 * hf + r) * ld] = (KER == DWFMM_K_GAUSS) ? v * tfac : v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Dynamic shared memory of one CTA.  At least 80 KB, so that no more than two
// CTAs (2 x 256 TMEM columns = all 512) are ever resident on one SM and
// tcgen05.alloc never has to wait for columns.
size_t tc_smem(int D, int ld) {
  const size_t pad = static_cast<size_t>((D + 1) * kRow * 4);
  const size_t need = 2 * (pad + static_cast<size_t>(2 * 16 * ld * 4)) + 1024 + 16384;   // + Kahan sums
  return need < 80 * 1024 ? 80 * 1024 : need;
}

template <int D>
void tc_launch_d(int kernel, const TcArgs& a, int grid, size_t smem, cudaStream_t s) {
  switch (kernel) {
    case DWFMM_K_EXP: k_sum_tc<D, DWFMM_K_EXP><<<grid, kTcThreads, smem, s>>>(a); break;
    case DWFMM_K_MATERN32: k_sum_tc<D, DWFMM_K_MATERN32><<<grid, kTcThreads, smem, s>>>(a); break;
    default: k_sum_tc<D, DWFMM_K_GAUSS><<<grid, kTcThreads, smem, s>>>(a);
  }
}

template <int D>
void tc_attrs_d() {
  const int big = 200 * 1024;
  cudaFuncSetAttribute(k_sum_tc<D, DWFMM_K_EXP>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_sum_tc<D, DWFMM_K_MATERN32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_sum_tc<D, DWFMM_K_GAUSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

std::atomic<uint64_t> g_tc_attrs_dev{0};   // devices whose kernel attributes are set

}  // namespace

// Tensor-core kernel summation over (target group, source group) lists.
// bq_scratch receives the TF32 hi/lo charge blocks.  Returns false when the
// shape is not covered (the caller then runs the CUDA-core kernel): a
// Gaussian needs gauss_factored, i.e. every scaled squared norm |x'|^2 of
// the sites and nodes small enough that 2^(2 x'.s') and 2^(-|s'|^2) stay
// well inside the float32 range.
bool sum_tc(int D, int kernel, const float* tgt, int64_t tgt_gstride, const float* src, int64_t src_gstride,
            const float* xq16, int64_t groups_src, DBuf<float>& bq_scratch, float* out, int64_t out_gstride,
            const int32_t* rowptr, const int32_t* col, const int32_t* count, int count_off, int count_const,
            int first, int ngroups, int ld, int Rc, bool gauss_factored, int* err, cudaStream_t s) {
  if (ld % 8 != 0 || ld > kRow || (D != 4 && D != 8 && D != 10 && D != 12 && D != 16 && D != 20)) return false;
  const bool gauss = kernel == DWFMM_K_GAUSS;
  if (gauss && !gauss_factored) return false;
  const size_t smem = tc_smem(D, ld);
  if (smem > 200 * 1024) return false;
  const uint64_t dbit = device_bit();
  if (!(g_tc_attrs_dev.load() & dbit)) {
    tc_attrs_d<4>();
    tc_attrs_d<8>();
    tc_attrs_d<10>();
    tc_attrs_d<12>();
    tc_attrs_d<16>();
    tc_attrs_d<20>();
    DW_CUDA(cudaGetLastError());
    g_tc_attrs_dev.fetch_or(dbit);
  }
  bq_scratch.alloc(static_cast<size_t>(groups_src) * 2 * 16 * ld);
  const int64_t nq = groups_src * ld * 16;
  k_make_bq<<<ceil_div(nq, 256), 256, 0, s>>>(xq16, groups_src, ld, src, src_gstride, D, gauss ? 1 : 0,
                                               bq_scratch.p);
  TcArgs a{};
  a.tgt = tgt;
  a.tgt_gstride = tgt_gstride;
  a.src = src;
  a.src_gstride = src_gstride;
  a.bq = bq_scratch.p;
  a.out = out;
  a.out_gstride = out_gstride;
  a.rowptr = rowptr;
  a.col = col;
  a.count = count;
  a.count_off = count_off;
  a.count_const = count_const;
  a.first = first;
  a.ld = ld;
  a.halves = (ld + 127) / 128;
  a.Rc = Rc;
  a.err = err;
  const int grid = ngroups * a.halves;
  if (grid <= 0) return true;
  switch (D) {
    case 4: tc_launch_d<4>(kernel, a, grid, smem, s); break;
    case 8: tc_launch_d<8>(kernel, a, grid, smem, s); break;
    case 10: tc_launch_d<10>(kernel, a, grid, smem, s); break;
    case 12: tc_launch_d<12>(kernel, a, grid, smem, s); break;
    case 16: tc_launch_d<16>(kernel, a, grid, smem, s); break;
    default: tc_launch_d<20>(kernel, a, grid, smem, s); break;
  }
  DW_CUDA(cudaGetLastError());
  return true;
}

}  // namespace dw
