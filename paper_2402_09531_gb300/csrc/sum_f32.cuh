// Float32 kernel summation, y_i = sum_j phi(|x_i - x_j| / sigma) q_j over a
// CSR list of source blocks (the P2P near field and the M2L couplings of
// Sec. 5.2), as a device function over one target group.  Shared by the
// one-CTA-per-group kernel (k_sum_f32) and the persistent batch kernel,
// whose CTAs split into several such groups.
//
//  - Source blocks (scaled coordinates plus a norm row, then R charge rows)
//    are contiguous and 32-byte aligned in HBM, so each block is two 1-D
//    bulk copies (cp.async.bulk, mbarrier completion) into a double-buffered
//    shared-memory stage; the group's first thread issues, every thread waits
//    with a bounded try_wait loop that raises an error flag instead of hanging.
//  - Each thread owns kTT targets; sources are read as float4 broadcasts from
//    shared memory, 4 sources per step; arithmetic is packed (f32x2).
//  - Per source block the contributions are summed in float32 partials, then
//    folded into per-target running sums with Kahan compensation (kept in
//    shared memory).
#pragma once

#include <cstdint>

#include "dwfmm_internal.cuh"

namespace dw {
namespace sk {

constexpr int kThreadsMax = 128;
constexpr int kTT = 2;
constexpr long long kWaitLimit = 1ll << 24;   // ~ seconds of polling: a copy never takes that long

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait for phase `parity` of the barrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}


template <int KER>
__device__ __forceinline__ float phi_scaled(float a) {
  // a = the kernel's argument after scaling: Gaussian: exponent; exp/Matern: r'^2
  if (KER == DWFMM_K_GAUSS) return ex2_approx(a);
  const float r = sqrt_approx(a);
  if (KER == DWFMM_K_EXP) return ex2_approx(-r);
  const float e = ex2_approx(-1.4426950408889634f * r);
  return fmaf(r, e, e);
}

// Packed float32 pairs (fma/add/sub .f32x2): one instruction, two lanes of work.
typedef unsigned long long u64;

__device__ __forceinline__ u64 pk2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(u64 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 fadd2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fsub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Element t of the interleaved charges: row layout src[g][16][ld] ->
// dst[g][ld][RC] (first RC rows), t < groups * ld * RC.
__device__ __forceinline__ void interleave_elem(const float* src, int ld, int RC, float* dst, int64_t t) {
  const int r = static_cast<int>(t % RC);
  const int64_t gi = t / RC;
  const int i = static_cast<int>(gi % ld);
  const int64_t g = gi / ld;
  dst[t] = src[(g * kRC + r) * ld + i];
}

// A group of threads that works on one target group: `tid` its thread index
// within the group, `size` its thread count (a multiple of 32), `bar` the
// hardware barrier it synchronises on (0 with size = blockDim.x: the CTA).
struct Grp {
  int tid, size, bar;
};

__device__ __forceinline__ void grp_sync(const Grp& G) {
  asm volatile("bar.sync %0, %1;" ::"r"(G.bar), "r"(G.size) : "memory");
}

// Barrier of the group that also returns whether any of its threads passed p.
__device__ __forceinline__ bool grp_or(const Grp& G, bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(p)), "r"(G.bar), "r"(G.size)
      : "memory");
  return r != 0;
}

// Stage and compensation bytes of one group of `threads` threads.
__host__ __device__ constexpr size_t group_stage_bytes(int D, int RC, int ld, int threads) {
  return 2 * static_cast<size_t>((D + 1) * ld + RC * ld) * sizeof(float) +
         static_cast<size_t>(kTT) * (RC >= 2 ? RC / 2 : 1) * threads * sizeof(unsigned long long);
}

// Target group g (all of its targets, kTT * G.size per pass) against its
// list a.rowptr[g] .. a.rowptr[g + 1].  `smem` holds the group's two stages
// and its compensation array (group_stage_bytes), `full` its two stage
// barriers, initialised with count 1; `tile_base` counts the stages the
// barriers have completed so far and is advanced.  Returns false (after
// setting *a.err = 3) when a copy did not land within the wait limit.

// Charge blocks are interleaved per source, [g][ld][RC], so RHS pairs are
// adjacent: (acc_r, acc_r+1) += (phi, phi) * (q_r, q_r+1) is one fma.f32x2.
// Distances pair up consecutive sources: (e_j, e_j+1) += (2x_k, 2x_k) * (s_jk, s_j+1,k).
template <int D, int RC, int KER>
__device__ __forceinline__ bool sum_block(const SumArgs& a, int g, const Grp& G, unsigned char* smem, uint64_t* full,
                                          int& tile_base) {
  constexpr int RP = RC >= 2 ? RC / 2 : 1;   // packed accumulators per target
  const int ld = a.ld;
  const int stage_floats = (D + 1) * ld + RC * ld;
  float* stage0 = reinterpret_cast<float*>(smem);
  // Kahan compensation, [kTT * RP][group size] packed pairs (or floats when RC == 1)
  u64* comp = reinterpret_cast<u64*>(stage0 + 2 * stage_floats);
  const int rb = a.rowptr[g], re = a.rowptr[g + 1];
  const uint32_t coord_bytes = static_cast<uint32_t>((D + 1) * ld * sizeof(float));
  const uint32_t q_bytes = static_cast<uint32_t>(RC * ld * sizeof(float));

  // tiles are numbered across all target passes (and, in a persistent
  // kernel, across the group's earlier groups): stage = tile & 1, completion
  // parity of that stage's barrier = (tile >> 1) & 1
  auto issue = [&](int e, int tile) {
    const int s = a.col[e];
    float* st = stage0 + (tile & 1) * stage_floats;
    uint64_t* bar = &full[tile & 1];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, coord_bytes + q_bytes);
    bulk_copy(st, a.src + s * a.src_gstride, coord_bytes, bar);
    bulk_copy(st + (D + 1) * ld, a.q + s * a.q_gstride, q_bytes, bar);
  };

  for (int tb = 0; tb < ld; tb += kTT * G.size) {
    u64 xt2[kTT][D];   // (c x_k, c x_k), c = 2 for the Gaussian, else 1
    u64 mnt2[kTT];     // (-|x|^2, -|x|^2) for the Gaussian
    int ti[kTT];
#pragma unroll
    for (int t = 0; t < kTT; ++t) {
      ti[t] = tb + G.tid + t * G.size;
      const int i = ti[t] < ld ? ti[t] : 0;
      const float* tp = a.tgt + g * a.tgt_gstride + i;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float v = (KER == DWFMM_K_GAUSS) ? 2.0f * tp[k * ld] : tp[k * ld];
        xt2[t][k] = pk2(v, v);
      }
      const float nt = (KER == DWFMM_K_GAUSS) ? -tp[D * ld] : 0.0f;
      mnt2[t] = pk2(nt, nt);
    }
    u64 acc[kTT][RP];
    float acc1[kTT];
#pragma unroll
    for (int t = 0; t < kTT; ++t) {
      acc1[t] = 0.0f;
#pragma unroll
      for (int p = 0; p < RP; ++p) {
        acc[t][p] = 0ull;
        comp[(t * RP + p) * G.size + G.tid] = 0ull;
      }
    }

    if (G.tid == 0) {
      if (rb < re) issue(rb, tile_base);
      if (rb + 1 < re) issue(rb + 1, tile_base + 1);
    }
    bool timeout = false;
    for (int e = rb; e < re; ++e) {
      const int tile = tile_base + (e - rb);
      const int sidx = tile & 1;
      const uint32_t parity = static_cast<uint32_t>((tile >> 1) & 1);
      if (!mbar_wait(&full[sidx], parity)) timeout = true;
      const float* sc = stage0 + sidx * stage_floats;
      const float* sq = sc + (D + 1) * ld;
      const int scnt = a.count ? a.count[a.count_off + a.col[e]] : a.count_const;
      const int s4 = timeout ? 0 : ((scnt + 3) & ~3);
      u64 part[kTT][RP];
      float part1[kTT];
#pragma unroll
      for (int t = 0; t < kTT; ++t) {
        part1[t] = 0.0f;
#pragma unroll
        for (int p = 0; p < RP; ++p) part[t][p] = 0ull;
      }
      for (int j = 0; j < s4; j += 4) {
        u64 ph01[kTT], ph23[kTT];
        if (KER == DWFMM_K_GAUSS) {
          const ulonglong2 ns = *reinterpret_cast<const ulonglong2*>(sc + D * ld + j);
#pragma unroll
          for (int t = 0; t < kTT; ++t) {
            ph01[t] = fsub2(mnt2[t], ns.x);
            ph23[t] = fsub2(mnt2[t], ns.y);
          }
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const ulonglong2 sv = *reinterpret_cast<const ulonglong2*>(sc + k * ld + j);
#pragma unroll
            for (int t = 0; t < kTT; ++t) {
              ph01[t] = ffma2(xt2[t][k], sv.x, ph01[t]);
              ph23[t] = ffma2(xt2[t][k], sv.y, ph23[t]);
            }
          }
        } else {
#pragma unroll
          for (int t = 0; t < kTT; ++t) ph01[t] = ph23[t] = 0ull;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const ulonglong2 sv = *reinterpret_cast<const ulonglong2*>(sc + k * ld + j);
#pragma unroll
            for (int t = 0; t < kTT; ++t) {
              u64 df = fsub2(xt2[t][k], sv.x);
              ph01[t] = ffma2(df, df, ph01[t]);
              df = fsub2(xt2[t][k], sv.y);
              ph23[t] = ffma2(df, df, ph23[t]);
            }
          }
        }
        float ph[kTT][4];
#pragma unroll
        for (int t = 0; t < kTT; ++t) {
          up2(ph01[t], ph[t][0], ph[t][1]);
          up2(ph23[t], ph[t][2], ph[t][3]);
#pragma unroll
          for (int u = 0; u < 4; ++u) ph[t][u] = phi_scaled<KER>(ph[t][u]);
        }
        if constexpr (RC == 1) {
          const float4 qv = *reinterpret_cast<const float4*>(sq + j);
#pragma unroll
          for (int t = 0; t < kTT; ++t) {
            float p = part1[t];
            p = fmaf(ph[t][0], qv.x, p);
            p = fmaf(ph[t][1], qv.y, p);
            p = fmaf(ph[t][2], qv.z, p);
            p = fmaf(ph[t][3], qv.w, p);
            part1[t] = p;
          }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const ulonglong2* qrow = reinterpret_cast<const ulonglong2*>(sq + (j + u) * RC);
            u64 f2[kTT];
#pragma unroll
            for (int t = 0; t < kTT; ++t) f2[t] = pk2(ph[t][u], ph[t][u]);
#pragma unroll
            for (int rr = 0; rr < RC / 4; ++rr) {
              const ulonglong2 qv = qrow[rr];
#pragma unroll
              for (int t = 0; t < kTT; ++t) {
                part[t][2 * rr] = ffma2(f2[t], qv.x, part[t][2 * rr]);
                part[t][2 * rr + 1] = ffma2(f2[t], qv.y, part[t][2 * rr + 1]);
              }
            }
          }
        }
      }
      // Kahan: acc += part (compensation kept in shared memory)
#pragma unroll
      for (int t = 0; t < kTT; ++t) {
        if constexpr (RC == 1) {
          float* c1 = reinterpret_cast<float*>(comp) + t * G.size + G.tid;
          const float y = part1[t] - *c1;
          const float s = acc1[t] + y;
          *c1 = (s - acc1[t]) - y;
          acc1[t] = s;
        } else {
#pragma unroll
          for (int p = 0; p < RP; ++p) {
            u64* cp = comp + (t * RP + p) * G.size + G.tid;
            const u64 y = fsub2(part[t][p], *cp);
            const u64 s = fadd2(acc[t][p], y);
            *cp = fsub2(fsub2(s, acc[t][p]), y);
            acc[t][p] = s;
          }
        }
      }
      // every thread is done with this stage before it is refilled
      if (grp_or(G, timeout)) {
        if (G.tid == 0) {
          atomicExch(a.err, 3);
          // let the copy already issued for the next tile land before exiting
          if (e + 1 < re) (void)mbar_wait(&full[(tile + 1) & 1], static_cast<uint32_t>(((tile + 1) >> 1) & 1));
        }
        grp_sync(G);
        return false;
      }
      if (G.tid == 0 && e + 2 < re) issue(e + 2, tile + 2);
    }
    tile_base += re - rb;
#pragma unroll
    for (int t = 0; t < kTT; ++t) {
      if (ti[t] < ld) {
        float* op = a.out + g * a.out_gstride + ti[t];
        if constexpr (RC == 1) {
          if (a.Rc > 0) op[0] = acc1[t];
        } else {
#pragma unroll
          for (int p = 0; p < RP; ++p) {
            float lo, hi;
            up2(acc[t][p], lo, hi);
            if (2 * p < a.Rc) op[(2 * p) * ld] = lo;
            if (2 * p + 1 < a.Rc) op[(2 * p + 1) * ld] = hi;
          }
        }
      }
    }
    grp_sync(G);
  }
  return true;
}

}  // namespace sk
}  // namespace dw
