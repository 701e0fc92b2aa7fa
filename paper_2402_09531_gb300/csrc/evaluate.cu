// Evaluation of the kernel interpolant at new points (Sec. 2):
//   s(x_t) = sum_j phi(||x_t - x_j|| / sigma) c_j,  t = 1..n_t,
// the quantity whose error at test points is the prediction error of
// Sec. 6.2.  It is evaluated exactly: targets are blocked like leaves and
// every target block meets every source leaf in the kernel-summation engine
// (float32 tuned kernel or float64 generic kernel, by the plan's precision).
#include <algorithm>

#include "dwfmm_internal.cuh"

namespace dw {

namespace {

// Targets (row-major, leading dimension ld) -> blocks [G][d][m_pad]; padding
// slots repeat the block's first target.
__global__ void k_target_blocks(const double* t, int64_t nt, int64_t ld, int d, int m_pad, int G, double* blk) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(G) * m_pad) return;
  const int64_t g = i / m_pad;
  const int64_t src = i < nt ? i : g * m_pad;
  const int slot = static_cast<int>(i % m_pad);
  for (int k = 0; k < d; ++k) blk[(g * d + k) * m_pad + slot] = t[src * ld + k];
}

__global__ void k_full_lists(int G, int L, int32_t* rowptr, int32_t* col) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i <= G) rowptr[i] = static_cast<int32_t>(i * L);
  if (i < static_cast<int64_t>(G) * L) col[i] = static_cast<int32_t>(i % L);
}

template <typename T>
__global__ void k_eval_out(const T* out, int64_t nt, int m_pad, int r0, int Rc, double* y, int64_t ldy) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= nt * Rc) return;
  const int r = static_cast<int>(i / nt);
  const int64_t t = i % nt;
  const int64_t g = t / m_pad;
  const int slot = static_cast<int>(t % m_pad);
  y[(r0 + r) * ldy + t] = static_cast<double>(out[(g * kRC + r) * m_pad + slot]);
}

}  // namespace

void evaluate(Plan& P, const double* tgt, int64_t nt, int64_t ldt, const double* c, int64_t ldc, double* out,
              int64_t ldo, int R) {
  cudaStream_t s = P.stream;
  const bool fp64 = P.prec == DWFMM_P_FP64;
  const int m = P.m_pad;
  const int G = static_cast<int>((nt + m - 1) / m);
  DBuf<double> blk64;
  DBuf<int32_t> rowptr, col;
  blk64.alloc(static_cast<size_t>(G) * P.d * m);
  rowptr.alloc(G + 1);
  col.alloc(static_cast<size_t>(G) * P.L);
  k_target_blocks<<<ceil_div(static_cast<int64_t>(G) * m, 256), 256, 0, s>>>(tgt, nt, ldt, P.d, m, G, blk64.p);
  k_full_lists<<<ceil_div(static_cast<int64_t>(G) * P.L + 1, 256), 256, 0, s>>>(G, P.L, rowptr.p, col.p);
  ensure_workspace(P, fp64);
  DBuf<double> o64;
  DBuf<float> o32, blk32;
  if (fp64) o64.alloc(static_cast<size_t>(G) * kRC * m);
  else o32.alloc(static_cast<size_t>(G) * kRC * m);
  for (int r0 = 0; r0 < R; r0 += kRC) {
    const int Rc = std::min(kRC, R - r0);
    launch_gather(P, c, ldc, r0, Rc, fp64);
    if (fp64) {
      eval_f64(P, blk64.p, G, rowptr.p, col.p, Rc, o64.p, s);
      k_eval_out<double><<<ceil_div(nt * Rc, 256), 256, 0, s>>>(o64.p, nt, m, r0, Rc, out, ldo);
    } else {
      eval_f32(P, blk64.p, G, rowptr.p, col.p, Rc, o32.p, blk32, s);
      k_eval_out<float><<<ceil_div(nt * Rc, 256), 256, 0, s>>>(o32.p, nt, m, r0, Rc, out, ldo);
    }
  }
  DW_CUDA(cudaGetLastError());
  DW_CUDA(cudaStreamSynchronize(s));   // the local blocks are freed on return
}

}  // namespace dw
