// Conjugate gradients for (K_tilde + lambda I) c = f (Sec. 2 Eq. (2.2);
// Sec. 6.2 solves the kernel ridge system by CG to a relative tolerance).
// One independent CG per right-hand side column, float64 vectors, dot
// products reduced deterministically (fixed block partition, fixed order).
// The compressed matrix can be mildly indefinite (Sec. 5.3 error against a
// small ridge), so negative curvature p^T A p < 0 does not stop CG; a column
// breaks down only when p^T A p is zero or not finite.
// FP32/MIXED plans run iterative refinement: the outer residual uses the
// float64 operator, the inner CG the plan's reduced-precision operator.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dwfmm_internal.cuh"

namespace dw {

namespace {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 120;

__global__ void k_dot_partial(const double* a, const double* b, int64_t n, int64_t ld, double* part) {
  __shared__ double sh[kDotThreads / 32];
  const int r = blockIdx.y;
  const double* x = a + r * ld;
  const double* y = b + r * ld;
  double s = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    s += x[i] * y[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) t += sh[w];
    part[r * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_dot_final(const double* part, int nb, int R, double* out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += part[r * nb + b];
  out[r] = t;
}

// y[:, r] = a * x[:, r] + b * y[:, r] (+ lam * z[:, r] if z)
__global__ void k_axpby(const double* x, double* y, const double* z, const double* coef_a,
                        double coef_b_const, const double* coef_b, double lam, int64_t n, int64_t ld,
                        int R, double a_sign) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * R) return;
  const int r = static_cast<int>(t / n);
  const int64_t i = t % n;
  const int64_t o = r * ld + i;
  const double a = coef_a ? a_sign * coef_a[r] : a_sign;
  const double bb = coef_b ? coef_b[r] : coef_b_const;
  double v = a * x[o] + bb * y[o];
  if (z) v += lam * z[o];
  y[o] = v;
}

void dots(Plan& P, const double* a, const double* b, int64_t n, int64_t ld, int R, double* part,
          double* out_dev, double* out_host) {
  dim3 grid(kDotBlocks, R);
  k_dot_partial<<<grid, kDotThreads, 0, P.stream>>>(a, b, n, ld, part);
  k_dot_final<<<ceil_div(R, 64), 64, 0, P.stream>>>(part, kDotBlocks, R, out_dev);
  DW_CUDA(cudaMemcpyAsync(out_host, out_dev, R * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
  DW_CUDA(cudaStreamSynchronize(P.stream));
}

// A v = K_tilde v + lam v (into out); v, out: n x R, leading dimension n.
void apply_op(Plan& P, const double* v, double* out, int R, double lam, bool fp64) {
  const int64_t n = P.N;
  matvec_device(P, v, n, out, n, R, fp64);
  if (lam != 0.0)
    // out = lam * v + 1 * out  (a_sign carries lam, coef_b_const = 1)
    k_axpby<<<ceil_div(n * R, 256), 256, 0, P.stream>>>(v, out, nullptr, nullptr, 1.0, nullptr, 0.0, n, n, R, lam);
}

}  // namespace

// One refinement step with a minimal-residual length (defined with the
// device-side CG helpers below): c += alpha delta, r -= alpha (A64 delta).
void refine_step(Plan& P, double lam, double* c, const double* delta, double* r, int R, double* w,
                 double* part, double* dev3);

// CG from x = 0 on (K_tilde + lam I) x = b (device, compact) with the
// device-side iteration of dwfmm_cg_step (scalars on the GPU, iterations
// replayed from a captured graph), checking the status snapshot every
// kSolveChunk iterations; the solution stays in P.cg_c.  st per column:
// 0 converged, 1 breakdown, 2 not converged.  Returns the largest iteration
// count.
int cg_dev(Plan& P, const double* b, int R, double lam, double rtol, int maxit, std::vector<int>& st) {
  constexpr int kSolveChunk = 16;
  cg_begin(P, lam, b, R, P.N, rtol);
  CgState& S = P.cgs;
  st.assign(R, 2);
  int done = 0, its = 0;
  while (done < maxit) {
    const int k = std::min(kSolveChunk, maxit - done);
    cg_step(P, k);
    done += k;
    DW_CUDA(cudaEventSynchronize(S.ev));
    bool all = true;
    for (int r = 0; r < R; ++r) all &= S.h_snap[r] != 0;
    if (all) break;
  }
  for (int r = 0; r < R; ++r) {
    const int code = S.h_snap[r];
    st[r] = code == 1 ? 0 : (code == 2 ? 1 : 2);
    its = std::max(its, S.h_snap[R + r]);
  }
  return its;
}

dwfmm_status solve(Plan& P, double lam, const double* f, double* c, int R, int64_t ld, double rtol,
                   int maxit, int* iters, double* relres) {
  const int64_t n = P.N;
  const int64_t nr = n * R;
  if (n == 0) {
    if (iters) *iters = 0;
    if (relres)
      for (int r = 0; r < R; ++r) relres[r] = 0.0;
    return DWFMM_OK;
  }
  P.cg_tmp.alloc(nr);
  P.cg_dot.alloc(static_cast<size_t>(kDotBlocks) * R + 8 * R + 8);
  double* part = P.cg_dot.p;
  double* dot = part + static_cast<size_t>(kDotBlocks) * R;
  // f (compact) and the solution live outside the CG's own buffers
  DBuf<double> fc, x;
  fc.alloc(nr);
  x.alloc(nr);
  DW_CUDA(cudaMemcpy2DAsync(fc.p, n * sizeof(double), f, ld * sizeof(double), n * sizeof(double), R,
                            cudaMemcpyDeviceToDevice, P.stream));
  std::vector<double> fn2(R), res2(R);
  dots(P, fc.p, fc.p, n, n, R, part, dot, fn2.data());
  const bool fp64 = P.prec == DWFMM_P_FP64;
  int total_it = 0;
  std::vector<int> st;
  dwfmm_status status = DWFMM_OK;
  if (fp64) {
    total_it = cg_dev(P, fc.p, R, lam, rtol, maxit, st);
    DW_CUDA(cudaMemcpyAsync(x.p, P.cg_c.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
    for (int r = 0; r < R; ++r) {
      if (st[r] == 1) status = DWFMM_ERR_BREAKDOWN;
      else if (st[r] == 2 && status == DWFMM_OK) status = DWFMM_ERR_NOT_CONVERGED;
    }
  } else {
    // iterative refinement: delta = CG32(r), c += alpha delta, r -= alpha A64 delta
    // with alpha = 1 where that lowers the float64 residual, else the
    // minimal-residual length (when the float32 operator's error approaches
    // lambda a capped inner CG can return a correction that would raise it)
    DW_CUDA(cudaMemsetAsync(x.p, 0, nr * sizeof(double), P.stream));
    DBuf<double> rhs;
    rhs.alloc(nr);
    DW_CUDA(cudaMemcpyAsync(rhs.p, fc.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
    // Each inner CG (float32 operator) reduces the float64 residual by at most
    // 1e-3 within at most 400 iterations; the float64 residual then restarts
    // it.  With a small ridge the float32 rounding of the operator (~1e-7 of
    // ||K||) exceeds lambda, and one long float32 CG loses its way.
    const double inner_floor = 1e-3;
    const int inner_maxit = 400;
    status = DWFMM_ERR_NOT_CONVERGED;
    for (int outer = 0; outer < 100 && total_it < maxit; ++outer) {
      dots(P, rhs.p, rhs.p, n, n, R, part, dot, res2.data());
      bool done = true;
      double relmax = 0.0;
      for (int r = 0; r < R; ++r) {
        const double rel = fn2[r] > 0.0 ? std::sqrt(res2[r] / fn2[r]) : 0.0;
        done &= rel <= rtol;
        relmax = std::max(relmax, rel);
      }
      if (done) {
        status = DWFMM_OK;
        break;
      }
      double inner_tol = std::max(rtol, 0.5 * rtol / std::max(relmax, 1e-300));
      if (relmax > rtol / inner_floor) inner_tol = std::max(inner_tol, inner_floor);
      inner_tol = std::min(0.5, inner_tol);
      const int it = cg_dev(P, rhs.p, R, lam, inner_tol, std::min(inner_maxit, maxit - total_it), st);
      total_it += it;
      bool broke = false;
      for (int r = 0; r < R; ++r) broke |= st[r] == 1;
      double* dev3 = dot + 2 * R;
      refine_step(P, lam, x.p, P.cg_c.p, rhs.p, R, P.cg_tmp.p, part, dev3);
      if (broke) {
        // a breakdown of the inner CG is fatal only if its correction did not help
        std::vector<double> alpha(R);
        DW_CUDA(cudaMemcpyAsync(alpha.data(), dev3 + 2 * R, R * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
        DW_CUDA(cudaStreamSynchronize(P.stream));
        bool moved = false;
        for (int r = 0; r < R; ++r) moved |= alpha[r] != 0.0;
        if (!moved) {
          status = DWFMM_ERR_BREAKDOWN;
          break;
        }
      }
    }
    if (status == DWFMM_ERR_NOT_CONVERGED) {
      dots(P, rhs.p, rhs.p, n, n, R, part, dot, res2.data());
      bool done = true;
      for (int r = 0; r < R; ++r) done &= std::sqrt(res2[r]) <= rtol * std::sqrt(fn2[r]) || fn2[r] == 0.0;
      if (done) status = DWFMM_OK;
    }
  }
  // true residual with the float64 operator
  DBuf<double> res;
  res.alloc(nr);
  apply_op(P, x.p, P.cg_tmp.p, R, lam, true);
  DW_CUDA(cudaMemcpyAsync(res.p, fc.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  k_axpby<<<ceil_div(nr, 256), 256, 0, P.stream>>>(P.cg_tmp.p, res.p, nullptr, nullptr, 1.0, nullptr, 0.0, n, n, R, -1.0);
  dots(P, res.p, res.p, n, n, R, part, dot, res2.data());
  if (relres)
    for (int r = 0; r < R; ++r) relres[r] = fn2[r] > 0.0 ? std::sqrt(res2[r] / fn2[r]) : 0.0;
  if (iters) *iters = total_it;
  DW_CUDA(cudaMemcpy2DAsync(c, ld * sizeof(double), x.p, n * sizeof(double), n * sizeof(double), R,
                            cudaMemcpyDeviceToDevice, P.stream));
  DW_CUDA(cudaStreamSynchronize(P.stream));
  return status;
}

}  // namespace dw

// ---------------------------------------------------------------------------
// Incremental CG with every scalar on the device (for many solves in flight).
// One iteration is a fixed sequence of launches on the plan's stream with no
// host synchronisation: Ap = K_tilde p + lambda p, pAp, alpha, x/r update,
// rr_new, beta (convergence and breakdown decided per column on the device),
// p update.  A non-blocking poll reads a status snapshot copied to pinned
// host memory after each batch of iterations.
// ---------------------------------------------------------------------------

namespace dw {

namespace {

// state layout (doubles): rr[R], pap[R], coef[R], bn2[R]; ints: status[R], iters[R]
// rtol^2 goes to device memory, so that captured iterations read it there
// (refinement rounds change the tolerance, not the graph).
__global__ void k_cg_init(const double* rr, int R, double* st_rr, double* st_bn2, int* status, int* iters,
                          double rtol, double* st_rtol2) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  st_rr[r] = rr[r];
  st_bn2[r] = rr[r];
  iters[r] = 0;
  status[r] = (rr[r] == 0.0) ? 1 : 0;   // 0 running, 1 converged, 2 breakdown
  if (r == 0) *st_rtol2 = rtol * rtol;
}

__global__ void k_cg_alpha(const double* pap, const double* rr, int* status, double* alpha, int R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double a = 0.0;
  if (status[r] == 0) {
    if (pap[r] == 0.0 || !isfinite(pap[r])) status[r] = 2;   // negative curvature is tolerated
    else a = rr[r] / pap[r];
  }
  alpha[r] = a;
}

__global__ void k_cg_beta(const double* rr_new, double* rr, const double* bn2, int* status, int* iters,
                          double* beta, int R, const double* rtol2) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double b = 0.0;
  if (status[r] == 0) {
    iters[r] += 1;
    if (rr_new[r] <= *rtol2 * bn2[r]) status[r] = 1;
    b = rr_new[r] / rr[r];
    rr[r] = rr_new[r];
  }
  beta[r] = b;
}

void dots_dev(Plan& P, const double* a, const double* b, int64_t n, int R, double* part, double* out) {
  dim3 grid(kDotBlocks, R);
  k_dot_partial<<<grid, kDotThreads, 0, P.stream>>>(a, b, n, n, part);
  k_dot_final<<<ceil_div(R, 64), 64, 0, P.stream>>>(part, kDotBlocks, R, out);
}

// Step length per column from a* = (r, w) / (w, w): the plain refinement
// step 1 whenever it lowers ||r - alpha w|| (a* > 1/2), else a*; 0 when
// w = 0 or a* is not finite.  Either way ||r - alpha w|| <= ||r||.
__global__ void k_minres_alpha(const double* num, const double* den, double* alpha, int R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double a = den[r] > 0.0 ? num[r] / den[r] : 0.0;
  if (!isfinite(a)) a = 0.0;
  alpha[r] = a > 0.5 ? 1.0 : a;
}

}  // namespace

// c += alpha delta and r -= alpha w with w = (K64 + lam I) delta and alpha
// per column from k_minres_alpha (never raising ||r||); r must hold f - (K64 + lam I) c on
// entry and holds the same for the new c on return.  All buffers compact
// (leading dimension N); w: N x R scratch; part: dot partials; dev3: 3R
// doubles (numerators, denominators, alpha).  No host synchronisation.
void refine_step(Plan& P, double lam, double* c, const double* delta, double* r, int R, double* w,
                 double* part, double* dev3) {
  const int64_t n = P.N;
  const int64_t nr = n * R;
  apply_op(P, delta, w, R, lam, true);
  dots_dev(P, r, w, n, R, part, dev3);
  dots_dev(P, w, w, n, R, part, dev3 + R);
  k_minres_alpha<<<ceil_div(R, 64), 64, 0, P.stream>>>(dev3, dev3 + R, dev3 + 2 * R, R);
  k_axpby<<<ceil_div(nr, 256), 256, 0, P.stream>>>(delta, c, nullptr, dev3 + 2 * R, 1.0, nullptr, 0.0, n, n, R, 1.0);
  k_axpby<<<ceil_div(nr, 256), 256, 0, P.stream>>>(w, r, nullptr, dev3 + 2 * R, 1.0, nullptr, 0.0, n, n, R, -1.0);
  DW_CUDA(cudaGetLastError());
}

// Device pointers of a plan's incremental CG state (for the batched step).
CgPtrs cg_ptrs(Plan& P) {
  CgState& S = P.cgs;
  const int R = S.R;
  double* part = P.cg_dot.p;
  CgPtrs c;
  std::memset(&c, 0, sizeof(c));   // padding too: batches compare the bytes
  c.p = P.cg_p.p;
  c.ap = P.cg_ap.p;
  c.c = P.cg_c.p;
  c.r = P.cg_r.p;
  c.rr = part + kDotBlocks * R;
  c.pap = c.rr + R;
  c.coef = c.pap + R;
  c.bn2 = c.coef + R;
  c.tmp = c.bn2 + R;
  c.rtol2 = c.tmp + R;
  c.status = S.d_int.p;
  c.iters = S.d_int.p + R;
  c.n = P.N;
  c.R = R;
  c.lam = S.lam;
  return c;
}

// Status snapshot of the plan's CG for dwfmm_cg_poll, on stream s.
void cg_snapshot(Plan& P, cudaStream_t s) {
  CgState& S = P.cgs;
  const int R = S.R;
  double* rr = P.cg_dot.p + kDotBlocks * R;
  DW_CUDA(cudaMemcpyAsync(S.h_snap, S.d_int.p, 2 * R * sizeof(int), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(S.h_snap) + 128 * sizeof(int), rr, R * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaEventRecord(S.ev, s));
  S.stepped = true;
}

void cg_begin(Plan& P, double lam, const double* f, int R, int64_t ld, double rtol) {
  const int64_t n = P.N;
  const int64_t nr = n * R;
  CgState& S = P.cgs;
  S.R = R;
  S.lam = lam;
  S.rtol = rtol;
  S.active = true;
  S.stepped = false;   // the previous status snapshot belongs to the previous solve
  P.cg_r.alloc(nr);
  P.cg_p.alloc(nr);
  P.cg_ap.alloc(nr);
  P.cg_c.alloc(nr);
  P.cg_f.alloc(nr);
  P.cg_dot.alloc(static_cast<size_t>(kDotBlocks) * R + 8 * R + 8);
  S.d_int.alloc(2 * R);
  if (!S.h_snap) DW_CUDA(cudaMallocHost(reinterpret_cast<void**>(&S.h_snap), 64 * (2 * sizeof(int) + sizeof(double))));
  if (!S.ev) DW_CUDA(cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming));
  double* part = P.cg_dot.p;
  double* rr = part + kDotBlocks * R;
  double* pap = rr + R;
  double* coef = pap + R;
  double* bn2 = coef + R;
  double* tmp = bn2 + R;
  DW_CUDA(cudaMemcpy2DAsync(P.cg_f.p, n * sizeof(double), f, ld * sizeof(double), n * sizeof(double), R,
                            cudaMemcpyDeviceToDevice, P.stream));
  DW_CUDA(cudaMemsetAsync(P.cg_c.p, 0, nr * sizeof(double), P.stream));
  DW_CUDA(cudaMemcpyAsync(P.cg_r.p, P.cg_f.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  DW_CUDA(cudaMemcpyAsync(P.cg_p.p, P.cg_f.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  dots_dev(P, P.cg_r.p, P.cg_r.p, n, R, part, tmp);
  k_cg_init<<<1, 64, 0, P.stream>>>(tmp, R, rr, bn2, S.d_int.p, S.d_int.p + R, rtol, tmp + R);
  DW_CUDA(cudaGetLastError());
}

// One CG iteration for every column on P.stream; nothing here waits for the
// host, so a run of iterations can be captured into a CUDA graph.
static void cg_iteration(Plan& P) {
  CgState& S = P.cgs;
  const int64_t n = P.N;
  const int R = S.R;
  const int64_t nr = n * R;
  double* part = P.cg_dot.p;
  double* rr = part + kDotBlocks * R;
  double* pap = rr + R;
  double* coef = pap + R;
  double* bn2 = coef + R;
  double* tmp = bn2 + R;
  double* rtol2 = tmp + R;
  int* status = S.d_int.p;
  int* its = S.d_int.p + R;
  const bool fp64 = P.prec == DWFMM_P_FP64;
  apply_op(P, P.cg_p.p, P.cg_ap.p, R, S.lam, fp64);
  dots_dev(P, P.cg_p.p, P.cg_ap.p, n, R, part, pap);
  k_cg_alpha<<<1, 64, 0, P.stream>>>(pap, rr, status, coef, R);
  k_axpby<<<ceil_div(nr, 256), 256, 0, P.stream>>>(P.cg_p.p, P.cg_c.p, nullptr, coef, 1.0, nullptr, 0.0, n, n, R, 1.0);
  k_axpby<<<ceil_div(nr, 256), 256, 0, P.stream>>>(P.cg_ap.p, P.cg_r.p, nullptr, coef, 1.0, nullptr, 0.0, n, n, R, -1.0);
  dots_dev(P, P.cg_r.p, P.cg_r.p, n, R, part, tmp);
  k_cg_beta<<<1, 64, 0, P.stream>>>(tmp, rr, bn2, status, its, coef, R, rtol2);
  k_axpby<<<ceil_div(nr, 256), 256, 0, P.stream>>>(P.cg_r.p, P.cg_p.p, nullptr, nullptr, 0.0, coef, 0.0, n, n, R, 1.0);
}

// Run `iters` iterations from a captured graph when possible: the launch
// sequence of an iteration is fixed for a tree, R, shift and buffer set, and
// small problems are bound by the host's launch rate, not by the GPU.  The
// first step with a new key runs plainly (it allocates whatever the matvec
// allocates on first use), the second captures, later steps replay.  Returns
// false when the caller should launch plainly (legacy default stream, phase
// timers on, first step of a key, or a capture that failed once).
static bool cg_step_graph(Plan& P, int iters) {
  CgState& S = P.cgs;
  if (iters <= 0 || P.stream == nullptr || P.tm.on || S.graphs_off) return false;
  CgGraphKey key;
  key.tree_gen = P.tree_gen;
  key.R = S.R;
  key.iters = iters;
  key.lam = S.lam;
  key.fp64 = P.prec == DWFMM_P_FP64;
  key.stream = P.stream;
  const void* bufs[6] = {P.cg_p.p, P.cg_ap.p, P.cg_c.p, P.cg_r.p, P.cg_dot.p, S.d_int.p};
  for (int i = 0; i < 6; ++i) key.bufs[i] = bufs[i];
  if (S.exec && S.graph_key == key) {
    DW_CUDA(cudaGraphLaunch(S.exec, P.stream));
    return true;
  }
  if (!(S.warm_key == key)) {
    S.warm_key = key;
    return false;
  }
  if (S.exec) cudaGraphExecDestroy(S.exec);
  if (S.graph) cudaGraphDestroy(S.graph);
  S.exec = nullptr;
  S.graph = nullptr;
  if (cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    (void)cudaGetLastError();
    S.graphs_off = true;
    return false;
  }
  try {
    for (int k = 0; k < iters; ++k) cg_iteration(P);
  } catch (...) {
    // a call in the path refused capture: nothing ran; launch plainly from now on
    cudaGraph_t g = nullptr;
    (void)cudaStreamEndCapture(P.stream, &g);
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    S.graphs_off = true;
    return false;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(P.stream, &g) != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    S.graphs_off = true;
    return false;   // nothing was enqueued: the caller launches plainly
  }
  cudaGraphExec_t e = nullptr;
  if (cudaGraphInstantiate(&e, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    (void)cudaGetLastError();
    S.graphs_off = true;
    return false;
  }
  S.graph = g;
  S.exec = e;
  S.graph_key = key;
  DW_CUDA(cudaGraphLaunch(S.exec, P.stream));
  return true;
}

void cg_step(Plan& P, int iters) {
  CgState& S = P.cgs;
  const int R = S.R;
  double* rr = P.cg_dot.p + kDotBlocks * R;
  if (!cg_step_graph(P, iters))
    for (int k = 0; k < iters; ++k) cg_iteration(P);
  // status snapshot for the non-blocking poll
  DW_CUDA(cudaMemcpyAsync(S.h_snap, S.d_int.p, 2 * R * sizeof(int), cudaMemcpyDeviceToHost, P.stream));
  DW_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(S.h_snap) + 128 * sizeof(int), rr, R * sizeof(double),
                          cudaMemcpyDeviceToHost, P.stream));
  DW_CUDA(cudaEventRecord(S.ev, P.stream));
  S.stepped = true;
  DW_CUDA(cudaGetLastError());
}

// Returns true when the snapshot of the last cg_step is available.
bool cg_poll(Plan& P, int* status, int* iters, double* rr) {
  CgState& S = P.cgs;
  if (!S.stepped) return false;
  const cudaError_t e = cudaEventQuery(S.ev);
  if (e == cudaErrorNotReady) return false;
  DW_CUDA(e);
  const int R = S.R;
  for (int r = 0; r < R; ++r) {
    if (status) status[r] = S.h_snap[r];
    if (iters) iters[r] = S.h_snap[R + r];
    if (rr) rr[r] = reinterpret_cast<const double*>(reinterpret_cast<const char*>(S.h_snap) + 128 * sizeof(int))[r];
  }
  return true;
}

void cg_result(Plan& P, double* c, int64_t ld) {
  const int64_t n = P.N;
  DW_CUDA(cudaMemcpy2DAsync(c, ld * sizeof(double), P.cg_c.p, n * sizeof(double), n * sizeof(double), P.cgs.R,
                            cudaMemcpyDefault, P.stream));
}

}  // namespace dw

namespace dw {

// r = f - (K64 c + lam c); relres per column.  f, c, r: device, leading dimension n.
void residual64(Plan& P, double lam, const double* f, const double* c, double* r, int R, double* relres) {
  const int64_t n = P.N;
  const int64_t nr = n * R;
  P.cg_tmp.alloc(nr);
  P.cg_dot.alloc(static_cast<size_t>(kDotBlocks) * R + 8 * R + 8);
  apply_op(P, c, P.cg_tmp.p, R, lam, true);
  DW_CUDA(cudaMemcpyAsync(r, f, nr * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  k_axpby<<<ceil_div(nr, 256), 256, 0, P.stream>>>(P.cg_tmp.p, r, nullptr, nullptr, 1.0, nullptr, 0.0, n, n, R, -1.0);
  std::vector<double> rn(R), fn(R);
  double* part = P.cg_dot.p;
  double* out = part + kDotBlocks * R;
  dots(P, r, r, n, n, R, part, out, rn.data());
  dots(P, f, f, n, n, R, part, out, fn.data());
  for (int k = 0; k < R; ++k) relres[k] = fn[k] > 0.0 ? std::sqrt(rn[k] / fn[k]) : 0.0;
}

// refine_step on compact device buffers, then alpha and ||r|| / ||f|| per
// column to the host.  Synchronises the plan's stream.
void refine64(Plan& P, double lam, const double* f, double* c, const double* delta, double* r, int R,
              double* alpha, double* relres) {
  const int64_t n = P.N;
  const int64_t nr = n * R;
  P.cg_tmp.alloc(nr);
  P.cg_dot.alloc(static_cast<size_t>(kDotBlocks) * R + 8 * R + 8);
  double* part = P.cg_dot.p;
  double* dev3 = part + static_cast<size_t>(kDotBlocks) * R + 2 * R;
  refine_step(P, lam, c, delta, r, R, P.cg_tmp.p, part, dev3);
  DW_CUDA(cudaMemcpyAsync(alpha, dev3 + 2 * R, R * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
  std::vector<double> rn(R), fn(R);
  double* out = part + static_cast<size_t>(kDotBlocks) * R;
  dots(P, r, r, n, n, R, part, out, rn.data());
  dots(P, f, f, n, n, R, part, out, fn.data());
  for (int k = 0; k < R; ++k) relres[k] = fn[k] > 0.0 ? std::sqrt(rn[k] / fn[k]) : 0.0;
}

}  // namespace dw
