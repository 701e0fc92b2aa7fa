// Expansion setup of the DW-FMM: weights, weighted total-degree index set,
// approximate Fekete nodes and V^{-1}.
//
//  - weights omega_k: Lemma 4.1 / Thm 4.6 / Sec. 6.2 (host, float64)
//  - Lambda_{omega,q,d} = {alpha : sum_k omega_k alpha_k <= q} (Sec. 4; host)
//  - Halton candidates, Vandermonde on the candidates, greedy column-pivoted
//    QR (Sec. 5.4), V = [p_hat_alpha'(xi_alpha)] (Eq. (5.3)) and its inverse:
//    GPU kernels in float64.
//
// This file is compiled with -fmad=false: every product and sum is rounded
// separately, so the candidate Vandermonde values and the residual norms of
// the pivoted QR are the same numbers a plain float64 evaluation gives.
#include <cmath>
#include <cstring>

#include "dwfmm_internal.cuh"

namespace dw {

// ---------------------------------------------------------------------------
// Host: weights and index set
// ---------------------------------------------------------------------------

static double rho_of_tau(double t) { return 2.0 * t + std::sqrt(1.0 + 4.0 * t * t); }

static std::vector<double> make_weights(const Plan& P) {
  std::vector<double> w(P.d);
  if (P.wrule == DWFMM_W_INV_GAMMA) {
    for (int k = 0; k < P.d; ++k) w[k] = P.gamma[0] / P.gamma[k];
  } else if (P.wrule == DWFMM_W_PAPER_LOGRHO) {
    // Sec. 6.2: tau_k^{-1} = eta b_k with b_k = 2 gamma_k; rho_k normalised
    // by rho_1 and scaled by e so that omega_1 = log e = 1.
    std::vector<double> tau(P.d);
    for (int k = 0; k < P.d; ++k) tau[k] = 1.0 / (P.eta * (2.0 * P.gamma[k]));
    const double r1 = rho_of_tau(tau[0]);
    for (int k = 0; k < P.d; ++k) w[k] = std::log(M_E * rho_of_tau(tau[k]) / r1);
  } else {
    w = P.w;
  }
  return w;
}

// Lexicographic enumeration (alpha_1 most significant).  Total degree: the
// partial sums s_k = s_{k-1} + omega_k alpha_k are accumulated left to right;
// tensor: every term omega_k alpha_k alone is bounded.  The test is inclusive
// with a 1e-12 relative slack.
static void enumerate(const std::vector<double>& w, double tol, bool tensor, int k, double s,
                      std::vector<int32_t>& alpha, std::vector<int32_t>& out, size_t cap) {
  const int d = static_cast<int>(w.size());
  if (k == d) {
    if (out.size() / d >= cap) fail(DWFMM_ERR_INVALID_ARG, "index set larger than 4096");
    out.insert(out.end(), alpha.begin(), alpha.end());
    return;
  }
  for (int a = 0;; ++a) {
    const double term = w[k] * static_cast<double>(a);
    const double t = tensor ? term : s + term;
    if (t > tol) break;
    alpha[k] = a;
    enumerate(w, tol, tensor, k + 1, tensor ? 0.0 : t, alpha, out, cap);
  }
  alpha[k] = 0;
}

static void make_index_set(Plan& P) {
  P.w = make_weights(P);
  for (int k = 0; k < P.d; ++k)
    if (!(P.w[k] > 0.0) || !std::isfinite(P.w[k])) fail(DWFMM_ERR_INVALID_ARG, "weights must be positive");
  const double tol = P.q * (1.0 + 1e-12);
  std::vector<int32_t> alpha(P.d, 0), out;
  enumerate(P.w, tol, P.iset == DWFMM_I_TENSOR, 0, 0.0, alpha, out, 4096);
  P.lam = out;
  P.n = static_cast<int>(out.size() / P.d);
  P.n_pad = round_up(P.n, 8);
  P.qk.assign(P.d, 0);
  for (int a = 0; a < P.n; ++a)
    for (int k = 0; k < P.d; ++k) P.qk[k] = std::max(P.qk[k], P.lam[a * P.d + k]);
  P.loff.assign(P.d, 0);
  int off = 0;
  for (int k = 0; k < P.d; ++k) {
    P.loff[k] = off;
    off += P.qk[k] + 1;
  }
  P.lsum = off;
  int nnz_max = 1;
  for (int a = 0; a < P.n; ++a) {
    int z = 0;
    for (int k = 0; k < P.d; ++k) z += P.lam[a * P.d + k] > 0;
    nnz_max = std::max(nnz_max, z);
  }
  P.nnz_max = nnz_max;
  std::vector<int16_t> fac(static_cast<size_t>(P.n) * nnz_max, int16_t(-1));
  for (int a = 0; a < P.n; ++a) {
    int z = 0;
    for (int k = 0; k < P.d; ++k) {
      const int ak = P.lam[a * P.d + k];
      if (ak > 0) fac[a * nnz_max + z++] = static_cast<int16_t>(P.loff[k] + ak);
    }
  }
  P.d_fac.alloc(fac.size());
  P.d_qk.alloc(P.d);
  P.d_loff.alloc(P.d);
  P.d_lam.alloc(P.lam.size());
  DW_CUDA(cudaMemcpy(P.d_fac.p, fac.data(), fac.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
  DW_CUDA(cudaMemcpy(P.d_qk.p, P.qk.data(), P.d * sizeof(int32_t), cudaMemcpyHostToDevice));
  DW_CUDA(cudaMemcpy(P.d_loff.p, P.loff.data(), P.d * sizeof(int32_t), cudaMemcpyHostToDevice));
  DW_CUDA(cudaMemcpy(P.d_lam.p, P.lam.data(), P.lam.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
}

// ---------------------------------------------------------------------------
// Device: Legendre tables and the tensor basis in float64 (Sec. 5.2)
// ---------------------------------------------------------------------------

constexpr int kMaxLsum = 256;

// p_hat_j(t) = sqrt(2j+1) P_j(2t-1), j = 0..qk, written to tab[loff + j].
__device__ void legendre_row64(double t, int qk, double* tab) {
  const double u = 2.0 * t - 1.0;
  double pm = 1.0, pc = u;
  tab[0] = 1.0;
  if (qk >= 1) tab[1] = u;
  for (int j = 1; j < qk; ++j) {
    const double pn = (static_cast<double>(2 * j + 1) * u * pc - static_cast<double>(j) * pm) /
                      static_cast<double>(j + 1);
    tab[j + 1] = pn;
    pm = pc;
    pc = pn;
  }
  for (int j = 1; j <= qk; ++j) tab[j] = tab[j] * sqrt(2.0 * j + 1.0);
}

// Product of the nonzero-degree factors in k order (factors of degree 0
// equal 1.0 exactly and are skipped without changing the rounding).
__device__ __forceinline__ double basis_value64(const double* tab, const int16_t* fac, int nnz) {
  double v = 1.0;
  for (int z = 0; z < nnz; ++z) {
    const int o = fac[z];
    if (o < 0) break;
    v = v * tab[o];
  }
  return v;
}

// Radical inverse of i in `base` as the correctly rounded ratio num / base^k.
__device__ double radical_inverse(long long i, long long base) {
  unsigned long long num = 0, den = 1;
  while (i > 0) {
    const long long digit = i % base;
    i /= base;
    num = num * base + digit;
    den *= base;
  }
  return static_cast<double>(num) / static_cast<double>(den);
}

// Candidates h_i (i = 1..M) and A[alpha][i] = p_hat_alpha(h_i).
__global__ void k_halton_vandermonde(int M, int d, const int32_t* primes, ExpDev e, double* H,
                                     double* A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double tab[kMaxLsum];
  for (int k = 0; k < d; ++k) {
    const double h = radical_inverse(static_cast<long long>(i) + 1, primes[k]);
    H[static_cast<int64_t>(i) * d + k] = h;
    legendre_row64(h, e.qk[k], tab + e.loff[k]);
  }
  for (int a = 0; a < e.n; ++a)
    A[static_cast<int64_t>(a) * M + i] = basis_value64(tab, e.fac + a * e.nnz_max, e.nnz_max);
}

// ---------------------------------------------------------------------------
// Greedy column-pivoted QR on A (n x M, row-major, columns = candidates).
// Step s: pick the live column with the largest residual norm (ties: lowest
// index), normalise it to q, project q out of every live column, recompute
// the norms.  Each block owns a contiguous range of columns; the pivot column
// is never written after it is picked, so all blocks can read it.
// ---------------------------------------------------------------------------

struct ArgMax {
  double v;
  int i;
};

__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i && b.i >= 0)) return b;
  return a;
}

__device__ ArgMax block_argmax(ArgMax m) {
  __shared__ double sv[32];
  __shared__ int si[32];
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax t{__shfl_down_sync(0xffffffffu, m.v, o), __shfl_down_sync(0xffffffffu, m.i, o)};
    m = better(m, t);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sv[wid] = m.v;
    si[wid] = m.i;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    m = lane < nw ? ArgMax{sv[lane], si[lane]} : ArgMax{-1.0, -1};
    for (int o = 16; o > 0; o >>= 1) {
      ArgMax t{__shfl_down_sync(0xffffffffu, m.v, o), __shfl_down_sync(0xffffffffu, m.i, o)};
      m = better(m, t);
    }
  }
  __syncthreads();
  return m;  // valid in thread 0
}

constexpr int kQrThreads = 256;

__device__ double column_norm2(const double* A, int n, int M, int i) {
  double s = 0.0;
  for (int a = 0; a < n; ++a) {
    const double v = A[static_cast<int64_t>(a) * M + i];
    s = s + v * v;
  }
  return s;
}

__global__ void k_qr_init(const double* A, int n, int M, unsigned char* alive, double* pv, int* pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  ArgMax m{-1.0, -1};
  if (i < M) {
    alive[i] = 1;
    m = ArgMax{column_norm2(A, n, M, i), i};
  }
  m = block_argmax(m);
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = m.v;
    pi[blockIdx.x] = m.i;
  }
}

__global__ void k_qr_step(double* A, int n, int M, int s, unsigned char* alive, const double* pv_in,
                          const int* pi_in, double* pv_out, int* pi_out, int nblocks,
                          int32_t* pivots, int* err) {
  extern __shared__ double qv[];
  __shared__ ArgMax best;
  __shared__ int bad;
  if (threadIdx.x == 0) {
    ArgMax m{-1.0, -1};
    for (int b = 0; b < nblocks; ++b) m = better(m, ArgMax{pv_in[b], pi_in[b]});
    best = m;
    bad = (*err != 0) || !(m.v > 0.0) || m.i < 0;
    if (blockIdx.x == 0) {
      if (bad && *err == 0) *err = 1;
      pivots[s] = bad ? -1 : m.i;
    }
  }
  __syncthreads();
  if (bad) return;
  const int p = best.i;
  const double nrm = sqrt(best.v);
  for (int a = threadIdx.x; a < n; a += blockDim.x) qv[a] = A[static_cast<int64_t>(a) * M + p] / nrm;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  ArgMax m{-1.0, -1};
  if (i < M) {
    if (i == p) alive[i] = 0;
    if (alive[i]) {
      double c = 0.0;
      for (int a = 0; a < n; ++a) c = c + qv[a] * A[static_cast<int64_t>(a) * M + i];
      double s2 = 0.0;
      for (int a = 0; a < n; ++a) {
        const int64_t o = static_cast<int64_t>(a) * M + i;
        const double v = A[o] - qv[a] * c;
        A[o] = v;
        s2 = s2 + v * v;
      }
      m = ArgMax{s2, i};
    }
  }
  m = block_argmax(m);
  if (threadIdx.x == 0) {
    pv_out[blockIdx.x] = m.v;
    pi_out[blockIdx.x] = m.i;
  }
}

__global__ void k_gather_nodes(const double* H, const int32_t* piv, int n, int d, double* nodes) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * d) return;
  const int s = t / d, k = t % d;
  const int p = piv[s];
  nodes[t] = p >= 0 ? H[static_cast<int64_t>(p) * d + k] : 0.0;
}

// Augmented [V | I] with V[s][alpha'] = p_hat_alpha'(xi_s) (Eq. (5.3)).
__global__ void k_vandermonde_aug(const double* nodes, ExpDev e, double* aug) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= e.n) return;
  double tab[kMaxLsum];
  for (int k = 0; k < e.d; ++k) legendre_row64(nodes[s * e.d + k], e.qk[k], tab + e.loff[k]);
  const int w = 2 * e.n;
  for (int a = 0; a < e.n; ++a) {
    aug[static_cast<int64_t>(s) * w + a] = basis_value64(tab, e.fac + a * e.nnz_max, e.nnz_max);
    aug[static_cast<int64_t>(s) * w + e.n + a] = (a == s) ? 1.0 : 0.0;
  }
}

// Gauss-Jordan elimination with partial pivoting (largest |pivot|, ties:
// lowest row) on the n x 2n augmented matrix, one block.
__global__ void k_gauss_jordan(double* aug, int n, int* err) {
  const int w = 2 * n;
  __shared__ ArgMax red;
  for (int col = 0; col < n; ++col) {
    ArgMax m{-1.0, -1};
    for (int r = col + threadIdx.x; r < n; r += blockDim.x) m = better(m, ArgMax{fabs(aug[static_cast<int64_t>(r) * w + col]), r});
    m = block_argmax(m);
    if (threadIdx.x == 0) red = m;
    __syncthreads();
    const int pr = red.i;
    if (!(red.v > 0.0) || pr < 0) {
      if (threadIdx.x == 0) *err = 2;
      return;
    }
    if (pr != col)
      for (int c = threadIdx.x; c < w; c += blockDim.x) {
        const double t = aug[static_cast<int64_t>(pr) * w + c];
        aug[static_cast<int64_t>(pr) * w + c] = aug[static_cast<int64_t>(col) * w + c];
        aug[static_cast<int64_t>(col) * w + c] = t;
      }
    __syncthreads();
    const double piv = aug[static_cast<int64_t>(col) * w + col];
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += blockDim.x) aug[static_cast<int64_t>(col) * w + c] /= piv;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * w; idx += blockDim.x) {
      const int r = idx / w, c = idx % w;
      if (r == col || c == col) continue;
      const double f = aug[static_cast<int64_t>(r) * w + col];
      if (f != 0.0) aug[idx] -= f * aug[static_cast<int64_t>(col) * w + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != col) aug[static_cast<int64_t>(r) * w + col] = 0.0;
    __syncthreads();
  }
}

__global__ void k_extract_vinv(const double* aug, int n, int n_pad, double* vinv, float* vinv32) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pad * n_pad) return;
  const int r = t / n_pad, c = t % n_pad;
  const double v = (r < n && c < n) ? aug[static_cast<int64_t>(r) * 2 * n + n + c] : 0.0;
  vinv[t] = v;
  vinv32[t] = static_cast<float>(v);
}

static std::vector<int32_t> primes(int d) {
  std::vector<int32_t> out;
  for (int c = 2; static_cast<int>(out.size()) < d; ++c) {
    bool ok = true;
    for (int p : out) {
      if (p * p > c) break;
      if (c % p == 0) {
        ok = false;
        break;
      }
    }
    if (ok) out.push_back(c);
  }
  return out;
}

void setup_vinv_from_nodes(Plan& P) {
  cudaStream_t s = P.stream;
  const ExpDev e = P.exp_dev();
  DBuf<double> aug;
  DBuf<int> err;
  aug.alloc(static_cast<size_t>(P.n) * 2 * P.n);
  err.alloc(1);
  DW_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_vandermonde_aug<<<ceil_div(P.n, 64), 64, 0, s>>>(P.d_nodes.p, e, aug.p);
  k_gauss_jordan<<<1, 1024, 0, s>>>(aug.p, P.n, err.p);
  P.d_vinv.alloc(static_cast<size_t>(P.n_pad) * P.n_pad);
  P.d_vinv32.alloc(static_cast<size_t>(P.n_pad) * P.n_pad);
  P.far_vt_ok = false;
  k_extract_vinv<<<ceil_div(static_cast<int64_t>(P.n_pad) * P.n_pad, 256), 256, 0, s>>>(
      aug.p, P.n, P.n_pad, P.d_vinv.p, P.d_vinv32.p);
  DW_CUDA(cudaGetLastError());
  int h_err = 0;
  DW_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  aug.release();
  err.release();
  if (h_err) fail(DWFMM_ERR_SINGULAR, "Vandermonde matrix of the nodes is singular");
  P.have_nodes = true;
}

void setup_expansion(Plan& P) {
  make_index_set(P);
  if (P.lsum > kMaxLsum) fail(DWFMM_ERR_INVALID_ARG, "degrees too large for the Legendre table");
  const int n = P.n, d = P.d;
  const int M = P.M > 0 ? P.M : std::max(2000, 10 * n);
  if (M < n) fail(DWFMM_ERR_INVALID_ARG, "fewer Halton candidates than polynomials");
  P.M = M;
  cudaStream_t s = P.stream;
  const ExpDev e = P.exp_dev();
  const std::vector<int32_t> pr = primes(d);
  DBuf<int32_t> d_pr, d_piv;
  DBuf<double> H, A, pv0, pv1;
  DBuf<int> pi0, pi1, err;
  DBuf<unsigned char> alive;
  const int nb = ceil_div(M, kQrThreads);
  d_pr.alloc(d);
  d_piv.alloc(n);
  H.alloc(static_cast<size_t>(M) * d);
  A.alloc(static_cast<size_t>(M) * n);
  pv0.alloc(nb);
  pv1.alloc(nb);
  pi0.alloc(nb);
  pi1.alloc(nb);
  err.alloc(1);
  alive.alloc(M);
  DW_CUDA(cudaMemcpyAsync(d_pr.p, pr.data(), d * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  DW_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_halton_vandermonde<<<ceil_div(M, 64), 64, 0, s>>>(M, d, d_pr.p, e, H.p, A.p);
  k_qr_init<<<nb, kQrThreads, 0, s>>>(A.p, n, M, alive.p, pv0.p, pi0.p);
  for (int st = 0; st < n; ++st) {
    const bool even = (st % 2) == 0;
    k_qr_step<<<nb, kQrThreads, n * sizeof(double), s>>>(
        A.p, n, M, st, alive.p, even ? pv0.p : pv1.p, even ? pi0.p : pi1.p, even ? pv1.p : pv0.p,
        even ? pi1.p : pi0.p, nb, d_piv.p, err.p);
  }
  P.d_nodes.alloc(static_cast<size_t>(n) * d);
  k_gather_nodes<<<ceil_div(n * d, 128), 128, 0, s>>>(H.p, d_piv.p, n, d, P.d_nodes.p);
  DW_CUDA(cudaGetLastError());
  int h_err = 0;
  P.pivots.assign(n, -1);
  DW_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaMemcpyAsync(P.pivots.data(), d_piv.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  d_pr.release();
  d_piv.release();
  H.release();
  A.release();
  pv0.release();
  pv1.release();
  pi0.release();
  pi1.release();
  err.release();
  alive.release();
  if (h_err) fail(DWFMM_ERR_SINGULAR, "Halton candidates are not unisolvent for the index set");
  setup_vinv_from_nodes(P);
}

}  // namespace dw
