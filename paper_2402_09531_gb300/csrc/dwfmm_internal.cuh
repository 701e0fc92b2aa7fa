// Internal declarations of the GB300 DW-FMM library (not part of the ABI).
//
// Data layout in HBM (all arrays owned by the plan):
//   clusters   heap order: level j holds clusters 2^j-1 .. 2^{j+1}-2,
//              children of c are 2c+1, 2c+2; the leaves are level J.
//   sites      leaf-blocked SoA: pts[leaf][k][m_pad], m_pad a multiple of 8
//              (every leaf block starts on a 32-byte boundary, so one
//              leaf is one contiguous bulk copy); slots past the leaf's
//              count hold copies of its first site and zero charges.
//   charges    xb[leaf][r][m_pad]      (right-hand sides, tree order)
//   nodes      ynode[c][k][n_pad]      (a_c(xi_alpha), Sec. 5.2)
//   moments    mom[c][r][n_pad]        (V^{-T} P_c^T x: charges at the nodes)
//   locals     loc[c][r][n_pad]        (sum_s S_{c,s} mom_s: potentials at the nodes)
//              lco[c][r][n_pad]        (V^{-1} loc + inherited: Legendre coefficients)
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dwfmm.h"

namespace dw {

constexpr int kMaxDim = 32;
constexpr int kRC = 16;  // right-hand sides per kernel pass

struct CudaError {
  cudaError_t err;
  const char* what;
};

#define DW_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t _e = (call);                                                   \
    if (_e != cudaSuccess) throw ::dw::CudaError{_e, #call};                   \
  } while (0)

struct ApiError {
  dwfmm_status status;
  std::string msg;
};

inline void fail(dwfmm_status s, const std::string& m) { throw ApiError{s, m}; }

// Device buffer with explicit lifetime (freed by the plan).
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    if (count <= n && p) return;
    release();
    if (count == 0) return;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      (void)cudaGetLastError();
      fail(DWFMM_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    n = count;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// Expansion tables shared by all clusters (device pointers).
struct ExpDev {
  int n;            // |Lambda|
  int n_pad;        // n rounded up to a multiple of 8
  int d;
  int lsum;         // sum_k (q_k + 1): Legendre values per point
  int nnz_max;      // max nonzeros of a multi-index
  const int16_t* fac;   // [n][nnz_max] offsets into a point's Legendre table, -1 = none
  const int32_t* qk;    // [d] max degree per dimension
  const int32_t* loff;  // [d] offset of dimension k in a point's Legendre table
};

// One problem of a batch, float32 (device table entry).  Arrays marked
// "slice" point into the batch's concatenated buffers.
struct ProbF32 {
  ExpDev e;
  int L, J, jmin, m_pad, R;
  const int32_t* count;   // [C] sites per cluster
  const int32_t* perm;    // tree position -> caller index
  const int32_t* begin;   // [C]
  const float* pts;       // [L][d][m_pad]
  const float* ynode;     // [C][d][n_pad]
  const float* lo;        // [C][d]
  const float* iext;      // [C][d]
  const float* vinv;      // [n_pad][n_pad]
  float* xb;              // slice [L][16][m_pad]
  float* mom;             // slice [C][16][n_pad]
  float* loc;             // slice
  float* lco;             // slice
  float* yfar;            // slice [L][16][m_pad]
  const double* x;        // caller, column-major, ldx
  double* y;
  int64_t ldx, ldy;
};

// Arguments of the float32 kernel summation (P2P and M2L), see p2p_f32.cu.
struct SumArgs {
  const float* tgt;        // target blocks [g][D+1][ld] (scaled coords, norm row)
  int64_t tgt_gstride;
  const float* src;        // source blocks [g][D+1][ld]
  int64_t src_gstride;
  const float* q;          // charges [g][ld][RC] (interleaved per source)
  int64_t q_gstride;
  float* out;              // [g][16][ld]
  int64_t out_gstride;
  const int32_t* rowptr;   // CSR over target groups (indexed by first + blockIdx.x)
  const int32_t* col;      // source group ids
  const int32_t* count;    // group sizes (count[count_off + g]); nullptr -> count_const
  int count_off;
  int count_const;
  int first;               // first target group
  int ld;                  // m_pad or n_pad (multiple of 8)
  int Rc;                  // right-hand sides actually written (<= RC)
  int* err;
};

// The persistent batch matvec (one cooperative launch, farfield.cu): the
// phases of the batch's fused matvec as work items of one kernel, separated
// by grid-wide barriers with bounded waits.
constexpr int kPersistThreads = 128;
constexpr int kPersistMaxSeg = 4;     // right-hand-side classes
constexpr int kPersistMaxLev = 32;    // tree heights / levels
constexpr int kPersistSync = 2 * kPersistMaxLev + 8;   // barrier counters, then the two queue heads

// One right-hand-side class of the near field or of the couplings: its
// summation arguments (a.first = the class's first target group), padded
// right-hand sides, and target-group count.  The class's charges are
// interleaved first from the row layout of every group, ilv_src
// [group][16][a.ld], into a.q ([group][a.ld][rc]), groups a.first ..
// a.first + count - 1.
struct PersistSeg {
  SumArgs a;
  int rc;
  int count;
  const float* ilv_src;
};

struct PersistArgs {
  const ProbF32* probs;
  const int* leaf_off;
  const int2* work;           // upward items by height, then downward items by level
  int P, Ltot, ld;
  float* xb;                  // gathered right-hand sides [Ltot][16][ld]
  const float* ynear;
  const float* yfar;
  int nup, ndown;
  int up_off[kPersistMaxLev], up_cnt[kPersistMaxLev];
  int down_off[kPersistMaxLev], down_cnt[kPersistMaxLev];
  int nnear, nm2l;
  PersistSeg near[kPersistMaxSeg], m2l[kPersistMaxSeg];
  int near_total, m2l_total;
  int gs_near, gs_m2l;                      // threads per target group (32, 64, 128)
  int near_group_bytes, m2l_group_bytes;    // shared-memory stage bytes per group
  unsigned* sync;             // [kPersistSync], zero at launch
  int* err;
  int io;                     // 1: gather the callers' x first and scatter to their y last
};


struct TreeDev {
  int64_t N;
  int J;
  int L;        // 2^J leaves
  int C;        // 2^{J+1} - 1 clusters
  int m_pad;
  const int32_t* begin;   // [C] first tree position
  const int32_t* count;   // [C] sites
};

struct TimerRec {
  int phase;
  cudaEvent_t a, b;
  int launches;
};

struct Timers {
  bool on = false;
  bool serialize = false;
  std::vector<cudaEvent_t> open;
  std::vector<TimerRec> recs;
  double ms[8] = {0};
  int64_t launches[8] = {0};
};

// Incremental CG state (device scalars; pinned status snapshot for polling).
// What a captured CG-iteration graph depends on: replayed only while all of
// it is unchanged (tree, right-hand sides, shift, iteration count,
// precision, stream and the Krylov buffers).
struct CgGraphKey {
  int tree_gen = -1, R = 0, iters = 0;
  double lam = 0.0;
  bool fp64 = false;
  cudaStream_t stream = nullptr;
  const void* bufs[6] = {};
  bool operator==(const CgGraphKey& o) const {
    if (tree_gen != o.tree_gen || R != o.R || iters != o.iters || lam != o.lam || fp64 != o.fp64 ||
        stream != o.stream)
      return false;
    for (int i = 0; i < 6; ++i)
      if (bufs[i] != o.bufs[i]) return false;
    return true;
  }
};

struct CgState {
  int R = 0;
  double lam = 0.0, rtol = 1e-6;
  bool active = false, stepped = false;
  DBuf<int> d_int;              // status[R], iters[R]
  int* h_snap = nullptr;        // pinned: status[R], iters[R] | rr[R] at byte 128*4
  cudaEvent_t ev = nullptr;
  // CUDA graph of `iters` CG iterations (cg_step): the first step with a new
  // key runs uncaptured (it sizes every buffer), the next captures, later
  // steps replay.
  CgGraphKey warm_key, graph_key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graphs_off = false;      // capture failed once: plain launches from then on
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    graph_key = CgGraphKey{};
    warm_key = CgGraphKey{};
  }
};

struct Plan {
  // configuration
  int d = 0, kernel = 0, wrule = 0, leaf = 0, M = 0, prec = 0, max_rhs = 0;
  int iset = 0;   // dwfmm_index_set
  int tree_gen = 0;   // incremented by every tree build
  double sigma = 1.0, q = 0.0, eta = 1.0;
  std::vector<double> gamma, w;
  cudaStream_t stream = nullptr;   // stream of the last call
  cudaStream_t side = nullptr;     // near field runs here, concurrently with the far field
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int device = 0;
  std::string last_error;

  // expansion (Sec. 4, 5.2, 5.4)
  int n = 0, n_pad = 0, lsum = 0, nnz_max = 0;
  std::vector<int32_t> lam;       // [n][d]
  std::vector<int32_t> qk, loff;
  std::vector<int32_t> pivots;    // [n], -1 if set by the caller
  DBuf<int16_t> d_fac;
  DBuf<int32_t> d_qk, d_loff, d_lam;
  DBuf<double> d_nodes;           // [n][d]
  DBuf<double> d_vinv;            // [n_pad][n_pad] row-major, zero padded
  DBuf<float> d_vinv32;
  bool have_nodes = false;

  // tree (Sec. 5.1)
  bool have_tree = false;
  // Gaussian kernel with every scaled squared norm |x'|^2 of the root box at
  // most 30: the tensor-core near field may evaluate it in factored form
  bool gauss_fact = false;
  double gauss_bound = 0.0;   // that bound (Gaussian kernel)
  int64_t N = 0;
  int J = -1, L = 0, C = 0, m_pad = 0, jmin = 0;
  std::vector<int32_t> h_begin, h_count;
  DBuf<int32_t> d_begin, d_count;
  DBuf<int32_t> d_perm;           // tree position -> caller index
  DBuf<double> d_lo, d_hi, d_ext;  // [C][d]
  DBuf<float> d_lo32, d_iext32;    // [C][d]
  DBuf<double> d_iext;             // [C][d]
  DBuf<double> d_pts64;           // [L][d][m_pad]
  DBuf<float> d_pts32;
  DBuf<double> d_ynode64;         // [C][d][n_pad]
  DBuf<float> d_ynode32;
  // lists (Eq. (5.1)), CSR by target
  int64_t nfar = 0, nnear = 0;
  std::vector<int64_t> far_level_count;
  DBuf<int32_t> d_far_rowptr, d_far_col;    // [C+1], [nfar]  (sources: cluster ids)
  DBuf<int32_t> d_near_rowptr, d_near_col;  // [L+1], [nnear] (sources: leaf index)
  DBuf<int32_t> d_far_pairs, d_near_pairs;  // for export: [nfar][2], [nnear][2]

  // matvec workspace, float64 and float32 variants
  DBuf<double> xb64, ynear64, yfar64, mom64, loc64, lco64;
  DBuf<float> xb32, ynear32, yfar32, mom32, loc32, lco32;
  DBuf<double> stage_in, stage_out;   // host-pointer staging
  // solve workspace
  DBuf<double> cg_r, cg_p, cg_ap, cg_c, cg_f, cg_dot, cg_tmp;

  // scratch for tree build
  DBuf<unsigned char> scratch;

  // tuned float32 kernel summation: scaled blocks [g][dpad+1][ld]
  int dpad = -1;
  DBuf<float> d_ptsk, d_ynodek;
  DBuf<float> xq32, momq32;   // charges interleaved per source, [g][ld][RC]
  DBuf<float> bq32;           // TF32 hi/lo charge blocks for the tensor-core P2P
  DBuf<float> bqm32;          // the same for the tensor-core M2L (moments at the nodes)
  DBuf<double> near_parts64;  // partial near-field sums of small float64 problems (split lists)
  // symmetric float64 near field: upper entries (T, S >= T) of the near list,
  // per-leaf rows of the upper and lower lists, slots of the lower entries,
  // forward and transposed partial sums
  DBuf<int32_t> sym_t, sym_s, sym_uprow, sym_lorow, sym_loslot;
  DBuf<double> sym_pf, sym_pt;
  int64_t sym_nup = 0;
  bool sym_ok = false;
  // symmetric tensor-core near field (MIXED): target leaves by decreasing
  // upper-row length, FP16 hi/lo charge blocks, forward sums, fixed-point
  // transposed sums, per-column largest |q'| (float bits)
  DBuf<int32_t> sym_order;
  DBuf<uint16_t> sym_bq16;
  DBuf<float> sym_fwd;
  DBuf<unsigned long long> sym_acc;
  DBuf<unsigned> sym_colmax;
  DBuf<uint16_t> sym_xa16, sym_xb16;   // FP16 hi/lo coordinate blocks (2x' and x') of the Gaussian path
  bool sym_x16_ok = false;
  int near_engine = -1;   // engine of the last near field (dwfmm_near_engine)
  // symmetric tensor-core M2L (MIXED): upper entries (t, s > t) of the far
  // list by target cluster, target clusters by decreasing upper-row length
  // (the first fsym_rows have entries), node coordinates in 128-slot
  // blocks, FP16 charge blocks, forward and fixed-point transposed sums
  DBuf<int32_t> fsym_uprow, fsym_s, fsym_order;
  int fsym_rows = 0;
  bool fsym_ok = false;
  DBuf<float> m2l_crd;
  int m2l_crd_D = -1;
  DBuf<uint16_t> m2l_xa16, m2l_xb16;   // FP16 hi/lo node coordinates (2y', y') of the Gaussian path
  int m2l_x16_D = -1;
  DBuf<uint16_t> m2l_bq16;
  DBuf<float> m2l_fwd;
  DBuf<unsigned long long> m2l_acc;
  DBuf<unsigned> m2l_colmax;
  int m2l_engine = -1;    // engine of the last M2L (dwfmm_m2l_engine)
  int m2l_pref = -1;      // engine chosen by the caller (dwfmm_plan_set_m2l_engine), -1 = timed
  int m2l_tuned = -1;     // engine the timing chose for this tree (-1 = not yet timed)
  double m2l_tune_ms[2] = {-1.0, -1.0};   // symmetric, ordered
  // tensor-core far field (MIXED): FP16 hi/lo tiles of V^{-T} and V^{-1}
  // scaled by 2^-far_vexp, valid for the current node set
  DBuf<uint16_t> far_vt;
  DBuf<int> far_vexp;
  bool far_vt_ok = false;
  int far_engine = -1;    // engine of the last far field (dwfmm_far_engine)
  cudaEvent_t ev_scaled = nullptr;
  DBuf<int> d_err;   // device error flag (3 = a bounded wait timed out)

  Timers tm;
  CgState cgs;

  ExpDev exp_dev() const {
    return ExpDev{n, n_pad, d, lsum, nnz_max, d_fac.p, d_qk.p, d_loff.p};
  }
  TreeDev tree_dev() const { return TreeDev{N, J, L, C, m_pad, d_begin.p, d_count.p}; }
  void free_tree();
  void free_all();
};

// ---- setup (setup.cu) ----
void setup_expansion(Plan& P);              // weights, Lambda, tables (host) + nodes/V^{-1} (GPU)
void setup_vinv_from_nodes(Plan& P);         // V and V^{-1} on the GPU from d_nodes

// ---- tree and lists (tree.cu) ----
void build_tree(Plan& P, const double* pts_dev, int64_t n, int64_t ld);
void build_lists(Plan& P);
void build_cluster_data(Plan& P);           // extents, nodes, leaf-blocked sites

// ---- matvec (farfield.cu, nearfield.cu, matvec.cu) ----
// x, y: device, caller order, column-major.
void matvec_device(Plan& P, const double* x, int64_t ldx, double* y, int64_t ldy, int R, bool fp64);
void ensure_workspace(Plan& P, bool fp64);
void farfield_set_smem_limits(Plan& P);
size_t farfield_smem_need(const Plan& P, bool fp64);
void launch_gather(Plan& P, const double* x, int64_t ldx, int r0, int Rc, bool fp64);
void launch_scatter(Plan& P, double* y, int64_t ldy, int r0, int Rc, bool fp64);
void launch_farfield(Plan& P, int Rc, bool fp64);
bool farfield_tc_eligible(const Plan& P);   // farfield_tc.cu
void farfield_tc(Plan& P, int Rc);
void launch_m2l(Plan& P, int Rc, bool fp64);
void launch_nearfield(Plan& P, int Rc, bool fp64, cudaStream_t s);
// Bit of the current device in a per-device mask (kernel attributes are set
// per device); devices beyond 63 get no bit, so their setup simply repeats.
uint64_t device_bit();
void build_sym_lists(Plan& P);              // upper / lower near lists (symmetric float64 P2P)
void sym_tc_order(Plan& P, const std::vector<int>& upper_counts);
bool m2l_sym_tc(Plan& P, int D, int Rc, cudaStream_t s);   // p2p_sym.cu
void m2l_autotune(Plan& P, int Rc);                         // p2p_f32.cu
void build_far_sym_lists(Plan& P);                          // nearfield.cu
bool near_sym_tc(Plan& P, int D, int Rc, cudaStream_t s);   // symmetric tensor-core P2P (MIXED, 9..16 RHS)
int sm_count();
bool p2p_f32_tuned(Plan& P, int Rc, cudaStream_t s);
bool m2l_f32_tuned(Plan& P, int Rc);
void check_device_error(Plan& P);
// batches (batch.cu uses these)
void batch_far_attrs();
size_t batch_far_smem(int lsum, int n_pad);
void launch_moments_batched(const ProbF32* probs, const int2* work, int items, size_t smem, cudaStream_t s);
void launch_downward_batched(const ProbF32* probs, const int2* work, int items, size_t smem, cudaStream_t s);
void launch_gather_batched(const ProbF32* probs, const int* leaf_off, int P, int Ltot, int ld, float* xb,
                           cudaStream_t s);
void launch_scatter_batched(const ProbF32* probs, const int* leaf_off, int P, int Ltot, int ld, const float* ynear,
                            const float* yfar, cudaStream_t s);
// persistent batch matvec: dynamic shared memory and resident CTAs per SM
// for a launch, and the cooperative launch itself (false if the launch was
// refused, e.g. by a stream capture that cannot hold it)
size_t persist_group_bytes(int D, int RC, int ld, int threads);
int persist_blocks_per_sm(int D, int kernel, size_t smem);
cudaError_t launch_batch_persistent(int D, int kernel, const PersistArgs& pa, int grid, size_t smem, cudaStream_t s);
int sum_padded_dim(int d);
int sum_padded_rc(int r);
size_t sum_stage_bytes(int D, int RC, int ld);
void launch_sum_f32(int D, int kernel, int RC, const SumArgs& a, int groups, int threads, size_t smem,
                    cudaStream_t s);
void launch_interleave(const float* src, int64_t groups, int ld, int RC, float* dst, cudaStream_t s);
void launch_scaled_blocks(const double* src, int64_t groups, int d, int D, int ld, int kernel, double sigma,
                          float* dst, cudaStream_t s);
void ensure_sum_attrs();
bool sum_tc(int D, int kernel, const float* tgt, int64_t tgt_gstride, const float* src, int64_t src_gstride,
            const float* xq16, int64_t groups_src, DBuf<float>& bq_scratch, float* out, int64_t out_gstride,
            const int32_t* rowptr, const int32_t* col, const int32_t* count, int count_off, int count_const,
            int first, int ngroups, int ld, int Rc, bool gauss_factored, int* err, cudaStream_t s);
void evaluate(Plan& P, const double* tgt, int64_t nt, int64_t ldt, const double* c, int64_t ldc, double* out,
              int64_t ldo, int R);
void eval_f64(Plan& P, const double* tgt64, int G, const int32_t* rowptr, const int32_t* col, int Rc, double* out,
              cudaStream_t s);
void eval_f32(Plan& P, const double* tgt64, int G, const int32_t* rowptr, const int32_t* col, int Rc, float* out,
              DBuf<float>& scratch, cudaStream_t s);
struct Batch;
Batch* batch_new();
void batch_delete(Batch* b);
void batch_create(Batch& B, Plan* const* plans, const int32_t* nrhs, int count);
void batch_matvec(Batch& B, const double* const* x, double* const* y, cudaStream_t s);
void batch_info(const Batch& B, int32_t* split, double* tune_ms, int64_t* leaves);
void batch_shape(const Batch& B, int32_t* shape);
void batch_engine(const Batch& B, int32_t* engine, double* ms, int32_t* launch);
void batch_set_engine(Batch& B, int persistent);
dwfmm_status direct_sum_noalloc(int kernel, double sigma, const double* pts, int64_t n, int d, int64_t ldp,
                                const double* x, double* y, int R, int64_t ldx, int64_t ldy,
                                cudaStream_t s);

// ---- solve (solve.cu) ----
// device state of one plan's incremental CG (layout of cg_begin)
struct CgPtrs {
  double *p, *ap, *c, *r;
  double *rr, *pap, *coef, *bn2, *tmp;
  const double* rtol2;
  int *status, *iters;
  int64_t n;
  int R;
  double lam;
};
CgPtrs cg_ptrs(Plan& P);
void cg_snapshot(Plan& P, cudaStream_t s);
void batch_cg_step(Batch& B, int iters, cudaStream_t s);
dwfmm_status solve(Plan& P, double lambda, const double* f, double* c, int R, int64_t ld,
                   double rtol, int maxit, int* iters, double* relres);
void cg_begin(Plan& P, double lam, const double* f, int R, int64_t ld, double rtol);
void cg_step(Plan& P, int iters);
bool cg_poll(Plan& P, int* status, int* iters, double* rr);
void cg_result(Plan& P, double* c, int64_t ld);
void residual64(Plan& P, double lam, const double* f, const double* c, double* r, int R, double* relres);
void refine_step(Plan& P, double lam, double* c, const double* delta, double* r, int R, double* w,
                 double* part, double* dev3);
void refine64(Plan& P, double lam, const double* f, double* c, const double* delta, double* r, int R,
              double* alpha, double* relres);

inline int ceil_div(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }
inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// timers (matvec.cu): CUDA events on the launching stream, per phase
void timer_begin(Plan& P, int phase, cudaStream_t s);
void timer_end(Plan& P, int phase, cudaStream_t s, int launches);
void timers_collect(Plan& P);

}  // namespace dw

struct dwfmm_plan_s {
  dw::Plan P;
};
