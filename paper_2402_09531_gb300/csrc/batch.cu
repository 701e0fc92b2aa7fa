// Many uneven DW-FMM problems in one fused matvec (float32).
//
// A batch concatenates the problems' scaled source blocks, charges, outputs
// and far/near lists into single arrays with global CSR lists, so that the
// near field (P2P) of every problem is one launch of the kernel-summation
// engine and the couplings (M2L) of every problem another; the upward and
// downward passes are one launch per tree height / level over a work list of
// (problem, cluster) items that reads each problem's arrays from a device
// table.  The whole sequence is captured once into a CUDA graph and replayed.
//
// Autotuning: the problems are ordered by their padded right-hand-side class
// (1, 4, 8, 16); at creation the P2P+M2L work is timed both as one launch
// padded to the largest class and as one launch per class, and the faster
// shape is captured.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "dwfmm_internal.cuh"

namespace dw {

struct Batch {
  std::vector<Plan*> plans;   // internal order
  std::vector<int> order;     // internal index -> caller index
  std::vector<int> R;
  int P = 0, D = 0, ld = 0, n = 0, n_pad = 0, kernel = 0, RCmax = 1;
  std::vector<int> leaf_off, clus_off;
  int Ltot = 0, Ctot = 0;
  DBuf<float> ptsk, ynodek, xb, xq, ynear, yfar, mom, momq, loc, lco;
  DBuf<int32_t> near_rowptr, near_col, far_rowptr, far_col, counts;
  DBuf<int> d_leaf_off, err;
  DBuf<ProbF32> probs;
  ProbF32* h_probs = nullptr;   // pinned
  DBuf<int2> work;
  std::vector<int> up_off, up_cnt, down_off, down_cnt;
  size_t far_smem = 0;
  struct Cls {
    int RC, leaf_first, leaf_count, clus_first, clus_count;
  };
  std::vector<Cls> classes;
  bool split = false;            // near field: one launch per right-hand-side class
  double tune_ms[2] = {0, 0};    // best padded / best per-class time of near field + couplings
  // tile shapes chosen by the autotuner: CTA width (targets per pass = 2 x
  // threads) and right-hand-side grouping, separately for the fused near
  // field and the fused couplings
  int thr_near = 0, thr_m2l = 0;
  bool split_m2l = false;
  cudaStream_t stream = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_copy = nullptr;
  bool copied = false;
  DBuf<char> cg_tab;     // batched CG: problem, segment and block tables
  DBuf<double> cg_part;  // batched CG: partial inner products
  std::vector<char> cg_host;     // content of cg_tab (uploaded only when it changes)
  char* cg_pinned = nullptr;     // pinned staging of the upload
  size_t cg_pinned_n = 0;
  cudaEvent_t cg_ev = nullptr;   // the last upload is done
  bool cg_copied = false;
  cudaGraph_t cg_graph = nullptr;        // `cg_iters` batched CG iterations
  cudaGraphExec_t cg_exec = nullptr;
  int cg_iters = -1, cg_nseg = -1, cg_nblk = -1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // persistent engine: the whole matvec as one cooperative launch
  bool persist_tried = false;    // the persistent engine was tuned
  bool persist_ok = false;       // eligible (launch and capture worked, no wait gave up)
  bool persistent = false;       // the engine in use
  PersistArgs pa{};
  int pgrid = 0;
  size_t psmem = 0;
  DBuf<unsigned> psync;
  double engine_ms[2] = {-1.0, -1.0};   // best timed matvec: launches in a graph, persistent
  cudaGraph_t pgraph = nullptr;
  cudaGraphExec_t pexec = nullptr;

  void release() {
    if (cg_exec) cudaGraphExecDestroy(cg_exec);
    if (cg_graph) cudaGraphDestroy(cg_graph);
    if (cg_pinned) cudaFreeHost(cg_pinned);
    if (cg_ev) cudaEventDestroy(cg_ev);
    cg_exec = nullptr;
    cg_graph = nullptr;
    cg_pinned = nullptr;
    cg_pinned_n = 0;
    cg_ev = nullptr;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (pexec) cudaGraphExecDestroy(pexec);
    if (pgraph) cudaGraphDestroy(pgraph);
    pexec = nullptr;
    pgraph = nullptr;
    if (h_probs) cudaFreeHost(h_probs);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_copy) cudaEventDestroy(ev_copy);
    if (stream) cudaStreamDestroy(stream);
    if (side) cudaStreamDestroy(side);
    exec = nullptr;
    graph = nullptr;
    h_probs = nullptr;
    ev_fork = ev_join = ev_copy = nullptr;
    stream = side = nullptr;
  }
};

namespace {

SumArgs p2p_args(Batch& B, int RC, int leaf_first) {
  SumArgs a{};
  a.tgt = B.ptsk.p;
  a.tgt_gstride = static_cast<int64_t>(B.D + 1) * B.ld;
  a.src = B.ptsk.p;
  a.src_gstride = a.tgt_gstride;
  a.q = B.xq.p;   // class regions are disjoint: [leaf_first*ld*RC, (leaf_first+count)*ld*RC)
  a.q_gstride = static_cast<int64_t>(RC) * B.ld;
  a.out = B.ynear.p;
  a.out_gstride = static_cast<int64_t>(kRC) * B.ld;
  a.rowptr = B.near_rowptr.p;
  a.col = B.near_col.p;
  a.count = B.counts.p;
  a.count_off = 0;
  a.count_const = 0;
  a.first = leaf_first;
  a.ld = B.ld;
  a.Rc = RC;
  a.err = B.err.p;
  return a;
}

SumArgs m2l_args(Batch& B, int RC, int clus_first) {
  SumArgs a{};
  a.tgt = B.ynodek.p;
  a.tgt_gstride = static_cast<int64_t>(B.D + 1) * B.n_pad;
  a.src = B.ynodek.p;
  a.src_gstride = a.tgt_gstride;
  a.q = B.momq.p;
  a.q_gstride = static_cast<int64_t>(RC) * B.n_pad;
  a.out = B.loc.p;
  a.out_gstride = static_cast<int64_t>(kRC) * B.n_pad;
  a.rowptr = B.far_rowptr.p;
  a.col = B.far_col.p;
  a.count = nullptr;
  a.count_off = 0;
  a.count_const = B.n;
  a.first = clus_first;
  a.ld = B.n_pad;
  a.Rc = RC;
  a.err = B.err.p;
  return a;
}

int threads_for(int ld) { return std::min(128, round_up((ld + 1) / 2, 32)); }

// The fused near-field work: interleave charges, P2P launch(es) with
// `threads` per CTA.
void enqueue_near(Batch& B, bool split, int threads, cudaStream_t s) {
  if (!split) {
    launch_interleave(B.xb.p, B.Ltot, B.ld, B.RCmax, B.xq.p, s);
    launch_sum_f32(B.D, B.kernel, B.RCmax, p2p_args(B, B.RCmax, 0), B.Ltot, threads,
                   sum_stage_bytes(B.D, B.RCmax, B.ld), s);
    return;
  }
  for (const auto& c : B.classes) {
    launch_interleave(B.xb.p + static_cast<int64_t>(c.leaf_first) * kRC * B.ld, c.leaf_count, B.ld, c.RC,
                      B.xq.p + static_cast<int64_t>(c.leaf_first) * B.ld * c.RC, s);
    launch_sum_f32(B.D, B.kernel, c.RC, p2p_args(B, c.RC, c.leaf_first), c.leaf_count, threads,
                   sum_stage_bytes(B.D, c.RC, B.ld), s);
  }
}

// The fused couplings (M2L) with `threads` per CTA.
void enqueue_m2l(Batch& B, bool split, int threads, cudaStream_t s) {
  if (!split) {
    launch_interleave(B.mom.p, B.Ctot, B.n_pad, B.RCmax, B.momq.p, s);
    launch_sum_f32(B.D, B.kernel, B.RCmax, m2l_args(B, B.RCmax, 0), B.Ctot, threads,
                   sum_stage_bytes(B.D, B.RCmax, B.n_pad), s);
    return;
  }
  for (const auto& c : B.classes) {
    launch_interleave(B.mom.p + static_cast<int64_t>(c.clus_first) * kRC * B.n_pad, c.clus_count, B.n_pad, c.RC,
                      B.momq.p + static_cast<int64_t>(c.clus_first) * B.n_pad * c.RC, s);
    launch_sum_f32(B.D, B.kernel, c.RC, m2l_args(B, c.RC, c.clus_first), c.clus_count, threads,
                   sum_stage_bytes(B.D, c.RC, B.n_pad), s);
  }
}

// io = false leaves out the gather of the callers' x and the scatter to their
// y (for timing at creation, before any caller buffer is known).
cudaError_t enqueue_persistent(Batch& B, cudaStream_t s, bool io) {
  const cudaError_t e = cudaMemsetAsync(B.psync.p, 0, sizeof(unsigned) * kPersistSync, s);
  if (e != cudaSuccess) return e;
  PersistArgs a = B.pa;
  a.io = io ? 1 : 0;
  return launch_batch_persistent(B.D, B.kernel, a, B.pgrid, B.psmem, s);
}

void enqueue_matvec(Batch& B, bool io = true) {
  if (B.persistent) {
    DW_CUDA(enqueue_persistent(B, B.stream, io));
    return;
  }
  cudaStream_t s = B.stream;
  if (io) launch_gather_batched(B.probs.p, B.d_leaf_off.p, B.P, B.Ltot, B.ld, B.xb.p, s);
  DW_CUDA(cudaEventRecord(B.ev_fork, s));
  DW_CUDA(cudaStreamWaitEvent(B.side, B.ev_fork, 0));
  enqueue_near(B, B.split, B.thr_near, B.side);
  DW_CUDA(cudaEventRecord(B.ev_join, B.side));
  for (size_t h = 0; h < B.up_off.size(); ++h)
    launch_moments_batched(B.probs.p, B.work.p + B.up_off[h], B.up_cnt[h], B.far_smem, s);
  enqueue_m2l(B, B.split_m2l, B.thr_m2l, s);
  for (size_t j = 0; j < B.down_off.size(); ++j)
    launch_downward_batched(B.probs.p, B.work.p + B.down_off[j], B.down_cnt[j], B.far_smem, s);
  DW_CUDA(cudaStreamWaitEvent(s, B.ev_join, 0));
  if (io) launch_scatter_batched(B.probs.p, B.d_leaf_off.p, B.P, B.Ltot, B.ld, B.ynear.p, B.yfar.p, s);
  DW_CUDA(cudaGetLastError());
}

// Best of two timed runs of one launch shape of the near field (which = 0)
// or the couplings (which = 1).
double time_shape(Batch& B, int which, bool split, int threads) {
  cudaEvent_t a, b;
  DW_CUDA(cudaEventCreate(&a));
  DW_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  for (int rep = 0; rep < 2; ++rep) {
    DW_CUDA(cudaEventRecord(a, B.stream));
    if (which == 0) enqueue_near(B, split, threads, B.stream);
    else enqueue_m2l(B, split, threads, B.stream);
    DW_CUDA(cudaEventRecord(b, B.stream));
    DW_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    DW_CUDA(cudaEventElapsedTime(&ms, a, b));
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

// Autotuner: every candidate shape (CTA width 32, 64, 128 threads up to the
// widest useful one for the group's slots, and that one; one padded launch
// or one per right-hand-side class) of the near field and of the couplings
// is timed on the batch's own data, and the fastest of each is kept.  Each
// thread sums its targets' sources in the same order whatever the width,
// so the choice changes no result.
void tune_shapes(Batch& B) {
  const bool can_split = B.classes.size() > 1;
  double best_pad = 0.0, best_split = 0.0;
  for (int which = 0; which < 2; ++which) {
    const int widest = threads_for(which == 0 ? B.ld : B.n_pad);
    double best = 1e30, bp = 1e30, bs = 1e30;
    bool bsplit = false;
    int bthr = widest;
    for (int thr = 32; thr <= widest; thr = (thr * 2 > widest && thr < widest) ? widest : thr * 2) {
      for (int sp = 0; sp < (can_split ? 2 : 1); ++sp) {
        const double ms = time_shape(B, which, sp != 0, thr);
        if (sp) bs = std::min(bs, ms);
        else bp = std::min(bp, ms);
        if (ms < best) {
          best = ms;
          bsplit = sp != 0;
          bthr = thr;
        }
      }
    }
    if (which == 0) {
      B.split = bsplit;
      B.thr_near = bthr;
    } else {
      B.split_m2l = bsplit;
      B.thr_m2l = bthr;
    }
    best_pad += bp;
    best_split += can_split ? bs : bp;
  }
  B.tune_ms[0] = best_pad;
  B.tune_ms[1] = best_split;
}

// --- persistent engine -------------------------------------------------------

// Fused near-field + coupling time (ms, from the launch tuner) from which the
// persistent engine is tuned at creation.
constexpr double kPersistTuneMinMs = 2.0;

int pow2_width(int t) { return t <= 32 ? 32 : t <= 64 ? 64 : 128; }

// Arguments of the persistent kernel with near-field groups of gs_near threads
// and coupling groups of gs_m2l; its shared memory and grid (every CTA
// resident).  False if the batch does not fit the kernel's tables or an SM.
bool build_persist_args(Batch& B, int gs_near, int gs_m2l) {
  if (B.up_off.size() > static_cast<size_t>(kPersistMaxLev) ||
      B.down_off.size() > static_cast<size_t>(kPersistMaxLev) ||
      B.classes.size() > static_cast<size_t>(kPersistMaxSeg))
    return false;
  PersistArgs& a = B.pa;
  a = PersistArgs{};
  a.probs = B.probs.p;
  a.leaf_off = B.d_leaf_off.p;
  a.work = B.work.p;
  a.P = B.P;
  a.Ltot = B.Ltot;
  a.ld = B.ld;
  a.xb = B.xb.p;
  a.ynear = B.ynear.p;
  a.yfar = B.yfar.p;
  a.nup = static_cast<int>(B.up_off.size());
  a.ndown = static_cast<int>(B.down_off.size());
  for (int h = 0; h < a.nup; ++h) {
    a.up_off[h] = B.up_off[h];
    a.up_cnt[h] = B.up_cnt[h];
  }
  for (int j = 0; j < a.ndown; ++j) {
    a.down_off[j] = B.down_off[j];
    a.down_cnt[j] = B.down_cnt[j];
  }
  int rcn = 1, rcm = 1;
  // the largest right-hand-side class first: the longest items leave the queue first
  for (auto it = B.classes.rbegin(); it != B.classes.rend(); ++it) {
    const Batch::Cls& c = *it;
    if (c.leaf_count > 0) {
      PersistSeg& sg = a.near[a.nnear++];
      sg.a = p2p_args(B, c.RC, c.leaf_first);
      sg.rc = c.RC;
      sg.count = c.leaf_count;
      sg.ilv_src = B.xb.p;
      a.near_total += c.leaf_count;
      rcn = std::max(rcn, c.RC);
    }
    if (c.clus_count > 0) {
      PersistSeg& sg = a.m2l[a.nm2l++];
      sg.a = m2l_args(B, c.RC, c.clus_first);
      sg.rc = c.RC;
      sg.count = c.clus_count;
      sg.ilv_src = B.mom.p;
      a.m2l_total += c.clus_count;
      rcm = std::max(rcm, c.RC);
    }
  }
  a.gs_near = gs_near;
  a.gs_m2l = gs_m2l;
  const size_t gn = persist_group_bytes(B.D, rcn, B.ld, gs_near), gm = persist_group_bytes(B.D, rcm, B.n_pad, gs_m2l);
  a.near_group_bytes = static_cast<int>(gn);
  a.m2l_group_bytes = static_cast<int>(gm);
  a.sync = B.psync.p;
  a.err = B.err.p;
  B.psmem = std::max({B.far_smem, static_cast<size_t>(kPersistThreads / gs_near) * gn,
                      static_cast<size_t>(kPersistThreads / gs_m2l) * gm});
  if (B.psmem > 227 * 1024) return false;
  const int per_sm = persist_blocks_per_sm(B.D, B.kernel, B.psmem);
  if (per_sm < 1) return false;
  B.pgrid = per_sm * sm_count();
  return true;
}

// One matvec of either engine captured on the batch's stream (graph and
// executable); false if the capture or the instantiation is refused.
bool capture_engine(Batch& B, bool persistent, bool io, cudaGraph_t* graph, cudaGraphExec_t* exec) {
  *graph = nullptr;
  *exec = nullptr;
  if (cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  const bool keep = B.persistent;
  B.persistent = persistent;
  cudaError_t le = cudaSuccess;
  if (persistent) le = enqueue_persistent(B, B.stream, io);
  else enqueue_matvec(B, io);
  B.persistent = keep;
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(B.stream, &g);
  if (le != cudaSuccess || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    return false;
  }
  cudaGraphExec_t e = nullptr;
  if (cudaGraphInstantiate(&e, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    (void)cudaGetLastError();
    return false;
  }
  *graph = g;
  *exec = e;
  return true;
}

void drop_graph(cudaGraph_t* g, cudaGraphExec_t* e) {
  if (*e) cudaGraphExecDestroy(*e);
  if (*g) cudaGraphDestroy(*g);
  *e = nullptr;
  *g = nullptr;
}

// Best of two timed replays of a captured matvec (after one untimed); -1 if
// a launch or the timing failed (the events are released either way).
double time_exec(Batch& B, cudaGraphExec_t e) {
  cudaEvent_t a = nullptr, b = nullptr;
  float best = 1e30f;
  bool ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess &&
            cudaGraphLaunch(e, B.stream) == cudaSuccess;
  for (int rep = 0; ok && rep < 2; ++rep) {
    float ms = 0.f;
    ok = cudaEventRecord(a, B.stream) == cudaSuccess && cudaGraphLaunch(e, B.stream) == cudaSuccess &&
         cudaEventRecord(b, B.stream) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
         cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    if (ok) best = std::min(best, ms);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return ok ? best : -1.0;
}

// Reads and clears the batch's error flag (a bounded device wait gave up).
bool take_device_error(Batch& B) {
  int e = 0;
  DW_CUDA(cudaMemcpy(&e, B.err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) DW_CUDA(cudaMemset(B.err.p, 0, sizeof(int)));
  return e != 0;
}

// Times the persistent engine at each near-field group width (32, 64, 128
// threads up to the widest the leaves use; the couplings keep the width the
// launch tuner chose) against the captured launches, and keeps the faster.
// Both are timed without the gather and the scatter (no caller buffers
// exist yet; those two phases are the same elementwise work in both).
void tune_persistent(Batch& B) {
  B.persist_tried = true;
  B.persist_ok = false;
  B.persistent = false;
  int dev = 0, coop = 0;
  DW_CUDA(cudaGetDevice(&dev));
  DW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  if (!capture_engine(B, false, false, &g, &e)) fail(DWFMM_ERR_CUDA, "capture of the batch matvec failed");
  B.engine_ms[0] = time_exec(B, e);
  drop_graph(&g, &e);
  if (B.engine_ms[0] < 0.0) fail(DWFMM_ERR_CUDA, "the batch matvec failed while it was timed");
  if (!coop) return;
  B.psync.alloc(kPersistSync);
  const int gs_m2l = pow2_width(B.thr_m2l);
  const int widest = pow2_width(threads_for(B.ld));
  double best = 1e30;
  int best_gs = 0;
  for (int gs = 32; gs <= widest; gs *= 2) {
    if (!build_persist_args(B, gs, gs_m2l)) continue;
    if (!capture_engine(B, true, false, &g, &e)) return;
    const double ms = time_exec(B, e);
    drop_graph(&g, &e);
    // a launch the device refuses leaves the engine unavailable (a fault is
    // sticky and ends the creation at the next checked call)
    if (ms < 0.0) {
      (void)cudaGetLastError();
      return;
    }
    if (take_device_error(B)) return;
    if (ms < best) {
      best = ms;
      best_gs = gs;
    }
  }
  if (!best_gs || !build_persist_args(B, best_gs, gs_m2l)) return;
  if (!capture_engine(B, true, true, &B.pgraph, &B.pexec)) return;
  B.persist_ok = true;
  B.engine_ms[1] = best;
  B.persistent = best < B.engine_ms[0];
}

}  // namespace

void batch_create(Batch& B, Plan* const* plans, const int32_t* nrhs, int count) {
  if (count < 1) fail(DWFMM_ERR_INVALID_ARG, "empty batch");
  Plan& P0 = *plans[0];
  for (int i = 0; i < count; ++i) {
    Plan& p = *plans[i];
    if (!p.have_tree || p.N == 0) fail(DWFMM_ERR_STATE, "every plan needs a non-empty tree");
    if (p.prec == DWFMM_P_FP64) fail(DWFMM_ERR_INVALID_ARG, "batches run float32 plans");
    if (p.kernel != P0.kernel || p.n != P0.n || p.m_pad != P0.m_pad)
      fail(DWFMM_ERR_INVALID_ARG, "plans differ in kernel, |Lambda| or leaf block size");
    if (sum_padded_dim(p.d) < 0) fail(DWFMM_ERR_INVALID_ARG, "batches need d <= 16");
    if (nrhs[i] < 1 || nrhs[i] > kRC || nrhs[i] > p.max_rhs) fail(DWFMM_ERR_INVALID_ARG, "nrhs outside 1..16");
  }
  B.P = count;
  B.order.resize(count);
  std::iota(B.order.begin(), B.order.end(), 0);
  std::stable_sort(B.order.begin(), B.order.end(),
                   [&](int a, int b) { return sum_padded_rc(nrhs[a]) < sum_padded_rc(nrhs[b]); });
  for (int i : B.order) {
    B.plans.push_back(plans[i]);
    B.R.push_back(nrhs[i]);
  }
  B.kernel = P0.kernel;
  B.n = P0.n;
  B.n_pad = P0.n_pad;
  B.ld = P0.m_pad;
  B.D = 0;
  int lsum_max = 0, Rmax = 1;
  for (int i = 0; i < count; ++i) {
    B.D = std::max(B.D, sum_padded_dim(B.plans[i]->d));
    lsum_max = std::max(lsum_max, B.plans[i]->lsum);
    Rmax = std::max(Rmax, B.R[i]);
  }
  B.RCmax = sum_padded_rc(Rmax);
  B.leaf_off.assign(count + 1, 0);
  B.clus_off.assign(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    B.leaf_off[i + 1] = B.leaf_off[i] + B.plans[i]->L;
    B.clus_off[i + 1] = B.clus_off[i] + B.plans[i]->C;
  }
  B.Ltot = B.leaf_off[count];
  B.Ctot = B.clus_off[count];
  DW_CUDA(cudaStreamCreateWithFlags(&B.stream, cudaStreamNonBlocking));
  DW_CUDA(cudaStreamCreateWithFlags(&B.side, cudaStreamNonBlocking));
  DW_CUDA(cudaEventCreateWithFlags(&B.ev_fork, cudaEventDisableTiming));
  DW_CUDA(cudaEventCreateWithFlags(&B.ev_join, cudaEventDisableTiming));
  DW_CUDA(cudaEventCreateWithFlags(&B.ev_copy, cudaEventDisableTiming));
  cudaStream_t s = B.stream;
  const size_t nl = static_cast<size_t>(B.Ltot) * kRC * B.ld;
  const size_t nc = static_cast<size_t>(B.Ctot) * kRC * B.n_pad;
  B.ptsk.alloc(static_cast<size_t>(B.Ltot) * (B.D + 1) * B.ld);
  B.ynodek.alloc(static_cast<size_t>(B.Ctot) * (B.D + 1) * B.n_pad);
  B.xb.alloc(nl);
  B.ynear.alloc(nl);
  B.yfar.alloc(nl);
  B.xq.alloc(static_cast<size_t>(B.Ltot) * B.ld * B.RCmax);
  B.mom.alloc(nc);
  B.loc.alloc(nc);
  B.lco.alloc(nc);
  B.momq.alloc(static_cast<size_t>(B.Ctot) * B.n_pad * B.RCmax);
  B.err.alloc(1);
  DW_CUDA(cudaMemsetAsync(B.err.p, 0, sizeof(int), s));
  DW_CUDA(cudaMemsetAsync(B.xb.p, 0, nl * sizeof(float), s));
  DW_CUDA(cudaMemsetAsync(B.mom.p, 0, nc * sizeof(float), s));
  // scaled blocks at the common padded dimension; global CSR lists
  std::vector<int32_t> nr(B.Ltot + 1, 0), fr(B.Ctot + 1, 0), ncol, fcol, cnt(B.Ltot);
  for (int i = 0; i < count; ++i) {
    Plan& p = *B.plans[i];
    launch_scaled_blocks(p.d_pts64.p, p.L, p.d, B.D, B.ld, B.kernel, p.sigma,
                         B.ptsk.p + static_cast<size_t>(B.leaf_off[i]) * (B.D + 1) * B.ld, s);
    launch_scaled_blocks(p.d_ynode64.p, p.C, p.d, B.D, B.n_pad, B.kernel, p.sigma,
                         B.ynodek.p + static_cast<size_t>(B.clus_off[i]) * (B.D + 1) * B.n_pad, s);
    std::vector<int32_t> rp(p.L + 1), cl(std::max<int64_t>(p.nnear, 1)), frp(p.C + 1), fcl(std::max<int64_t>(p.nfar, 1));
    DW_CUDA(cudaMemcpy(rp.data(), p.d_near_rowptr.p, sizeof(int32_t) * (p.L + 1), cudaMemcpyDeviceToHost));
    if (p.nnear) DW_CUDA(cudaMemcpy(cl.data(), p.d_near_col.p, sizeof(int32_t) * p.nnear, cudaMemcpyDeviceToHost));
    DW_CUDA(cudaMemcpy(frp.data(), p.d_far_rowptr.p, sizeof(int32_t) * (p.C + 1), cudaMemcpyDeviceToHost));
    if (p.nfar) DW_CUDA(cudaMemcpy(fcl.data(), p.d_far_col.p, sizeof(int32_t) * p.nfar, cudaMemcpyDeviceToHost));
    for (int l = 0; l < p.L; ++l) {
      nr[B.leaf_off[i] + l + 1] = rp[l + 1] - rp[l];
      cnt[B.leaf_off[i] + l] = p.h_count[p.L - 1 + l];
    }
    for (int64_t e = 0; e < p.nnear; ++e) ncol.push_back(cl[e] + B.leaf_off[i]);
    for (int c = 0; c < p.C; ++c) fr[B.clus_off[i] + c + 1] = frp[c + 1] - frp[c];
    for (int64_t e = 0; e < p.nfar; ++e) fcol.push_back(fcl[e] + B.clus_off[i]);
  }
  for (int l = 0; l < B.Ltot; ++l) nr[l + 1] += nr[l];
  for (int c = 0; c < B.Ctot; ++c) fr[c + 1] += fr[c];
  B.near_rowptr.alloc(nr.size());
  B.near_col.alloc(std::max<size_t>(ncol.size(), 1));
  B.far_rowptr.alloc(fr.size());
  B.far_col.alloc(std::max<size_t>(fcol.size(), 1));
  B.counts.alloc(cnt.size());
  DW_CUDA(cudaMemcpy(B.near_rowptr.p, nr.data(), sizeof(int32_t) * nr.size(), cudaMemcpyHostToDevice));
  if (!ncol.empty()) DW_CUDA(cudaMemcpy(B.near_col.p, ncol.data(), sizeof(int32_t) * ncol.size(), cudaMemcpyHostToDevice));
  DW_CUDA(cudaMemcpy(B.far_rowptr.p, fr.data(), sizeof(int32_t) * fr.size(), cudaMemcpyHostToDevice));
  if (!fcol.empty()) DW_CUDA(cudaMemcpy(B.far_col.p, fcol.data(), sizeof(int32_t) * fcol.size(), cudaMemcpyHostToDevice));
  DW_CUDA(cudaMemcpy(B.counts.p, cnt.data(), sizeof(int32_t) * cnt.size(), cudaMemcpyHostToDevice));
  B.d_leaf_off.alloc(count + 1);
  DW_CUDA(cudaMemcpy(B.d_leaf_off.p, B.leaf_off.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice));
  // problem table (pinned host copy: x/y pointers change per call)
  DW_CUDA(cudaMallocHost(reinterpret_cast<void**>(&B.h_probs), sizeof(ProbF32) * count));
  for (int i = 0; i < count; ++i) {
    Plan& p = *B.plans[i];
    ProbF32 q{};
    q.e = p.exp_dev();
    q.L = p.L;
    q.J = p.J;
    q.jmin = p.jmin;
    q.m_pad = B.ld;
    q.R = B.R[i];
    q.count = p.d_count.p;
    q.perm = p.d_perm.p;
    q.begin = p.d_begin.p;
    q.pts = p.d_pts32.p;
    q.ynode = p.d_ynode32.p;
    q.lo = p.d_lo32.p;
    q.iext = p.d_iext32.p;
    q.vinv = p.d_vinv32.p;
    q.xb = B.xb.p + static_cast<size_t>(B.leaf_off[i]) * kRC * B.ld;
    q.yfar = B.yfar.p + static_cast<size_t>(B.leaf_off[i]) * kRC * B.ld;
    q.mom = B.mom.p + static_cast<size_t>(B.clus_off[i]) * kRC * B.n_pad;
    q.loc = B.loc.p + static_cast<size_t>(B.clus_off[i]) * kRC * B.n_pad;
    q.lco = B.lco.p + static_cast<size_t>(B.clus_off[i]) * kRC * B.n_pad;
    q.x = nullptr;
    q.y = nullptr;
    q.ldx = q.ldy = p.N;
    B.h_probs[i] = q;
  }
  B.probs.alloc(count);
  DW_CUDA(cudaMemcpy(B.probs.p, B.h_probs, sizeof(ProbF32) * count, cudaMemcpyHostToDevice));
  // work lists: upward by height above the leaves, downward by level
  std::vector<int2> w;
  int maxJ = 0;
  for (auto* p : B.plans) maxJ = std::max(maxJ, p->J);
  for (int h = 0; h <= maxJ; ++h) {
    const int off = static_cast<int>(w.size());
    for (int i = 0; i < count; ++i) {
      Plan& p = *B.plans[i];
      const int lev = p.J - h;
      if (lev < 0 || lev < p.jmin) continue;
      for (int g = (1 << lev) - 1; g < (1 << (lev + 1)) - 1; ++g) w.push_back(make_int2(i, g));
    }
    if (static_cast<int>(w.size()) > off) {
      B.up_off.push_back(off);
      B.up_cnt.push_back(static_cast<int>(w.size()) - off);
    }
  }
  for (int j = 0; j <= maxJ; ++j) {
    const int off = static_cast<int>(w.size());
    for (int i = 0; i < count; ++i) {
      Plan& p = *B.plans[i];
      if (j < p.jmin || j > p.J) continue;
      for (int g = (1 << j) - 1; g < (1 << (j + 1)) - 1; ++g) w.push_back(make_int2(i, g));
    }
    if (static_cast<int>(w.size()) > off) {
      B.down_off.push_back(off);
      B.down_cnt.push_back(static_cast<int>(w.size()) - off);
    }
  }
  B.work.alloc(std::max<size_t>(w.size(), 1));
  if (!w.empty()) DW_CUDA(cudaMemcpy(B.work.p, w.data(), sizeof(int2) * w.size(), cudaMemcpyHostToDevice));
  B.far_smem = batch_far_smem(lsum_max, B.n_pad);
  if (B.far_smem > 200 * 1024) fail(DWFMM_ERR_INVALID_ARG, "index sets too large for a batch");
  batch_far_attrs();
  ensure_sum_attrs();
  // right-hand-side classes (contiguous in the internal order)
  for (int i = 0; i < count;) {
    const int rc = sum_padded_rc(B.R[i]);
    int k = i;
    while (k < count && sum_padded_rc(B.R[k]) == rc) ++k;
    B.classes.push_back(Batch::Cls{rc, B.leaf_off[i], B.leaf_off[k] - B.leaf_off[i], B.clus_off[i],
                                   B.clus_off[k] - B.clus_off[i]});
    i = k;
  }
  DW_CUDA(cudaStreamSynchronize(s));
  // autotune the P2P/M2L launch shape, then capture the whole matvec
  tune_shapes(B);
  DW_CUDA(cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal));
  enqueue_matvec(B);
  DW_CUDA(cudaStreamEndCapture(B.stream, &B.graph));
  DW_CUDA(cudaGraphInstantiate(&B.exec, B.graph, 0));
  // then the persistent engine against it, for batches whose fused work
  // takes long enough to repay the tuning (a serving loop rebuilds small
  // batches often; there the engine is tuned only when asked for)
  if (std::min(B.tune_ms[0], B.tune_ms[1]) >= kPersistTuneMinMs) tune_persistent(B);
}

void batch_matvec(Batch& B, const double* const* x, double* const* y, cudaStream_t s) {
  // the pinned table may still be the source of the previous call's copy
  if (B.copied) DW_CUDA(cudaEventSynchronize(B.ev_copy));
  for (int i = 0; i < B.P; ++i) {
    const int c = B.order[i];
    if (!x[c] || !y[c]) fail(DWFMM_ERR_INVALID_ARG, "NULL buffer in batch");
    B.h_probs[i].x = x[c];
    B.h_probs[i].y = y[c];
  }
  // the table lives in device memory; order it before the graph on the caller's stream
  DW_CUDA(cudaMemcpyAsync(B.probs.p, B.h_probs, sizeof(ProbF32) * B.P, cudaMemcpyHostToDevice, s));
  DW_CUDA(cudaEventRecord(B.ev_copy, s));
  B.copied = true;
  DW_CUDA(cudaGraphLaunch(B.persistent ? B.pexec : B.exec, s));
  DW_CUDA(cudaGetLastError());
}

void batch_set_engine(Batch& B, int persistent) {
  if (persistent && !B.persist_tried) {
    // the tuning runs overwrite the batch's buffers: nothing may be in flight
    DW_CUDA(cudaDeviceSynchronize());
    tune_persistent(B);
    B.persistent = false;
  }
  if (persistent && !B.persist_ok) fail(DWFMM_ERR_STATE, "the persistent engine is not available for this batch");
  if (B.persistent == (persistent != 0)) return;
  B.persistent = persistent != 0;
  // captured CG iterations hold the other engine
  if (B.cg_exec) cudaGraphExecDestroy(B.cg_exec);
  if (B.cg_graph) cudaGraphDestroy(B.cg_graph);
  B.cg_exec = nullptr;
  B.cg_graph = nullptr;
}

void batch_engine(const Batch& B, int32_t* engine, double* ms, int32_t* launch) {
  engine[0] = B.persistent ? 1 : 0;
  engine[1] = B.persist_ok ? 1 : 0;
  ms[0] = B.engine_ms[0];
  ms[1] = B.engine_ms[1];
  launch[0] = B.persist_ok ? B.pgrid : 0;
  launch[1] = B.persist_ok ? B.pa.gs_near : 0;
  launch[2] = B.persist_ok ? B.pa.gs_m2l : 0;
}

}  // namespace dw

namespace dw {

Batch* batch_new() { return new Batch(); }
void batch_delete(Batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  b->release();
  delete b;
}
void batch_shape(const Batch& B, int32_t* shape) {
  shape[0] = B.split ? 1 : 0;
  shape[1] = B.thr_near;
  shape[2] = B.split_m2l ? 1 : 0;
  shape[3] = B.thr_m2l;
}

void batch_info(const Batch& B, int32_t* split, double* tune_ms, int64_t* leaves) {
  if (split) *split = B.split ? 1 : 0;
  if (tune_ms) {
    tune_ms[0] = B.tune_ms[0];
    tune_ms[1] = B.tune_ms[1];
  }
  if (leaves) *leaves = B.Ltot;
}

}  // namespace dw

// ---------------------------------------------------------------------------
// Batched CG: one iteration advances the incremental CG (dwfmm_cg_begin) of
// every problem of the batch.  Ap = K_tilde p of all problems is the batch's
// fused matvec (its captured graph); the shift, the inner products, the
// x / r / p updates and the per-column scalar decisions (the same as the
// single-plan iteration: breakdown on pAp = 0 or not finite, convergence on
// ||r||^2 <= rtol^2 ||f||^2) are fused kernels over all problems.  Inner
// products are computed in a fixed partition (block partials, then their
// sum in block order), so results do not depend on timing.
// ---------------------------------------------------------------------------

namespace dw {

namespace {

constexpr int kBcgThreads = 256;
constexpr int64_t kBcgPerBlock = 8192;   // elements of one column per partial block

struct BcgSeg {   // one (problem, column): its partial blocks
  int item, col, first, nblk;
};

// Partial inner products of every (problem, column).  mode 0: ap += lam p and
// partial sum of p . ap; mode 1: c += alpha p, r -= alpha ap and partial sum
// of r . r (alpha = coef).
__global__ void k_bcg_partial(const CgPtrs* items, const BcgSeg* segs, const int2* blk, int mode, double* part) {
  __shared__ double sh[kBcgThreads / 32];
  const int2 bs = blk[blockIdx.x];                 // (segment, block within it)
  const BcgSeg g = segs[bs.x];
  const CgPtrs it = items[g.item];
  const int64_t n = it.n;
  const int64_t lo = static_cast<int64_t>(bs.y) * kBcgPerBlock;
  const int64_t hi = lo + kBcgPerBlock < n ? lo + kBcgPerBlock : n;
  const int64_t off = static_cast<int64_t>(g.col) * n;
  double acc = 0.0;
  if (mode == 0) {
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBcgThreads) {
      const double pv = it.p[off + i];
      const double v = it.ap[off + i] + it.lam * pv;
      it.ap[off + i] = v;
      acc += pv * v;
    }
  } else {
    const double a = it.coef[g.col];
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBcgThreads) {
      it.c[off + i] += a * it.p[off + i];
      const double rv = it.r[off + i] - a * it.ap[off + i];
      it.r[off + i] = rv;
      acc += rv * rv;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBcgThreads / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// Per (problem, column): the inner product from its partials in block
// order, then the scalar step.  mode 0: alpha = rr / pAp; mode 1: the new
// rr, convergence, beta.
__global__ void k_bcg_scalar(const CgPtrs* items, const BcgSeg* segs, int nseg, int mode, const double* part) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nseg) return;
  const BcgSeg g = segs[k];
  const CgPtrs it = items[g.item];
  double v = 0.0;
  for (int b = 0; b < g.nblk; ++b) v += part[g.first + b];
  const int r = g.col;
  if (mode == 0) {
    double a = 0.0;
    if (it.status[r] == 0) {
      if (v == 0.0 || !isfinite(v)) it.status[r] = 2;
      else a = it.rr[r] / v;
    }
    it.pap[r] = v;
    it.coef[r] = a;
  } else {
    double b = 0.0;
    if (it.status[r] == 0) {
      it.iters[r] += 1;
      if (v <= *it.rtol2 * it.bn2[r]) it.status[r] = 1;
      b = v / it.rr[r];
      it.rr[r] = v;
    }
    it.tmp[r] = v;
    it.coef[r] = b;
  }
}

// p = r + beta p for every problem and column.
__global__ void k_bcg_p(const CgPtrs* items, const BcgSeg* segs, const int2* blk) {
  const int2 bs = blk[blockIdx.x];
  const BcgSeg g = segs[bs.x];
  const CgPtrs it = items[g.item];
  const int64_t n = it.n;
  const int64_t lo = static_cast<int64_t>(bs.y) * kBcgPerBlock;
  const int64_t hi = lo + kBcgPerBlock < n ? lo + kBcgPerBlock : n;
  const int64_t off = static_cast<int64_t>(g.col) * n;
  const double b = it.coef[g.col];
  for (int64_t i = lo + threadIdx.x; i < hi; i += kBcgThreads) it.p[off + i] = it.r[off + i] + b * it.p[off + i];
}

}  // namespace

void batch_cg_step(Batch& B, int iters, cudaStream_t s) {
  if (iters < 0) fail(DWFMM_ERR_INVALID_ARG, "iters must be >= 0");
  std::vector<CgPtrs> items(B.P);
  std::vector<const double*> xs(B.P);
  std::vector<double*> ys(B.P);
  std::vector<BcgSeg> segs;
  std::vector<int2> blk;
  for (int i = 0; i < B.P; ++i) {
    Plan& P = *B.plans[i];
    if (!P.cgs.active || !P.cg_p.p) fail(DWFMM_ERR_STATE, "every plan of the batch needs dwfmm_cg_begin first");
    if (P.cgs.R != B.R[i]) fail(DWFMM_ERR_INVALID_ARG, "a plan's CG right-hand sides differ from its batch nrhs");
    items[i] = cg_ptrs(P);
    const int c = B.order[i];
    xs[c] = P.cg_p.p;
    ys[c] = P.cg_ap.p;
    const int nb = static_cast<int>((P.N + kBcgPerBlock - 1) / kBcgPerBlock);
    for (int r = 0; r < B.R[i]; ++r) {
      const int seg = static_cast<int>(segs.size());
      segs.push_back(BcgSeg{i, r, static_cast<int>(blk.size()), nb});
      for (int b = 0; b < nb; ++b) blk.push_back(make_int2(seg, b));
    }
  }
  // device tables: uploaded on the stream only when their content changed
  // (a pinned staging buffer, reused once its previous copy is done)
  const size_t bi = sizeof(CgPtrs) * items.size(), bs = sizeof(BcgSeg) * segs.size(), bb = sizeof(int2) * blk.size();
  std::vector<char> host(bi + bs + bb);
  std::memcpy(host.data(), items.data(), bi);
  std::memcpy(host.data() + bi, segs.data(), bs);
  std::memcpy(host.data() + bi + bs, blk.data(), bb);
  const int nseg = static_cast<int>(segs.size()), nblk = static_cast<int>(blk.size());
  if (host != B.cg_host) {
    if (B.cg_copied) DW_CUDA(cudaEventSynchronize(B.cg_ev));
    if (B.cg_pinned_n < host.size()) {
      if (B.cg_pinned) cudaFreeHost(B.cg_pinned);
      B.cg_pinned = nullptr;
      B.cg_pinned_n = 0;
      DW_CUDA(cudaMallocHost(reinterpret_cast<void**>(&B.cg_pinned), host.size()));
      B.cg_pinned_n = host.size();
    }
    if (!B.cg_ev) DW_CUDA(cudaEventCreateWithFlags(&B.cg_ev, cudaEventDisableTiming));
    const bool grow = B.cg_tab.n < host.size() || B.cg_part.n < blk.size();
    if (grow && B.cg_exec) {   // the captured iterations point at the old tables
      cudaGraphExecDestroy(B.cg_exec);
      cudaGraphDestroy(B.cg_graph);
      B.cg_exec = nullptr;
      B.cg_graph = nullptr;
    }
    B.cg_tab.alloc(host.size());
    B.cg_part.alloc(blk.size());
    std::memcpy(B.cg_pinned, host.data(), host.size());
    DW_CUDA(cudaMemcpyAsync(B.cg_tab.p, B.cg_pinned, host.size(), cudaMemcpyHostToDevice, s));
    DW_CUDA(cudaEventRecord(B.cg_ev, s));
    B.cg_copied = true;
    B.cg_host.swap(host);
    // the matvec's problem table (x = p, y = Ap of every problem)
    if (B.copied) DW_CUDA(cudaEventSynchronize(B.ev_copy));
    for (int i = 0; i < B.P; ++i) {
      const int c = B.order[i];
      B.h_probs[i].x = xs[c];
      B.h_probs[i].y = ys[c];
    }
    DW_CUDA(cudaMemcpyAsync(B.probs.p, B.h_probs, sizeof(ProbF32) * B.P, cudaMemcpyHostToDevice, s));
    DW_CUDA(cudaEventRecord(B.ev_copy, s));
    B.copied = true;
  }
  const CgPtrs* d_items = reinterpret_cast<const CgPtrs*>(B.cg_tab.p);
  const BcgSeg* d_segs = reinterpret_cast<const BcgSeg*>(B.cg_tab.p + bi);
  const int2* d_blk = reinterpret_cast<const int2*>(B.cg_tab.p + bi + bs);
  // `iters` iterations captured once per (iteration count, table shape) on the
  // batch's stream and replayed on the caller's
  if (iters > 0 && (!B.cg_exec || B.cg_iters != iters || B.cg_nseg != nseg || B.cg_nblk != nblk)) {
    if (B.cg_exec) cudaGraphExecDestroy(B.cg_exec);
    if (B.cg_graph) cudaGraphDestroy(B.cg_graph);
    B.cg_exec = nullptr;
    B.cg_graph = nullptr;
    cudaStream_t bst = B.stream;
    DW_CUDA(cudaStreamBeginCapture(bst, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < iters; ++k) {
      enqueue_matvec(B);
      k_bcg_partial<<<nblk, kBcgThreads, 0, bst>>>(d_items, d_segs, d_blk, 0, B.cg_part.p);
      k_bcg_scalar<<<ceil_div(nseg, 64), 64, 0, bst>>>(d_items, d_segs, nseg, 0, B.cg_part.p);
      k_bcg_partial<<<nblk, kBcgThreads, 0, bst>>>(d_items, d_segs, d_blk, 1, B.cg_part.p);
      k_bcg_scalar<<<ceil_div(nseg, 64), 64, 0, bst>>>(d_items, d_segs, nseg, 1, B.cg_part.p);
      k_bcg_p<<<nblk, kBcgThreads, 0, bst>>>(d_items, d_segs, d_blk);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(bst, &g);
    if (ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      DW_CUDA(ce);
      fail(DWFMM_ERR_CUDA, "capture of the batched CG iterations failed");
    }
    cudaGraphExec_t e = nullptr;
    if (cudaGraphInstantiate(&e, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      (void)cudaGetLastError();
      fail(DWFMM_ERR_CUDA, "instantiation of the batched CG iterations failed");
    }
    B.cg_graph = g;
    B.cg_exec = e;
    B.cg_iters = iters;
    B.cg_nseg = nseg;
    B.cg_nblk = nblk;
  }
  if (iters > 0) DW_CUDA(cudaGraphLaunch(B.cg_exec, s));
  DW_CUDA(cudaGetLastError());
  for (int i = 0; i < B.P; ++i) cg_snapshot(*B.plans[i], s);
}

}  // namespace dw
