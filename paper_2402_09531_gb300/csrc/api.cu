// extern "C" entry points of include/dwfmm.h.  Validates arguments, stages
// host buffers through device memory, and maps internal errors to status
// codes; every numerical step is a kernel launched from the other files.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "dwfmm_internal.cuh"

using dw::ApiError;
using dw::CudaError;
using dw::Plan;

namespace dw {

void Plan::free_tree() {
  have_tree = false;
  N = 0;
  J = -1;
  d_begin.release();
  d_count.release();
  d_perm.release();
  d_lo.release();
  d_hi.release();
  d_ext.release();
  d_iext.release();
  d_lo32.release();
  d_iext32.release();
  d_pts64.release();
  d_pts32.release();
  d_ynode64.release();
  d_ynode32.release();
  d_far_rowptr.release();
  d_far_col.release();
  d_near_rowptr.release();
  d_near_col.release();
  d_far_pairs.release();
  d_near_pairs.release();
  xb64.release();
  ynear64.release();
  yfar64.release();
  mom64.release();
  loc64.release();
  lco64.release();
  xb32.release();
  ynear32.release();
  yfar32.release();
  mom32.release();
  loc32.release();
  lco32.release();
  cg_r.release();
  cg_p.release();
  cg_ap.release();
  cg_c.release();
  cg_f.release();
  cg_dot.release();
  cg_tmp.release();
  scratch.release();
  d_ptsk.release();
  d_ynodek.release();
  xq32.release();
  momq32.release();
  bq32.release();
  bqm32.release();
  near_parts64.release();
  sym_t.release();
  sym_s.release();
  sym_uprow.release();
  sym_lorow.release();
  sym_loslot.release();
  sym_pf.release();
  sym_pt.release();
  sym_nup = 0;
  sym_ok = false;
  sym_order.release();
  sym_bq16.release();
  sym_fwd.release();
  sym_acc.release();
  sym_colmax.release();
  sym_xa16.release();
  sym_xb16.release();
  sym_x16_ok = false;
  fsym_uprow.release();
  fsym_s.release();
  fsym_order.release();
  fsym_rows = 0;
  fsym_ok = false;
  m2l_crd.release();
  m2l_crd_D = -1;
  m2l_xa16.release();
  m2l_xb16.release();
  m2l_x16_D = -1;
  m2l_bq16.release();
  m2l_fwd.release();
  m2l_acc.release();
  m2l_colmax.release();
  m2l_tuned = -1;
  m2l_tune_ms[0] = m2l_tune_ms[1] = -1.0;
  dpad = -1;
}

// Report a bounded device wait that gave up (raised by the tuned kernels).
void check_device_error(Plan& P) {
  if (!P.d_err.p) return;
  int e = 0;
  DW_CUDA(cudaMemcpy(&e, P.d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    DW_CUDA(cudaMemset(P.d_err.p, 0, sizeof(int)));
    fail(DWFMM_ERR_TIMEOUT, "a bounded wait on a shared-memory copy gave up");
  }
}

void Plan::free_all() {
  free_tree();
  d_fac.release();
  d_qk.release();
  d_loff.release();
  d_lam.release();
  d_nodes.release();
  d_vinv.release();
  d_vinv32.release();
  far_vt.release();
  far_vexp.release();
  far_vt_ok = false;
  d_err.release();
  stage_in.release();
  stage_out.release();
  for (auto& r : tm.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  tm.recs.clear();
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (ev_scaled) cudaEventDestroy(ev_scaled);
  ev_scaled = nullptr;
  cgs.drop_graph();
  cgs.d_int.release();
  if (cgs.h_snap) cudaFreeHost(cgs.h_snap);
  cgs.h_snap = nullptr;
  if (cgs.ev) cudaEventDestroy(cgs.ev);
  cgs.ev = nullptr;
  if (side) cudaStreamDestroy(side);
  ev_fork = ev_join = nullptr;
  side = nullptr;
}

}  // namespace dw

namespace {

template <class F>
dwfmm_status guarded(Plan* P, F&& f) {
  try {
    if (P) P->last_error.clear();
    return f();
  } catch (const ApiError& e) {
    if (P) P->last_error = e.msg;
    return e.status;
  } catch (const CudaError& e) {
    if (P) P->last_error = std::string(e.what) + ": " + cudaGetErrorString(e.err);
    (void)cudaGetLastError();
    return e.err == cudaErrorMemoryAllocation ? DWFMM_ERR_OOM : DWFMM_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    if (P) P->last_error = "host allocation failed";
    return DWFMM_ERR_OOM;
  } catch (...) {
    if (P) P->last_error = "unexpected error";
    return DWFMM_ERR_CUDA;
  }
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void bind_stream(Plan& P, void* stream) {
  P.stream = static_cast<cudaStream_t>(stream);
  DW_CUDA(cudaSetDevice(P.device));
}

}  // namespace

extern "C" {

const char* dwfmm_status_string(dwfmm_status s) {
  switch (s) {
    case DWFMM_OK: return "ok";
    case DWFMM_ERR_INVALID_ARG: return "invalid argument";
    case DWFMM_ERR_OOM: return "out of device memory";
    case DWFMM_ERR_CUDA: return "CUDA error";
    case DWFMM_ERR_BREAKDOWN: return "CG breakdown (p^T A p == 0 or not finite)";
    case DWFMM_ERR_NOT_CONVERGED: return "CG did not converge";
    case DWFMM_ERR_TIMEOUT: return "device wait timed out";
    case DWFMM_ERR_STATE: return "call out of order";
    case DWFMM_ERR_SINGULAR: return "interpolation nodes not unisolvent";
  }
  return "unknown status";
}

const char* dwfmm_last_error(dwfmm_plan plan) { return plan ? plan->P.last_error.c_str() : ""; }

dwfmm_status dwfmm_plan_create(const dwfmm_config* cfg, void* stream, dwfmm_plan* out) {
  if (!cfg || !out) return DWFMM_ERR_INVALID_ARG;
  *out = nullptr;
  dwfmm_plan h = new (std::nothrow) dwfmm_plan_s();
  if (!h) return DWFMM_ERR_OOM;
  Plan& P = h->P;
  dwfmm_status st = guarded(&P, [&]() -> dwfmm_status {
    using dw::fail;
    if (cfg->d < 1 || cfg->d > dw::kMaxDim) fail(DWFMM_ERR_INVALID_ARG, "d must be in 1..32");
    if (cfg->kernel < 0 || cfg->kernel > 2) fail(DWFMM_ERR_INVALID_ARG, "unknown kernel");
    if (!(cfg->sigma > 0.0) || !std::isfinite(cfg->sigma)) fail(DWFMM_ERR_INVALID_ARG, "sigma must be > 0");
    if (!cfg->gamma) fail(DWFMM_ERR_INVALID_ARG, "gamma is NULL");
    if (cfg->weight_rule < 0 || cfg->weight_rule > 2) fail(DWFMM_ERR_INVALID_ARG, "unknown weight rule");
    if (cfg->weight_rule == DWFMM_W_EXPLICIT && !cfg->weights) fail(DWFMM_ERR_INVALID_ARG, "weights is NULL");
    if (!(cfg->q >= 0.0) || !std::isfinite(cfg->q)) fail(DWFMM_ERR_INVALID_ARG, "q must be >= 0");
    if (!(cfg->eta > 0.0) || !std::isfinite(cfg->eta)) fail(DWFMM_ERR_INVALID_ARG, "eta must be > 0");
    if (cfg->leaf_size < 2 || cfg->leaf_size > 1024) fail(DWFMM_ERR_INVALID_ARG, "leaf_size must be in 2..1024");
    if (cfg->precision < 0 || cfg->precision > 2) fail(DWFMM_ERR_INVALID_ARG, "unknown precision");
    if (cfg->max_rhs < 1 || cfg->max_rhs > 64) fail(DWFMM_ERR_INVALID_ARG, "max_rhs must be in 1..64");
    if (cfg->index_set < 0 || cfg->index_set > 1) fail(DWFMM_ERR_INVALID_ARG, "unknown index set");
    P.d = cfg->d;
    P.kernel = cfg->kernel;
    P.sigma = cfg->sigma;
    P.gamma.assign(cfg->gamma, cfg->gamma + cfg->d);
    for (double g : P.gamma)
      if (!(g > 0.0) || !std::isfinite(g)) fail(DWFMM_ERR_INVALID_ARG, "gamma_k must be > 0");
    P.wrule = cfg->weight_rule;
    if (cfg->weight_rule == DWFMM_W_EXPLICIT) P.w.assign(cfg->weights, cfg->weights + cfg->d);
    P.q = cfg->q;
    P.eta = cfg->eta;
    P.leaf = cfg->leaf_size;
    P.M = cfg->halton_candidates;
    P.prec = cfg->precision;
    P.max_rhs = cfg->max_rhs;
    P.iset = cfg->index_set;
    DW_CUDA(cudaGetDevice(&P.device));
    bind_stream(P, stream);
    DW_CUDA(cudaStreamCreateWithFlags(&P.side, cudaStreamNonBlocking));
    DW_CUDA(cudaEventCreateWithFlags(&P.ev_fork, cudaEventDisableTiming));
    DW_CUDA(cudaEventCreateWithFlags(&P.ev_join, cudaEventDisableTiming));
    DW_CUDA(cudaEventCreateWithFlags(&P.ev_scaled, cudaEventDisableTiming));
    P.d_err.alloc(1);
    DW_CUDA(cudaMemset(P.d_err.p, 0, sizeof(int)));
    dw::setup_expansion(P);
    if (dw::farfield_smem_need(P, true) > 220 * 1024)
      fail(DWFMM_ERR_INVALID_ARG, "index set too large for the far-field kernels");
    dw::farfield_set_smem_limits(P);
    return DWFMM_OK;
  });
  if (st != DWFMM_OK) {
    P.free_all();
    delete h;
    return st;
  }
  *out = h;
  return DWFMM_OK;
}

dwfmm_status dwfmm_plan_set_nodes(dwfmm_plan plan, const double* nodes, int64_t n, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!nodes || n != P.n) dw::fail(DWFMM_ERR_INVALID_ARG, "nodes must be n x d with n = |Lambda|");
    if (P.have_tree) dw::fail(DWFMM_ERR_STATE, "set nodes before building the tree");
    bind_stream(P, stream);
    DW_CUDA(cudaMemcpyAsync(P.d_nodes.p, nodes, sizeof(double) * P.n * P.d, cudaMemcpyHostToDevice, P.stream));
    P.pivots.assign(P.n, -1);
    dw::setup_vinv_from_nodes(P);
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_tree_build(dwfmm_plan plan, const double* pts, int64_t n, int64_t ld, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (n < 0 || n > (int64_t(1) << 30)) dw::fail(DWFMM_ERR_INVALID_ARG, "N must be in 0..2^30");
    if (n > 0 && (!pts || ld < P.d)) dw::fail(DWFMM_ERR_INVALID_ARG, "pts is NULL or ld < d");
    bind_stream(P, stream);
    P.free_tree();
    P.cgs.drop_graph();
    ++P.tree_gen;
    const double* dev = pts;
    int64_t ld_dev = ld;
    dw::DBuf<double> staged;
    if (n > 0 && !is_device_pointer(pts)) {
      // the d used columns of each row only (a host buffer may end right after them)
      staged.alloc(static_cast<size_t>(n) * P.d);
      DW_CUDA(cudaMemcpy2DAsync(staged.p, sizeof(double) * P.d, pts, sizeof(double) * ld, sizeof(double) * P.d, n,
                                cudaMemcpyHostToDevice, P.stream));
      dev = staged.p;
      ld_dev = P.d;
    }
    dw::build_tree(P, dev, n, ld_dev);
    dw::build_lists(P);
    dw::build_cluster_data(P);
    dw::build_sym_lists(P);
    if (P.prec == DWFMM_P_MIXED) dw::build_far_sym_lists(P);
    // bound of |x'|^2 = |x|^2 log2(e) / (2 sigma^2) over the root box, which
    // holds every site and every interpolation node
    P.gauss_fact = false;
    P.gauss_bound = 0.0;
    if (P.kernel == DWFMM_K_GAUSS && n > 0) {
      std::vector<double> lo(P.d), hi(P.d);
      DW_CUDA(cudaMemcpyAsync(lo.data(), P.d_lo.p, sizeof(double) * P.d, cudaMemcpyDeviceToHost, P.stream));
      DW_CUDA(cudaMemcpyAsync(hi.data(), P.d_hi.p, sizeof(double) * P.d, cudaMemcpyDeviceToHost, P.stream));
      DW_CUDA(cudaStreamSynchronize(P.stream));
      const double s2 = 1.4426950408889634 / (2.0 * P.sigma * P.sigma);
      double b = 0.0;
      for (int k = 0; k < P.d; ++k) {
        const double m = std::max(std::fabs(lo[k]), std::fabs(hi[k]));
        b += m * m * s2;
      }
      P.gauss_fact = b <= 30.0;
      P.gauss_bound = b;
    }
    P.have_tree = true;
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_matvec(dwfmm_plan plan, const double* x, double* y, int32_t nrhs, int64_t ldx,
                          int64_t ldy, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.have_tree) dw::fail(DWFMM_ERR_STATE, "matvec before tree_build");
    if (nrhs < 1 || nrhs > P.max_rhs) dw::fail(DWFMM_ERR_INVALID_ARG, "nrhs outside 1..max_rhs");
    if (P.N == 0) return DWFMM_OK;
    if (!x || !y || ldx < P.N || ldy < P.N) dw::fail(DWFMM_ERR_INVALID_ARG, "NULL buffer or ld < N");
    bind_stream(P, stream);
    const bool fp64 = P.prec == DWFMM_P_FP64;
    const double* xd = x;
    double* yd = y;
    int64_t lx = ldx, ly = ldy;
    const bool xh = !is_device_pointer(x), yh = !is_device_pointer(y);
    const size_t bytes = sizeof(double) * P.N * nrhs;
    if (xh) {
      P.stage_in.alloc(static_cast<size_t>(P.N) * P.max_rhs);
      DW_CUDA(cudaMemcpy2DAsync(P.stage_in.p, P.N * sizeof(double), x, ldx * sizeof(double),
                                P.N * sizeof(double), nrhs, cudaMemcpyHostToDevice, P.stream));
      xd = P.stage_in.p;
      lx = P.N;
    }
    if (yh) {
      P.stage_out.alloc(static_cast<size_t>(P.N) * P.max_rhs);
      yd = P.stage_out.p;
      ly = P.N;
    }
    (void)bytes;
    dw::matvec_device(P, xd, lx, yd, ly, nrhs, fp64);
    if (yh) {
      DW_CUDA(cudaMemcpy2DAsync(y, ldy * sizeof(double), yd, P.N * sizeof(double), P.N * sizeof(double),
                                nrhs, cudaMemcpyDeviceToHost, P.stream));
      DW_CUDA(cudaStreamSynchronize(P.stream));
      dw::check_device_error(P);
    }
    DW_CUDA(cudaGetLastError());
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_solve(dwfmm_plan plan, double lambda, const double* f, double* c, int32_t nrhs,
                         int64_t ld, double rtol, int32_t maxit, int32_t* iters_out, double* relres_out,
                         void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.have_tree) dw::fail(DWFMM_ERR_STATE, "solve before tree_build");
    if (nrhs < 1 || nrhs > P.max_rhs) dw::fail(DWFMM_ERR_INVALID_ARG, "nrhs outside 1..max_rhs");
    if (!(lambda >= 0.0) || !(rtol > 0.0) || maxit < 1) dw::fail(DWFMM_ERR_INVALID_ARG, "lambda, rtol or maxit");
    if (P.N > 0 && (!f || !c || ld < P.N)) dw::fail(DWFMM_ERR_INVALID_ARG, "NULL buffer or ld < N");
    bind_stream(P, stream);
    const double* fd = f;
    double* cd = c;
    int64_t l = ld;
    dw::DBuf<double> fs, cs;
    const bool fh = P.N > 0 && !is_device_pointer(f), ch = P.N > 0 && !is_device_pointer(c);
    if (fh) {
      fs.alloc(static_cast<size_t>(P.N) * nrhs);
      DW_CUDA(cudaMemcpy2DAsync(fs.p, P.N * sizeof(double), f, ld * sizeof(double), P.N * sizeof(double),
                                nrhs, cudaMemcpyHostToDevice, P.stream));
      fd = fs.p;
    }
    if (ch) {
      cs.alloc(static_cast<size_t>(P.N) * nrhs);
      cd = cs.p;
    }
    const int64_t lf = fh ? P.N : ld;
    // solve() takes one leading dimension: stage to compact buffers when they differ
    dw::DBuf<double> fc;
    if (!fh && lf != P.N) {
      fc.alloc(static_cast<size_t>(P.N) * nrhs);
      DW_CUDA(cudaMemcpy2DAsync(fc.p, P.N * sizeof(double), f, ld * sizeof(double), P.N * sizeof(double),
                                nrhs, cudaMemcpyDeviceToDevice, P.stream));
      fd = fc.p;
    }
    l = P.N;
    dw::DBuf<double> cc;
    double* ctarget = cd;
    if (!ch && ld != P.N) {
      cc.alloc(static_cast<size_t>(P.N) * nrhs);
      ctarget = cc.p;
    }
    int its = 0;
    const dwfmm_status s = dw::solve(P, lambda, fd, ctarget, nrhs, l, rtol, maxit, &its, relres_out);
    if (ctarget != cd)
      DW_CUDA(cudaMemcpy2DAsync(cd, ld * sizeof(double), ctarget, P.N * sizeof(double), P.N * sizeof(double),
                                nrhs, cudaMemcpyDeviceToDevice, P.stream));
    if (ch)
      DW_CUDA(cudaMemcpy2DAsync(c, ld * sizeof(double), cs.p, P.N * sizeof(double), P.N * sizeof(double),
                                nrhs, cudaMemcpyDeviceToHost, P.stream));
    DW_CUDA(cudaStreamSynchronize(P.stream));
    dw::check_device_error(P);
    if (iters_out) *iters_out = its;
    if (s != DWFMM_OK) P.last_error = dwfmm_status_string(s);
    return s;
  });
}

dwfmm_status dwfmm_plan_destroy(dwfmm_plan plan) {
  if (!plan) return DWFMM_OK;
  Plan& P = plan->P;
  if (P.stream) (void)cudaStreamSynchronize(P.stream);
  if (P.side) (void)cudaStreamSynchronize(P.side);
  P.free_all();
  delete plan;
  return DWFMM_OK;
}

dwfmm_status dwfmm_near_engine(dwfmm_plan plan, int32_t* engine) {
  if (!plan || !engine) return DWFMM_ERR_INVALID_ARG;
  *engine = plan->P.near_engine;
  return DWFMM_OK;
}

dwfmm_status dwfmm_m2l_engine(dwfmm_plan plan, int32_t* engine) {
  if (!plan || !engine) return DWFMM_ERR_INVALID_ARG;
  *engine = plan->P.m2l_engine;
  return DWFMM_OK;
}

dwfmm_status dwfmm_plan_set_m2l_engine(dwfmm_plan plan, int32_t engine) {
  if (!plan || (engine != -1 && engine != 2 && engine != 3)) return DWFMM_ERR_INVALID_ARG;
  plan->P.m2l_pref = engine;
  return DWFMM_OK;
}

dwfmm_status dwfmm_m2l_tune_ms(dwfmm_plan plan, double* ms) {
  if (!plan || !ms) return DWFMM_ERR_INVALID_ARG;
  ms[0] = plan->P.m2l_tune_ms[0];
  ms[1] = plan->P.m2l_tune_ms[1];
  return DWFMM_OK;
}

dwfmm_status dwfmm_far_engine(dwfmm_plan plan, int32_t* engine) {
  if (!plan || !engine) return DWFMM_ERR_INVALID_ARG;
  *engine = plan->P.far_engine;
  return DWFMM_OK;
}

dwfmm_status dwfmm_plan_info(dwfmm_plan plan, int64_t* n_x, int64_t* n_far, int64_t* n_near, int32_t* depth) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  const Plan& P = plan->P;
  if (n_x) *n_x = P.n;
  if (n_far) *n_far = P.have_tree ? P.nfar : 0;
  if (n_near) *n_near = P.have_tree ? P.nnear : 0;
  if (depth) *depth = P.have_tree ? P.J : -1;
  return DWFMM_OK;
}

dwfmm_status dwfmm_plan_export(dwfmm_plan plan, double* weights, int32_t* lam, double* nodes, int32_t* pivots,
                               double* vinv) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (weights) std::memcpy(weights, P.w.data(), sizeof(double) * P.d);
    if (lam) std::memcpy(lam, P.lam.data(), sizeof(int32_t) * P.lam.size());
    if (pivots) std::memcpy(pivots, P.pivots.data(), sizeof(int32_t) * P.n);
    if (nodes) DW_CUDA(cudaMemcpy(nodes, P.d_nodes.p, sizeof(double) * P.n * P.d, cudaMemcpyDeviceToHost));
    if (vinv) {
      std::vector<double> tmp(static_cast<size_t>(P.n_pad) * P.n_pad);
      DW_CUDA(cudaMemcpy(tmp.data(), P.d_vinv.p, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost));
      for (int r = 0; r < P.n; ++r)
        for (int c = 0; c < P.n; ++c) vinv[r * P.n + c] = tmp[static_cast<size_t>(r) * P.n_pad + c];
    }
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_tree_export(dwfmm_plan plan, int64_t* perm, int64_t* begin, int64_t* end, double* lo,
                               double* hi) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.have_tree) dw::fail(DWFMM_ERR_STATE, "no tree");
    if (perm && P.N > 0) {
      std::vector<int32_t> t(P.N);
      DW_CUDA(cudaMemcpy(t.data(), P.d_perm.p, sizeof(int32_t) * P.N, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < P.N; ++i) perm[i] = t[i];
    }
    for (int c = 0; c < P.C; ++c) {
      if (begin) begin[c] = P.h_begin[c];
      if (end) end[c] = P.h_begin[c] + P.h_count[c];
    }
    if (lo) DW_CUDA(cudaMemcpy(lo, P.d_lo.p, sizeof(double) * P.C * P.d, cudaMemcpyDeviceToHost));
    if (hi) DW_CUDA(cudaMemcpy(hi, P.d_hi.p, sizeof(double) * P.C * P.d, cudaMemcpyDeviceToHost));
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_lists_export(dwfmm_plan plan, int32_t* far, int32_t* near) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.have_tree) dw::fail(DWFMM_ERR_STATE, "no tree");
    if (far && P.nfar > 0)
      DW_CUDA(cudaMemcpy(far, P.d_far_pairs.p, sizeof(int32_t) * 2 * P.nfar, cudaMemcpyDeviceToHost));
    if (near && P.nnear > 0)
      DW_CUDA(cudaMemcpy(near, P.d_near_pairs.p, sizeof(int32_t) * 2 * P.nnear, cudaMemcpyDeviceToHost));
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_set_profiling(dwfmm_plan plan, int32_t enable) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  plan->P.tm.on = enable != 0;
  plan->P.tm.serialize = enable == 2;
  return DWFMM_OK;
}

dwfmm_status dwfmm_phase_times(dwfmm_plan plan, double* ms, int64_t* launches, int32_t reset) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    dw::timers_collect(P);
    dw::check_device_error(P);
    for (int i = 0; i < 7; ++i) {
      if (ms) ms[i] = P.tm.ms[i];
      if (launches) launches[i] = P.tm.launches[i];
    }
    if (reset)
      for (int i = 0; i < 8; ++i) {
        P.tm.ms[i] = 0.0;
        P.tm.launches[i] = 0;
      }
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_cg_begin(dwfmm_plan plan, double lambda, const double* f, int32_t nrhs, int64_t ld,
                            double rtol, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.have_tree) dw::fail(DWFMM_ERR_STATE, "cg_begin before tree_build");
    if (nrhs < 1 || nrhs > P.max_rhs || nrhs > 64) dw::fail(DWFMM_ERR_INVALID_ARG, "nrhs outside 1..max_rhs");
    if (!(lambda >= 0.0) || !(rtol > 0.0)) dw::fail(DWFMM_ERR_INVALID_ARG, "lambda or rtol");
    if (P.N == 0) dw::fail(DWFMM_ERR_INVALID_ARG, "empty problem");
    if (!f || ld < P.N || !is_device_pointer(f)) dw::fail(DWFMM_ERR_INVALID_ARG, "f must be a device buffer, ld >= N");
    bind_stream(P, stream);
    dw::cg_begin(P, lambda, f, nrhs, ld, rtol);
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_cg_step(dwfmm_plan plan, int32_t iters, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.cgs.active) dw::fail(DWFMM_ERR_STATE, "cg_step before cg_begin");
    if (iters < 0) dw::fail(DWFMM_ERR_INVALID_ARG, "iters < 0");
    bind_stream(P, stream);
    dw::cg_step(P, iters);
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_cg_poll(dwfmm_plan plan, int32_t* ready, int32_t* status, int32_t* iters, double* rr) {
  if (!plan || !ready) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.cgs.active) dw::fail(DWFMM_ERR_STATE, "cg_poll before cg_begin");
    *ready = dw::cg_poll(P, status, iters, rr) ? 1 : 0;
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_cg_result(dwfmm_plan plan, double* c, int64_t ld, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.cgs.active) dw::fail(DWFMM_ERR_STATE, "cg_result before cg_begin");
    if (!c || ld < P.N) dw::fail(DWFMM_ERR_INVALID_ARG, "NULL buffer or ld < N");
    bind_stream(P, stream);
    dw::cg_result(P, c, ld);
    if (!is_device_pointer(c)) DW_CUDA(cudaStreamSynchronize(P.stream));
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_residual(dwfmm_plan plan, double lambda, const double* f, const double* c, double* r,
                            int32_t nrhs, int64_t ld, double* relres, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.have_tree) dw::fail(DWFMM_ERR_STATE, "residual before tree_build");
    if (nrhs < 1 || nrhs > P.max_rhs) dw::fail(DWFMM_ERR_INVALID_ARG, "nrhs outside 1..max_rhs");
    if (P.N == 0) return DWFMM_OK;
    if (!f || !c || ld < P.N) dw::fail(DWFMM_ERR_INVALID_ARG, "NULL buffer or ld < N");
    bind_stream(P, stream);
    const int64_t n = P.N;
    const size_t nr = static_cast<size_t>(n) * nrhs;
    dw::DBuf<double> fd, cd, rd;
    fd.alloc(nr);
    cd.alloc(nr);
    rd.alloc(nr);
    DW_CUDA(cudaMemcpy2DAsync(fd.p, n * sizeof(double), f, ld * sizeof(double), n * sizeof(double), nrhs,
                              cudaMemcpyDefault, P.stream));
    DW_CUDA(cudaMemcpy2DAsync(cd.p, n * sizeof(double), c, ld * sizeof(double), n * sizeof(double), nrhs,
                              cudaMemcpyDefault, P.stream));
    std::vector<double> rel(nrhs);
    dw::residual64(P, lambda, fd.p, cd.p, rd.p, nrhs, rel.data());
    if (r)
      DW_CUDA(cudaMemcpy2DAsync(r, ld * sizeof(double), rd.p, n * sizeof(double), n * sizeof(double), nrhs,
                                cudaMemcpyDefault, P.stream));
    DW_CUDA(cudaStreamSynchronize(P.stream));
    dw::check_device_error(P);
    if (relres)
      for (int k = 0; k < nrhs; ++k) relres[k] = rel[k];
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_refine(dwfmm_plan plan, double lambda, const double* f, double* c, const double* delta,
                          double* r, int32_t nrhs, int64_t ld, double* alpha, double* relres, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.have_tree) dw::fail(DWFMM_ERR_STATE, "refine before tree_build");
    if (nrhs < 1 || nrhs > P.max_rhs) dw::fail(DWFMM_ERR_INVALID_ARG, "nrhs outside 1..max_rhs");
    if (P.N == 0) return DWFMM_OK;
    if (!f || !c || !delta || !r || ld < P.N) dw::fail(DWFMM_ERR_INVALID_ARG, "NULL buffer or ld < N");
    bind_stream(P, stream);
    const int64_t n = P.N;
    const size_t nr = static_cast<size_t>(n) * nrhs;
    dw::DBuf<double> cd, dd, rd, fd;
    cd.alloc(nr);
    dd.alloc(nr);
    rd.alloc(nr);
    fd.alloc(nr);
    auto in = [&](double* dst, const double* src) {
      DW_CUDA(cudaMemcpy2DAsync(dst, n * sizeof(double), src, ld * sizeof(double), n * sizeof(double), nrhs,
                                cudaMemcpyDefault, P.stream));
    };
    in(cd.p, c);
    in(dd.p, delta);
    in(rd.p, r);
    in(fd.p, f);
    std::vector<double> al(nrhs), rel(nrhs);
    dw::refine64(P, lambda, fd.p, cd.p, dd.p, rd.p, nrhs, al.data(), rel.data());
    auto out = [&](double* dst, const double* src) {
      DW_CUDA(cudaMemcpy2DAsync(dst, ld * sizeof(double), src, n * sizeof(double), n * sizeof(double), nrhs,
                                cudaMemcpyDefault, P.stream));
    };
    out(c, cd.p);
    out(r, rd.p);
    DW_CUDA(cudaStreamSynchronize(P.stream));
    dw::check_device_error(P);
    for (int k = 0; k < nrhs; ++k) {
      if (alpha) alpha[k] = al[k];
      if (relres) relres[k] = rel[k];
    }
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_evaluate(dwfmm_plan plan, const double* targets, int64_t nt, int64_t ld_t, const double* c,
                            int64_t ld_c, double* out, int64_t ld_o, int32_t nrhs, void* stream) {
  if (!plan) return DWFMM_ERR_INVALID_ARG;
  Plan& P = plan->P;
  return guarded(&P, [&]() -> dwfmm_status {
    if (!P.have_tree) dw::fail(DWFMM_ERR_STATE, "evaluate before tree_build");
    if (nrhs < 1 || nrhs > P.max_rhs) dw::fail(DWFMM_ERR_INVALID_ARG, "nrhs outside 1..max_rhs");
    if (nt < 0) dw::fail(DWFMM_ERR_INVALID_ARG, "nt < 0");
    if (nt == 0 || P.N == 0) return DWFMM_OK;
    if (!targets || !c || !out || ld_t < P.d || ld_c < P.N || ld_o < nt)
      dw::fail(DWFMM_ERR_INVALID_ARG, "NULL buffer or leading dimension too small");
    bind_stream(P, stream);
    const size_t ntr = static_cast<size_t>(nt) * nrhs;
    dw::DBuf<double> ts, cs, os;
    const double* td = targets;
    const double* cd = c;
    double* od = out;
    int64_t lt = ld_t, lc = ld_c, lo = ld_o;
    if (!is_device_pointer(targets)) {
      // the d used columns of each row only (a host buffer may end right after them)
      ts.alloc(static_cast<size_t>(nt) * P.d);
      DW_CUDA(cudaMemcpy2DAsync(ts.p, sizeof(double) * P.d, targets, sizeof(double) * ld_t, sizeof(double) * P.d, nt,
                                cudaMemcpyHostToDevice, P.stream));
      td = ts.p;
      lt = P.d;
    }
    if (!is_device_pointer(c)) {
      cs.alloc(static_cast<size_t>(P.N) * nrhs);
      DW_CUDA(cudaMemcpy2DAsync(cs.p, P.N * sizeof(double), c, ld_c * sizeof(double), P.N * sizeof(double), nrhs,
                                cudaMemcpyHostToDevice, P.stream));
      cd = cs.p;
      lc = P.N;
    }
    const bool oh = !is_device_pointer(out);
    if (oh) {
      os.alloc(ntr);
      od = os.p;
      lo = nt;
    }
    dw::evaluate(P, td, nt, lt, cd, lc, od, lo, nrhs);
    if (oh)
      DW_CUDA(cudaMemcpy2DAsync(out, ld_o * sizeof(double), od, nt * sizeof(double), nt * sizeof(double), nrhs,
                                cudaMemcpyDeviceToHost, P.stream));
    DW_CUDA(cudaStreamSynchronize(P.stream));
    dw::check_device_error(P);
    return DWFMM_OK;
  });
}

struct dwfmm_batch_s {
  dw::Batch* B = nullptr;
};

dwfmm_status dwfmm_batch_create(const dwfmm_plan* plans, const int32_t* nrhs, int32_t count, void* stream,
                                dwfmm_batch* out) {
  if (!plans || !nrhs || !out || count < 1) return DWFMM_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<Plan*> ps(count);
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) return DWFMM_ERR_INVALID_ARG;
    ps[i] = &plans[i]->P;
  }
  dw::Batch* b = dw::batch_new();
  const dwfmm_status st = guarded(ps[0], [&]() -> dwfmm_status {
    if (stream) DW_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    dw::batch_create(*b, ps.data(), nrhs, count);
    return DWFMM_OK;
  });
  if (st != DWFMM_OK) {
    dw::batch_delete(b);
    return st;
  }
  *out = new dwfmm_batch_s{b};
  return DWFMM_OK;
}

dwfmm_status dwfmm_batch_matvec(dwfmm_batch batch, const double* const* x, double* const* y, void* stream) {
  if (!batch || !x || !y) return DWFMM_ERR_INVALID_ARG;
  return guarded(nullptr, [&]() -> dwfmm_status {
    dw::batch_matvec(*batch->B, x, y, static_cast<cudaStream_t>(stream));
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_batch_cg_step(dwfmm_batch batch, int32_t iters, void* stream) {
  if (!batch) return DWFMM_ERR_INVALID_ARG;
  return guarded(nullptr, [&]() -> dwfmm_status {
    dw::batch_cg_step(*batch->B, iters, static_cast<cudaStream_t>(stream));
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_batch_info(dwfmm_batch batch, int32_t* split, double* tune_ms, int64_t* leaves) {
  if (!batch) return DWFMM_ERR_INVALID_ARG;
  dw::batch_info(*batch->B, split, tune_ms, leaves);
  return DWFMM_OK;
}

dwfmm_status dwfmm_batch_shape(dwfmm_batch batch, int32_t* shape) {
  if (!batch || !shape) return DWFMM_ERR_INVALID_ARG;
  dw::batch_shape(*batch->B, shape);
  return DWFMM_OK;
}

dwfmm_status dwfmm_batch_engine(dwfmm_batch batch, int32_t* engine, double* ms, int32_t* launch) {
  if (!batch || !engine || !ms || !launch) return DWFMM_ERR_INVALID_ARG;
  dw::batch_engine(*batch->B, engine, ms, launch);
  return DWFMM_OK;
}

dwfmm_status dwfmm_batch_set_engine(dwfmm_batch batch, int32_t engine) {
  if (!batch || engine < 0 || engine > 1) return DWFMM_ERR_INVALID_ARG;
  return guarded(nullptr, [&]() -> dwfmm_status {
    dw::batch_set_engine(*batch->B, engine);
    return DWFMM_OK;
  });
}

dwfmm_status dwfmm_batch_destroy(dwfmm_batch batch) {
  if (!batch) return DWFMM_OK;
  dw::batch_delete(batch->B);
  delete batch;
  return DWFMM_OK;
}

dwfmm_status dwfmm_direct_sum_noalloc(int32_t kernel, double sigma, const double* pts, int64_t n, int32_t d,
                                      int64_t ld_pts, const double* x, double* y, int32_t nrhs, int64_t ldx,
                                      int64_t ldy, void* stream) {
  return guarded(nullptr, [&]() -> dwfmm_status {
    return dw::direct_sum_noalloc(kernel, sigma, pts, n, d, ld_pts, x, y, nrhs, ldx, ldy,
                                  static_cast<cudaStream_t>(stream));
  });
}

}  // extern "C"
