// Orchestration of one DW-FMM matvec y = K_tilde x (Eq. (5.4)):
//   gather x into leaf blocks -> fork
//     side stream: P2P over the nearfield
//     main stream: P2M, M2M (levels J..jmin), M2L, L2L + L2P (levels jmin..J)
//   -> join -> scatter near + far into the caller's order.
// Right-hand sides are processed in passes of kRC columns.
#include <algorithm>

#include "dwfmm_internal.cuh"

namespace dw {

void timer_begin(Plan& P, int phase, cudaStream_t s) {
  if (!P.tm.on) return;
  cudaEvent_t a;
  DW_CUDA(cudaEventCreate(&a));
  DW_CUDA(cudaEventRecord(a, s));
  if (static_cast<int>(P.tm.open.size()) < 8) P.tm.open.assign(8, nullptr);
  P.tm.open[phase] = a;
}

void timer_end(Plan& P, int phase, cudaStream_t s, int launches) {
  if (!P.tm.on || P.tm.open.empty() || !P.tm.open[phase]) return;
  cudaEvent_t b;
  DW_CUDA(cudaEventCreate(&b));
  DW_CUDA(cudaEventRecord(b, s));
  P.tm.recs.push_back(TimerRec{phase, P.tm.open[phase], b, launches});
  P.tm.open[phase] = nullptr;
}

void timers_collect(Plan& P) {
  for (auto& r : P.tm.recs) {
    DW_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    DW_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    P.tm.ms[r.phase] += ms;
    P.tm.launches[r.phase] += r.launches;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  P.tm.recs.clear();
}

void ensure_workspace(Plan& P, bool fp64) {
  const size_t nl = static_cast<size_t>(P.L) * kRC * P.m_pad;
  const size_t nc = static_cast<size_t>(P.C) * kRC * P.n_pad;
  if (fp64) {
    P.xb64.alloc(nl);
    P.ynear64.alloc(nl);
    P.yfar64.alloc(nl);
    P.mom64.alloc(nc);
    P.loc64.alloc(nc);
    P.lco64.alloc(nc);
  } else {
    P.xb32.alloc(nl);
    P.ynear32.alloc(nl);
    P.yfar32.alloc(nl);
    P.mom32.alloc(nc);
    P.loc32.alloc(nc);
    P.lco32.alloc(nc);
  }
}

void matvec_device(Plan& P, const double* x, int64_t ldx, double* y, int64_t ldy, int R, bool fp64) {
  if (P.N == 0 || R == 0) return;
  ensure_workspace(P, fp64);
  cudaStream_t s = P.stream;
  timer_begin(P, 6, s);
  for (int r0 = 0; r0 < R; r0 += kRC) {
    const int Rc = std::min(kRC, R - r0);
    timer_begin(P, 0, s);
    launch_gather(P, x, ldx, r0, Rc, fp64);
    timer_end(P, 0, s, 1);
    if (!fp64) m2l_autotune(P, Rc);   // once per tree, before the near field starts
    if (P.tm.on && P.tm.serialize) {  // every phase alone on the caller's stream
      launch_farfield(P, Rc, fp64);
      timer_begin(P, 4, s);
      launch_nearfield(P, Rc, fp64, s);
      timer_end(P, 4, s, 1);
    } else {
      DW_CUDA(cudaEventRecord(P.ev_fork, s));
      DW_CUDA(cudaStreamWaitEvent(P.side, P.ev_fork, 0));
      timer_begin(P, 4, P.side);
      launch_nearfield(P, Rc, fp64, P.side);
      timer_end(P, 4, P.side, 1);
      DW_CUDA(cudaEventRecord(P.ev_join, P.side));
      launch_farfield(P, Rc, fp64);
      DW_CUDA(cudaStreamWaitEvent(s, P.ev_join, 0));
    }
    timer_begin(P, 5, s);
    launch_scatter(P, y, ldy, r0, Rc, fp64);
    timer_end(P, 5, s, 1);
  }
  timer_end(P, 6, s, 0);
}

}  // namespace dw
