// C ABI of the library (declared in include/sipg.h): handle and workspace
// management, the V-cycle of Sec. 3 and the flexible CG outer solver.
// All device memory is caller-owned; every kernel launch is ordered on the
// caller's stream (or, for CUDA-graph replay, on an internal stream joined to
// it by events).
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <tuple>
#include <vector>

#include "sipg_internal.cuh"

cudaError_t smem_opt_in(const void* kernel, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::set<std::tuple<const void*, int, int>> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(std::make_tuple(kernel, dev, bytes))) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert(std::make_tuple(kernel, dev, bytes));
  return e;
}

cudaError_t smem_opt_in_occupancy(const void* kernel, int threads, int bytes, int* ctas_per_sm) {
  cudaError_t e = smem_opt_in(kernel, bytes);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, int>, int> known;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(kernel, dev, threads, bytes);
  auto it = known.find(key);
  if (it != known.end()) {
    *ctas_per_sm = it->second;
    return cudaSuccess;
  }
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, (size_t)bytes);
  if (e != cudaSuccess) return e;
  known[key] = nb;
  *ctas_per_sm = nb;
  return cudaSuccess;
}

namespace {

const char* kVersion = "sipg-gb300 0.1 (sm_103a)";

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

sipg_status fail(sipg_handle* h, sipg_status st, const char* msg) {
  if (h) h->err = msg;
  return st;
}

sipg_status cuda_fail(sipg_handle* h, cudaError_t e, const char* where) {
  if (h) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    h->err = buf;
  }
  return SIPG_ECUDA;
}

#define SIPG_CHECK(expr, where)                 \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

sipg_status need_bound(sipg_handle* h) {
  if (!h) return SIPG_EINVAL;
  if (!h->bound) return fail(h, SIPG_ESTATE, "workspace not bound");
  return SIPG_OK;
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

size_t vec_bytes(const sipg_handle* h, int level, size_t elem) {
  return align256(h->lv[level].ndofs * (size_t)h->prm.nrhs * elem);
}

// ------------------------------------------------------------------ V-cycle
template <typename T>
sipg_status smooth_T(sipg_handle* h, int level, int reverse, const T* b, T* x, cudaStream_t s) {
  int nl = 0;
  SIPG_CHECK(launch_smooth_step<T>(h, level, reverse, b, x, s, &nl), "smoother");
  h->launches += nl;
  return SIPG_OK;
}

template <typename T>
sipg_status vcycle_T(sipg_handle* h, const T* bL, T* xL, cudaStream_t s) {
  const int L = h->L;
  const int nr = h->prm.nrhs;
  auto bvec = [&](int l) -> T* { return (l == L) ? const_cast<T*>(bL) : reinterpret_cast<T*>(h->vb(l)); };
  auto xvec = [&](int l) -> T* { return (l == L) ? xL : reinterpret_cast<T*>(h->vx(l)); };
  for (int l = L; l >= 1; --l) {
    T* b = bvec(l);
    T* x = xvec(l);
    SIPG_CHECK(cudaMemsetAsync(x, 0, h->lv[l].ndofs * nr * sizeof(T), s), "memset");
    sipg_status st = smooth_T<T>(h, l, 0, b, x, s);
    if (st) return st;
    cudaError_t e = launch_residual_restrict<T>(h, l, b, x, bvec(l - 1), s);
    if (e == cudaSuccess) {
      h->launches += 1;
      continue;
    }
    if (e != cudaErrorNotSupported) return cuda_fail(h, e, "residual and restriction");
    cudaGetLastError();
    T* r = reinterpret_cast<T*>(h->vr(l));
    SIPG_CHECK(launch_apply<T>(h, l, APPLY_RESIDUAL, b, x, r, s), "residual");
    SIPG_CHECK(launch_restrict<T>(h, l, r, bvec(l - 1), s), "restrict");
    h->launches += 2;
  }
  SIPG_CHECK(launch_coarse_solve<T>(h, bvec(0), xvec(0), s), "coarse solve");
  h->launches += 1;
  for (int l = 1; l <= L; ++l) {
    SIPG_CHECK(launch_prolongate_add<T>(h, l, xvec(l - 1), xvec(l), s), "prolongate");
    h->launches += 1;
    sipg_status st = smooth_T<T>(h, l, 1, bvec(l), xvec(l), s);
    if (st) return st;
  }
  return SIPG_OK;
}

// z = B r for the Krylov residual in kr(); leaves the preconditioned vector
// either in kz() (FP64 V-cycle) or in the FP32 finest-level buffer.
sipg_status precondition(sipg_handle* h, int first, cudaStream_t s) {
  sipg_status st;
  if (h->prm.vcycle_precision == SIPG_FP32) {
    float* bL = reinterpret_cast<float*>(h->ws + h->off_bL);
    float* xL = reinterpret_cast<float*>(h->ws + h->off_xL);
    if (first) {
      SIPG_CHECK(convert_d2f(h->kr(), bL, h->lv[h->L].ndofs * h->prm.nrhs, s), "convert");
      h->launches += 1;
    }
    st = vcycle_T<float>(h, bL, xL, s);
    if (st) return st;
    SIPG_CHECK(krylov_after_precond(h, first, h->kr(), xL, 1, s), "precond post");
  } else {
    st = vcycle_T<double>(h, h->kr(), h->kz(), s);
    if (st) return st;
    SIPG_CHECK(krylov_after_precond(h, first, h->kr(), h->kz(), 0, s), "precond post");
  }
  return SIPG_OK;
}

// q = A p, alpha, x += alpha p, r -= alpha q, ||r||^2 (and the FP32 copy of r).
sipg_status step_update(sipg_handle* h, double* x, cudaStream_t s) {
  SIPG_CHECK(launch_apply<double>(h, h->L, APPLY_Y, nullptr, h->kp(), h->kq(), s), "apply");
  h->launches += 1;
  SIPG_CHECK(krylov_after_apply(h, s), "pq");
  if (h->prm.vcycle_precision == SIPG_FP32)
    SIPG_CHECK(krylov_update_xr(h, x, h->ws + h->off_bL, 1, s), "update");
  else
    SIPG_CHECK(krylov_update_xr(h, x, nullptr, 0, s), "update");
  return SIPG_OK;
}

sipg_status iteration_body(sipg_handle* h, double* x, cudaStream_t s) {
  sipg_status st = precondition(h, 0, s);
  if (st) return st;
  return step_update(h, x, s);
}

// Capture one iteration body as a CUDA graph (on the internal stream).
sipg_status ensure_graph(sipg_handle* h, double* x) {
  // (the tolerance is a kernel argument of the captured convergence test)
  if (h->iter_exec && h->g_x == x && h->g_rtol2 == h->rtol2) return SIPG_OK;
  if (h->iter_exec) {
    cudaGraphExecDestroy(h->iter_exec);
    h->iter_exec = nullptr;
  }
  if (!h->gstream) SIPG_CHECK(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking), "stream");
  if (!h->ev_a) SIPG_CHECK(cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming), "event");
  if (!h->ev_b) SIPG_CHECK(cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming), "event");
  uint64_t before = h->launches;
  SIPG_CHECK(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal), "begin capture");
  sipg_status st = iteration_body(h, x, h->gstream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->gstream, &graph);
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
  e = cudaGraphInstantiate(&h->iter_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
  h->graph_launches = h->launches - before;
  h->launches = before;
  h->g_x = x;
  h->g_rtol2 = h->rtol2;
  return SIPG_OK;
}

sipg_status run_body(sipg_handle* h, double* x, cudaStream_t s) {
  if (!h->prm.use_graphs) return iteration_body(h, x, s);
  sipg_status st = ensure_graph(h, x);
  if (st) return st;
  SIPG_CHECK(cudaEventRecord(h->ev_a, s), "event record");
  SIPG_CHECK(cudaStreamWaitEvent(h->gstream, h->ev_a, 0), "stream wait");
  SIPG_CHECK(cudaGraphLaunch(h->iter_exec, h->gstream), "graph launch");
  SIPG_CHECK(cudaEventRecord(h->ev_b, h->gstream), "event record");
  SIPG_CHECK(cudaStreamWaitEvent(s, h->ev_b, 0), "stream wait");
  h->launches += h->graph_launches;
  return SIPG_OK;
}

// Flexible CG as a state machine, so that several independent problems (a
// batch) can advance in lockstep, each on its own stream: every step launches
// GPU work and an asynchronous copy of the Krylov scalars, the driver waits
// once for all pending problems, then each problem takes its host decision.
// For one problem the launch sequence is: true residual; first direction;
// iterations until convergence, breakdown or maxit; true residual again
// (restarting, at most 4 times, if the recursively updated residual drifted
// below the true one).
struct FcgRun {
  sipg_handle* h = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  cudaStream_t s = nullptr;
  int maxit = 0;
  sipg_info* info = nullptr;
  enum Phase { INITIAL, FIRST, ITERATE, VERIFY, DONE } phase = INITIAL;
  bool pending = false;     // GPU work in flight whose scalars must be read
  int it = 0, restarts = 0;
  sipg_status result = SIPG_OK;
  std::vector<double> hist;
  bool zero_start = false;  // x = 0 on entry: the first residual is b
  // optional copy of x to host memory overlapped with the final true
  // residual: issued on out_stream as soon as the iteration ends; a restart
  // waits for it before it changes x, and marks it stale
  double* out_host = nullptr;
  size_t out_bytes = 0;
  cudaStream_t out_stream = nullptr;
  cudaEvent_t out_ready = nullptr, out_done = nullptr;
  bool out_valid = false;  // the copy in flight holds the x the run ends with
};

sipg_status copy_out(FcgRun& r) {
  sipg_handle* h = r.h;
  SIPG_CHECK(cudaEventRecord(r.out_ready, r.s), "event record");
  SIPG_CHECK(cudaStreamWaitEvent(r.out_stream, r.out_ready, 0), "stream wait");
  SIPG_CHECK(cudaMemcpyAsync(r.out_host, r.x, r.out_bytes, cudaMemcpyDeviceToHost, r.out_stream), "D2H");
  SIPG_CHECK(cudaEventRecord(r.out_done, r.out_stream), "event record");
  r.out_valid = true;
  return SIPG_OK;
}

bool run_any(const sipg_handle* h, bool (*pred)(const KrylovScalars&)) {
  for (int c = 0; c < h->prm.nrhs; ++c)
    if (pred(h->pinned[c])) return true;
  return false;
}
bool is_active(const KrylovScalars& k) { return k.active != 0; }
bool is_broken(const KrylovScalars& k) { return k.breakdown != 0; }

sipg_status queue_scalars(FcgRun& r) {
  sipg_handle* h = r.h;
  SIPG_CHECK(cudaMemcpyAsync(h->pinned, h->scalars(), sizeof(KrylovScalars) * h->prm.nrhs, cudaMemcpyDeviceToHost,
                             r.s),
             "scalars D2H");
  r.pending = true;
  return SIPG_OK;
}

sipg_status launch_true_residual(FcgRun& r) {
  sipg_handle* h = r.h;
  if (r.zero_start && r.phase == FcgRun::INITIAL) {
    // x = 0: r = b without an operator apply
    const size_t bytes = h->lv[h->L].ndofs * h->prm.nrhs * sizeof(double);
    SIPG_CHECK(cudaMemsetAsync(r.x, 0, bytes, r.s), "memset");
    SIPG_CHECK(cudaMemcpyAsync(h->kr(), r.b, bytes, cudaMemcpyDeviceToDevice, r.s), "copy");
  } else {
    SIPG_CHECK(launch_apply<double>(h, h->L, APPLY_RESIDUAL, r.b, r.x, h->kr(), r.s), "residual");
    h->launches += 1;
  }
  SIPG_CHECK(krylov_init_norms(h, r.b, h->kr(), r.s), "norms");
  return queue_scalars(r);
}

// Host decisions after the scalars of the last step arrived; launches the
// next step (or finishes the run).
sipg_status advance(FcgRun& r) {
  sipg_handle* h = r.h;
  sipg_status st = SIPG_OK;
  switch (r.phase) {
    case FcgRun::INITIAL:
      if (!r.pending) return launch_true_residual(r);
      r.pending = false;
      r.hist.push_back(sqrt(h->pinned[0].rr));
      r.phase = FcgRun::VERIFY;
      r.restarts = -1;  // the initial residual is not a restart
      return advance(r);
    case FcgRun::VERIFY:
      // true residual known: finish, or (re)start the iteration
      r.pending = false;
      ++r.restarts;
      if (run_any(h, is_broken)) {
        r.result = SIPG_EBREAKDOWN;
        r.phase = FcgRun::DONE;
        return SIPG_OK;
      }
      if (!run_any(h, is_active) || r.it >= r.maxit || r.restarts >= 4) {
        r.phase = FcgRun::DONE;
        return SIPG_OK;
      }
      if (r.out_valid) {  // x changes again: the copy in flight is stale
        SIPG_CHECK(cudaStreamWaitEvent(r.s, r.out_done, 0), "stream wait");
        r.out_valid = false;
      }
      st = precondition(h, 1, r.s);  // z_0 = B r_0, p_0 = z_0
      if (st) return st;
      st = step_update(h, r.x, r.s);
      if (st) return st;
      r.phase = FcgRun::FIRST;
      return queue_scalars(r);
    case FcgRun::FIRST:
    case FcgRun::ITERATE:
      r.pending = false;
      ++r.it;
      r.hist.push_back(sqrt(h->pinned[0].rr));
      if (run_any(h, is_broken)) {
        r.result = SIPG_EBREAKDOWN;
        r.phase = FcgRun::DONE;
        return SIPG_OK;
      }
      if (run_any(h, is_active) && r.it < r.maxit) {
        st = run_body(h, r.x, r.s);
        if (st) return st;
        r.phase = FcgRun::ITERATE;
        return queue_scalars(r);
      }
      r.phase = FcgRun::VERIFY;
      if (r.out_host) {
        st = copy_out(r);
        if (st) return st;
      }
      return launch_true_residual(r);
    case FcgRun::DONE:
      return SIPG_OK;
  }
  return SIPG_OK;
}

sipg_status finish(FcgRun& r) {
  sipg_handle* h = r.h;
  const int nr = h->prm.nrhs;
  const KrylovScalars* sc = h->pinned;
  sipg_status result = r.result;
  if (result == SIPG_OK && run_any(h, is_broken)) result = SIPG_EBREAKDOWN;
  double worst = 0.0;
  bool all_conv = true;
  for (int c = 0; c < nr; ++c) {
    double rel = sc[c].bb > 0.0 ? sqrt(sc[c].rr / sc[c].bb) : 0.0;
    worst = std::max(worst, rel);
    if (sc[c].active) all_conv = false;
  }
  if (result == SIPG_OK && !all_conv) result = SIPG_ENOCONV;
  sipg_info* info = r.info;
  if (info) {
    info->iterations = r.it;
    info->status = result;
    info->rel_residual = worst;
    double nu = 0.0;
    if (r.it > 0 && r.hist.size() > 1 && r.hist.front() > 0.0) {
      double rbar = pow(r.hist.back() / r.hist.front(), 1.0 / (double)(r.hist.size() - 1));
      nu = (rbar > 0.0 && rbar < 1.0) ? -8.0 / log10(rbar) : INFINITY;
    }
    info->nu = nu;
    int cnt = 0;
    if (info->history && info->history_capacity > 0) {
      cnt = std::min((int)r.hist.size(), info->history_capacity);
      for (int i = 0; i < cnt; ++i) info->history[i] = r.hist[i];
    }
    info->history_len = cnt;
  }
  {
    // a bounded grid-barrier wait that ran out (fused smoothing steps)
    int status = 0;
    SIPG_CHECK(cudaMemcpyAsync(&status, h->ws + h->off_sync + 2 * sizeof(unsigned int), sizeof(int),
                               cudaMemcpyDeviceToHost, r.s),
               "status D2H");
    SIPG_CHECK(cudaStreamSynchronize(r.s), "sync");
    if (status != 0) {
      SIPG_CHECK(cudaMemsetAsync(h->ws + h->off_sync, 0, 256, r.s), "memset");
      h->err = "a bounded grid-barrier wait in the smoother timed out";
      if (info) info->status = SIPG_ETIMEOUT;
      return SIPG_ETIMEOUT;
    }
  }
  if (result == SIPG_ENOCONV) h->err = "solver reached maxit before rtol";
  if (result == SIPG_EBREAKDOWN) h->err = "Krylov breakdown (non-finite or non-positive scalar)";
  return result;
}

// Drive several runs to completion; the first CUDA-level failure aborts.
sipg_status drive(std::vector<FcgRun>& runs) {
  for (auto& r : runs) {
    sipg_status st = advance(r);
    if (st) return st;
  }
  for (;;) {
    bool any = false;
    for (auto& r : runs) {
      if (!r.pending) continue;
      any = true;
      cudaError_t e = cudaStreamSynchronize(r.s);
      if (e != cudaSuccess) return cuda_fail(r.h, e, "sync");
    }
    if (!any) break;
    for (auto& r : runs) {
      if (!r.pending) continue;
      sipg_status st = advance(r);
      if (st) return st;
    }
  }
  return SIPG_OK;
}

// out_host: also copy the final x there (out_stream, events: see FcgRun);
// on return *out_copied says whether a copy of the final x was issued (the
// caller then waits for out_stream, else copies x itself).
sipg_status fcg_solve(sipg_handle* h, const double* b, double* x, double rtol, int maxit,
                      sipg_info* info, cudaStream_t s, bool zero_start = false, double* out_host = nullptr,
                      cudaStream_t out_stream = nullptr, cudaEvent_t out_ready = nullptr,
                      cudaEvent_t out_done = nullptr, bool* out_copied = nullptr) {
  h->rtol2 = rtol * rtol;
  std::vector<FcgRun> runs(1);
  runs[0].zero_start = zero_start;
  runs[0].h = h;
  runs[0].b = b;
  runs[0].x = x;
  runs[0].s = s;
  runs[0].maxit = maxit;
  runs[0].info = info;
  if (out_host) {
    runs[0].out_host = out_host;
    runs[0].out_bytes = h->lv[h->L].ndofs * h->prm.nrhs * sizeof(double);
    runs[0].out_stream = out_stream;
    runs[0].out_ready = out_ready;
    runs[0].out_done = out_done;
  }
  sipg_status st = drive(runs);
  if (out_copied) *out_copied = runs[0].out_valid;
  if (st) return st;
  return finish(runs[0]);
}

// ------------------------------------------------------------------ GMRES
// Caller-owned workspace of sipg_gmres_solve: Arnoldi vectors V_0..V_m and
// preconditioned vectors Z_0..Z_{m-1} (finest level, FP64, each 256-byte
// aligned), reduction partials for m+1 simultaneous dot products, m+1
// device scalars, the device state of one restart cycle.
struct GmresLayout {
  size_t vec = 0, off_z = 0, off_part = 0, off_dev = 0, off_state = 0, total = 0;
};

GmresLayout gmres_layout(const sipg_handle* h, int m) {
  GmresLayout g;
  g.vec = align256(h->lv[h->L].ndofs * sizeof(double));
  g.off_z = (size_t)(m + 1) * g.vec;
  g.off_part = g.off_z + (size_t)m * g.vec;
  g.off_dev = g.off_part + align256(sizeof(double) * (size_t)(m + 1) * h->n_partials);
  g.off_state = g.off_dev + align256(sizeof(double) * (size_t)(m + 1));
  g.total = g.off_state + align256(sizeof(GmresCycleState));
  return g;
}

// z = B v, one V-cycle: FP32 through the finest-level buffers, or FP64.
sipg_status gmres_precond(sipg_handle* h, const double* v, double* z, cudaStream_t s) {
  const size_t n = h->lv[h->L].ndofs;
  if (h->prm.vcycle_precision == SIPG_FP32) {
    float* bL = reinterpret_cast<float*>(h->ws + h->off_bL);
    float* xL = reinterpret_cast<float*>(h->ws + h->off_xL);
    SIPG_CHECK(convert_d2f(v, bL, n, s), "convert");
    h->launches += 1;
    sipg_status st = vcycle_T<float>(h, bL, xL, s);
    if (st) return st;
    SIPG_CHECK(convert_f2d(xL, z, n, s), "convert");
    h->launches += 1;
    return SIPG_OK;
  }
  return vcycle_T<double>(h, v, z, s);
}

struct GmresVectors {
  sipg_handle* h;
  cudaStream_t s;
  long long n, ld;  // vector length, distance between consecutive vectors
  double* V;
  double* Z;
  double* part;
  double* dev;
  double* v(int j) const { return V + (long long)j * ld; }
  double* z(int j) const { return Z + (long long)j * ld; }
  // out[i] = <Vb + i ld, w> for i < cnt, copied to the host
  sipg_status dots(const double* Vb, int cnt, const double* w, double* out) {
    SIPG_CHECK(gmres_mdot(h, Vb, ld, cnt, w, n, part, dev, s), "dot");
    SIPG_CHECK(cudaMemcpyAsync(out, dev, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s), "D2H");
    SIPG_CHECK(cudaStreamSynchronize(s), "sync");
    return SIPG_OK;
  }
  bool left = false;  // preconditioned from the left: the residual is B (b - A x)
  // V_0 = b - A x (left: B (b - A x), through Z_0), *beta = ||V_0||_2
  sipg_status residual(const double* b, const double* x, double* beta) {
    SIPG_CHECK(launch_apply<double>(h, h->L, APPLY_RESIDUAL, b, x, V, s), "residual");
    h->launches += 1;
    if (left) {
      sipg_status st = gmres_precond(h, V, Z, s);
      if (st) return st;
      SIPG_CHECK(cudaMemcpyAsync(V, Z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s), "copy");
    }
    double rr = 0.0;
    sipg_status st = dots(V, 1, V, &rr);
    if (st) return st;
    *beta = sqrt(rr);
    return SIPG_OK;
  }
};

// One Arnoldi step of a device-resident cycle (j read from st by every
// kernel).  Right: z_j = B v_j into Z_j, w = A z_j; left: w = B A v_j.  The
// finest-level Krylov vectors of the handle (unused by GMRES otherwise) are
// the scratch: T0, T1 = w, T2.  Then classical Gram-Schmidt applied twice,
// ||w||^2, the rotations on the device, v_{j+1} = w / ||w||.
sipg_status gmres_step_body(sipg_handle* h, const GmresVectors& g, int m, GmresCycleState* st,
                            cudaGraphConditionalHandle cond, cudaStream_t s) {
  double* T0 = h->kp();
  double* T1 = h->kq();
  double* T2 = h->kz();
  const long long n = g.n;
  const bool f32 = h->prm.vcycle_precision == SIPG_FP32;
  float* bL = reinterpret_cast<float*>(h->ws + h->off_bL);
  float* xL = reinterpret_cast<float*>(h->ws + h->off_xL);
  sipg_status st_ = SIPG_OK;
  if (!g.left) {
    if (f32) {
      SIPG_CHECK(gmres_gather(h, g.V, g.ld, st, bL, true, n, s), "gather");
      st_ = vcycle_T<float>(h, bL, xL, s);
      if (st_) return st_;
      SIPG_CHECK(gmres_put(h, xL, true, g.Z, g.ld, st, T0, n, s), "put");
    } else {
      SIPG_CHECK(gmres_gather(h, g.V, g.ld, st, T0, false, n, s), "gather");
      st_ = vcycle_T<double>(h, T0, T2, s);
      if (st_) return st_;
      SIPG_CHECK(gmres_put(h, T2, false, g.Z, g.ld, st, nullptr, n, s), "put");
    }
    SIPG_CHECK(launch_apply<double>(h, h->L, APPLY_Y, nullptr, f32 ? T0 : T2, T1, s), "apply");
    h->launches += 1;
  } else {
    SIPG_CHECK(gmres_gather(h, g.V, g.ld, st, T0, false, n, s), "gather");
    SIPG_CHECK(launch_apply<double>(h, h->L, APPLY_Y, nullptr, T0, T2, s), "apply");
    h->launches += 1;
    st_ = gmres_precond(h, T2, T1, s);
    if (st_) return st_;
  }
  for (int pass = 0; pass < 2; ++pass) {
    double* c = pass ? st->hc2 : st->hc1;
    SIPG_CHECK(gmres_mdot_dev(h, g.V, g.ld, st, m, T1, n, g.part, c, s), "dot");
    SIPG_CHECK(gmres_maxpy_dev(h, T1, g.V, g.ld, st, c, n, s), "axpy");
  }
  SIPG_CHECK(gmres_mdot(h, T1, g.ld, 1, T1, n, g.part, &st->nrm, s), "dot");
  SIPG_CHECK(gmres_rotate(h, st, cond, s), "rotate");
  SIPG_CHECK(gmres_next(h, T1, g.V, g.ld, st, n, s), "next");
  return SIPG_OK;
}

// The cycle graph: one conditional while node (condition 1 at launch) whose
// body, recorded by stream capture, is one Arnoldi step; the rotation kernel
// sets the condition.  Recorded once per workspace, restart length and side.
sipg_status gmres_ensure_graph(sipg_handle* h, const GmresVectors& g, int m, GmresCycleState* st) {
  const char* work = reinterpret_cast<const char*>(g.V);
  if (h->gm_exec && h->gm_work == work && h->gm_m == m && h->gm_left == g.left) return SIPG_OK;
  if (h->gm_exec) {
    cudaGraphExecDestroy(h->gm_exec);
    h->gm_exec = nullptr;
  }
  if (!h->gstream) SIPG_CHECK(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking), "stream");
  if (!h->ev_a) SIPG_CHECK(cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming), "event");
  if (!h->ev_b) SIPG_CHECK(cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming), "event");
  cudaGraph_t graph = nullptr;
  SIPG_CHECK(cudaGraphCreate(&graph, 0), "graph create");
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(h, e, "conditional node");
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const uint64_t before = h->launches;
  e = cudaStreamBeginCaptureToGraph(h->gstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(h, e, "begin capture");
  }
  sipg_status st_ = gmres_step_body(h, g, m, st, cond, h->gstream);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(h->gstream, &captured);
  if (st_ || e != cudaSuccess) {
    cudaGraphDestroy(graph);
    h->launches = before;
    if (st_) return st_;
    return cuda_fail(h, e, "end capture");
  }
  e = cudaGraphInstantiate(&h->gm_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->gm_exec = nullptr;
    h->launches = before;
    return cuda_fail(h, e, "graph instantiate");
  }
  h->gm_launches = h->launches - before;
  h->launches = before;
  h->gm_work = work;
  h->gm_m = m;
  h->gm_left = g.left;
  return SIPG_OK;
}

// One restart cycle on the device: clear the state, run the cycle graph,
// read the state back (the only host synchronisation of the cycle).
sipg_status gmres_device_cycle(sipg_handle* h, const GmresVectors& g, int m, GmresCycleState* st, double beta,
                               double thr, int budget, GmresCycleState* out) {
  sipg_status r = gmres_ensure_graph(h, g, m, st);
  if (r) return r;
  cudaStream_t s = g.s;
  SIPG_CHECK(gmres_cycle_setup(h, st, beta, thr, budget, s), "cycle setup");
  SIPG_CHECK(cudaEventRecord(h->ev_a, s), "event record");
  SIPG_CHECK(cudaStreamWaitEvent(h->gstream, h->ev_a, 0), "stream wait");
  SIPG_CHECK(cudaGraphLaunch(h->gm_exec, h->gstream), "graph launch");
  SIPG_CHECK(cudaEventRecord(h->ev_b, h->gstream), "event record");
  SIPG_CHECK(cudaStreamWaitEvent(s, h->ev_b, 0), "stream wait");
  SIPG_CHECK(cudaMemcpyAsync(out, st, sizeof(GmresCycleState), cudaMemcpyDeviceToHost, s), "D2H");
  SIPG_CHECK(cudaStreamSynchronize(s), "sync");
  h->launches += h->gm_launches * (uint64_t)std::max(out->runs, 0);
  return SIPG_OK;
}

sipg_status gmres_run(sipg_handle* h, const double* b, double* x, double rtol, int maxit, int m, char* work,
                      sipg_info* info, cudaStream_t s, bool left = false) {
  const GmresLayout lay = gmres_layout(h, m);
  GmresVectors g{h, s, (long long)h->lv[h->L].ndofs, (long long)(lay.vec / sizeof(double)),
                 reinterpret_cast<double*>(work), reinterpret_cast<double*>(work + lay.off_z),
                 reinterpret_cast<double*>(work + lay.off_part), reinterpret_cast<double*>(work + lay.off_dev)};
  g.left = left;
  double bb = 0.0, beta = 0.0;
  sipg_status st;
  if (left) {  // the norm the stopping test refers to: ||B b||
    st = gmres_precond(h, b, g.z(0), s);
    if (st) return st;
    st = g.dots(g.z(0), 1, g.z(0), &bb);
  } else {
    st = g.dots(b, 1, b, &bb);
  }
  if (st) return st;
  const double bnorm = sqrt(bb);
  st = g.residual(b, x, &beta);
  if (st) return st;
  std::vector<double> hist{beta};
  sipg_status result = (isfinite(bnorm) && isfinite(beta)) ? SIPG_OK : SIPG_EBREAKDOWN;
  bool conv = !(bnorm > 0.0) || beta <= rtol * bnorm;
  int steps = 0;
  // Hessenberg matrix (row-major, (m+1) x m), rotations, right-hand side
  std::vector<double> H((size_t)(m + 1) * m), gv(m + 1), cs(m), sn(m), y(m), hc(m + 1), tmp(m + 1);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  // with CUDA graphs on, every cycle runs on the device (one graph launch,
  // one host synchronisation per cycle); else the host drives every step
  const bool on_device = h->prm.use_graphs != 0;
  GmresCycleState* st_dev = reinterpret_cast<GmresCycleState*>(work + lay.off_state);
  std::unique_ptr<GmresCycleState> hs;
  if (on_device) hs.reset(new GmresCycleState());
  while (!conv && result == SIPG_OK && steps < maxit) {
    const int mc = std::min(m, maxit - steps);
    SIPG_CHECK(gmres_scale(h, g.v(0), 1.0 / beta, g.n, s), "scale");
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;  // completed steps of this cycle
    if (on_device) {
      st = gmres_device_cycle(h, g, m, st_dev, beta, rtol * bnorm, mc, hs.get());
      if (st) return st;
      j = std::min(std::max(hs->j, 0), mc);
      for (int i = 0; i < j; ++i) hist.push_back(hs->hist[i]);
      steps += j;
      if (hs->brk) result = SIPG_EBREAKDOWN;
      for (int i = 0; i <= j; ++i) {
        gv[i] = hs->g[i];
        for (int q = 0; q < j; ++q) Hat(i, q) = hs->H[i * SIPG_GMRES_MAXM + q];
      }
    }
    while (!on_device && j < mc) {
      if (left) {  // v_{j+1} = B A v_j (A v_j in Z_j)
        SIPG_CHECK(launch_apply<double>(h, h->L, APPLY_Y, nullptr, g.v(j), g.z(j), s), "apply");
        h->launches += 1;
        st = gmres_precond(h, g.z(j), g.v(j + 1), s);
        if (st) return st;
      } else {     // z_j = B v_j, v_{j+1} = A z_j
        st = gmres_precond(h, g.v(j), g.z(j), s);
        if (st) return st;
        SIPG_CHECK(launch_apply<double>(h, h->L, APPLY_Y, nullptr, g.z(j), g.v(j + 1), s), "apply");
        h->launches += 1;
      }
      // classical Gram-Schmidt, applied twice: w -= sum_i <V_i, w> V_i
      std::fill(hc.begin(), hc.end(), 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        SIPG_CHECK(gmres_mdot(h, g.V, g.ld, j + 1, g.v(j + 1), g.n, g.part, g.dev, s), "dot");
        SIPG_CHECK(gmres_maxpy(h, g.v(j + 1), g.V, g.ld, j + 1, g.dev, nullptr, -1.0, g.n, s), "axpy");
        SIPG_CHECK(cudaMemcpyAsync(tmp.data(), g.dev, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s),
                   "D2H");
        SIPG_CHECK(cudaStreamSynchronize(s), "sync");
        for (int i = 0; i <= j; ++i) hc[i] += tmp[i];
      }
      double ww = 0.0;
      st = g.dots(g.v(j + 1), 1, g.v(j + 1), &ww);
      if (st) return st;
      const double hn = sqrt(ww);
      bool finite = isfinite(hn);
      for (int i = 0; i <= j; ++i) finite = finite && isfinite(hc[i]);
      if (!finite) {
        result = SIPG_EBREAKDOWN;
        break;
      }
      for (int i = 0; i <= j; ++i) Hat(i, j) = hc[i];
      Hat(j + 1, j) = hn;
      if (hn > 0.0) SIPG_CHECK(gmres_scale(h, g.v(j + 1), 1.0 / hn, g.n, s), "scale");
      for (int i = 0; i < j; ++i) {  // rotations of the earlier steps
        const double a = Hat(i, j), c = Hat(i + 1, j);
        Hat(i, j) = cs[i] * a + sn[i] * c;
        Hat(i + 1, j) = -sn[i] * a + cs[i] * c;
      }
      const double den = hypot(Hat(j, j), Hat(j + 1, j));
      if (!(den > 0.0)) {
        result = SIPG_EBREAKDOWN;
        break;
      }
      cs[j] = Hat(j, j) / den;
      sn[j] = Hat(j + 1, j) / den;
      Hat(j, j) = den;
      Hat(j + 1, j) = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++j;
      ++steps;
      hist.push_back(fabs(gv[j]));
      if (fabs(gv[j]) <= rtol * bnorm || hn == 0.0) break;  // converged, or exact
    }
    if (j == 0) break;
    // y = R^{-1} g (back substitution), x += Z y, true residual
    for (int i = j - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int q = i + 1; q < j; ++q) acc -= Hat(i, q) * y[q];
      y[i] = acc / Hat(i, i);
    }
    SIPG_CHECK(gmres_maxpy(h, x, left ? g.V : g.Z, g.ld, j, nullptr, y.data(), 1.0, g.n, s), "update");
    st = g.residual(b, x, &beta);
    if (st) return st;
    hist.back() = beta;  // the true residual ends every cycle
    if (!isfinite(beta)) result = SIPG_EBREAKDOWN;
    conv = beta <= rtol * bnorm;
  }
  if (result == SIPG_OK && !conv) result = SIPG_ENOCONV;
  {
    // a bounded grid-barrier wait that ran out (fused smoothing steps)
    int status = 0;
    SIPG_CHECK(cudaMemcpyAsync(&status, h->ws + h->off_sync + 2 * sizeof(unsigned int), sizeof(int),
                               cudaMemcpyDeviceToHost, s),
               "status D2H");
    SIPG_CHECK(cudaStreamSynchronize(s), "sync");
    if (status != 0) {
      SIPG_CHECK(cudaMemsetAsync(h->ws + h->off_sync, 0, 256, s), "memset");
      result = SIPG_ETIMEOUT;
    }
  }
  if (info) {
    info->iterations = steps;
    info->status = result;
    info->rel_residual = bnorm > 0.0 ? beta / bnorm : 0.0;
    double nu = 0.0;
    if (hist.size() > 1 && hist.front() > 0.0) {
      double rbar = pow(hist.back() / hist.front(), 1.0 / (double)(hist.size() - 1));
      nu = (rbar > 0.0 && rbar < 1.0) ? -8.0 / log10(rbar) : INFINITY;
    }
    info->nu = nu;
    int cnt = 0;
    if (info->history && info->history_capacity > 0) {
      cnt = std::min((int)hist.size(), info->history_capacity);
      for (int i = 0; i < cnt; ++i) info->history[i] = hist[i];
    }
    info->history_len = cnt;
  }
  if (result == SIPG_ETIMEOUT) h->err = "a bounded grid-barrier wait in the smoother timed out";
  if (result == SIPG_ENOCONV) h->err = "GMRES reached maxit before rtol";
  if (result == SIPG_EBREAKDOWN) h->err = "GMRES breakdown (non-finite scalar)";
  return result;
}

// Autotuning of the smoothing step, per level: time each candidate launch
// path (colour by colour with the default or the half interior tile, or one
// fused launch where that applies) on the level's workspace vectors (zeroed;
// the arithmetic does not depend on the values) and keep the fastest.
template <typename T>
sipg_status tune_T(sipg_handle* h, cudaStream_t s) {
  const int pi = sizeof(T) == 4 ? 1 : 0;
  const int nl = h->L + 1;
  h->tune_path[pi].assign(nl, -1);
  h->tune_tile[pi].assign(nl, 0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SIPG_CHECK(cudaEventCreate(&e0), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(h, SIPG_ECUDA, "event");
  }
  sipg_status result = SIPG_OK;
  for (int l = 1; l <= h->L && result == SIPG_OK; ++l) {
    T* b = reinterpret_cast<T*>(h->vb(l));
    T* x = reinterpret_cast<T*>(h->vx(l));
    const size_t bytes = h->lv[l].ndofs * (size_t)h->prm.nrhs * sizeof(T);
    if (cudaMemsetAsync(b, 0, bytes, s) != cudaSuccess || cudaMemsetAsync(x, 0, bytes, s) != cudaSuccess) {
      result = fail(h, SIPG_ECUDA, "memset");
      break;
    }
    struct Cand {
      int path, tile;
    };
    std::vector<Cand> cands = {{1, 0}};
    if (h->prm.dim == 3 && sizeof(T) == 4) {
      cands.push_back({1, 1});
      cands.push_back({1, 2});
      cands.push_back({1, 3});
      cands.push_back({1, 4});
    }
    if (h->fuse_small_levels) cands.push_back({0, 0});
    float best = 1e30f;
    Cand pick = {-1, 0};
    for (const Cand& c : cands) {
      h->tune_path[pi][l] = c.path;
      h->tune_tile[pi][l] = c.tile;
      int launches = 0;
      cudaError_t e = launch_smooth_step<T>(h, l, 0, b, x, s, &launches);  // warm-up
      if (e != cudaSuccess) {
        result = cuda_fail(h, e, "autotune");
        break;
      }
      if (c.path == 0 && launches != 1) continue;  // no fused launch on this level
      float ms = 0.f;
      int reps = 1;
      for (int round = 0; round < 2; ++round) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_smooth_step<T>(h, l, 0, b, x, s, &launches);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        // second round: enough repetitions for about 0.3 ms
        reps = std::max(2, std::min(20, (int)(0.3f / std::max(ms / reps, 1e-4f))));
      }
      if (e != cudaSuccess) {
        result = cuda_fail(h, e, "autotune");
        break;
      }
      const float t = ms / reps;
      if (t < best) {
        best = t;
        pick = c;
      }
    }
    h->tune_path[pi][l] = pick.path;
    h->tune_tile[pi][l] = pick.tile;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != SIPG_OK) return result;
  // a fused launch whose bounded grid barrier gave up: keep colour-by-colour
  int status = 0;
  SIPG_CHECK(cudaMemcpyAsync(&status, h->ws + h->off_sync + 2 * sizeof(unsigned int), sizeof(int),
                             cudaMemcpyDeviceToHost, s),
             "status D2H");
  SIPG_CHECK(cudaStreamSynchronize(s), "sync");
  if (status != 0) {
    SIPG_CHECK(cudaMemsetAsync(h->ws + h->off_sync, 0, 256, s), "memset");
    for (int l = 1; l < nl; ++l) h->tune_path[pi][l] = 1;
  }
  return SIPG_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

const char* sipg_version(void) { return kVersion; }

sipg_status sipg_create(const sipg_params* p, sipg_handle** out) {
  if (!out) return SIPG_EINVAL;
  *out = nullptr;
  if (!p) return SIPG_EINVAL;
  if (p->dim != 2 && p->dim != 3) return SIPG_EINVAL;
  if (p->degree < 1 || p->degree > 7) return SIPG_EINVAL;
  if (p->log2_cells < 1 || p->log2_cells > (p->dim == 2 ? 14 : 10)) return SIPG_EINVAL;
  if (p->n_levels < 1 || p->n_levels > p->log2_cells) return SIPG_EINVAL;
  if (!(p->kappa > 0.0) || !isfinite(p->kappa)) return SIPG_EINVAL;
  if (!(p->penalty_factor > 0.0) || !isfinite(p->penalty_factor)) return SIPG_EINVAL;
  if (p->vcycle_precision != SIPG_FP64 && p->vcycle_precision != SIPG_FP32 && p->vcycle_precision != SIPG_TF32)
    return SIPG_EINVAL;
  if (p->smoother != SIPG_SMOOTHER_CONSISTENT && p->smoother != SIPG_SMOOTHER_PAPER &&
      p->smoother != SIPG_SMOOTHER_FULL && p->smoother != SIPG_SMOOTHER_CLAMPED)
    return SIPG_EINVAL;
  if (p->smoother == SIPG_SMOOTHER_CLAMPED && p->degree < 2) return SIPG_EINVAL;  // empty clamped space
  if (p->nrhs < 1 || p->nrhs > 65535) return SIPG_EINVAL;
  const int n = p->degree + 1;
  const int L = p->n_levels - 1;
  const int N = 1 << p->log2_cells;
  const int N0 = N >> L;
  if (N0 < 2) return SIPG_EINVAL;
  const int m0 = N0 * n;
  if (m0 > SIPG_MAXM0) return SIPG_EUNSUPPORTED;
  if (p->dim == 3 && m0 * m0 * m0 > 4096) return SIPG_EUNSUPPORTED;
  if (p->dim == 2 && m0 * m0 > 4096) return SIPG_EUNSUPPORTED;

  sipg_handle* h = new sipg_handle();
  h->prm = *p;
  // TF32: the FP32 V-cycle with tensor-core local solves where a kernel for
  // them exists; every other code path treats the handle as FP32
  h->tf32 = p->vcycle_precision == SIPG_TF32;
  if (h->tf32) h->prm.vcycle_precision = SIPG_FP32;
  // tuning knobs: SIPG_FUSED_SMOOTHING=0 launches small levels colour by
  // colour; SIPG_AUTOTUNE=0 skips the bind-time timing of the launch paths
  if (const char* env = getenv("SIPG_FUSED_SMOOTHING")) h->fuse_small_levels = atoi(env) != 0;
  if (const char* env = getenv("SIPG_AUTOTUNE")) h->autotune = atoi(env) != 0;
  if (const char* env = getenv("SIPG_BOUNDARY_FIRST")) h->bnd_first = atoi(env) != 0;
  if (const char* env = getenv("SIPG_TILE")) {
    const int t = atoi(env);
    h->force_tile = (t >= 0 && t <= 4) ? t : 0;
  }
  h->n = n;
  h->L = L;
  for (int l = 0; l <= L; ++l) {
    LevelInfo li;
    li.N = N >> (L - l);
    li.ncells = 1;
    for (int e = 0; e < p->dim; ++e) li.ncells *= (size_t)li.N;
    size_t nd = 1;
    for (int e = 0; e < p->dim; ++e) nd *= (size_t)n;
    li.ndofs = li.ncells * nd;
    h->lv.push_back(li);
  }
  // workspace layout
  size_t off = 0;
  const int nl = L + 1;
  h->off_const64 = off;
  off += align256(sizeof(LevelConst<double>) * nl);
  h->off_const32 = off;
  off += align256(sizeof(LevelConst<float>) * nl);
  h->off_scratch_setup = off;
  off += align256(256 + 5 * SIPG_MAXM0 * SIPG_MAXM0 * sizeof(double));
  h->n_partials = 1024;
  h->off_partials = off;
  off += align256(sizeof(double) * 3 * h->n_partials * p->nrhs);
  h->off_scalars = off;
  off += align256(sizeof(KrylovScalars) * p->nrhs);
  h->off_sync = off;
  off += 256;
  h->off_kr = off;
  off += vec_bytes(h, L, 8);
  h->off_kz = off;
  off += vec_bytes(h, L, 8);
  h->off_kp = off;
  off += vec_bytes(h, L, 8);
  h->off_kq = off;
  off += vec_bytes(h, L, 8);
  h->off_hb = off;
  off += vec_bytes(h, L, 8);
  h->off_hx = off;
  off += vec_bytes(h, L, 8);
  h->off_b.resize(nl);
  h->off_x.resize(nl);
  h->off_r.resize(nl);
  // level vectors sized for FP64 so that any precision can use them
  for (int l = 0; l <= L; ++l) {
    h->off_b[l] = off;
    off += vec_bytes(h, l, 8);
    h->off_x[l] = off;
    off += vec_bytes(h, l, 8);
    h->off_r[l] = off;
    off += vec_bytes(h, l, 8);
  }
  h->off_bL = h->off_b[L];
  h->off_xL = h->off_x[L];
  h->ws_bytes = off;
  *out = h;
  return SIPG_OK;
}

void sipg_destroy(sipg_handle* h) {
  if (!h) return;
  if (h->iter_exec) cudaGraphExecDestroy(h->iter_exec);
  if (h->gm_exec) cudaGraphExecDestroy(h->gm_exec);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  if (h->ev_a) cudaEventDestroy(h->ev_a);
  if (h->ev_b) cudaEventDestroy(h->ev_b);
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  delete h;
}

const char* sipg_last_error(const sipg_handle* h) { return h ? h->err.c_str() : "null handle"; }

size_t sipg_workspace_bytes(const sipg_handle* h) { return h ? h->ws_bytes : 0; }

size_t sipg_ndofs(const sipg_handle* h, int level) {
  if (!h || level < 0 || level > h->L) return 0;
  return h->lv[level].ndofs;
}

uint64_t sipg_launch_count(const sipg_handle* h) { return h ? h->launches : 0; }

sipg_status sipg_bind_workspace(sipg_handle* h, void* dev_ptr, size_t bytes, void* stream) {
  if (!h) return SIPG_EINVAL;
  if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255))
    return fail(h, SIPG_EINVAL, "workspace pointer null or not 256-byte aligned");
  if (bytes < h->ws_bytes) return fail(h, SIPG_ENOMEM_WORKSPACE, "workspace too small");
  if (h->iter_exec) {
    cudaGraphExecDestroy(h->iter_exec);
    h->iter_exec = nullptr;
  }
  if (h->gm_exec) {
    cudaGraphExecDestroy(h->gm_exec);
    h->gm_exec = nullptr;
  }
  h->ws = reinterpret_cast<char*>(dev_ptr);
  h->bound = true;
  cudaStream_t s = S(stream);
  {
    int dev = 0;
    SIPG_CHECK(cudaGetDevice(&dev), "device");
    SIPG_CHECK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  }
  if (!h->pinned)  // page-locked host memory for the per-iteration scalar read-back
    SIPG_CHECK(cudaHostAlloc(reinterpret_cast<void**>(&h->pinned), sizeof(KrylovScalars) * h->prm.nrhs,
                             cudaHostAllocDefault),
               "pinned host buffer");
  if (!h->side) {
    SIPG_CHECK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking), "side stream");
    int least = 0, greatest = 0;
    SIPG_CHECK(cudaDeviceGetStreamPriorityRange(&least, &greatest), "priority range");
    h->prio_hi = greatest;
    SIPG_CHECK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "event");
    SIPG_CHECK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "event");
  }
  SIPG_CHECK(cudaMemsetAsync(h->ws + h->off_sync, 0, 256, s), "memset");
  SIPG_CHECK(launch_setup(h, s), "setup");
  int status = 0;
  SIPG_CHECK(cudaMemcpyAsync(&status, h->ws + h->off_scratch_setup, sizeof(int), cudaMemcpyDeviceToHost, s),
             "setup status");
  SIPG_CHECK(cudaStreamSynchronize(s), "setup sync");
  if (status != 0) {
    h->bound = false;
    return fail(h, SIPG_EINVAL, "setup: a mass matrix was not positive definite");
  }
  const int nl = h->L + 1;
  h->hc64.resize(nl);
  h->hc32.resize(nl);
  SIPG_CHECK(cudaMemcpyAsync(h->hc64.data(), h->c64(0), sizeof(LevelConst<double>) * nl, cudaMemcpyDeviceToHost, s),
             "constants D2H");
  SIPG_CHECK(cudaMemcpyAsync(h->hc32.data(), h->c32(0), sizeof(LevelConst<float>) * nl, cudaMemcpyDeviceToHost, s),
             "constants D2H");
  SIPG_CHECK(cudaStreamSynchronize(s), "setup sync");
  // the full and clamped kernels have one launch path
  if (h->autotune && h->prm.smoother != SIPG_SMOOTHER_FULL && h->prm.smoother != SIPG_SMOOTHER_CLAMPED) {
    const sipg_status st = h->prm.vcycle_precision == SIPG_FP32 ? tune_T<float>(h, s) : tune_T<double>(h, s);
    if (st) return st;
  }
  return SIPG_OK;
}

sipg_status sipg_rhs(sipg_handle* h, const double* f, double* b, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (!f || !b) return fail(h, SIPG_EINVAL, "null vector");
  SIPG_CHECK(launch_mass(h, f, b, S(stream)), "mass");
  h->launches += 1;
  return SIPG_OK;
}

sipg_status sipg_manufactured_source(sipg_handle* h, double* f, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (!f) return fail(h, SIPG_EINVAL, "null vector");
  SIPG_CHECK(launch_manufactured(h, f, S(stream)), "manufactured");
  h->launches += 1;
  return SIPG_OK;
}

static sipg_status check_level_prec(sipg_handle* h, int level, int prec) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (level < 0 || level > h->L) return fail(h, SIPG_EINVAL, "level out of range");
  if (prec != SIPG_FP64 && prec != SIPG_FP32) return fail(h, SIPG_EINVAL, "bad precision");
  return SIPG_OK;
}

sipg_status sipg_apply(sipg_handle* h, int level, int prec, const void* x, void* y, void* stream) {
  sipg_status st = check_level_prec(h, level, prec);
  if (st) return st;
  if (!x || !y || x == y) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  cudaError_t e = prec == SIPG_FP64
                      ? launch_apply<double>(h, level, APPLY_Y, nullptr, (const double*)x, (double*)y, S(stream))
                      : launch_apply<float>(h, level, APPLY_Y, nullptr, (const float*)x, (float*)y, S(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "apply");
  h->launches += 1;
  return SIPG_OK;
}

sipg_status sipg_residual(sipg_handle* h, int level, int prec, const void* b, const void* x, void* r,
                          void* stream) {
  sipg_status st = check_level_prec(h, level, prec);
  if (st) return st;
  if (!b || !x || !r || x == r) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  cudaError_t e = prec == SIPG_FP64
                      ? launch_apply<double>(h, level, APPLY_RESIDUAL, (const double*)b, (const double*)x,
                                             (double*)r, S(stream))
                      : launch_apply<float>(h, level, APPLY_RESIDUAL, (const float*)b, (const float*)x,
                                            (float*)r, S(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "residual");
  h->launches += 1;
  return SIPG_OK;
}

sipg_status sipg_apply_penalty(sipg_handle* h, const double* x, double* y, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (!x || !y || x == y) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  SIPG_CHECK(launch_apply<double>(h, h->L, APPLY_PENALTY, nullptr, x, y, S(stream)), "apply penalty");
  h->launches += 1;
  return SIPG_OK;
}

sipg_status sipg_smooth_colour(sipg_handle* h, int level, int prec, int colour, const void* b, void* x,
                               void* stream) {
  sipg_status st = check_level_prec(h, level, prec);
  if (st) return st;
  if (colour < 0 || colour >= (1 << h->prm.dim)) return fail(h, SIPG_EINVAL, "bad colour");
  if (!b || !x || b == x) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  cudaError_t e = prec == SIPG_FP64
                      ? launch_smooth_colour<double>(h, level, colour, (const double*)b, (double*)x, S(stream))
                      : launch_smooth_colour<float>(h, level, colour, (const float*)b, (float*)x, S(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "smoother");
  const bool fp32_3d = h->prm.dim == 3 && prec == SIPG_FP32;
  const bool full = h->prm.smoother == SIPG_SMOOTHER_FULL || (h->prm.smoother == SIPG_SMOOTHER_CLAMPED && !fp32_3d);
  // full kernel: the residual apply, then the patch kernel (3D FP32: one per
  // patch set, interior and boundary)
  h->launches += full ? (fp32_3d ? 1 + colour_kernels(3, h->lv[level].N, colour) : 2)
                      : colour_kernels(h->prm.dim, h->lv[level].N, colour);
  return SIPG_OK;
}

sipg_status sipg_smooth(sipg_handle* h, int level, int prec, int reverse, const void* b, void* x,
                        void* stream) {
  sipg_status st = check_level_prec(h, level, prec);
  if (st) return st;
  if (!b || !x || b == x) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  if (prec == SIPG_FP64) return smooth_T<double>(h, level, reverse, (const double*)b, (double*)x, S(stream));
  return smooth_T<float>(h, level, reverse, (const float*)b, (float*)x, S(stream));
}

sipg_status sipg_restrict(sipg_handle* h, int fine_level, int prec, const void* rf, void* rc, void* stream) {
  sipg_status st = check_level_prec(h, fine_level, prec);
  if (st) return st;
  if (fine_level < 1) return fail(h, SIPG_EINVAL, "fine_level must be >= 1");
  if (!rf || !rc) return fail(h, SIPG_EINVAL, "null vector");
  cudaError_t e = prec == SIPG_FP64
                      ? launch_restrict<double>(h, fine_level, (const double*)rf, (double*)rc, S(stream))
                      : launch_restrict<float>(h, fine_level, (const float*)rf, (float*)rc, S(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "restrict");
  h->launches += 1;
  return SIPG_OK;
}

sipg_status sipg_prolongate_add(sipg_handle* h, int fine_level, int prec, const void* ec, void* xf,
                                void* stream) {
  sipg_status st = check_level_prec(h, fine_level, prec);
  if (st) return st;
  if (fine_level < 1) return fail(h, SIPG_EINVAL, "fine_level must be >= 1");
  if (!ec || !xf) return fail(h, SIPG_EINVAL, "null vector");
  cudaError_t e = prec == SIPG_FP64
                      ? launch_prolongate_add<double>(h, fine_level, (const double*)ec, (double*)xf, S(stream))
                      : launch_prolongate_add<float>(h, fine_level, (const float*)ec, (float*)xf, S(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "prolongate");
  h->launches += 1;
  return SIPG_OK;
}

sipg_status sipg_coarse_solve(sipg_handle* h, int prec, const void* b0, void* x0, void* stream) {
  sipg_status st = check_level_prec(h, 0, prec);
  if (st) return st;
  if (!b0 || !x0) return fail(h, SIPG_EINVAL, "null vector");
  cudaError_t e = prec == SIPG_FP64
                      ? launch_coarse_solve<double>(h, (const double*)b0, (double*)x0, S(stream))
                      : launch_coarse_solve<float>(h, (const float*)b0, (float*)x0, S(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "coarse solve");
  h->launches += 1;
  return SIPG_OK;
}

sipg_status sipg_vcycle(sipg_handle* h, int prec, const void* b, void* x, void* stream) {
  sipg_status st = check_level_prec(h, h->L, prec);
  if (st) return st;
  if (!b || !x || b == x) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  if (prec == SIPG_FP64) return vcycle_T<double>(h, (const double*)b, (double*)x, S(stream));
  return vcycle_T<float>(h, (const float*)b, (float*)x, S(stream));
}

sipg_status sipg_solve(sipg_handle* h, const double* b, double* x, double rtol, int maxit, sipg_info* info,
                       void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (!b || !x || b == x) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  if (!(rtol > 0.0) || maxit < 0) return fail(h, SIPG_EINVAL, "bad rtol or maxit");
  return fcg_solve(h, b, x, rtol, maxit, info, S(stream));
}

sipg_status sipg_solve_zero(sipg_handle* h, const double* b, double* x, double rtol, int maxit,
                            sipg_info* info, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (!b || !x || b == x) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  if (!(rtol > 0.0) || maxit < 0) return fail(h, SIPG_EINVAL, "bad rtol or maxit");
  return fcg_solve(h, b, x, rtol, maxit, info, S(stream), true);
}

size_t sipg_gmres_workspace_bytes(const sipg_handle* h, int restart) {
  if (!h || restart < 1 || restart > SIPG_GMRES_MAX_RESTART) return 0;
  return gmres_layout(h, restart).total;
}

sipg_status sipg_gmres_solve(sipg_handle* h, const double* b, double* x, double rtol, int maxit, int restart,
                             void* work, size_t work_bytes, sipg_info* info, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (h->prm.nrhs != 1) return fail(h, SIPG_EUNSUPPORTED, "GMRES solves one right-hand side (nrhs = 1)");
  if (!b || !x || b == x) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  if (!(rtol > 0.0) || maxit < 0) return fail(h, SIPG_EINVAL, "bad rtol or maxit");
  if (restart < 1 || restart > SIPG_GMRES_MAX_RESTART) return fail(h, SIPG_EINVAL, "restart out of range");
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255) != 0)
    return fail(h, SIPG_EINVAL, "GMRES workspace must be 256-byte aligned");
  if (work_bytes < gmres_layout(h, restart).total) return fail(h, SIPG_EINVAL, "GMRES workspace too small");
  return gmres_run(h, b, x, rtol, maxit, restart, static_cast<char*>(work), info, S(stream));
}

sipg_status sipg_gmres_solve_left(sipg_handle* h, const double* b, double* x, double rtol, int maxit, int restart,
                                  void* work, size_t work_bytes, sipg_info* info, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (h->prm.nrhs != 1) return fail(h, SIPG_EUNSUPPORTED, "GMRES solves one right-hand side (nrhs = 1)");
  if (!b || !x || b == x) return fail(h, SIPG_EINVAL, "null or aliased vectors");
  if (!(rtol > 0.0) || maxit < 0) return fail(h, SIPG_EINVAL, "bad rtol or maxit");
  if (restart < 1 || restart > SIPG_GMRES_MAX_RESTART) return fail(h, SIPG_EINVAL, "restart out of range");
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255) != 0)
    return fail(h, SIPG_EINVAL, "GMRES workspace must be 256-byte aligned");
  if (work_bytes < gmres_layout(h, restart).total) return fail(h, SIPG_EINVAL, "GMRES workspace too small");
  return gmres_run(h, b, x, rtol, maxit, restart, static_cast<char*>(work), info, S(stream), true);
}

sipg_status sipg_adjoint_solve(sipg_handle* h, const double* g, double* lambda, double rtol, int maxit,
                               sipg_info* info, void* stream) {
  // A is symmetric (Sec. 2, Eq. bilinear_form), so A^T lambda = g is the
  // same system.
  return sipg_solve(h, g, lambda, rtol, maxit, info, stream);
}

sipg_status sipg_solve_host(sipg_handle* h, const double* f_host, double* u_host, double rtol, int maxit,
                            sipg_info* info, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (!f_host || !u_host) return fail(h, SIPG_EINVAL, "null host buffer");
  cudaStream_t s = S(stream);
  const size_t bytes = h->lv[h->L].ndofs * h->prm.nrhs * sizeof(double);
  double* db = reinterpret_cast<double*>(h->ws + h->off_hb);
  double* dx = reinterpret_cast<double*>(h->ws + h->off_hx);
  SIPG_CHECK(cudaMemcpyAsync(dx, f_host, bytes, cudaMemcpyHostToDevice, s), "H2D");
  SIPG_CHECK(launch_mass(h, dx, db, s), "mass");
  h->launches += 1;
  // the copy of u back to the host runs beside the final true residual (a
  // second stream of this call)
  cudaStream_t os = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
  auto release = [&]() {
    if (os) cudaStreamDestroy(os);
    if (ready) cudaEventDestroy(ready);
    if (done) cudaEventDestroy(done);
  };
  if (cudaStreamCreateWithFlags(&os, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
    release();
    return fail(h, SIPG_ECUDA, "stream or event creation");
  }
  bool copied = false;
  sipg_status r = fcg_solve(h, db, dx, rtol, maxit, info, s, true, u_host, os, ready, done, &copied);
  cudaError_t e = cudaStreamSynchronize(os);  // a copy in flight ends before x or u goes
  if (r == SIPG_OK || r == SIPG_ENOCONV) {
    if (e == cudaSuccess && !copied) e = cudaMemcpyAsync(u_host, dx, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  release();
  if (r != SIPG_OK && r != SIPG_ENOCONV) return r;
  if (e != cudaSuccess) return cuda_fail(h, e, "D2H");
  return r;
}

sipg_status sipg_dot(sipg_handle* h, const double* a, const double* b, double* out, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (!a || !b || !out) return fail(h, SIPG_EINVAL, "null vector");
  SIPG_CHECK(launch_dot(h, a, b, out, S(stream)), "dot");
  return SIPG_OK;
}

sipg_status sipg_selftest_barrier(sipg_handle* h, int extra, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (extra < 0 || extra > 1024) return fail(h, SIPG_EINVAL, "extra out of range");
  cudaStream_t s = S(stream);
  SIPG_CHECK(cudaMemsetAsync(h->ws + h->off_sync, 0, 256, s), "memset");
  SIPG_CHECK(launch_barrier_selftest(h, extra, s), "barrier self test");
  h->launches += 1;
  int status = 0;
  SIPG_CHECK(cudaMemcpyAsync(&status, h->ws + h->off_sync + 2 * sizeof(unsigned int), sizeof(int),
                             cudaMemcpyDeviceToHost, s),
             "status D2H");
  SIPG_CHECK(cudaStreamSynchronize(s), "sync");
  SIPG_CHECK(cudaMemsetAsync(h->ws + h->off_sync, 0, 256, s), "memset");
  SIPG_CHECK(cudaStreamSynchronize(s), "sync");
  if (status != 0) return fail(h, SIPG_ETIMEOUT, "barrier wait timed out (self test)");
  return SIPG_OK;
}

sipg_status sipg_selftest_mma_tf32(sipg_handle* h, const float* a, const float* b, float* d, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (!a || !b || !d) return fail(h, SIPG_EINVAL, "null pointer");
  cudaStream_t s = S(stream);
  SIPG_CHECK(cudaMemsetAsync(h->ws + h->off_sync, 0, 256, s), "memset");
  SIPG_CHECK(launch_tc_selftest(h, a, b, d, s), "tensor-core self test");
  h->launches += 1;
  int status = 0;
  SIPG_CHECK(cudaMemcpyAsync(&status, h->ws + h->off_sync + 2 * sizeof(unsigned int), sizeof(int),
                             cudaMemcpyDeviceToHost, s),
             "status D2H");
  SIPG_CHECK(cudaStreamSynchronize(s), "sync");
  SIPG_CHECK(cudaMemsetAsync(h->ws + h->off_sync, 0, 256, s), "memset");
  SIPG_CHECK(cudaStreamSynchronize(s), "sync");
  if (status != 0) return fail(h, SIPG_ETIMEOUT, "tensor-core completion wait timed out (self test)");
  return SIPG_OK;
}

sipg_status sipg_get_constants(sipg_handle* h, int level, int which, int type, double* host_out, int cap,
                               int* count, void* stream) {
  sipg_status st = need_bound(h);
  if (st) return st;
  if (level < 0 || level > h->L || !host_out || !count || type < 0 || type > 3)
    return fail(h, SIPG_EINVAL, "bad argument");
  LevelConst<double> c;
  cudaStream_t s = S(stream);
  SIPG_CHECK(cudaMemcpyAsync(&c, h->c64(level), sizeof(c), cudaMemcpyDeviceToHost, s), "D2H");
  SIPG_CHECK(cudaStreamSynchronize(s), "sync");
  const int n = h->n;
  std::vector<double> v;
  switch (which) {
    case 0:
      for (int t = 0; t < 3; ++t)
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) v.push_back(c.Lself[t][i][j]);
      break;
    case 1:
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          v.push_back((i == 0 ? c.alo[j] : 0.0) + (j == n - 1 ? c.glo[i] : 0.0));
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          v.push_back((i == n - 1 ? c.ahi[j] : 0.0) + (j == 0 ? c.ghi[i] : 0.0));
      break;
    case 2:
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) v.push_back(c.M[i][j]);
      break;
    case 3:
      for (int i = 0; i < c.p[type]; ++i)
        for (int j = 0; j < c.p[type]; ++j) v.push_back(c.S[type][i][j]);
      break;
    case 4:
      for (int i = 0; i < c.p[type]; ++i) v.push_back(c.lam[type][i]);
      break;
    case 5:
      for (int o = 0; o < 2; ++o)
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) v.push_back(c.Pc[o][i][j]);
      break;
    case 6:
      for (int i = 0; i < c.m0; ++i)
        for (int j = 0; j < c.m0; ++j) v.push_back(c.S0[i][j]);
      break;
    case 7:
      for (int i = 0; i < c.m0; ++i) v.push_back(c.lam0[i]);
      break;
    case 8:
      for (int i = 0; i < n; ++i) v.push_back(c.nodes[i]);
      break;
    default:
      return fail(h, SIPG_EINVAL, "bad 'which'");
  }
  int cnt = std::min((int)v.size(), cap);
  for (int i = 0; i < cnt; ++i) host_out[i] = v[i];
  *count = (int)v.size();
  return SIPG_OK;
}

sipg_status sipg_tuning(const sipg_handle* h, int level, int precision, int* path, int* tile) {
  if (!h || !path || !tile) return SIPG_EINVAL;
  if (level < 0 || level > h->L || (precision != SIPG_FP64 && precision != SIPG_FP32 && precision != SIPG_TF32))
    return SIPG_EINVAL;
  const int pi = precision != SIPG_FP64 ? 1 : 0;
  *path = h->tuned_path(pi, level);
  *tile = h->tuned_tile(pi, level);
  return SIPG_OK;
}

// ------------------------------------------------------------------ ragged batch
struct sipg_batch {
  std::vector<sipg_handle*> hs;
  std::vector<size_t> off;
  size_t ws_bytes = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start = nullptr;
  std::string err;
  // fused path (2D FP32 batches): batched smoothing stages, one CUDA graph per
  // FCG iteration of the whole batch
  bool fused = false;
  size_t off_plan = 0;
  BatchPlan2* plan = nullptr;
  cudaStream_t gs = nullptr;                         // capture / launch stream
  std::vector<cudaEvent_t> fork;                     // capture-time fork and join events
  cudaGraphExec_t g_first = nullptr, g_iter = nullptr;
  std::vector<double*> g_x;                          // solution vectors the graphs were captured with
  double g_rtol2 = -1.0;
};

sipg_status sipg_batch_create(const sipg_params* params, int count, sipg_batch** out) {
  if (!out) return SIPG_EINVAL;
  *out = nullptr;
  if (!params || count < 1 || count > 4096) return SIPG_EINVAL;
  sipg_batch* bt = new sipg_batch();
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    sipg_handle* h = nullptr;
    sipg_status st = sipg_create(&params[i], &h);
    if (st != SIPG_OK) {
      for (auto* g : bt->hs) sipg_destroy(g);
      delete bt;
      return st;
    }
    // the members' kernels run concurrently on separate streams, so no member
    // relies on a cooperative launch having the whole GPU to itself
    h->fuse_small_levels = false;
    bt->hs.push_back(h);
    bt->off.push_back(off);
    off += align256(sipg_workspace_bytes(h));
  }
  // the fused path (batched smoothing stages) is opt-in: measured on GB300 it
  // is slower than the members on their own streams, whose kernels overlap
  // across members and levels
  bt->fused = false;
  if (const char* env = getenv("SIPG_BATCH_FUSED")) bt->fused = atoi(env) != 0 && batch2_supported(bt->hs);
  if (bt->fused) {
    bt->off_plan = off;
    off += align256(batch2_plan_bytes(bt->hs));
  }
  bt->ws_bytes = off;
  *out = bt;
  return SIPG_OK;
}

void sipg_batch_destroy(sipg_batch* bt) {
  if (!bt) return;
  if (bt->g_first) cudaGraphExecDestroy(bt->g_first);
  if (bt->g_iter) cudaGraphExecDestroy(bt->g_iter);
  for (auto e : bt->fork) cudaEventDestroy(e);
  if (bt->gs) cudaStreamDestroy(bt->gs);
  if (bt->plan) batch2_plan_free(bt->plan);
  for (auto* h : bt->hs) sipg_destroy(h);
  for (auto s : bt->streams) cudaStreamDestroy(s);
  for (auto e : bt->done) cudaEventDestroy(e);
  if (bt->start) cudaEventDestroy(bt->start);
  delete bt;
}

const char* sipg_batch_last_error(const sipg_batch* bt) { return bt ? bt->err.c_str() : "null batch"; }

size_t sipg_batch_workspace_bytes(const sipg_batch* bt) { return bt ? bt->ws_bytes : 0; }

int sipg_batch_count(const sipg_batch* bt) { return bt ? (int)bt->hs.size() : 0; }

sipg_handle* sipg_batch_member(sipg_batch* bt, int i) {
  if (!bt || i < 0 || i >= (int)bt->hs.size()) return nullptr;
  return bt->hs[i];
}

sipg_status sipg_batch_bind_workspace(sipg_batch* bt, void* dev_ptr, size_t bytes, void* stream) {
  if (!bt) return SIPG_EINVAL;
  if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255) || bytes < bt->ws_bytes) {
    bt->err = "workspace pointer null, misaligned or too small";
    return dev_ptr ? SIPG_ENOMEM_WORKSPACE : SIPG_EINVAL;
  }
  for (size_t i = 0; i < bt->hs.size(); ++i) {
    sipg_handle* h = bt->hs[i];
    sipg_status st = sipg_bind_workspace(h, static_cast<char*>(dev_ptr) + bt->off[i], sipg_workspace_bytes(h),
                                         stream);
    if (st != SIPG_OK) {
      bt->err = "member " + std::to_string(i) + ": " + h->err;
      return st;
    }
  }
  if (bt->streams.empty()) {
    bt->streams.resize(bt->hs.size());
    bt->done.resize(bt->hs.size());
    for (size_t i = 0; i < bt->hs.size(); ++i) {
      if (cudaStreamCreateWithFlags(&bt->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&bt->done[i], cudaEventDisableTiming) != cudaSuccess) {
        bt->err = "stream or event creation failed";
        return SIPG_ECUDA;
      }
    }
    if (cudaEventCreateWithFlags(&bt->start, cudaEventDisableTiming) != cudaSuccess) {
      bt->err = "event creation failed";
      return SIPG_ECUDA;
    }
  }
  if (bt->fused && !bt->plan) {
    // the members' level constants are on the host now: build the batched
    // smoothing plan in the batch workspace
    cudaError_t e = batch2_plan_build(bt->hs, static_cast<char*>(dev_ptr) + bt->off_plan, &bt->plan);
    if (e != cudaSuccess) {
      bt->err = std::string("batched smoothing plan: ") + cudaGetErrorString(e);
      return SIPG_ECUDA;
    }
    if (cudaStreamCreateWithFlags(&bt->gs, cudaStreamNonBlocking) != cudaSuccess) {
      bt->err = "stream creation failed";
      return SIPG_ECUDA;
    }
  }
  return SIPG_OK;
}

// ---------------------------------------------------------- fused ragged batch
// (CUDA failures here name the batch: BATCH_CHECK records the message in the
// batch and returns SIPG_ECUDA)
#define BATCH_CHECK(expr, where)                                                       \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      bt->err = std::string(where) + ": " + cudaGetErrorString(e_);                  \
      return SIPG_ECUDA;                                                             \
    }                                                                                \
  } while (0)
// Fork the member streams off `s` (every member stream waits for s) and join
// them back (s waits for every member stream); captured into the batch graphs
// as dependency edges.
sipg_status batch_fork(sipg_batch* bt, cudaStream_t s, int slot) {
  cudaEvent_t e = bt->fork[slot];
  BATCH_CHECK(cudaEventRecord(e, s), "fork record");
  for (auto ms : bt->streams) BATCH_CHECK(cudaStreamWaitEvent(ms, e, 0), "fork wait");
  return SIPG_OK;
}
sipg_status batch_join(sipg_batch* bt, cudaStream_t s) {
  for (size_t i = 0; i < bt->streams.size(); ++i) {
    BATCH_CHECK(cudaEventRecord(bt->done[i], bt->streams[i]), "join record");
    BATCH_CHECK(cudaStreamWaitEvent(s, bt->done[i], 0), "join wait");
  }
  return SIPG_OK;
}

// One FP32 V-cycle of every member (finest-level buffers bL -> xL), level by
// level: per-member work (zeroing, residual and restriction, coarse solve,
// prolongation) on the member streams, every smoothing step of a level as
// one batched cooperative launch on s.
sipg_status batch_vcycle(sipg_batch* bt, cudaStream_t s, int& slot) {
  const int levels = batch2_levels(bt->plan);
  const size_t nm = bt->hs.size();
  auto bvec = [&](sipg_handle* h, int l) -> float* {
    return l == h->L ? reinterpret_cast<float*>(h->ws + h->off_bL) : reinterpret_cast<float*>(h->vb(l));
  };
  auto xvec = [&](sipg_handle* h, int l) -> float* {
    return l == h->L ? reinterpret_cast<float*>(h->ws + h->off_xL) : reinterpret_cast<float*>(h->vx(l));
  };
  sipg_status st;
  for (int l = levels - 1; l >= 1; --l) {
    if ((st = batch_fork(bt, s, slot++))) return st;
    for (size_t i = 0; i < nm; ++i) {
      sipg_handle* h = bt->hs[i];
      if (l > h->L) continue;
      BATCH_CHECK(cudaMemsetAsync(xvec(h, l), 0, h->lv[l].ndofs * sizeof(float), bt->streams[i]), "memset");
    }
    if ((st = batch_join(bt, s))) return st;
    BATCH_CHECK(batch2_step(bt->plan, l, 0, s), "batched smoothing");
    if ((st = batch_fork(bt, s, slot++))) return st;
    for (size_t i = 0; i < nm; ++i) {
      sipg_handle* h = bt->hs[i];
      if (l > h->L) continue;
      float* r = reinterpret_cast<float*>(h->vr(l));
      BATCH_CHECK(launch_apply<float>(h, l, APPLY_RESIDUAL, bvec(h, l), xvec(h, l), r, bt->streams[i]), "residual");
      BATCH_CHECK(launch_restrict<float>(h, l, r, bvec(h, l - 1), bt->streams[i]), "restrict");
      if (l == 1) BATCH_CHECK(launch_coarse_solve<float>(h, bvec(h, 0), xvec(h, 0), bt->streams[i]), "coarse solve");
    }
  }
  for (int l = 1; l < levels; ++l) {
    if (l > 1 && (st = batch_fork(bt, s, slot++))) return st;
    for (size_t i = 0; i < nm; ++i) {
      sipg_handle* h = bt->hs[i];
      if (l > h->L) continue;
      BATCH_CHECK(launch_prolongate_add<float>(h, l, xvec(h, l - 1), xvec(h, l), bt->streams[i]), "prolongate");
    }
    if ((st = batch_join(bt, s))) return st;
    BATCH_CHECK(batch2_step(bt->plan, l, 1, s), "batched smoothing");
  }
  return SIPG_OK;
}

// One FCG iteration of every member: V-cycle (batched), then per member the
// preconditioned-direction update, q = A p, the step and the scalars' copy to
// the host.  first: z_0 = B r_0 from the FP64 residual, p_0 = z_0.
sipg_status batch_iteration(sipg_batch* bt, const std::vector<double*>& xs, bool first, cudaStream_t s) {
  int slot = 0;
  sipg_status st;
  const size_t nm = bt->hs.size();
  if (first) {
    if ((st = batch_fork(bt, s, slot++))) return st;
    for (size_t i = 0; i < nm; ++i) {
      sipg_handle* h = bt->hs[i];
      BATCH_CHECK(convert_d2f(h->kr(), reinterpret_cast<float*>(h->ws + h->off_bL), h->lv[h->L].ndofs, bt->streams[i]),
                 "convert");
    }
    if ((st = batch_join(bt, s))) return st;
  }
  if ((st = batch_vcycle(bt, s, slot))) return st;
  if ((st = batch_fork(bt, s, slot++))) return st;
  for (size_t i = 0; i < nm; ++i) {
    sipg_handle* h = bt->hs[i];
    cudaStream_t ms = bt->streams[i];
    BATCH_CHECK(krylov_after_precond(h, first ? 1 : 0, h->kr(), h->ws + h->off_xL, 1, ms), "precond post");
    BATCH_CHECK(launch_apply<double>(h, h->L, APPLY_Y, nullptr, h->kp(), h->kq(), ms), "apply");
    BATCH_CHECK(krylov_after_apply(h, ms), "pq");
    BATCH_CHECK(krylov_update_xr(h, xs[i], h->ws + h->off_bL, 1, ms), "update");
    BATCH_CHECK(cudaMemcpyAsync(h->pinned, h->scalars(), sizeof(KrylovScalars), cudaMemcpyDeviceToHost, ms),
               "scalars D2H");
  }
  return batch_join(bt, s);
}

sipg_status batch_capture(sipg_batch* bt, const std::vector<double*>& xs, bool first, cudaGraphExec_t* out) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  BATCH_CHECK(cudaStreamBeginCapture(bt->gs, cudaStreamCaptureModeThreadLocal), "begin capture");
  sipg_status st = batch_iteration(bt, xs, first, bt->gs);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(bt->gs, &graph);
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return bt->err = "end capture", SIPG_ECUDA;
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bt->err = "graph instantiate", SIPG_ECUDA;
  return SIPG_OK;
}

// Lockstep flexible CG over all members with the batched V-cycle: the true
// residual per member, then iterations of the whole batch (two CUDA graphs:
// the first iteration and the others) until no member is active or maxit;
// members whose recursively updated residual converged keep their x (the
// Krylov kernels skip inactive columns).  The final true residual of each
// member is verified by the per-member path (which restarts a member whose
// residual drifted).
sipg_status batch_solve_fused(sipg_batch* bt, const double* const* b, double* const* x, double rtol, int maxit,
                              sipg_info* infos, cudaStream_t cs) {
  const size_t nm = bt->hs.size();
  std::vector<double*> xs(x, x + nm);
  if (bt->fork.size() < 64) {
    const size_t old = bt->fork.size();
    bt->fork.resize(64);
    for (size_t i = old; i < bt->fork.size(); ++i)
      if (cudaEventCreateWithFlags(&bt->fork[i], cudaEventDisableTiming) != cudaSuccess)
        return bt->err = "event creation failed", SIPG_ECUDA;
  }
  const double rtol2 = rtol * rtol;
  if (!bt->g_iter || bt->g_x != xs || bt->g_rtol2 != rtol2) {
    for (auto* h : bt->hs) h->rtol2 = rtol2;
    sipg_status st = batch_capture(bt, xs, true, &bt->g_first);
    if (!st) st = batch_capture(bt, xs, false, &bt->g_iter);
    if (st) return st;
    bt->g_x = xs;
    bt->g_rtol2 = rtol2;
  }
  // initial true residuals and norms, on the member streams after cs
  if (cudaEventRecord(bt->start, cs) != cudaSuccess) return SIPG_ECUDA;
  std::vector<FcgRun> runs(nm);
  for (size_t i = 0; i < nm; ++i) {
    sipg_handle* h = bt->hs[i];
    h->rtol2 = rtol2;
    if (cudaStreamWaitEvent(bt->streams[i], bt->start, 0) != cudaSuccess) return SIPG_ECUDA;
    runs[i].h = h;
    runs[i].b = b[i];
    runs[i].x = x[i];
    runs[i].s = bt->streams[i];
    runs[i].maxit = maxit;
    runs[i].info = infos ? &infos[i] : nullptr;
    sipg_status st = launch_true_residual(runs[i]);
    if (st) return bt->err = "member " + std::to_string(i) + ": " + h->err, st;
  }
  for (size_t i = 0; i < nm; ++i)
    if (cudaStreamSynchronize(bt->streams[i]) != cudaSuccess) return bt->err = "sync", SIPG_ECUDA;
  for (size_t i = 0; i < nm; ++i) {
    runs[i].pending = false;
    runs[i].hist.push_back(sqrt(bt->hs[i]->pinned[0].rr));
  }
  auto any_active = [&]() {
    for (auto* h : bt->hs)
      if (h->pinned[0].active && !h->pinned[0].breakdown) return true;
    return false;
  };
  // the graphs wait for the member streams' initial work through gs
  for (size_t i = 0; i < nm; ++i) {
    if (cudaEventRecord(bt->done[i], bt->streams[i]) != cudaSuccess ||
        cudaStreamWaitEvent(bt->gs, bt->done[i], 0) != cudaSuccess)
      return SIPG_ECUDA;
  }
  int it = 0;
  std::vector<bool> was_active(nm);
  while (any_active() && it < maxit) {
    for (size_t i = 0; i < nm; ++i) was_active[i] = bt->hs[i]->pinned[0].active && !bt->hs[i]->pinned[0].breakdown;
    if (cudaGraphLaunch(it == 0 ? bt->g_first : bt->g_iter, bt->gs) != cudaSuccess)
      return bt->err = "graph launch", SIPG_ECUDA;
    if (cudaStreamSynchronize(bt->gs) != cudaSuccess) return bt->err = "sync", SIPG_ECUDA;
    ++it;
    for (size_t i = 0; i < nm; ++i) {
      if (!was_active[i]) continue;
      runs[i].it = it;
      runs[i].hist.push_back(sqrt(bt->hs[i]->pinned[0].rr));
    }
  }
  {
    int status = 0;
    if (cudaMemcpy(&status, batch2_status(bt->plan), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return SIPG_ECUDA;
    if (status != 0) {
      cudaMemset(batch2_status(bt->plan) - 2, 0, 3 * sizeof(int));
      bt->err = "a bounded grid-barrier wait of the batched smoother timed out";
      return SIPG_ETIMEOUT;
    }
  }
  // verify: the per-member state machine from its VERIFY phase (true
  // residual; a restart if it drifted; the members' own V-cycles then)
  for (size_t i = 0; i < nm; ++i) {
    runs[i].phase = FcgRun::VERIFY;
    runs[i].restarts = -1;
    if (cudaStreamWaitEvent(bt->streams[i], bt->start, 0) != cudaSuccess) return SIPG_ECUDA;
    sipg_status st = launch_true_residual(runs[i]);
    if (st) return st;
  }
  sipg_status st = SIPG_OK;
  for (;;) {
    bool any = false;
    for (auto& r : runs) {
      if (!r.pending) continue;
      any = true;
      if (cudaStreamSynchronize(r.s) != cudaSuccess) return SIPG_ECUDA;
    }
    if (!any) break;
    for (auto& r : runs) {
      if (!r.pending) continue;
      st = advance(r);
      if (st) return st;
    }
  }
  sipg_status worst = SIPG_OK;
  for (size_t i = 0; i < nm; ++i) {
    sipg_status si = finish(runs[i]);
    if (si != SIPG_OK && worst == SIPG_OK) {
      worst = si;
      bt->err = "member " + std::to_string(i) + ": " + bt->hs[i]->err;
    }
  }
  for (size_t i = 0; i < nm; ++i) {
    cudaEventRecord(bt->done[i], bt->streams[i]);
    cudaStreamWaitEvent(cs, bt->done[i], 0);
  }
  return worst;
}

sipg_status sipg_batch_solve(sipg_batch* bt, const double* const* b, double* const* x, double rtol, int maxit,
                             sipg_info* infos, void* stream) {
  if (!bt || !b || !x || !(rtol > 0.0) || maxit < 0) return SIPG_EINVAL;
  const size_t n = bt->hs.size();
  for (size_t i = 0; i < n; ++i) {
    if (!bt->hs[i]->bound || bt->streams.empty()) {
      bt->err = "workspace not bound";
      return SIPG_ESTATE;
    }
    if (!b[i] || !x[i] || b[i] == x[i]) {
      bt->err = "member " + std::to_string(i) + ": null or aliased vectors";
      return SIPG_EINVAL;
    }
  }
  cudaStream_t cs = S(stream);
  if (bt->plan) return batch_solve_fused(bt, b, x, rtol, maxit, infos, cs);
  if (cudaEventRecord(bt->start, cs) != cudaSuccess) return SIPG_ECUDA;
  std::vector<FcgRun> runs(n);
  for (size_t i = 0; i < n; ++i) {
    if (cudaStreamWaitEvent(bt->streams[i], bt->start, 0) != cudaSuccess) return SIPG_ECUDA;
    bt->hs[i]->rtol2 = rtol * rtol;
    runs[i].h = bt->hs[i];
    runs[i].b = b[i];
    runs[i].x = x[i];
    runs[i].s = bt->streams[i];
    runs[i].maxit = maxit;
    runs[i].info = infos ? &infos[i] : nullptr;
  }
  sipg_status st = drive(runs);
  sipg_status worst = st;
  for (size_t i = 0; i < n && st == SIPG_OK; ++i) {
    sipg_status si = finish(runs[i]);
    if (si != SIPG_OK && worst == SIPG_OK) {
      worst = si;
      bt->err = "member " + std::to_string(i) + ": " + bt->hs[i]->err;
    }
  }
  if (st != SIPG_OK) {
    for (size_t i = 0; i < n; ++i)
      if (!bt->hs[i]->err.empty()) bt->err = "member " + std::to_string(i) + ": " + bt->hs[i]->err;
  }
  for (size_t i = 0; i < n; ++i) {
    cudaEventRecord(bt->done[i], bt->streams[i]);
    cudaStreamWaitEvent(cs, bt->done[i], 0);
  }
  return worst;
}

}  // extern "C"
