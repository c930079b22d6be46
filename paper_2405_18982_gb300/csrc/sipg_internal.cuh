// Internal declarations shared by the CUDA translation units of the SIPG
// multigrid library (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/sipg.h"

#define SIPG_MAXN 8    // n = k+1 <= 8
#define SIPG_MAXP 16   // 1D patch size 2n
#define SIPG_MAXPE 18  // 2n plus one halo node on each side
#define SIPG_MAXM0 64  // 1D size of the coarsest level, N_0 * n
#define SIPG_GMRES_MAXM SIPG_GMRES_MAX_RESTART

// Per-level constants, written by the device setup kernel (FP64) and copied
// to an FP32 twin.  All 1D operators include kappa; physical cell size h.
// Index convention: [test row][trial column].
template <typename T>
struct LevelConst {
  int N;      // cells per direction
  int n;      // nodes per direction per cell (k+1)
  int m0;     // N * n on the coarsest level, 0 elsewhere
  int pad_;
  T h, gamma;
  // 1D SIPG self block of a cell: stiffness + its two faces.  Type 0: both
  // faces interior; 1: low face on the boundary; 2: high face on the boundary.
  T Lself[3][SIPG_MAXN][SIPG_MAXN];
  // Coupling to the low neighbour (test in c, trial in c-1) is rank two:
  //   l_lo[i][j] = delta_{i0} alo[j] + delta_{jk} glo[i]
  // and to the high neighbour (trial in c+1):
  //   l_hi[i][j] = delta_{ik} ahi[j] + delta_{j0} ghi[i].
  T alo[SIPG_MAXN], glo[SIPG_MAXN], ahi[SIPG_MAXN], ghi[SIPG_MAXN];
  // Same objects for dA/dgamma (unit penalty, times kappa).
  T Pself[3][SIPG_MAXN][SIPG_MAXN];
  T palo[SIPG_MAXN], pglo[SIPG_MAXN], pahi[SIPG_MAXN], pghi[SIPG_MAXN];
  T M[SIPG_MAXN][SIPG_MAXN];  // 1D cell mass h * Mhat
  // The exact mass on Gauss-Lobatto nodes is diagonal plus rank one: the
  // (2n-3)-exact GLL rule integrates phi_i phi_j up to a multiple of the
  // product of the leading coefficients a_i a_j, so
  //   M = diag(Mw) + Mu Ma^T   (Mw = h w_gll, Ma = a, Mu = h e a).
  T Mw[SIPG_MAXN], Ma[SIPG_MAXN], Mu[SIPG_MAXN];
  // Vertex-patch 1D data per type t (bit 0: low end on the domain boundary,
  // bit 1: high end).  Patch-local 1D node a = o*n + i, o in {0,1}.  V_j keeps
  // a in [first, first+p).  Lr/Mr are the rows V_j of the 1D patch matrices
  // over the extended columns (0 = low halo node, 1..2n = patch, 2n+1 = high
  // halo node); Mr has zero halo columns.
  int p[4], first[4];
  T Lr[4][SIPG_MAXP][SIPG_MAXPE];
  T Mr[4][SIPG_MAXP][SIPG_MAXPE];
  T S[4][SIPG_MAXP][SIPG_MAXP];  // M-orthonormal generalised eigenvectors (columns)
  T lam[4][SIPG_MAXP];
  // Full-kernel patch (all 2n nodes) of type t: eigenpairs of the 1D patch
  // matrices Lp S = Mp S Lambda, S M-orthonormal (columns).
  T Sf[4][SIPG_MAXP][SIPG_MAXP];
  T lamf[4][SIPG_MAXP];
  // Canonical embedding: Pc[o][i][j] = phi_j((o + xi_i) / 2).
  T Pc[2][SIPG_MAXN][SIPG_MAXN];
  T nodes[SIPG_MAXN];  // Gauss-Lobatto nodes on [0,1]
  // Coarsest level only: global 1D eigenpairs L S0 = M S0 Lambda0.
  T S0[SIPG_MAXM0][SIPG_MAXM0];
  T lam0[SIPG_MAXM0];
};

// Per-rhs scalars of the flexible CG (device memory).
struct KrylovScalars {
  double rho;      // <r_i, z_i>
  double alpha;
  double beta;
  double pq;       // <p_i, q_i>
  double rr;       // ||r||^2
  double bb;       // ||b||^2
  double zq;       // <z_{i+1}, q_i>
  int active;      // 1 while this column has not converged
  int breakdown;   // set when a scalar is non-finite or <p,q> <= 0
};

// Device-resident state of one GMRES restart cycle (Sec. 3.3), read and
// written by the step kernels so that a whole cycle runs as one graph launch
// without host round trips: the Hessenberg matrix (row-major, row stride
// SIPG_GMRES_MAXM), the plane rotations, the rotated right-hand side g, the
// Gram-Schmidt coefficients of the two passes, the squared norm of the new
// direction and |g_{j+1}| after every step.
struct GmresCycleState {
  int j;       // completed steps of this cycle
  int budget;  // steps allowed in this cycle
  int conv;    // |g_j| <= thr, or an exactly zero new direction
  int brk;     // a non-finite scalar or a zero rotation denominator
  int runs;    // step bodies executed (bounds the loop on its own)
  int pad_[3];
  double thr;  // rtol ||b|| (left preconditioning: rtol ||B b||)
  double nrm;  // ||w||^2 of the current step's new direction
  double hn;   // ||w||: the subdiagonal entry of the current column
  double pad2_;
  double H[(SIPG_GMRES_MAXM + 1) * SIPG_GMRES_MAXM];
  double cs[SIPG_GMRES_MAXM], sn[SIPG_GMRES_MAXM], g[SIPG_GMRES_MAXM + 1];
  double hc1[SIPG_GMRES_MAXM + 1], hc2[SIPG_GMRES_MAXM + 1];
  double hist[SIPG_GMRES_MAXM];
};

struct LevelInfo {
  int N;
  size_t ndofs;    // one rhs
  size_t ncells;
};

struct sipg_handle {
  sipg_params prm;
  int n;           // k+1
  int L;           // finest level index
  std::vector<LevelInfo> lv;
  std::string err;
  uint64_t launches = 0;

  // workspace layout (byte offsets)
  size_t ws_bytes = 0;
  size_t off_const64 = 0, off_const32 = 0, off_scratch_setup = 0;
  std::vector<size_t> off_b, off_x, off_r;   // level vectors, vcycle precision
  size_t off_bL = 0, off_xL = 0;             // finest-level V-cycle vectors
  size_t off_kr = 0, off_kz = 0, off_kp = 0, off_kq = 0;  // Krylov vectors FP64
  size_t off_hb = 0, off_hx = 0;             // device b and x of sipg_solve_host
  size_t off_partials = 0, off_scalars = 0;
  size_t off_sync = 0;                       // grid-barrier state [count, generation] + status word
  int n_partials = 0;                        // reduction blocks per rhs
  double rtol2 = 0.0;                        // squared relative tolerance of the running solve
  size_t vec_elem = 8;                       // bytes per element of level vectors

  char* ws = nullptr;
  bool bound = false;
  int num_sms = 0;                           // of the device the workspace lives on
  KrylovScalars* pinned = nullptr;           // page-locked host copy of the scalars (nrhs)
  bool fuse_small_levels = true;             // one cooperative launch per smoothing step when it fits one wave
  // autotuned choices per precision (0 FP64, 1 FP32) and level, measured at
  // bind time unless SIPG_AUTOTUNE=0: smoothing-step path (-1 not tuned,
  // 0 fused launch, 1 colour by colour) and interior tile of the 3D FP32
  // colour pass (0 default patches per CTA, 1 half as many, 2 / 3 the default
  // with b and x loaded ahead, at four / three CTAs per SM)
  bool autotune = true;
  std::vector<int> tune_path[2], tune_tile[2];
  int tuned_path(int prec, int l) const {
    return l >= 0 && l < (int)tune_path[prec].size() ? tune_path[prec][l] : -1;
  }
  bool tf32 = false;                         // tensor-core (TF32) local solves where available
  int force_tile = -1;                       // SIPG_TILE: this interior tile on every level (tests)
  int tuned_tile(int prec, int l) const {
    if (force_tile >= 0) return force_tile;
    return l >= 0 && l < (int)tune_tile[prec].size() ? tune_tile[prec][l] : 0;
  }
  // second stream for the boundary-patch kernel of a colour pass, forked
  // from and joined to the calling stream with these events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int prio_hi = 0;  // greatest launch priority of the device: the interior kernel of a colour pass
  // colour passes: the boundary-patch kernel is launched first and at
  // prio_hi, the interior one fills the SMs behind it (SIPG_BOUNDARY_FIRST=0:
  // the other way round)
  bool bnd_first = true;
  // host copies of the device-computed level constants (read back once at
  // bind time; kernels receive the small 1D operators as launch parameters)
  std::vector<LevelConst<double>> hc64;
  std::vector<LevelConst<float>> hc32;
  template <typename T> const LevelConst<T>& hcst(int l) const;

  // CUDA graph of one Krylov iteration (optional)
  cudaGraphExec_t iter_exec = nullptr;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  double* g_x = nullptr;
  double g_rtol2 = -1.0;  // the tolerance the captured iteration was recorded with
  uint64_t graph_launches = 0;               // kernels inside one graph launch
  // CUDA graph of one GMRES restart cycle: a conditional while node whose
  // body is one Arnoldi step, recorded for one workspace, restart length
  // and side of preconditioning
  cudaGraphExec_t gm_exec = nullptr;
  const char* gm_work = nullptr;
  int gm_m = 0;
  bool gm_left = false;
  uint64_t gm_launches = 0;                  // kernels in one step body

  LevelConst<double>* c64(int l) const { return reinterpret_cast<LevelConst<double>*>(ws + off_const64) + l; }
  LevelConst<float>* c32(int l) const { return reinterpret_cast<LevelConst<float>*>(ws + off_const32) + l; }
  template <typename T> LevelConst<T>* cst(int l) const;
  void* vb(int l) const { return ws + off_b[l]; }
  void* vx(int l) const { return ws + off_x[l]; }
  void* vr(int l) const { return ws + off_r[l]; }
  double* kr() const { return reinterpret_cast<double*>(ws + off_kr); }
  double* kz() const { return reinterpret_cast<double*>(ws + off_kz); }
  double* kp() const { return reinterpret_cast<double*>(ws + off_kp); }
  double* kq() const { return reinterpret_cast<double*>(ws + off_kq); }
  double* partials() const { return reinterpret_cast<double*>(ws + off_partials); }
  KrylovScalars* scalars() const { return reinterpret_cast<KrylovScalars*>(ws + off_scalars); }
};
template <> inline LevelConst<double>* sipg_handle::cst<double>(int l) const { return c64(l); }
template <> inline LevelConst<float>* sipg_handle::cst<float>(int l) const { return c32(l); }
template <> inline const LevelConst<double>& sipg_handle::hcst<double>(int l) const { return hc64[l]; }
template <> inline const LevelConst<float>& sipg_handle::hcst<float>(int l) const { return hc32[l]; }

// ---------------------------------------------------------------- launchers
// Each returns cudaGetLastError() after its launches; `nrhs` columns of
// length `ndofs` are processed.
cudaError_t launch_setup(sipg_handle* h, cudaStream_t s);
template <typename T>
cudaError_t launch_apply(const sipg_handle* h, int level, int mode, const T* b, const T* x, T* y,
                         cudaStream_t s);
cudaError_t launch_mass(const sipg_handle* h, const double* f, double* b, cudaStream_t s);
cudaError_t launch_manufactured(const sipg_handle* h, double* f, cudaStream_t s);
template <typename T>
cudaError_t launch_smooth_colour(const sipg_handle* h, int level, int colour, const T* b, T* x,
                                 cudaStream_t s);
// Full-kernel colour pass (smooth_full.cu): r = b - A x on the whole level
// into the level's residual buffer, then every patch of the colour adds
// A_j^{-1} R_j r.  Reports its launches.
template <typename T>
cudaError_t launch_full_colour(const sipg_handle* h, int level, int colour, const T* b, T* x, cudaStream_t s,
                               int* launches);
// One smoothing step (all colours, reversed order if `reverse`); reports the
// number of kernels it launched.
template <typename T>
cudaError_t launch_smooth_step(const sipg_handle* h, int level, int reverse, const T* b, T* x, cudaStream_t s,
                               int* launches);
cudaError_t launch_barrier_selftest(const sipg_handle* h, int extra, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(const sipg_handle* h, int fine_level, const T* rf, T* rc, cudaStream_t s);
template <typename T>
cudaError_t launch_prolongate_add(const sipg_handle* h, int fine_level, const T* ec, T* xf,
                                  cudaStream_t s);
// b_{level-1} = P^T (b - A x) on `level` without storing the fine residual;
// cudaErrorNotSupported where the fused kernel does not apply.
template <typename T>
cudaError_t launch_residual_restrict(const sipg_handle* h, int level, const T* b, const T* x, T* rc,
                                     cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve(const sipg_handle* h, const T* b0, T* x0, cudaStream_t s);

// apply modes
enum { APPLY_Y = 0, APPLY_RESIDUAL = 1, APPLY_PENALTY = 2 };

// Krylov kernels (krylov.cu)
cudaError_t launch_dot(sipg_handle* h, const double* a, const double* b, double* out,
                       cudaStream_t s);
cudaError_t krylov_init_norms(sipg_handle* h, const double* b, const double* r, cudaStream_t s);
cudaError_t krylov_after_precond(sipg_handle* h, int first, const double* r, const void* zsrc,
                                 int zsrc_is_float, cudaStream_t s);
cudaError_t krylov_after_apply(sipg_handle* h, cudaStream_t s);
cudaError_t krylov_update_xr(sipg_handle* h, double* x, void* bL, int bL_is_float, cudaStream_t s);
// GMRES vector kernels (krylov.cu); nrhs = 1.  out[i] = <V_i, w> for
// i < cnt (V_i = V + i * ld), deterministic two-stage sums (partials holds
// cnt * n_partials doubles); w += sign * sum_q c_q V_q with c in device
// memory (cdev) or copied from the host into the launch parameters (chost);
// w *= a.
cudaError_t gmres_mdot(sipg_handle* h, const double* V, long long ld, int cnt, const double* w, long long n,
                       double* partials, double* out, cudaStream_t s);
cudaError_t gmres_maxpy(sipg_handle* h, double* w, const double* V, long long ld, int cnt, const double* cdev,
                        const double* chost, double sign, long long n, cudaStream_t s);
cudaError_t gmres_scale(sipg_handle* h, double* w, double a, long long n, cudaStream_t s);
// Device-resident cycle (GmresCycleState st; j = st->j when the kernel runs):
// setup: st cleared, g_0 = beta, thr and budget set; gather: out = V_j
// (converted to float when out_float); put: Z_j = in (float or double
// input) and, if copy is not null, copy = the same values; mdot_dev:
// out[i] = <V_i, w> for i <= j (grid sized for m + 1 vectors); maxpy_dev:
// w -= sum_{i <= j} c_i V_i; rotate: the new Hessenberg column from hc1 +
// hc2 and sqrt(nrm), the earlier rotations, the new rotation, g, hist, the
// stopping flags, j += 1, and the loop condition of the cycle graph set to
// continue or stop; next: V_j = w / ||w|| (j already advanced; nothing after
// a breakdown).
cudaError_t gmres_cycle_setup(sipg_handle* h, GmresCycleState* st, double beta, double thr, int budget,
                              cudaStream_t s);
cudaError_t gmres_gather(sipg_handle* h, const double* V, long long ld, const GmresCycleState* st, void* out,
                         bool out_float, long long n, cudaStream_t s);
cudaError_t gmres_put(sipg_handle* h, const void* in, bool in_float, double* Z, long long ld,
                      const GmresCycleState* st, double* copy, long long n, cudaStream_t s);
cudaError_t gmres_mdot_dev(sipg_handle* h, const double* V, long long ld, const GmresCycleState* st, int m,
                           const double* w, long long n, double* partials, double* out, cudaStream_t s);
cudaError_t gmres_maxpy_dev(sipg_handle* h, double* w, const double* V, long long ld, const GmresCycleState* st,
                            const double* c, long long n, cudaStream_t s);
cudaError_t gmres_rotate(sipg_handle* h, GmresCycleState* st, cudaGraphConditionalHandle cond, cudaStream_t s);
cudaError_t gmres_next(sipg_handle* h, const double* w, double* V, long long ld, const GmresCycleState* st,
                       long long n, cudaStream_t s);
cudaError_t convert_d2f(const double* a, float* b, size_t n, cudaStream_t s);
cudaError_t convert_f2d(const float* a, double* b, size_t n, cudaStream_t s);
cudaError_t copy_or_zero(void* dst, size_t bytes, cudaStream_t s);
// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per (kernel, device, bytes).  cudaFuncSetAttribute acts on the
// current device only, so the record is kept per device; a mutex guards it
// against concurrent first calls from several host threads.
cudaError_t smem_opt_in(const void* kernel, int bytes);
// Kernels one Dirichlet- or clamped-kernel colour pass launches on a level of
// N cells per direction (interior and domain-boundary patches).
int colour_kernels(int dim, int N, int colour);
// Interior patches of a 3D FP32 colour pass with the fast-diagonalisation
// sweeps on the tensor cores (TF32); cudaErrorNotSupported where that kernel
// does not apply (the caller then launches the FP32 kernel).
cudaError_t launch_tc3(const sipg_handle* h, int level, int colour, const float* b, float* x, cudaStream_t s);
// Ragged 2D batches: batched smoothing stages (smooth_batch2.cu).
struct BatchPlan2;
bool batch2_supported(const std::vector<sipg_handle*>& hs);
size_t batch2_plan_bytes(const std::vector<sipg_handle*>& hs);
cudaError_t batch2_plan_build(const std::vector<sipg_handle*>& hs, char* dev, BatchPlan2** out);
void batch2_plan_free(BatchPlan2* p);
int batch2_levels(const BatchPlan2* p);
cudaError_t batch2_step(const BatchPlan2* p, int level, int reverse, cudaStream_t s);
int* batch2_status(const BatchPlan2* p);
cudaError_t launch_tc_selftest(const sipg_handle* h, const float* A, const float* B, float* D, cudaStream_t s);
// smem_opt_in, then the kernel's resident CTAs per SM at that launch shape on
// the current device (cached per kernel, device and shape).
cudaError_t smem_opt_in_occupancy(const void* kernel, int threads, int bytes, int* ctas_per_sm);

static inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
