// FP64 vector kernels of the outer flexible CG: dot products with a
// deterministic two-stage reduction (warp shuffles inside a block, fixed-order
// sum of the per-block partials in a second kernel), device-resident Krylov
// scalars so that one iteration can be replayed as a CUDA graph without host
// round trips, and fused updates (x += alpha p, r -= alpha q, ||r||^2 and the
// FP64 -> FP32 conversion at V-cycle entry; the FP32 -> FP64 conversion of the
// V-cycle output fused with <r, z> and <z, q>).  Mixed precision: Sec. 5.2.
#include <math.h>

#include <algorithm>

#include "sipg_internal.cuh"

namespace {

constexpr int RB = 256;  // threads per reduction block

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of up to 3 values, fixed order; result valid in thread 0.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ]) {
  __shared__ double red[NQ][RB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) red[q][w] = s;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = (lane < RB / 32) ? red[q][lane] : 0.0;
      v[q] = warp_sum(s);
    }
  }
}

struct DotArgs {
  const double* a[3];
  const double* b[3];
};

template <int NQ>
__global__ void __launch_bounds__(RB) dot_partial_kernel(DotArgs args, long long n, double* partials) {
  const long long col = (long long)blockIdx.y * n;
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = fma(args.a[q][col + i], args.b[q][col + i], v[q]);
  }
  block_sum<NQ>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) partials[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 3 + q] = v[q];
  }
}

enum { FIN_INIT = 0, FIN_RHO_FIRST, FIN_RHO_NEXT, FIN_PQ, FIN_RR, FIN_OUT };

// One block per column: sums the nb partials of each quantity in a fixed
// order and updates the Krylov scalars of that column.
__global__ void __launch_bounds__(RB) finalize_kernel(int mode, KrylovScalars* sc, const double* partials,
                                                      int nb, double rtol2, double* out) {
  const int col = blockIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += RB) {
    const double* p = partials + ((long long)col * nb + i) * 3;
    v[0] += p[0];
    v[1] += p[1];
    v[2] += p[2];
  }
  block_sum<3>(v);
  if (threadIdx.x != 0) return;
  KrylovScalars& s = sc[col];
  switch (mode) {
    case FIN_INIT:
      s.bb = v[0];
      s.rr = v[1];
      s.rho = s.alpha = s.beta = s.pq = s.zq = 0.0;
      s.breakdown = !(isfinite(v[0]) && isfinite(v[1]));
      s.active = (!s.breakdown && v[0] > 0.0 && v[1] > rtol2 * v[0]) ? 1 : 0;
      break;
    case FIN_RHO_FIRST:
      s.rho = v[0];
      if (s.active && !isfinite(v[0])) {
        s.breakdown = 1;
        s.active = 0;
      }
      break;
    case FIN_RHO_NEXT: {
      // flexible CG: beta = <z_{i+1}, r_{i+1} - r_i> / <z_i, r_i>
      //                   = -alpha_i <z_{i+1}, q_i> / <z_i, r_i>   (r_{i+1} = r_i - alpha_i q_i)
      double beta = 0.0;
      if (s.active) {
        beta = -s.alpha * v[1] / s.rho;
        if (!isfinite(beta) || !isfinite(v[0])) {
          s.breakdown = 1;
          s.active = 0;
          beta = 0.0;
        }
      }
      s.beta = beta;
      s.zq = v[1];
      s.rho = v[0];
      break;
    }
    case FIN_PQ: {
      s.pq = v[0];
      double alpha = 0.0;
      if (s.active) {
        if (v[0] > 0.0 && isfinite(v[0]) && isfinite(s.rho)) {
          alpha = s.rho / v[0];
        } else {
          s.breakdown = 1;
          s.active = 0;
        }
      }
      s.alpha = alpha;
      break;
    }
    case FIN_RR:
      s.rr = v[0];
      if (s.active && !isfinite(v[0])) {
        s.breakdown = 1;
        s.active = 0;
      } else if (s.active && v[0] <= rtol2 * s.bb) {
        s.active = 0;
      }
      break;
    case FIN_OUT:
      out[col] = v[0];
      break;
  }
}

// partial <r, z> and <z, q> with z = double(zsrc); z is also stored when
// the pointer is given and differs from zsrc (an FP32 V-cycle output is read
// again by p_update_kernel instead).
template <typename TZ>
__global__ void __launch_bounds__(RB) precond_post_kernel(const TZ* zsrc, double* z, const double* r,
                                                          const double* q, long long n, double* partials,
                                                          int want_zq) {
  const long long col = (long long)blockIdx.y * n;
  double v[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) {
    double zi = (double)zsrc[col + i];
    if (z && (const void*)zsrc != (const void*)z) z[col + i] = zi;
    v[0] = fma(r[col + i], zi, v[0]);
    if (want_zq) v[1] = fma(zi, q[col + i], v[1]);
  }
  block_sum<3>(v);
  if (threadIdx.x == 0) {
    double* p = partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * 3;
    p[0] = v[0];
    p[1] = v[1];
    p[2] = 0.0;
  }
}

// p = z + beta p (p = z first), z = double(z_src)
template <typename TZ>
__global__ void __launch_bounds__(RB) p_update_kernel(int first, const TZ* z, double* p,
                                                      const KrylovScalars* sc, long long n) {
  const long long col = (long long)blockIdx.y * n;
  const double beta = first ? 0.0 : sc[blockIdx.y].beta;
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) {
    const double zi = (double)z[col + i];
    p[col + i] = first ? zi : fma(beta, p[col + i], zi);
  }
}

// x += alpha p, r -= alpha q, partial ||r||^2, optional V-cycle input bL = r.
template <typename TB>
__global__ void __launch_bounds__(RB) xr_update_kernel(double* x, double* r, const double* p, const double* q,
                                                       const KrylovScalars* sc, TB* bL, long long n,
                                                       double* partials) {
  const long long col = (long long)blockIdx.y * n;
  const double alpha = sc[blockIdx.y].alpha;
  double v[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) {
    const long long j = col + i;
    x[j] = fma(alpha, p[j], x[j]);
    double ri = fma(-alpha, q[j], r[j]);
    r[j] = ri;
    v[0] = fma(ri, ri, v[0]);
    if (bL) bL[j] = (TB)ri;
  }
  block_sum<3>(v);
  if (threadIdx.x == 0) {
    double* pp = partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * 3;
    pp[0] = v[0];
    pp[1] = 0.0;
    pp[2] = 0.0;
  }
}

__global__ void d2f_kernel(const double* a, float* b, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (float)a[i];
}
__global__ void f2d_kernel(const float* a, double* b, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (double)a[i];
}

// ---------------------------------------------------------------- GMRES
// partial <V_i, w> of vector i = blockIdx.y (V_i starts at V + i * ld)
__global__ void __launch_bounds__(RB) mdot_partial_kernel(const double* V, long long ld, const double* w,
                                                          long long n, double* partials) {
  const double* v = V + (long long)blockIdx.y * ld;
  double acc[1] = {0.0};
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) acc[0] = fma(v[i], w[i], acc[0]);
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = acc[0];
}

// partials of <V_i, w> for every i <= *lim in one launch (one block per
// partial, vectors in turn): the same element-to-partial mapping as
// mdot_partial_kernel with gridDim.x blocks, so the sums are the same
__global__ void __launch_bounds__(RB) mdot_multi_partial_kernel(const double* V, long long ld, const double* w,
                                                                long long n, double* partials, const int* lim) {
  const int cnt = *lim + 1;
  const long long stride = (long long)gridDim.x * RB;
  for (int q = 0; q < cnt; ++q) {
    const double* v = V + (long long)q * ld;
    double acc[1] = {0.0};
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) acc[0] = fma(v[i], w[i], acc[0]);
    block_sum<1>(acc);
    if (threadIdx.x == 0) partials[(long long)q * gridDim.x + blockIdx.x] = acc[0];
    __syncthreads();  // block_sum's shared slots are reused by the next vector
  }
}

// out[i] = the nb partials of vector i = blockIdx.x summed in a fixed order
__global__ void __launch_bounds__(RB) mdot_finalize_kernel(const double* partials, int nb, double* out,
                                                           const int* lim) {
  if (lim && (int)blockIdx.x > *lim) return;
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += RB) acc[0] += partials[(long long)blockIdx.x * nb + i];
  block_sum<1>(acc);
  if (threadIdx.x == 0) out[blockIdx.x] = acc[0];
}

struct GmresCoef {
  double c[SIPG_GMRES_MAXM + 1];
};

// w += sign * sum_{q < cnt} c_q V_q with c from device memory (cdev) or from
// the parameter block (cdev == nullptr); with cnt_dev, cnt = *cnt_dev + 1
__global__ void __launch_bounds__(RB) maxpy_kernel(double* w, const double* V, long long ld, int cnt,
                                                   const double* cdev, GmresCoef cpar, double sign, long long n,
                                                   const int* cnt_dev) {
  if (cnt_dev) cnt = *cnt_dev + 1;
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) {
    double acc = 0.0;
    for (int q = 0; q < cnt; ++q) acc = fma(cdev ? cdev[q] : cpar.c[q], V[q * ld + i], acc);
    w[i] = fma(sign, acc, w[i]);
  }
}

__global__ void __launch_bounds__(RB) scale_kernel(double* w, double a, long long n) {
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) w[i] *= a;
}

// ------------------------------------------- GMRES cycle on the device
__global__ void __launch_bounds__(RB) gmres_setup_kernel(GmresCycleState* st, double beta, double thr,
                                                         int budget) {
  constexpr int M = SIPG_GMRES_MAXM;
  for (int i = threadIdx.x; i < (M + 1) * M; i += RB) st->H[i] = 0.0;
  for (int i = threadIdx.x; i <= M; i += RB) {
    st->g[i] = 0.0;
    st->hc1[i] = 0.0;
    st->hc2[i] = 0.0;
    if (i < M) {
      st->cs[i] = 0.0;
      st->sn[i] = 0.0;
      st->hist[i] = 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->j = 0;
    st->budget = budget;
    st->conv = 0;
    st->brk = 0;
    st->runs = 0;
    st->thr = thr;
    st->nrm = 0.0;
    st->hn = 0.0;
    st->g[0] = beta;
  }
}

template <typename TO>
__global__ void __launch_bounds__(RB) gmres_gather_kernel(const double* V, long long ld, const GmresCycleState* st,
                                                          TO* out, long long n) {
  const double* v = V + (long long)st->j * ld;
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) out[i] = (TO)v[i];
}

template <typename TI>
__global__ void __launch_bounds__(RB) gmres_put_kernel(const TI* in, double* Z, long long ld,
                                                       const GmresCycleState* st, double* copy, long long n) {
  double* z = Z + (long long)st->j * ld;
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) {
    const double v = (double)in[i];
    z[i] = v;
    if (copy) copy[i] = v;
  }
}

// One thread: the step's Hessenberg column and rotations, the same
// arithmetic in the same order as the host loop of gmres_run.  Every path
// ends in exactly one cudaGraphSetConditional, and the loop stops at the
// latest after `budget` bodies (runs), whatever the flags say.
__global__ void gmres_rotate_kernel(GmresCycleState* st, cudaGraphConditionalHandle cond) {
  constexpr int M = SIPG_GMRES_MAXM;
  unsigned int more = 0;
  st->runs += 1;
  const int j = st->j;
  if (!st->conv && !st->brk && j < st->budget && j < M && st->runs <= st->budget) {
    double* H = st->H;
    const double hn = sqrt(st->nrm);
    bool finite = isfinite(hn);
    for (int i = 0; i <= j; ++i) finite = finite && isfinite(st->hc1[i] + st->hc2[i]);
    if (!finite) {
      st->brk = 1;
    } else {
      for (int i = 0; i <= j; ++i) H[i * M + j] = st->hc1[i] + st->hc2[i];
      H[(j + 1) * M + j] = hn;
      st->hn = hn;
      for (int i = 0; i < j; ++i) {
        const double a = H[i * M + j], c = H[(i + 1) * M + j];
        H[i * M + j] = st->cs[i] * a + st->sn[i] * c;
        H[(i + 1) * M + j] = -st->sn[i] * a + st->cs[i] * c;
      }
      const double den = hypot(H[j * M + j], H[(j + 1) * M + j]);
      if (!(den > 0.0)) {
        st->brk = 1;
      } else {
        st->cs[j] = H[j * M + j] / den;
        st->sn[j] = H[(j + 1) * M + j] / den;
        H[j * M + j] = den;
        H[(j + 1) * M + j] = 0.0;
        st->g[j + 1] = -st->sn[j] * st->g[j];
        st->g[j] = st->cs[j] * st->g[j];
        st->hist[j] = fabs(st->g[j + 1]);
        st->j = j + 1;
        if (fabs(st->g[j + 1]) <= st->thr || hn == 0.0) st->conv = 1;
        more = (!st->conv && st->j < st->budget) ? 1u : 0u;
      }
    }
  }
  cudaGraphSetConditional(cond, more);
}

__global__ void __launch_bounds__(RB) gmres_next_kernel(const double* w, double* V, long long ld,
                                                        const GmresCycleState* st, long long n) {
  if (st->brk) return;
  double* v = V + (long long)st->j * ld;
  const double hn = st->hn;
  const double a = hn > 0.0 ? 1.0 / hn : 1.0;
  const long long stride = (long long)gridDim.x * RB;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < n; i += stride) v[i] = w[i] * a;
}

}  // namespace

static inline long long fine_n(const sipg_handle* h) { return (long long)h->lv[h->L].ndofs; }

cudaError_t gmres_mdot(sipg_handle* h, const double* V, long long ld, int cnt, const double* w, long long n,
                       double* partials, double* out, cudaStream_t s) {
  if (cnt < 1 || cnt > SIPG_GMRES_MAXM + 1) return cudaErrorInvalidValue;
  dim3 grid(h->n_partials, cnt);
  mdot_partial_kernel<<<grid, RB, 0, s>>>(V, ld, w, n, partials);
  mdot_finalize_kernel<<<cnt, RB, 0, s>>>(partials, h->n_partials, out, nullptr);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t gmres_maxpy(sipg_handle* h, double* w, const double* V, long long ld, int cnt, const double* cdev,
                        const double* chost, double sign, long long n, cudaStream_t s) {
  if (cnt < 1 || cnt > SIPG_GMRES_MAXM + 1 || (!cdev && !chost)) return cudaErrorInvalidValue;
  GmresCoef cp;
  for (int q = 0; q <= SIPG_GMRES_MAXM; ++q) cp.c[q] = (!cdev && q < cnt) ? chost[q] : 0.0;
  const int blocks = std::min(ceil_div(n, RB), 64 * h->num_sms);
  maxpy_kernel<<<blocks, RB, 0, s>>>(w, V, ld, cnt, cdev, cp, sign, n, nullptr);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t gmres_scale(sipg_handle* h, double* w, double a, long long n, cudaStream_t s) {
  const int blocks = std::min(ceil_div(n, RB), 64 * h->num_sms);
  scale_kernel<<<blocks, RB, 0, s>>>(w, a, n);
  h->launches += 1;
  return cudaGetLastError();
}

static inline int vec_blocks(const sipg_handle* h, long long n) {
  return (int)std::min<long long>(ceil_div(n, RB), 64LL * h->num_sms);
}

cudaError_t gmres_cycle_setup(sipg_handle* h, GmresCycleState* st, double beta, double thr, int budget,
                              cudaStream_t s) {
  gmres_setup_kernel<<<1, RB, 0, s>>>(st, beta, thr, budget);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t gmres_gather(sipg_handle* h, const double* V, long long ld, const GmresCycleState* st, void* out,
                         bool out_float, long long n, cudaStream_t s) {
  if (out_float)
    gmres_gather_kernel<float><<<vec_blocks(h, n), RB, 0, s>>>(V, ld, st, static_cast<float*>(out), n);
  else
    gmres_gather_kernel<double><<<vec_blocks(h, n), RB, 0, s>>>(V, ld, st, static_cast<double*>(out), n);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t gmres_put(sipg_handle* h, const void* in, bool in_float, double* Z, long long ld,
                      const GmresCycleState* st, double* copy, long long n, cudaStream_t s) {
  if (in_float)
    gmres_put_kernel<float><<<vec_blocks(h, n), RB, 0, s>>>(static_cast<const float*>(in), Z, ld, st, copy, n);
  else
    gmres_put_kernel<double><<<vec_blocks(h, n), RB, 0, s>>>(static_cast<const double*>(in), Z, ld, st, copy, n);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t gmres_mdot_dev(sipg_handle* h, const double* V, long long ld, const GmresCycleState* st, int m,
                           const double* w, long long n, double* partials, double* out, cudaStream_t s) {
  if (m < 1 || m > SIPG_GMRES_MAXM) return cudaErrorInvalidValue;
  mdot_multi_partial_kernel<<<h->n_partials, RB, 0, s>>>(V, ld, w, n, partials, &st->j);
  mdot_finalize_kernel<<<m + 1, RB, 0, s>>>(partials, h->n_partials, out, &st->j);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t gmres_maxpy_dev(sipg_handle* h, double* w, const double* V, long long ld, const GmresCycleState* st,
                            const double* c, long long n, cudaStream_t s) {
  GmresCoef cp{};
  maxpy_kernel<<<vec_blocks(h, n), RB, 0, s>>>(w, V, ld, 0, c, cp, -1.0, n, &st->j);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t gmres_rotate(sipg_handle* h, GmresCycleState* st, cudaGraphConditionalHandle cond, cudaStream_t s) {
  gmres_rotate_kernel<<<1, 1, 0, s>>>(st, cond);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t gmres_next(sipg_handle* h, const double* w, double* V, long long ld, const GmresCycleState* st,
                       long long n, cudaStream_t s) {
  gmres_next_kernel<<<vec_blocks(h, n), RB, 0, s>>>(w, V, ld, st, n);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_dot(sipg_handle* h, const double* a, const double* b, double* out,
                       cudaStream_t s) {
  DotArgs args{{a, nullptr, nullptr}, {b, nullptr, nullptr}};
  dim3 grid(h->n_partials, h->prm.nrhs);
  dot_partial_kernel<1><<<grid, RB, 0, s>>>(args, fine_n(h), h->partials());
  finalize_kernel<<<h->prm.nrhs, RB, 0, s>>>(FIN_OUT, h->scalars(), h->partials(), h->n_partials,
                                             0.0, out);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t krylov_init_norms(sipg_handle* h, const double* b, const double* r, cudaStream_t s) {
  DotArgs args{{b, r, nullptr}, {b, r, nullptr}};
  dim3 grid(h->n_partials, h->prm.nrhs);
  dot_partial_kernel<2><<<grid, RB, 0, s>>>(args, fine_n(h), h->partials());
  finalize_kernel<<<h->prm.nrhs, RB, 0, s>>>(FIN_INIT, h->scalars(), h->partials(), h->n_partials,
                                             h->rtol2, nullptr);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t krylov_after_precond(sipg_handle* h, int first, const double* r, const void* zsrc,
                                 int zsrc_is_float, cudaStream_t s) {
  dim3 grid(h->n_partials, h->prm.nrhs);
  // an FP32 V-cycle output stays in its buffer: the dots and the direction
  // update convert it on the fly (no FP64 copy of z is written)
  if (zsrc_is_float)
    precond_post_kernel<float><<<grid, RB, 0, s>>>((const float*)zsrc, nullptr, r, h->kq(), fine_n(h),
                                                   h->partials(), first ? 0 : 1);
  else
    precond_post_kernel<double><<<grid, RB, 0, s>>>((const double*)zsrc, h->kz(), r, h->kq(), fine_n(h),
                                                    h->partials(), first ? 0 : 1);
  finalize_kernel<<<h->prm.nrhs, RB, 0, s>>>(first ? FIN_RHO_FIRST : FIN_RHO_NEXT, h->scalars(),
                                             h->partials(), h->n_partials, h->rtol2, nullptr);
  if (zsrc_is_float)
    p_update_kernel<float><<<grid, RB, 0, s>>>(first, (const float*)zsrc, h->kp(), h->scalars(), fine_n(h));
  else
    p_update_kernel<double><<<grid, RB, 0, s>>>(first, h->kz(), h->kp(), h->scalars(), fine_n(h));
  h->launches += 3;
  return cudaGetLastError();
}

cudaError_t krylov_after_apply(sipg_handle* h, cudaStream_t s) {
  DotArgs args{{h->kp(), nullptr, nullptr}, {h->kq(), nullptr, nullptr}};
  dim3 grid(h->n_partials, h->prm.nrhs);
  dot_partial_kernel<1><<<grid, RB, 0, s>>>(args, fine_n(h), h->partials());
  finalize_kernel<<<h->prm.nrhs, RB, 0, s>>>(FIN_PQ, h->scalars(), h->partials(), h->n_partials,
                                             h->rtol2, nullptr);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t krylov_update_xr(sipg_handle* h, double* x, void* bL, int bL_is_float, cudaStream_t s) {
  dim3 grid(h->n_partials, h->prm.nrhs);
  if (bL_is_float)
    xr_update_kernel<float><<<grid, RB, 0, s>>>(x, h->kr(), h->kp(), h->kq(), h->scalars(), (float*)bL,
                                                fine_n(h), h->partials());
  else
    xr_update_kernel<double><<<grid, RB, 0, s>>>(x, h->kr(), h->kp(), h->kq(), h->scalars(),
                                                 (double*)bL, fine_n(h), h->partials());
  finalize_kernel<<<h->prm.nrhs, RB, 0, s>>>(FIN_RR, h->scalars(), h->partials(), h->n_partials,
                                             h->rtol2, nullptr);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t convert_d2f(const double* a, float* b, size_t n, cudaStream_t s) {
  d2f_kernel<<<ceil_div((long long)n, 256 * 8), 256, 0, s>>>(a, b, (long long)n);
  return cudaGetLastError();
}
cudaError_t convert_f2d(const float* a, double* b, size_t n, cudaStream_t s) {
  f2d_kernel<<<ceil_div((long long)n, 256 * 8), 256, 0, s>>>(a, b, (long long)n);
  return cudaGetLastError();
}
