// Grid transfer between nested levels (Sec. 3, Sec. 4.2) and the exact
// coarse solve P_0^{-1} = A_0^{-1} (Sec. 3).
//
// Prolongation is the canonical embedding: fine cell f = 2C + o (o in
// {0,1}^d) receives (Pc[o_2] (x) Pc[o_1] (x) Pc[o_0]) e_C with
// Pc[o][i][j] = phi_j((o + xi_i)/2).  Restriction of residuals is its
// transpose.  Both loop over coarse (parent) cells and contract one direction
// at a time (Sec. 4.2: x first, then y, then z), so no two threads write the
// same fine DoF and no atomics are needed.
//
// Coarse solve: on the coarsest level A_0 = sum_e (x)(L, M) exactly, so
// A_0^{-1} = (S (x) S (x) S) (sum Lambda)^{-1} (S^T (x) S^T (x) S^T) with the
// global 1D eigenpairs of the coarsest level, applied in FP64 in one CTA in
// global lexicographic order.
#include "tensor_ops.cuh"

namespace {

template <int DIM, int NN>
constexpr int transfer_cpb() {
  return DIM == 2 ? 8 : (NN <= 4 ? 4 : (NN <= 6 ? 2 : 1));
}

// x_fine += P e_coarse
template <int DIM, int NN, typename T, int CPB>
__global__ void prolongate_kernel(const LevelConst<T>* __restrict__ lc, const T* __restrict__ ec,
                                  T* __restrict__ xf, int Nc, long long ncc, long long ndc,
                                  long long ndf) {
  using CS = CellShape<DIM, NN>;
  constexpr int ND = CS::dofs, NL = CS::lines;
  __shared__ T Pm[2][NN * NN];
  __shared__ T Ec[CPB * ND], T1[CPB * 2 * ND], T2[DIM == 3 ? CPB * 4 * ND : 1];
  const int tid = threadIdx.x, nth = blockDim.x;
  ec += (long long)blockIdx.y * ndc;
  xf += (long long)blockIdx.y * ndf;
  for (int o = 0; o < 2; ++o) copy_block<NN>(Pm[o], lc->Pc[o], tid, nth);
  const long long c0 = (long long)blockIdx.x * CPB;
  const int ncb = (int)min((long long)CPB, ncc - c0);
  for (int e = tid; e < ncb * ND; e += nth) Ec[e] = ec[c0 * ND + e];
  __syncthreads();
  // x-sweep: T1[cl][o0] = Pc[o0] along x
  for (int task = tid; task < ncb * 2 * NL; task += nth) {
    int cl = task / (2 * NL), rem = task % (2 * NL), o0 = rem / NL, l = rem % NL;
    int base, stride;
    CS::line(0, l, base, stride);
    T v[NN], w[NN];
    load_line<NN>(Ec + cl * ND + base, stride, v);
    matvec_line<NN>(Pm[o0], v, w);
    store_line<NN>(T1 + (cl * 2 + o0) * ND + base, stride, w);
  }
  __syncthreads();
  const int Nf = 2 * Nc;
  if (DIM == 2) {
    // y-sweep straight into the fine cells
    for (int task = tid; task < ncb * 4 * NL; task += nth) {
      int cl = task / (4 * NL), rem = task % (4 * NL), ch = rem / NL, l = rem % NL;
      int o0 = ch & 1, o1 = ch >> 1;
      int base, stride;
      CS::line(1, l, base, stride);
      T v[NN], w[NN];
      load_line<NN>(T1 + (cl * 2 + o0) * ND + base, stride, v);
      matvec_line<NN>(Pm[o1], v, w);
      long long C = c0 + cl;
      int cx = (int)(C % Nc), cy = (int)(C / Nc);
      long long f = (2 * cx + o0) + (long long)Nf * (2 * cy + o1);
      T* dst = xf + f * ND + base;
#pragma unroll
      for (int i = 0; i < NN; ++i) dst[i * stride] += w[i];
    }
  } else {
    for (int task = tid; task < ncb * 4 * NL; task += nth) {
      int cl = task / (4 * NL), rem = task % (4 * NL), ch = rem / NL, l = rem % NL;
      int o0 = ch & 1, o1 = ch >> 1;
      int base, stride;
      CS::line(1, l, base, stride);
      T v[NN], w[NN];
      load_line<NN>(T1 + (cl * 2 + o0) * ND + base, stride, v);
      matvec_line<NN>(Pm[o1], v, w);
      store_line<NN>(T2 + (cl * 4 + ch) * ND + base, stride, w);
    }
    __syncthreads();
    for (int task = tid; task < ncb * 8 * NL; task += nth) {
      int cl = task / (8 * NL), rem = task % (8 * NL), ch = rem / NL, l = rem % NL;
      int o01 = ch & 3, o2 = ch >> 2;
      int base, stride;
      CS::line(2, l, base, stride);
      T v[NN], w[NN];
      load_line<NN>(T2 + (cl * 4 + o01) * ND + base, stride, v);
      matvec_line<NN>(Pm[o2], v, w);
      long long C = c0 + cl;
      int cx = (int)(C % Nc), cy = (int)((C / Nc) % Nc), cz = (int)(C / ((long long)Nc * Nc));
      long long f = (2 * cx + (o01 & 1)) +
                    (long long)Nf * ((2 * cy + (o01 >> 1)) + (long long)Nf * (2 * cz + o2));
      T* dst = xf + f * ND + base;
#pragma unroll
      for (int i = 0; i < NN; ++i) dst[i * stride] += w[i];
    }
  }
}

// r_coarse = P^T r_fine
template <int DIM, int NN, typename T, int CPB>
__global__ void restrict_kernel(const LevelConst<T>* __restrict__ lc, const T* __restrict__ rf,
                                T* __restrict__ rc, int Nc, long long ncc, long long ndc,
                                long long ndf) {
  using CS = CellShape<DIM, NN>;
  constexpr int ND = CS::dofs, NL = CS::lines;
  constexpr int NU = (DIM == 2) ? 2 : 4;  // x-summed arrays per coarse cell
  __shared__ T PmT[2][NN * NN];           // transposed: PmT[o][j][i] = Pc[o][i][j]
  __shared__ T U[CPB * NU * ND], V[DIM == 3 ? CPB * 2 * ND : 1];
  const int tid = threadIdx.x, nth = blockDim.x;
  rf += (long long)blockIdx.y * ndf;
  rc += (long long)blockIdx.y * ndc;
  for (int e = tid; e < 2 * NN * NN; e += nth) {
    int o = e / (NN * NN), r = e % (NN * NN), j = r / NN, i = r % NN;
    PmT[o][j * NN + i] = lc->Pc[o][i][j];
  }
  __syncthreads();
  const long long c0 = (long long)blockIdx.x * CPB;
  const int ncb = (int)min((long long)CPB, ncc - c0);
  const int Nf = 2 * Nc;
  // x-sweep over the two x-children: U[cl][u] = sum_o0 Pc[o0]^T r_child (along x)
  for (int task = tid; task < ncb * NU * NL; task += nth) {
    int cl = task / (NU * NL), rem = task % (NU * NL), u = rem / NL, l = rem % NL;
    int base, stride;
    CS::line(0, l, base, stride);
    long long C = c0 + cl;
    int cx, cy, cz = 0;
    if (DIM == 2) {
      cx = (int)(C % Nc);
      cy = (int)(C / Nc);
    } else {
      cx = (int)(C % Nc);
      cy = (int)((C / Nc) % Nc);
      cz = (int)(C / ((long long)Nc * Nc));
    }
    int o1 = u & 1, o2 = u >> 1;
    T acc[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) acc[i] = T(0);
    for (int o0 = 0; o0 < 2; ++o0) {
      long long f = (2 * cx + o0) + (long long)Nf * ((2 * cy + o1) + (DIM == 3 ? (long long)Nf * (2 * cz + o2) : 0));
      T v[NN], w[NN];
      load_line<NN>(rf + f * ND + base, stride, v);
      matvec_line<NN>(PmT[o0], v, w);
#pragma unroll
      for (int i = 0; i < NN; ++i) acc[i] += w[i];
    }
    store_line<NN>(U + (cl * NU + u) * ND + base, stride, acc);
  }
  __syncthreads();
  if (DIM == 2) {
    for (int task = tid; task < ncb * NL; task += nth) {
      int cl = task / NL, l = task % NL;
      int base, stride;
      CS::line(1, l, base, stride);
      T acc[NN];
#pragma unroll
      for (int i = 0; i < NN; ++i) acc[i] = T(0);
      for (int o1 = 0; o1 < 2; ++o1) {
        T v[NN], w[NN];
        load_line<NN>(U + (cl * NU + o1) * ND + base, stride, v);
        matvec_line<NN>(PmT[o1], v, w);
#pragma unroll
        for (int i = 0; i < NN; ++i) acc[i] += w[i];
      }
      store_line<NN>(rc + (c0 + cl) * ND + base, stride, acc);
    }
  } else {
    for (int task = tid; task < ncb * 2 * NL; task += nth) {
      int cl = task / (2 * NL), rem = task % (2 * NL), o2 = rem / NL, l = rem % NL;
      int base, stride;
      CS::line(1, l, base, stride);
      T acc[NN];
#pragma unroll
      for (int i = 0; i < NN; ++i) acc[i] = T(0);
      for (int o1 = 0; o1 < 2; ++o1) {
        T v[NN], w[NN];
        load_line<NN>(U + (cl * NU + o1 + 2 * o2) * ND + base, stride, v);
        matvec_line<NN>(PmT[o1], v, w);
#pragma unroll
        for (int i = 0; i < NN; ++i) acc[i] += w[i];
      }
      store_line<NN>(V + (cl * 2 + o2) * ND + base, stride, acc);
    }
    __syncthreads();
    for (int task = tid; task < ncb * NL; task += nth) {
      int cl = task / NL, l = task % NL;
      int base, stride;
      CS::line(2, l, base, stride);
      T acc[NN];
#pragma unroll
      for (int i = 0; i < NN; ++i) acc[i] = T(0);
      for (int o2 = 0; o2 < 2; ++o2) {
        T v[NN], w[NN];
        load_line<NN>(V + (cl * 2 + o2) * ND + base, stride, v);
        matvec_line<NN>(PmT[o2], v, w);
#pragma unroll
        for (int i = 0; i < NN; ++i) acc[i] += w[i];
      }
      store_line<NN>(rc + (c0 + cl) * ND + base, stride, acc);
    }
  }
}

// x0 = A_0^{-1} b0 (one CTA, FP64 arithmetic, global lexicographic order).
template <int DIM, typename T>
__global__ void coarse_solve_kernel(const LevelConst<double>* __restrict__ lc, const T* __restrict__ b0,
                                    T* __restrict__ x0, int N0, int n, long long nd0) {
  extern __shared__ __align__(16) double cs_smem[];
  const int m = N0 * n;
  const int D = (DIM == 2) ? m * m : m * m * m;
  double* S = cs_smem;              // m x m
  double* A = S + m * m;            // D
  double* B = A + D;                // D
  const int tid = threadIdx.x, nth = blockDim.x;
  b0 += (long long)blockIdx.x * nd0;
  x0 += (long long)blockIdx.x * nd0;
  for (int e = tid; e < m * m; e += nth) S[e] = lc->S0[e / m][e % m];
  const int nd = (DIM == 2) ? n * n : n * n * n;
  // cell-wise -> lexicographic (X_0 fastest)
  for (int g = tid; g < D; g += nth) {
    int X[3] = {g % m, (g / m) % m, DIM == 3 ? g / (m * m) : 0};
    long long c = 0, loc = 0, cs = 1, ls = 1;
    for (int e = 0; e < DIM; ++e) {
      c += (X[e] / n) * cs;
      loc += (X[e] % n) * ls;
      cs *= N0;
      ls *= n;
    }
    A[g] = (double)b0[c * nd + loc];
  }
  __syncthreads();
  double* src = A;
  double* dst = B;
  // S^T along every axis
  for (int e = 0; e < DIM; ++e) {
    const int st = (e == 0) ? 1 : (e == 1 ? m : m * m);
    for (int g = tid; g < D; g += nth) {
      int row = (g / st) % m;
      int base = g - row * st;
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc = fma(S[j * m + row], src[base + j * st], acc);
      dst[g] = acc;
    }
    __syncthreads();
    double* t = src;
    src = dst;
    dst = t;
  }
  for (int g = tid; g < D; g += nth) {
    int X[3] = {g % m, (g / m) % m, DIM == 3 ? g / (m * m) : 0};
    double l = 0.0;
    for (int e = 0; e < DIM; ++e) l += lc->lam0[X[e]];
    src[g] = src[g] / l;
  }
  __syncthreads();
  for (int e = 0; e < DIM; ++e) {
    const int st = (e == 0) ? 1 : (e == 1 ? m : m * m);
    for (int g = tid; g < D; g += nth) {
      int row = (g / st) % m;
      int base = g - row * st;
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc = fma(S[row * m + j], src[base + j * st], acc);
      dst[g] = acc;
    }
    __syncthreads();
    double* t = src;
    src = dst;
    dst = t;
  }
  for (int g = tid; g < D; g += nth) {
    int X[3] = {g % m, (g / m) % m, DIM == 3 ? g / (m * m) : 0};
    long long c = 0, loc = 0, cs = 1, ls = 1;
    for (int e = 0; e < DIM; ++e) {
      c += (X[e] / n) * cs;
      loc += (X[e] % n) * ls;
      cs *= N0;
      ls *= n;
    }
    x0[c * nd + loc] = (T)src[g];
  }
}

template <typename T, int DIM, int NN>
cudaError_t transfer_dispatch2(const sipg_handle* h, int fine_level, int prolong, const T* in, T* out,
                               cudaStream_t s) {
  constexpr int CPB = transfer_cpb<DIM, NN>();
  const LevelInfo& lf = h->lv[fine_level];
  const LevelInfo& lc = h->lv[fine_level - 1];
  dim3 grid(ceil_div((long long)lc.ncells, CPB), h->prm.nrhs);
  const int threads = CPB * CellShape<DIM, NN>::lines * 2;
  if (prolong)
    prolongate_kernel<DIM, NN, T, CPB><<<grid, threads, 0, s>>>(
        h->cst<T>(fine_level), in, out, lc.N, (long long)lc.ncells, (long long)lc.ndofs,
        (long long)lf.ndofs);
  else
    restrict_kernel<DIM, NN, T, CPB><<<grid, threads, 0, s>>>(
        h->cst<T>(fine_level), in, out, lc.N, (long long)lc.ncells, (long long)lc.ndofs,
        (long long)lf.ndofs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t transfer_dispatch(const sipg_handle* h, int fine_level, int prolong, const T* in, T* out,
                              cudaStream_t s) {
  if (h->prm.dim == 2) {
    switch (h->n) {
      case 2: return transfer_dispatch2<T, 2, 2>(h, fine_level, prolong, in, out, s);
      case 3: return transfer_dispatch2<T, 2, 3>(h, fine_level, prolong, in, out, s);
      case 4: return transfer_dispatch2<T, 2, 4>(h, fine_level, prolong, in, out, s);
      case 5: return transfer_dispatch2<T, 2, 5>(h, fine_level, prolong, in, out, s);
      case 6: return transfer_dispatch2<T, 2, 6>(h, fine_level, prolong, in, out, s);
      case 7: return transfer_dispatch2<T, 2, 7>(h, fine_level, prolong, in, out, s);
      case 8: return transfer_dispatch2<T, 2, 8>(h, fine_level, prolong, in, out, s);
    }
  } else {
    switch (h->n) {
      case 2: return transfer_dispatch2<T, 3, 2>(h, fine_level, prolong, in, out, s);
      case 3: return transfer_dispatch2<T, 3, 3>(h, fine_level, prolong, in, out, s);
      case 4: return transfer_dispatch2<T, 3, 4>(h, fine_level, prolong, in, out, s);
      case 5: return transfer_dispatch2<T, 3, 5>(h, fine_level, prolong, in, out, s);
      case 6: return transfer_dispatch2<T, 3, 6>(h, fine_level, prolong, in, out, s);
      case 7: return transfer_dispatch2<T, 3, 7>(h, fine_level, prolong, in, out, s);
      case 8: return transfer_dispatch2<T, 3, 8>(h, fine_level, prolong, in, out, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

template <typename T>
cudaError_t launch_restrict(const sipg_handle* h, int fine_level, const T* rf, T* rc, cudaStream_t s) {
  return transfer_dispatch<T>(h, fine_level, 0, rf, rc, s);
}
template <typename T>
cudaError_t launch_prolongate_add(const sipg_handle* h, int fine_level, const T* ec, T* xf,
                                  cudaStream_t s) {
  return transfer_dispatch<T>(h, fine_level, 1, ec, xf, s);
}

template <typename T>
cudaError_t launch_coarse_solve(const sipg_handle* h, const T* b0, T* x0, cudaStream_t s) {
  const LevelInfo& l0 = h->lv[0];
  const int m = l0.N * h->n;
  const int D = (h->prm.dim == 2) ? m * m : m * m * m;
  const size_t smem = (size_t)(m * m + 2 * D) * sizeof(double);
  // the largest coarse problem (m^d <= 4096, m <= 64) needs at most
  // (64^2 + 2 * 4096) doubles; opt in once per instantiation
  const int max_smem = (SIPG_MAXM0 * SIPG_MAXM0 + 2 * 4096) * (int)sizeof(double);
  cudaError_t e;
  if (h->prm.dim == 2) {
    e = smem_opt_in(reinterpret_cast<const void*>(coarse_solve_kernel<2, T>), max_smem);
    if (e != cudaSuccess) return e;
    coarse_solve_kernel<2, T><<<h->prm.nrhs, 512, smem, s>>>(h->c64(0), b0, x0, l0.N, h->n,
                                                            (long long)l0.ndofs);
  } else {
    e = smem_opt_in(reinterpret_cast<const void*>(coarse_solve_kernel<3, T>), max_smem);
    if (e != cudaSuccess) return e;
    coarse_solve_kernel<3, T><<<h->prm.nrhs, 512, smem, s>>>(h->c64(0), b0, x0, l0.N, h->n,
                                                            (long long)l0.ndofs);
  }
  return cudaGetLastError();
}

template cudaError_t launch_restrict<double>(const sipg_handle*, int, const double*, double*, cudaStream_t);
template cudaError_t launch_restrict<float>(const sipg_handle*, int, const float*, float*, cudaStream_t);
template cudaError_t launch_prolongate_add<double>(const sipg_handle*, int, const double*, double*, cudaStream_t);
template cudaError_t launch_prolongate_add<float>(const sipg_handle*, int, const float*, float*, cudaStream_t);
template cudaError_t launch_coarse_solve<double>(const sipg_handle*, const double*, double*, cudaStream_t);
template cudaError_t launch_coarse_solve<float>(const sipg_handle*, const float*, float*, cudaStream_t);
