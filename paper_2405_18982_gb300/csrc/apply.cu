// Matrix-free SIPG operator apply (Sec. 2.2, K1) and the block-diagonal mass.
//
// On a uniform Cartesian mesh with constant kappa the SIPG matrix, faces
// included, is a Kronecker sum of 1D DG operators (Sec. 2.2):
//   A = sum_e  M (x) .. (x) Lhat_e (x) .. (x) M,
// where Lhat_e is the 1D SIPG operator along e.  Per cell c this reads
//   (A x)_c = sum_e (M (x) .. I_e .. (x) M) z_e,
//   z_e = Lself[type_e(c)] x_c + l_lo x_{c-e} + l_hi x_{c+e}   (along e),
// and the neighbour couplings are rank two (face node value and normal
// derivative), so only one dot product per neighbour line is needed.
//
// Kernel layout: one CTA handles CPB consecutive cells; one thread owns one
// line of a cell per direction (n^(d-1) lines) and keeps it in registers
// while contracting with the n x n 1D matrices held in shared memory
// (Sec. 4.1: 1D matrices in shared memory).  Phases (3D):
//   P1  Z_e = normal operator along e (with neighbour terms), e = 0..2
//   P2  X <- M_y Z_0 ;  W <- M_x Z_2
//   P3  X += M_x Z_1 ;  Z_0 <- M_y W
//   P4  y = M_z X + Z_0      (staged in shared memory, stored coalesced)
// = 3 normal + 5 mass contractions per DoF.
#include "tensor_ops.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

template <int DIM, int NN>
constexpr int apply_cpb() {
  return DIM == 2 ? (NN <= 4 ? 32 : 16)
                  : (NN == 2 ? 32 : NN == 3 ? 16 : NN <= 5 ? 8 : NN == 6 ? 4 : 2);
}

template <int NN, typename T>
struct ApplyConst {
  T Ls[3][NN * NN];
  T alo[NN], glo[NN], ahi[NN], ghi[NN];
  T Mw[NN], Ma[NN], Mu[NN];  // M = diag(Mw) + Mu Ma^T (GLL mass: diagonal plus rank one)
};

template <int DIM, int NN, typename T>
__device__ __forceinline__ void normal_line(const ApplyConst<NN, T>& C, const T* __restrict__ xg,
                                            const T* Xs, T* Zs, int e, int l, long long c,
                                            const int* cc, int N) {
  using CS = CellShape<DIM, NN>;
  constexpr int ND = CS::dofs;
  int base, stride;
  CS::line(e, l, base, stride);
  T v[NN], o[NN];
  load_line<NN>(Xs + base, stride, v);
  const int ty = cc[e] == 0 ? 1 : (cc[e] == N - 1 ? 2 : 0);
  matvec_line<NN>(C.Ls[ty], v, o);
  const long long est = (e == 0) ? 1 : (e == 1 ? (long long)N : (long long)N * N);
  if (cc[e] > 0) {
    const T* nb = xg + (c - est) * ND + base;
    T s = T(0), F = T(0);
#pragma unroll
    for (int j = 0; j < NN; ++j) {
      T w = __ldg(nb + j * stride);
      s = fma(C.alo[j], w, s);
      if (j == NN - 1) F = w;
    }
    o[0] += s;
#pragma unroll
    for (int i = 0; i < NN; ++i) o[i] = fma(C.glo[i], F, o[i]);
  }
  if (cc[e] < N - 1) {
    const T* nb = xg + (c + est) * ND + base;
    T s = T(0), F = T(0);
#pragma unroll
    for (int j = 0; j < NN; ++j) {
      T w = __ldg(nb + j * stride);
      s = fma(C.ahi[j], w, s);
      if (j == 0) F = w;
    }
    o[NN - 1] += s;
#pragma unroll
    for (int i = 0; i < NN; ++i) o[i] = fma(C.ghi[i], F, o[i]);
  }
  store_line<NN>(Zs + base, stride, o);
}

// dst (+)= M src along direction e for line l, with the mass as diagonal
// plus rank one: 3n FMAs per line instead of n^2
template <int DIM, int NN, typename T>
__device__ __forceinline__ void mass_line_r1(const ApplyConst<NN, T>& C, const T* src, T* dst, int e, int l,
                                             bool acc) {
  using CS = CellShape<DIM, NN>;
  int base, stride;
  CS::line(e, l, base, stride);
  T v[NN], o[NN];
  load_line<NN>(src + base, stride, v);
  T s = C.Ma[0] * v[0];
#pragma unroll
  for (int j = 1; j < NN; ++j) s = fma(C.Ma[j], v[j], s);
#pragma unroll
  for (int i = 0; i < NN; ++i) o[i] = fma(C.Mu[i], s, C.Mw[i] * v[i]);
  if (acc) {
#pragma unroll
    for (int i = 0; i < NN; ++i) o[i] += dst[base + i * stride];
  }
  store_line<NN>(dst + base, stride, o);
}

// dst (+)= M src along direction e for line l (dense n x n mass)
template <int DIM, int NN, typename T>
__device__ __forceinline__ void mass_line(const T* M, const T* src, T* dst, int e, int l, bool acc) {
  using CS = CellShape<DIM, NN>;
  int base, stride;
  CS::line(e, l, base, stride);
  T v[NN], o[NN];
  load_line<NN>(src + base, stride, v);
  matvec_line<NN>(M, v, o);
  if (acc) {
#pragma unroll
    for (int i = 0; i < NN; ++i) o[i] += dst[base + i * stride];
  }
  store_line<NN>(dst + base, stride, o);
}

template <int DIM, int NN, typename T, int CPB>
__global__ void __launch_bounds__(CPB * CellShape<DIM, NN>::lines)
    apply_kernel(const LevelConst<T>* __restrict__ lc, int mode, const T* bvec,
                 const T* __restrict__ x, T* y, int N, long long ncells, long long ndofs) {
  using CS = CellShape<DIM, NN>;
  constexpr int NL = CS::lines, ND = CS::dofs;
  __shared__ ApplyConst<NN, T> C;
  __shared__ T X[CPB * ND], Z0[CPB * ND], Z1[CPB * ND];
  __shared__ T Z2[DIM == 3 ? CPB * ND : 1], W[DIM == 3 ? CPB * ND : 1];
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long col = (long long)blockIdx.y * ndofs;
  x += col;
  y += col;
  if (bvec) bvec += col;
  const bool pen = (mode == APPLY_PENALTY);
  for (int t = 0; t < 3; ++t) copy_block<NN>(C.Ls[t], pen ? lc->Pself[t] : lc->Lself[t], tid, nth);
  if (tid < NN) {
    C.Mw[tid] = lc->Mw[tid];
    C.Ma[tid] = lc->Ma[tid];
    C.Mu[tid] = lc->Mu[tid];
    C.alo[tid] = pen ? lc->palo[tid] : lc->alo[tid];
    C.glo[tid] = pen ? lc->pglo[tid] : lc->glo[tid];
    C.ahi[tid] = pen ? lc->pahi[tid] : lc->ahi[tid];
    C.ghi[tid] = pen ? lc->pghi[tid] : lc->ghi[tid];
  }
  const long long c0 = (long long)blockIdx.x * CPB;
  const int ncb = (int)min((long long)CPB, ncells - c0);
  const T* xb = x + c0 * ND;
  for (int e = tid; e < ncb * ND; e += nth) X[e] = xb[e];
  __syncthreads();

  const int cl = tid / NL, l = tid % NL;
  const bool valid = cl < ncb;
  const long long c = c0 + cl;
  int cc[3];
  cc[0] = (int)(c % N);
  cc[1] = (int)((c / N) % N);
  cc[2] = (DIM == 3) ? (int)(c / ((long long)N * N)) : 0;
  const int off = cl * ND;
  if (valid) {
    normal_line<DIM, NN, T>(C, x, X + off, Z0 + off, 0, l, c, cc, N);
    normal_line<DIM, NN, T>(C, x, X + off, Z1 + off, 1, l, c, cc, N);
    if (DIM == 3) normal_line<DIM, NN, T>(C, x, X + off, Z2 + off, 2, l, c, cc, N);
  }
  __syncthreads();
  T* out;  // shared buffer holding A x for the block's cells
  if (DIM == 2) {
    // y = M_y Z_0 + M_x Z_1
    if (valid) mass_line_r1<DIM, NN, T>(C, Z0 + off, X + off, 1, l, false);
    __syncthreads();
    if (valid) mass_line_r1<DIM, NN, T>(C, Z1 + off, X + off, 0, l, true);
    out = X;
  } else {
    if (valid) {
      mass_line_r1<DIM, NN, T>(C, Z0 + off, X + off, 1, l, false);
      mass_line_r1<DIM, NN, T>(C, Z2 + off, W + off, 0, l, false);
    }
    __syncthreads();
    if (valid) {
      mass_line_r1<DIM, NN, T>(C, Z1 + off, X + off, 0, l, true);
      mass_line_r1<DIM, NN, T>(C, W + off, Z0 + off, 1, l, false);
    }
    __syncthreads();
    if (valid) mass_line_r1<DIM, NN, T>(C, X + off, Z0 + off, 2, l, true);
    out = Z0;
  }
  __syncthreads();
  T* yb = y + c0 * ND;
  if (mode == APPLY_RESIDUAL) {
    const T* bb = bvec + c0 * ND;
    for (int e = tid; e < ncb * ND; e += nth) yb[e] = bb[e] - out[e];
  } else {
    for (int e = tid; e < ncb * ND; e += nth) yb[e] = out[e];
  }
}

// b = (M (x) M (x) M) f cell by cell (FP64).
template <int DIM, int NN, int CPB>
__global__ void __launch_bounds__(CPB * CellShape<DIM, NN>::lines)
    mass_kernel(const LevelConst<double>* __restrict__ lc, const double* __restrict__ f,
                double* __restrict__ b, long long ncells, long long ndofs) {
  using CS = CellShape<DIM, NN>;
  constexpr int NL = CS::lines, ND = CS::dofs;
  __shared__ double Mm[NN * NN];
  __shared__ double X[CPB * ND], Y[CPB * ND];
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long col = (long long)blockIdx.y * ndofs;
  f += col;
  b += col;
  copy_block<NN>(Mm, lc->M, tid, nth);
  const long long c0 = (long long)blockIdx.x * CPB;
  const int ncb = (int)min((long long)CPB, ncells - c0);
  for (int e = tid; e < ncb * ND; e += nth) X[e] = f[c0 * ND + e];
  __syncthreads();
  const int cl = tid / NL, l = tid % NL;
  const bool valid = cl < ncb;
  const int off = cl * ND;
  if (valid) mass_line<DIM, NN, double>(Mm, X + off, Y + off, 0, l, false);
  __syncthreads();
  if (valid) mass_line<DIM, NN, double>(Mm, Y + off, X + off, 1, l, false);
  __syncthreads();
  double* res = X;
  if (DIM == 3) {
    if (valid) mass_line<DIM, NN, double>(Mm, X + off, Y + off, 2, l, false);
    __syncthreads();
    res = Y;
  }
  for (int e = tid; e < ncb * ND; e += nth) b[c0 * ND + e] = res[e];
}

template <int DIM, int NN>
__global__ void manufactured_kernel(const LevelConst<double>* __restrict__ lc, double* __restrict__ f,
                                    int N, long long ndofs, int nrhs) {
  constexpr int ND = CellShape<DIM, NN>::dofs;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndofs) return;
  const long long c = i / ND;
  const int loc = (int)(i % ND);
  const double h = 1.0 / N;
  int cc[3] = {(int)(c % N), (int)((c / N) % N), DIM == 3 ? (int)(c / ((long long)N * N)) : 0};
  int ii[3] = {loc % NN, (loc / NN) % NN, DIM == 3 ? loc / (NN * NN) : 0};
  double v = DIM * kPi * kPi;
  for (int e = 0; e < DIM; ++e) v *= sin(kPi * (cc[e] + lc->nodes[ii[e]]) * h);
  for (int r = 0; r < nrhs; ++r) f[(long long)r * ndofs + i] = v;
}

template <typename T, int DIM, int NN>
cudaError_t apply_dispatch2(const sipg_handle* h, int level, int mode, const T* b, const T* x, T* y,
                            cudaStream_t s) {
  constexpr int CPB = apply_cpb<DIM, NN>();
  const LevelInfo& li = h->lv[level];
  dim3 grid(ceil_div((long long)li.ncells, CPB), h->prm.nrhs);
  apply_kernel<DIM, NN, T, CPB><<<grid, CPB * CellShape<DIM, NN>::lines, 0, s>>>(
      h->cst<T>(level), mode, b, x, y, li.N, (long long)li.ncells, (long long)li.ndofs);
  return cudaGetLastError();
}

template <int DIM, int NN>
cudaError_t mass_dispatch2(const sipg_handle* h, const double* f, double* b, cudaStream_t s) {
  constexpr int CPB = apply_cpb<DIM, NN>();
  const LevelInfo& li = h->lv[h->L];
  dim3 grid(ceil_div((long long)li.ncells, CPB), h->prm.nrhs);
  mass_kernel<DIM, NN, CPB><<<grid, CPB * CellShape<DIM, NN>::lines, 0, s>>>(
      h->c64(h->L), f, b, (long long)li.ncells, (long long)li.ndofs);
  return cudaGetLastError();
}

template <int DIM, int NN>
cudaError_t manufactured_dispatch2(const sipg_handle* h, double* f, cudaStream_t s) {
  const LevelInfo& li = h->lv[h->L];
  manufactured_kernel<DIM, NN><<<ceil_div((long long)li.ndofs, 256), 256, 0, s>>>(
      h->c64(h->L), f, li.N, (long long)li.ndofs, h->prm.nrhs);
  return cudaGetLastError();
}

#include "apply3.cuh"

template <int NN, typename T>
cudaError_t apply3_try(const sipg_handle* h, int level, int mode, const T* b, const T* x, T* y, cudaStream_t s) {
  return launch_apply3<NN, T>(h, level, mode, b, x, y, s);
}

}  // namespace

#define SIPG_DISPATCH_N(FN, DIM, ...)                                  \
  switch (h->n) {                                                      \
    case 2: return FN<DIM, 2>(__VA_ARGS__);                            \
    case 3: return FN<DIM, 3>(__VA_ARGS__);                            \
    case 4: return FN<DIM, 4>(__VA_ARGS__);                            \
    case 5: return FN<DIM, 5>(__VA_ARGS__);                            \
    case 6: return FN<DIM, 6>(__VA_ARGS__);                            \
    case 7: return FN<DIM, 7>(__VA_ARGS__);                            \
    case 8: return FN<DIM, 8>(__VA_ARGS__);                            \
    default: return cudaErrorInvalidValue;                             \
  }

template <typename T>
static cudaError_t apply_dim(const sipg_handle* h, int level, int mode, const T* b, const T* x, T* y,
                             cudaStream_t s) {
  if (h->prm.dim == 2) {
    switch (h->n) {
      case 2: return apply_dispatch2<T, 2, 2>(h, level, mode, b, x, y, s);
      case 3: return apply_dispatch2<T, 2, 3>(h, level, mode, b, x, y, s);
      case 4: return apply_dispatch2<T, 2, 4>(h, level, mode, b, x, y, s);
      case 5: return apply_dispatch2<T, 2, 5>(h, level, mode, b, x, y, s);
      case 6: return apply_dispatch2<T, 2, 6>(h, level, mode, b, x, y, s);
      case 7: return apply_dispatch2<T, 2, 7>(h, level, mode, b, x, y, s);
      case 8: return apply_dispatch2<T, 2, 8>(h, level, mode, b, x, y, s);
    }
  } else {
    switch (h->n) {
      case 2: return apply_dispatch2<T, 3, 2>(h, level, mode, b, x, y, s);
      case 3: return apply_dispatch2<T, 3, 3>(h, level, mode, b, x, y, s);
      case 4: return apply_dispatch2<T, 3, 4>(h, level, mode, b, x, y, s);
      case 5: return apply_dispatch2<T, 3, 5>(h, level, mode, b, x, y, s);
      case 6: return apply_dispatch2<T, 3, 6>(h, level, mode, b, x, y, s);
      case 7: return apply_dispatch2<T, 3, 7>(h, level, mode, b, x, y, s);
      case 8: return apply_dispatch2<T, 3, 8>(h, level, mode, b, x, y, s);
    }
  }
  return cudaErrorInvalidValue;
}

// The coarse-cell-organised 3D kernel where it applies (FP32, 16-byte
// aligned vectors, N even with whole CTA groups), else the cell-block kernel.
// FP64 stays on the cell-block kernel: bound by the FP64 pipe, it is faster
// there (1.39 ms against 1.53 ms for 16.8M DoFs, Q3).
template <typename T>
static cudaError_t apply3_dim(const sipg_handle* h, int level, int mode, const T* b, const T* x, T* y,
                              cudaStream_t s) {
  if constexpr (sizeof(T) != 4) {
    return cudaErrorNotSupported;
  } else {
    if (h->prm.dim != 3) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(y)) % 16)
      return cudaErrorNotSupported;
    switch (h->n) {
      case 2: return apply3_try<2, T>(h, level, mode, b, x, y, s);
      case 3: return apply3_try<3, T>(h, level, mode, b, x, y, s);
      case 4: return apply3_try<4, T>(h, level, mode, b, x, y, s);
      case 5: return apply3_try<5, T>(h, level, mode, b, x, y, s);
      case 6: return apply3_try<6, T>(h, level, mode, b, x, y, s);
      case 7: return apply3_try<7, T>(h, level, mode, b, x, y, s);
      case 8: return apply3_try<8, T>(h, level, mode, b, x, y, s);
    }
    return cudaErrorNotSupported;
  }
}

template <typename T>
cudaError_t launch_apply(const sipg_handle* h, int level, int mode, const T* b, const T* x, T* y,
                         cudaStream_t s) {
  if (mode == APPLY_Y || mode == APPLY_RESIDUAL) {
    cudaError_t e = apply3_dim<T>(h, level, mode == APPLY_Y ? A3_APPLY : A3_RESIDUAL, b, x, y, s);
    if (e != cudaErrorNotSupported) return e;
  }
  return apply_dim<T>(h, level, mode, b, x, y, s);
}

template <typename T>
cudaError_t launch_residual_restrict(const sipg_handle* h, int level, const T* b, const T* x, T* rc,
                                     cudaStream_t s) {
  return apply3_dim<T>(h, level, A3_RESTRICT, b, x, rc, s);
}
template cudaError_t launch_residual_restrict<double>(const sipg_handle*, int, const double*, const double*,
                                                      double*, cudaStream_t);
template cudaError_t launch_residual_restrict<float>(const sipg_handle*, int, const float*, const float*, float*,
                                                     cudaStream_t);
template cudaError_t launch_apply<double>(const sipg_handle*, int, int, const double*, const double*,
                                          double*, cudaStream_t);
template cudaError_t launch_apply<float>(const sipg_handle*, int, int, const float*, const float*,
                                         float*, cudaStream_t);

cudaError_t launch_mass(const sipg_handle* h, const double* f, double* b, cudaStream_t s) {
  if (h->prm.dim == 2) {
    SIPG_DISPATCH_N(mass_dispatch2, 2, h, f, b, s)
  } else {
    SIPG_DISPATCH_N(mass_dispatch2, 3, h, f, b, s)
  }
}

cudaError_t launch_manufactured(const sipg_handle* h, double* f, cudaStream_t s) {
  if (h->prm.dim == 2) {
    SIPG_DISPATCH_N(manufactured_dispatch2, 2, h, f, s)
  } else {
    SIPG_DISPATCH_N(manufactured_dispatch2, 3, h, f, s)
  }
}
