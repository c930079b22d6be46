// Full-kernel vertex-patch smoother (Sec. 3.1, Table 1): the local space V_j
// is every DoF of the 2^d cells around an interior vertex, A_j the principal
// block of A on them, inverted by fast diagonalisation (Eqs. inverse2d,
// inverse3d) with the eigenpairs of the whole 2n-node 1D patch matrices.
// Its domain of dependence reaches the cells around the patch, so the
// residual is updated globally (as Sec. 3.1 decides for this kernel): one
// colour pass is r = b - A x on the whole level (the operator-apply kernel),
// then every patch of the colour adds A_j^{-1} R_j r.  Same-colour patches
// share faces but no DoFs, so their corrections are independent and the
// pass is race-free.
//
// The clamped kernel (Sec. 3.1) runs the same passes: its constants are the
// columns B S of the clamped subspace basis B times the eigenvectors of the
// projected 1D patch matrices, padded with zero columns (eigenvalue 1), so
// the patch kernel applies B (B^T A_D B)^{-1} B^T to the patch residual;
// same-colour clamped patches do not see each other's DoFs in their
// residuals, so one global residual per colour gives the multiplicative
// result.
//
// Patch kernel (FP64, and 2D): a patch's P^d residual values (P = 2n) are
// staged in shared memory in patch-lexicographic order (direction 0 fastest); each thread owns
// one line per direction and applies S^T along directions 0..d-1, the
// eigenvalue scaling, then S along each direction, and finally adds its
// direction-0 line to x.  The 1D eigenvectors are read from the level
// constants in global memory (a few KB, L1-resident).
#include "sipg_internal.cuh"

template <int NN>
cudaError_t full3_colour_n(const sipg_handle* h, int level, int colour, const float* r, float* x, cudaStream_t s);

namespace {

template <int DIM, int NN>
struct FullCfg {
  static constexpr int P = 2 * NN;
  static constexpr int LINES = DIM == 2 ? P : P * P;        // lines per direction and patch
  static constexpr int PPC = LINES >= 64 ? 1 : 64 / LINES;  // patches per CTA
  static constexpr int THREADS = LINES * PPC;
  static constexpr int VOL = DIM == 2 ? P * P : P * P * P;
};

template <int DIM, int NN, typename T>
__global__ void __launch_bounds__(FullCfg<DIM, NN>::THREADS)
    full_patch_kernel(const LevelConst<T>* __restrict__ lc, int N, int colour, int3 cnt, long long npatch,
                      const T* __restrict__ r, T* __restrict__ x, long long ndofs) {
  using C = FullCfg<DIM, NN>;
  constexpr int P = C::P;
  __shared__ T u[C::PPC][C::VOL];
  const int slot = threadIdx.x / C::LINES;
  const int t = threadIdx.x % C::LINES;
  const long long pid = (long long)blockIdx.x * C::PPC + slot;
  const bool active = pid < npatch;
  const long long col = (long long)blockIdx.y * ndofs;
  T* us = u[slot];

  // vertex of the patch: per direction the vertices 1..N-1 of parity bit e
  // of the colour, enumerated direction 0 fastest
  int v[3] = {1, 1, 1}, ty[3] = {0, 0, 0};
  {
    long long q = active ? pid : 0;
    const int cn[3] = {cnt.x, cnt.y, cnt.z};
#pragma unroll
    for (int e = 0; e < DIM; ++e) {
      const int qe = (int)(q % cn[e]);
      q /= cn[e];
      v[e] = ((colour >> e) & 1) ? 1 + 2 * qe : 2 + 2 * qe;
      ty[e] = (v[e] == 1 ? 1 : 0) | (v[e] == N - 1 ? 2 : 0);
    }
  }
  // global index of patch node a (patch-local coordinates 0..P-1)
  auto gidx = [&](int a0, int a1, int a2) -> long long {
    const int a[3] = {a0, a1, a2};
    long long cell = 0, cs = 1;
    int node = 0, ns = 1;
#pragma unroll
    for (int e = 0; e < DIM; ++e) {
      cell += (long long)(v[e] - 1 + a[e] / NN) * cs;
      cs *= N;
      node += (a[e] % NN) * ns;
      ns *= NN;
    }
    return cell * ns + node;
  };
  // this thread's line: direction-0 line (a1, a2) = (t % P, t / P) in 3D,
  // a1 = t in 2D
  const int l1 = DIM == 2 ? t : t % P;
  const int l2 = DIM == 2 ? 0 : t / P;

  if (active) {
#pragma unroll
    for (int a0 = 0; a0 < P; ++a0) us[a0 + P * t] = r[col + gidx(a0, l1, l2)];
  }
  __syncthreads();

  // one 1D transform along direction e: S^T (forward) or S (backward)
  auto sweep = [&](int e, bool forward) {
    if (active) {
      int base, stride;
      if (e == 0) {
        base = P * t;
        stride = 1;
      } else if (e == 1) {
        base = DIM == 2 ? t : (t % P) + P * P * (t / P);
        stride = P;
      } else {
        base = t;  // (a0, a1) = (t % P, t / P)
        stride = P * P;
      }
      const T* S = &lc->Sf[ty[e]][0][0];
      T in[P];
#pragma unroll
      for (int i = 0; i < P; ++i) in[i] = us[base + i * stride];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        T acc = T(0);
#pragma unroll
        for (int i = 0; i < P; ++i)
          acc = fma(forward ? S[i * SIPG_MAXP + j] : S[j * SIPG_MAXP + i], in[i], acc);
        us[base + j * stride] = acc;
      }
    }
    __syncthreads();
  };

#pragma unroll
  for (int e = 0; e < DIM; ++e) sweep(e, true);
  if (active) {
    T lam12 = lc->lamf[ty[1]][l1];
    if (DIM == 3) lam12 += lc->lamf[ty[2]][l2];
#pragma unroll
    for (int a0 = 0; a0 < P; ++a0) us[a0 + P * t] /= lc->lamf[ty[0]][a0] + lam12;
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < DIM; ++e) sweep(e, false);
  if (active) {
#pragma unroll
    for (int a0 = 0; a0 < P; ++a0) {
      const long long g = col + gidx(a0, l1, l2);
      x[g] += us[a0 + P * t];
    }
  }
}

template <int DIM, int NN, typename T>
cudaError_t full_patches(const sipg_handle* h, int level, int colour, const T* r, T* x, cudaStream_t s) {
  using C = FullCfg<DIM, NN>;
  const int N = h->lv[level].N;
  int cn[3] = {1, 1, 1};
  long long np = 1;
  for (int e = 0; e < DIM; ++e) {
    cn[e] = ((colour >> e) & 1) ? N / 2 : N / 2 - 1;
    np *= cn[e];
  }
  if (np <= 0) return cudaSuccess;
  dim3 grid((unsigned)((np + C::PPC - 1) / C::PPC), h->prm.nrhs);
  full_patch_kernel<DIM, NN, T><<<grid, C::THREADS, 0, s>>>(h->cst<T>(level), N, colour,
                                                             make_int3(cn[0], cn[1], cn[2]), np, r, x,
                                                             (long long)h->lv[level].ndofs);
  return cudaGetLastError();
}

template <int DIM, typename T>
cudaError_t full_dim(const sipg_handle* h, int level, int colour, const T* r, T* x, cudaStream_t s) {
  switch (h->n) {
    case 2: return full_patches<DIM, 2, T>(h, level, colour, r, x, s);
    case 3: return full_patches<DIM, 3, T>(h, level, colour, r, x, s);
    case 4: return full_patches<DIM, 4, T>(h, level, colour, r, x, s);
    case 5: return full_patches<DIM, 5, T>(h, level, colour, r, x, s);
    case 6: return full_patches<DIM, 6, T>(h, level, colour, r, x, s);
    case 7: return full_patches<DIM, 7, T>(h, level, colour, r, x, s);
    case 8: return full_patches<DIM, 8, T>(h, level, colour, r, x, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

template <typename T>
cudaError_t launch_full_colour(const sipg_handle* h, int level, int colour, const T* b, T* x, cudaStream_t s,
                               int* launches) {
  *launches = 0;
  T* r = reinterpret_cast<T*>(h->vr(level));
  cudaError_t e = launch_apply<T>(h, level, APPLY_RESIDUAL, b, x, r, s);
  if (e != cudaSuccess) return e;
  *launches = 1;
  if constexpr (sizeof(T) == 4) {
    // 3D FP32 full kernel: the register-direct all-rows patch kernels
    if (h->prm.dim == 3 && h->prm.smoother == SIPG_SMOOTHER_FULL) {
      const float* rf = reinterpret_cast<const float*>(r);
      float* xf = reinterpret_cast<float*>(x);
      switch (h->n) {
        case 2: e = full3_colour_n<2>(h, level, colour, rf, xf, s); break;
        case 3: e = full3_colour_n<3>(h, level, colour, rf, xf, s); break;
        case 4: e = full3_colour_n<4>(h, level, colour, rf, xf, s); break;
        case 5: e = full3_colour_n<5>(h, level, colour, rf, xf, s); break;
        case 6: e = full3_colour_n<6>(h, level, colour, rf, xf, s); break;
        case 7: e = full3_colour_n<7>(h, level, colour, rf, xf, s); break;
        default: e = full3_colour_n<8>(h, level, colour, rf, xf, s); break;
      }
      if (e == cudaSuccess) *launches = 1 + colour_kernels(3, h->lv[level].N, colour);
      return e;
    }
  }
  e = h->prm.dim == 2 ? full_dim<2, T>(h, level, colour, r, x, s) : full_dim<3, T>(h, level, colour, r, x, s);
  if (e == cudaSuccess) *launches = 2;
  return e;
}
template cudaError_t launch_full_colour<double>(const sipg_handle*, int, int, const double*, double*, cudaStream_t,
                                                int*);
template cudaError_t launch_full_colour<float>(const sipg_handle*, int, int, const float*, float*, cudaStream_t,
                                               int*);
