// One colour pass of the colourised multiplicative vertex-patch smoother
// (Algorithm 1, Sec. 3.1) with fast-diagonalisation local solvers (Sec. 3.2,
// Eqs. inverse2d, inverse3d, fast_inverse).
//
// Patch j = the 2^d cells around interior vertex v (v_e in 1..N-1), colour
// c = sum_e (v_e mod 2) 2^e.  Per direction the patch has 2n nodes a = o n + i
// (o = 0: cell v-1, o = 1: cell v); V_j keeps a in [first, first+p): the two
// patch-boundary nodes are dropped unless that end lies on the domain
// boundary (Dirichlet kernel).  The local residual on V_j needs, besides the
// patch cells, only the face-node layer of the cells across the patch faces
// (the -[[u]].{grad v} term; consistent residual), held as a one-node halo
// on each side of an extended (2n+2)^d tile:
//   r_j = b_j - sum_e ( (x)_{f != e} Mr_f (x) Lr_e ) x_ext,
// with Lr/Mr the p x (2n+2) rows of the 1D patch operators (Mr has zero halo
// columns).  Then
//   x[V_j] += (S_2 (x) S_1 (x) S_0) (sum_e Lambda_e)^{-1} (S_2^T (x) S_1^T (x) S_0^T) r_j.
// Same-colour patches share no V_j rows and do not couple through A, so one
// launch processes the whole colour in parallel (one CTA per patch).
#include "tensor_ops.cuh"

namespace {

// dst[o] (+)= sum_j A[i_e(o)][j] src[o with i_e -> j] (+ A2 * src2) for all o
// in a d0 x d1 x d2 box (axis 0 fastest).  A has leading dimension lda.
template <typename T>
__device__ __forceinline__ void contract(T* __restrict__ dst, const T* __restrict__ src,
                                         const T* __restrict__ A, const T* __restrict__ src2,
                                         const T* __restrict__ A2, int lda, int d0, int d1, int d2,
                                         int e, int K) {
  const int tot = d0 * d1 * d2;
  const int s0 = (e == 0) ? K : d0;
  const int s1 = (e == 1) ? K : d1;
  const int st = (e == 0) ? 1 : (e == 1 ? s0 : s0 * s1);
  for (int o = threadIdx.x; o < tot; o += blockDim.x) {
    int i0 = o % d0, i1 = (o / d0) % d1, i2 = o / (d0 * d1);
    int row = (e == 0) ? i0 : (e == 1 ? i1 : i2);
    int sb = (e == 0 ? 0 : i0) + s0 * ((e == 1 ? 0 : i1) + s1 * (e == 2 ? 0 : i2));
    const T* a = A + row * lda;
    T acc = T(0);
    for (int j = 0; j < K; ++j) acc = fma(a[j], src[sb + j * st], acc);
    if (src2) {
      const T* a2 = A2 + row * lda;
      for (int j = 0; j < K; ++j) acc = fma(a2[j], src2[sb + j * st], acc);
    }
    dst[o] = acc;
  }
}

// Transposed application for the fast-diagonalisation sweeps:
// dst[o] = sum_j S[j][i_e(o)] src[o with i_e -> j]  (S^T along e), p x p.
template <typename T>
__device__ __forceinline__ void contract_t(T* __restrict__ dst, const T* __restrict__ src,
                                           const T* __restrict__ S, int lds, int d0, int d1, int d2,
                                           int e) {
  const int tot = d0 * d1 * d2;
  const int K = (e == 0) ? d0 : (e == 1 ? d1 : d2);
  const int st = (e == 0) ? 1 : (e == 1 ? d0 : d0 * d1);
  for (int o = threadIdx.x; o < tot; o += blockDim.x) {
    int i0 = o % d0, i1 = (o / d0) % d1, i2 = o / (d0 * d1);
    int row = (e == 0) ? i0 : (e == 1 ? i1 : i2);
    int sb = o - row * st;
    T acc = T(0);
    for (int j = 0; j < K; ++j) acc = fma(S[j * lds + row], src[sb + j * st], acc);
    dst[o] = acc;
  }
}

template <int NN>
struct SmoothDims {
  static constexpr int P = 2 * NN;
  static constexpr int E = 2 * NN + 2;
};

template <typename T>
struct PatchConst1D {
  T Lr[SIPG_MAXP * SIPG_MAXPE];
  T Mr[SIPG_MAXP * SIPG_MAXPE];
  T S[SIPG_MAXP * SIPG_MAXP];
  T lam[SIPG_MAXP];
};

template <int DIM, int NN>
__host__ __device__ constexpr int smooth_buf_elems(int which) {
  // which: 1 = x_ext / A01 / FD temp, 2 = A0 / r, 3 = B0 / FD temp, 4 = C
  constexpr int P = 2 * NN, E = 2 * NN + 2;
  return DIM == 2 ? (which == 1 ? E * E : which == 4 ? 1 : P * E)
                  : (which == 1 ? E * E * E : which == 4 ? P * P * E : P * E * E);
}

template <int DIM, int NN, typename T>
__global__ void __launch_bounds__(256)
    smooth_colour_kernel(const LevelConst<T>* __restrict__ lc, int colour, const T* __restrict__ b,
                         T* x, int N, int consistent, long long ndofs) {
  constexpr int P = 2 * NN, E = 2 * NN + 2;
  constexpr int ND = CellShape<DIM, NN>::dofs;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PatchConst1D<T>* pc = reinterpret_cast<PatchConst1D<T>*>(smem_raw);
  T* buf1 = reinterpret_cast<T*>(pc + DIM);
  T* buf2 = buf1 + smooth_buf_elems<DIM, NN>(1);
  T* buf3 = buf2 + smooth_buf_elems<DIM, NN>(2);
  T* buf4 = buf3 + smooth_buf_elems<DIM, NN>(3);
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long col = (long long)blockIdx.y * ndofs;
  b += col;
  x += col;

  // patch of this colour: per direction v_e = 2 m_e + 1 (odd) or 2 m_e + 2 (even)
  int v[3] = {1, 1, 1}, t[3] = {0, 0, 0}, p[3] = {1, 1, 1}, first[3] = {0, 0, 0};
  {
    long long rest = blockIdx.x;
    for (int e = 0; e < DIM; ++e) {
      const int par = (colour >> e) & 1;
      const int cnt = par ? N / 2 : N / 2 - 1;
      const int m = (int)(rest % cnt);
      rest /= cnt;
      v[e] = par ? 2 * m + 1 : 2 * m + 2;
      t[e] = (v[e] == 1 ? 1 : 0) | (v[e] == N - 1 ? 2 : 0);
      p[e] = lc->p[t[e]];
      first[e] = lc->first[t[e]];
    }
  }
  for (int e = 0; e < DIM; ++e) {
    const int ty = t[e];
    for (int i = tid; i < SIPG_MAXP * SIPG_MAXPE; i += nth) {
      pc[e].Lr[i] = (&lc->Lr[ty][0][0])[i];
      pc[e].Mr[i] = (&lc->Mr[ty][0][0])[i];
    }
    for (int i = tid; i < SIPG_MAXP * SIPG_MAXP; i += nth) pc[e].S[i] = (&lc->S[ty][0][0])[i];
    for (int i = tid; i < SIPG_MAXP; i += nth) pc[e].lam[i] = lc->lam[ty][i];
  }
  // extended tile: a_e = 0 low halo, 1..P patch nodes, P+1 high halo
  const int ext_tot = (DIM == 2) ? E * E : E * E * E;
  for (int o = tid; o < ext_tot; o += nth) {
    int a[3] = {o % E, (o / E) % E, DIM == 3 ? o / (E * E) : 1};
    int nh = 0, hdir = -1;
    for (int e = 0; e < DIM; ++e)
      if (a[e] == 0 || a[e] == E - 1) {
        ++nh;
        hdir = e;
      }
    T val = T(0);
    if (nh == 0 || (nh == 1 && consistent)) {
      int cell[3] = {0, 0, 0}, node[3] = {0, 0, 0};
      bool ok = true;
      for (int e = 0; e < DIM; ++e) {
        if (e == hdir) {
          if (a[e] == 0) {
            cell[e] = v[e] - 2;
            node[e] = NN - 1;
          } else {
            cell[e] = v[e] + 1;
            node[e] = 0;
          }
          ok = ok && cell[e] >= 0 && cell[e] < N;
        } else {
          cell[e] = v[e] - 1 + (a[e] - 1) / NN;
          node[e] = (a[e] - 1) % NN;
        }
      }
      if (ok) {
        long long c = cell[0] + (long long)N * (cell[1] + (DIM == 3 ? (long long)N * cell[2] : 0));
        int loc = node[0] + NN * (node[1] + (DIM == 3 ? NN * node[2] : 0));
        val = x[c * ND + loc];
      }
    }
    buf1[o] = val;
  }
  __syncthreads();

  const int p0 = p[0], p1 = p[1], p2 = (DIM == 3) ? p[2] : 1;
  T* r;  // local residual, p0 x p1 (x p2)
  if (DIM == 2) {
    // A0 = Mr0 x_ext, B0 = Lr0 x_ext   (p0 x E)
    contract<T>(buf2, buf1, pc[0].Mr, nullptr, nullptr, SIPG_MAXPE, p0, E, 1, 0, E);
    contract<T>(buf3, buf1, pc[0].Lr, nullptr, nullptr, SIPG_MAXPE, p0, E, 1, 0, E);
    __syncthreads();
    // Ax = Lr1 A0 + Mr1 B0 (p0 x p1)
    contract<T>(buf1, buf2, pc[1].Lr, buf3, pc[1].Mr, SIPG_MAXPE, p0, p1, 1, 1, E);
    __syncthreads();
    r = buf1;
  } else {
    contract<T>(buf2, buf1, pc[0].Mr, nullptr, nullptr, SIPG_MAXPE, p0, E, E, 0, E);
    contract<T>(buf3, buf1, pc[0].Lr, nullptr, nullptr, SIPG_MAXPE, p0, E, E, 0, E);
    __syncthreads();
    // A01 = Mr1 A0 (buf1), C = Lr1 A0 + Mr1 B0 (buf4)   (p0 x p1 x E)
    contract<T>(buf1, buf2, pc[1].Mr, nullptr, nullptr, SIPG_MAXPE, p0, p1, E, 1, E);
    contract<T>(buf4, buf2, pc[1].Lr, buf3, pc[1].Mr, SIPG_MAXPE, p0, p1, E, 1, E);
    __syncthreads();
    // Ax = Lr2 A01 + Mr2 C  (p0 x p1 x p2)
    contract<T>(buf2, buf1, pc[2].Lr, buf4, pc[2].Mr, SIPG_MAXPE, p0, p1, p2, 2, E);
    __syncthreads();
    r = buf2;
  }
  // r = b_V - A x on V_j
  const int ntot = p0 * p1 * p2;
  for (int o = tid; o < ntot; o += nth) {
    int rr[3] = {o % p0, (o / p0) % p1, o / (p0 * p1)};
    int cell[3] = {0, 0, 0}, node[3] = {0, 0, 0};
    for (int e = 0; e < DIM; ++e) {
      int a = first[e] + rr[e];
      cell[e] = v[e] - 1 + a / NN;
      node[e] = a % NN;
    }
    long long c = cell[0] + (long long)N * (cell[1] + (DIM == 3 ? (long long)N * cell[2] : 0));
    int loc = node[0] + NN * (node[1] + (DIM == 3 ? NN * node[2] : 0));
    r[o] = b[c * ND + loc] - r[o];
  }
  __syncthreads();
  // fast diagonalisation: S^T sweeps, scale by 1 / sum lambda, S sweeps
  T* ta = (DIM == 2) ? buf2 : buf3;
  T* tb = (DIM == 2) ? buf3 : buf1;
  contract_t<T>(ta, r, pc[0].S, SIPG_MAXP, p0, p1, p2, 0);
  __syncthreads();
  contract_t<T>(tb, ta, pc[1].S, SIPG_MAXP, p0, p1, p2, 1);
  __syncthreads();
  T* cur = tb;
  T* oth = ta;
  if (DIM == 3) {
    contract_t<T>(oth, cur, pc[2].S, SIPG_MAXP, p0, p1, p2, 2);
    __syncthreads();
    T* tmp = cur;
    cur = oth;
    oth = tmp;
  }
  for (int o = tid; o < ntot; o += nth) {
    int rr[3] = {o % p0, (o / p0) % p1, o / (p0 * p1)};
    T lsum = pc[0].lam[rr[0]] + pc[1].lam[rr[1]] + (DIM == 3 ? pc[2].lam[rr[2]] : T(0));
    cur[o] = cur[o] / lsum;
  }
  __syncthreads();
  if (DIM == 3) {
    contract<T>(oth, cur, pc[2].S, nullptr, nullptr, SIPG_MAXP, p0, p1, p2, 2, p2);
    __syncthreads();
    T* tmp = cur;
    cur = oth;
    oth = tmp;
  }
  contract<T>(oth, cur, pc[1].S, nullptr, nullptr, SIPG_MAXP, p0, p1, p2, 1, p1);
  __syncthreads();
  contract<T>(cur, oth, pc[0].S, nullptr, nullptr, SIPG_MAXP, p0, p1, p2, 0, p0);
  __syncthreads();
  // x[V_j] += u
  for (int o = tid; o < ntot; o += nth) {
    int rr[3] = {o % p0, (o / p0) % p1, o / (p0 * p1)};
    int cell[3] = {0, 0, 0}, node[3] = {0, 0, 0};
    for (int e = 0; e < DIM; ++e) {
      int a = first[e] + rr[e];
      cell[e] = v[e] - 1 + a / NN;
      node[e] = a % NN;
    }
    long long c = cell[0] + (long long)N * (cell[1] + (DIM == 3 ? (long long)N * cell[2] : 0));
    int loc = node[0] + NN * (node[1] + (DIM == 3 ? NN * node[2] : 0));
    x[c * ND + loc] += cur[o];
  }
}

template <int DIM, int NN, typename T>
size_t smooth_smem_bytes() {
  size_t elems = (size_t)smooth_buf_elems<DIM, NN>(1) + smooth_buf_elems<DIM, NN>(2) +
                 smooth_buf_elems<DIM, NN>(3) + smooth_buf_elems<DIM, NN>(4);
  return DIM * sizeof(PatchConst1D<T>) + elems * sizeof(T);
}

template <typename T, int DIM, int NN>
cudaError_t smooth_dispatch2(const sipg_handle* h, int level, int colour, const T* b, T* x,
                             cudaStream_t s) {
  const LevelInfo& li = h->lv[level];
  const int N = li.N;
  long long npatch = 1;
  for (int e = 0; e < DIM; ++e) {
    int par = (colour >> e) & 1;
    npatch *= par ? N / 2 : N / 2 - 1;
  }
  if (npatch <= 0) return cudaSuccess;  // no patch of this colour (N = 2)
  const size_t smem = smooth_smem_bytes<DIM, NN, T>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(smooth_colour_kernel<DIM, NN, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((unsigned)npatch, h->prm.nrhs);
  smooth_colour_kernel<DIM, NN, T><<<grid, 256, smem, s>>>(
      h->cst<T>(level), colour, b, x, N, h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0,
      (long long)li.ndofs);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_smooth_colour(const sipg_handle* h, int level, int colour, const T* b, T* x,
                                 cudaStream_t s) {
  if (h->prm.dim == 2) {
    switch (h->n) {
      case 2: return smooth_dispatch2<T, 2, 2>(h, level, colour, b, x, s);
      case 3: return smooth_dispatch2<T, 2, 3>(h, level, colour, b, x, s);
      case 4: return smooth_dispatch2<T, 2, 4>(h, level, colour, b, x, s);
      case 5: return smooth_dispatch2<T, 2, 5>(h, level, colour, b, x, s);
      case 6: return smooth_dispatch2<T, 2, 6>(h, level, colour, b, x, s);
      case 7: return smooth_dispatch2<T, 2, 7>(h, level, colour, b, x, s);
      case 8: return smooth_dispatch2<T, 2, 8>(h, level, colour, b, x, s);
    }
  } else {
    switch (h->n) {
      case 2: return smooth_dispatch2<T, 3, 2>(h, level, colour, b, x, s);
      case 3: return smooth_dispatch2<T, 3, 3>(h, level, colour, b, x, s);
      case 4: return smooth_dispatch2<T, 3, 4>(h, level, colour, b, x, s);
      case 5: return smooth_dispatch2<T, 3, 5>(h, level, colour, b, x, s);
      case 6: return smooth_dispatch2<T, 3, 6>(h, level, colour, b, x, s);
      case 7: return smooth_dispatch2<T, 3, 7>(h, level, colour, b, x, s);
      case 8: return smooth_dispatch2<T, 3, 8>(h, level, colour, b, x, s);
    }
  }
  return cudaErrorInvalidValue;
}
template cudaError_t launch_smooth_colour<double>(const sipg_handle*, int, int, const double*,
                                                  double*, cudaStream_t);
template cudaError_t launch_smooth_colour<float>(const sipg_handle*, int, int, const float*, float*,
                                                 cudaStream_t);
