// Small tensor-product building blocks used by the kernels: 1D contractions
// of an n-point line held in registers against an n x n matrix in shared
// memory, and index helpers for the cell-wise lexicographic layout
// (Sec. 4.1: DoF (c, i) at c * n^d + i, i = i0 + n (i1 + n i2)).
#pragma once
#include "sipg_internal.cuh"

template <int DIM, int NN>
struct CellShape {
  static constexpr int n = NN;
  static constexpr int lines = (DIM == 2) ? NN : NN * NN;       // lines per direction
  static constexpr int dofs = (DIM == 2) ? NN * NN : NN * NN * NN;
  // base offset and stride of line `l` along direction e inside a cell
  __device__ static inline void line(int e, int l, int& base, int& stride) {
    if (DIM == 2) {
      if (e == 0) { base = l * NN; stride = 1; }
      else { base = l; stride = NN; }
    } else {
      if (e == 0) { base = l * NN; stride = 1; }                         // l = iy + n iz
      else if (e == 1) { base = (l % NN) + (l / NN) * NN * NN; stride = NN; }  // l = ix + n iz
      else { base = l; stride = NN * NN; }                                // l = ix + n iy
    }
  }
};

// out[i] (+)= sum_j A[i][j] v[j] for a line held in registers.
template <int NN, typename T>
__device__ __forceinline__ void matvec_line(const T* __restrict__ A, const T (&v)[NN], T (&o)[NN]) {
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    T s = A[i * NN] * v[0];
#pragma unroll
    for (int j = 1; j < NN; ++j) s = fma(A[i * NN + j], v[j], s);
    o[i] = s;
  }
}

template <int NN, typename T>
__device__ __forceinline__ void load_line(const T* __restrict__ p, int stride, T (&v)[NN]) {
#pragma unroll
  for (int j = 0; j < NN; ++j) v[j] = p[j * stride];
}

template <int NN, typename T>
__device__ __forceinline__ void store_line(T* __restrict__ p, int stride, const T (&v)[NN]) {
#pragma unroll
  for (int j = 0; j < NN; ++j) p[j * stride] = v[j];
}

// Copy an n x n block stored with leading dimension SIPG_MAXN into a compact
// n x n shared-memory array.
template <int NN, typename T>
__device__ __forceinline__ void copy_block(T* __restrict__ dst, const T (*src)[SIPG_MAXN], int tid,
                                           int nthreads) {
  for (int e = tid; e < NN * NN; e += nthreads) dst[e] = src[e / NN][e % NN];
}

// Smallest s >= m with s = r (mod 32): strides that place the lines of a
// shared-memory tile on chosen banks.
constexpr int i3_pad32(int m, int r) {
  int s = m;
  while (((s % 32) + 32) % 32 != ((r % 32) + 32) % 32) ++s;
  return s;
}
constexpr int i3_max(int a, int b) { return a > b ? a : b; }

// Vector width (elements) for loading a contiguous run of NN nodes of a
// cell-wise vector: 16-byte loads when every run is 16-byte aligned, else
// 8-byte, else scalar.
template <int NN, typename T>
constexpr int run_vw() {
  return (NN * (int)sizeof(T)) % 16 == 0 ? 16 / (int)sizeof(T)
                                         : ((NN * (int)sizeof(T)) % 8 == 0 ? 8 / (int)sizeof(T) : 1);
}

template <typename T, int V>
struct i3_vec;
template <> struct i3_vec<float, 4> { using t = float4; };
template <> struct i3_vec<float, 2> { using t = float2; };
template <> struct i3_vec<float, 1> { using t = float; };
template <> struct i3_vec<double, 2> { using t = double2; };
template <> struct i3_vec<double, 1> { using t = double; };

// One element / vector through the read-only path (NC) or a plain,
// coherent global load.
template <bool NC, typename V>
__device__ __forceinline__ V ld_elem(const V* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

// v[0..NN) = p[0..NN) by vector loads of width VW (read-only path if NC)
template <int NN, int VW, typename T, bool NC = true>
__device__ __forceinline__ void i3_ldrun(const T* __restrict__ p, T* v) {
  using V = typename i3_vec<T, VW>::t;
  const V* q = reinterpret_cast<const V*>(p);
#pragma unroll
  for (int j = 0; j < NN / VW; ++j) {
    const V w = ld_elem<NC>(q + j);
    const T* e = reinterpret_cast<const T*>(&w);
#pragma unroll
    for (int c = 0; c < VW; ++c) v[j * VW + c] = e[c];
  }
}

