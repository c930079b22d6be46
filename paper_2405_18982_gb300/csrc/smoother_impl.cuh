// Colour-pass kernels of the colourised multiplicative vertex-patch smoother
// (Algorithm 1, Sec. 3.1) with fast-diagonalisation local solves (Sec. 3.2,
// Eqs. inverse2d, inverse3d, fast_inverse).
//
// Patch j = the 2^d cells around interior vertex v (v_e in 1..N-1), colour
// c = sum_e (v_e mod 2) 2^e.  Per direction the patch has P = 2n nodes
// a = o n + i (o = 0: cell v-1, o = 1: cell v).  V_j drops the two
// patch-boundary nodes unless that end lies on the domain boundary (Dirichlet
// kernel).  With GLL bases the local residual on V_j needs, besides the patch
// cells, only the face-node layer of the cells across the patch faces (the
// -[[u]].{grad v} term), held here as six P^(d-1) halo faces:
//   r_j = b_j - sum_e ( (x)_{f != e} Mr_f (x) [Lr_e | hlo_e | hhi_e] ) [x_patch ; halos],
// Mr/Lr the rows V_j of the 1D patch mass / SIPG matrices (Mr block
// diagonal: its structural zeros are skipped).  Then
//   x[V_j] += (S_2 (x) S_1 (x) S_0) (sum_e Lambda_e)^{-1} (S_2^T (x) S_1^T (x) S_0^T) r_j.
// Same-colour patches share no V_j rows and do not couple through A, so a
// launch processes a whole colour in parallel.
//
// Kernel layout (GB300): a group of TPP threads owns one patch (one warp for
// k <= 3 in 3D, several patches per CTA); every contraction is a "line"
// operation: a thread holds one line of the tile in registers and applies a
// 1D operator whose coefficients sit in shared memory (broadcast reads).
// Lines read contiguously by one thread use odd strides (no bank conflicts).
// Phases (3D): load -> S1 (x) -> S2 (y) -> S3 (z, residual) -> F1 (S_x^T)
// -> F2 (S_y^T) -> F3 (S_z^T, scale, S_z) -> G2 (S_y) -> G1 (S_x, x += u).
// Interior patches (all directions away from the domain boundary, the vast
// majority) run with the exact size p = 2k; patches touching the boundary
// run a padded variant with p = 2n per direction, where the rows outside V_j
// have zero operators, the eigenvectors are padded by the identity and their
// residual is zeroed, so the update is exactly the local solve on V_j.
#pragma once
#include <algorithm>
#include <type_traits>
#include <utility>

#include "tensor_ops.cuh"

namespace {

template <int DIM, int NN, bool BND, typename T, bool WIDE = (sizeof(T) == 4)>
struct SC {
  static constexpr int P = 2 * NN;                   // patch nodes per direction
  static constexpr int PO = BND ? 2 * NN : 2 * NN - 2;  // rows per direction
  static constexpr int OFF = BND ? 0 : 1;            // patch node of row 0
  static constexpr int SX = P + 1;                   // odd stride of x-lines of length P
  static constexpr int SO = PO + 1;                  // odd stride of x-lines of length PO
  // threads per patch.  FP64 (bound by the FP64 pipe): 2 PO divides the line
  // counts of every phase (S2: PO (P+2), FD: PO^2), so no lane idles.  FP32
  // (bound by latency): PO^2 threads, one round for the residual and FD
  // phases and more resident warps per SM.
  static constexpr int TPP = DIM == 3 ? (WIDE ? PO * PO : 2 * PO) : PO;
  static constexpr bool WARP_SYNC = (32 % TPP) == 0;  // patches never straddle warps
  // shared memory per patch (elements)
  static constexpr int X_SZ = DIM == 3 ? P * P * SX : P * SX;
  static constexpr int HX_SZ = DIM == 3 ? 2 * P * P : 2 * P;     // x faces: scalars per line
  static constexpr int HYZ_SZ = DIM == 3 ? 4 * P * SX : 2 * SX;  // y (and z) faces as x-lines
  static constexpr int R1 = X_SZ + HX_SZ + HYZ_SZ;
  static constexpr int AB_SZ = DIM == 3 ? P * P * SO : P * SO;   // A and B
  static constexpr int AH_SZ = DIM == 3 ? 4 * P * SO : 2 * SO;   // Mx applied to y/z faces
  static constexpr int R2 = 2 * AB_SZ + AH_SZ;
  static constexpr int CD_SZ = DIM == 3 ? P * PO * PO : 1;       // C and D (3D only)
  static constexpr int CZ_SZ = DIM == 3 ? 2 * PO * PO : 1;
  static constexpr int R3 = DIM == 3 ? 2 * CD_SZ + CZ_SZ : 1;
  static constexpr int FD_SZ = DIM == 3 ? PO * PO * SO : PO * SO;  // FD arrays (x-lines padded)
  static constexpr int B_SZ = DIM == 3 ? PO * PO * PO : PO * PO;
  // region a: tile + halos (load, S1), then C/D (S2, S3), then FD ping;
  // region b: A/B (S1, S2), then the residual and FD pong
  static constexpr int RA_SZ = (R1 > R3 ? R1 : R3) > FD_SZ ? (R1 > R3 ? R1 : R3) : FD_SZ;
  static constexpr int RB_SZ = R2 > FD_SZ ? R2 : FD_SZ;
  static constexpr int PER_PATCH = RA_SZ + RB_SZ + B_SZ;
  static constexpr int NT = BND ? 4 : 1;                         // 1D types held in smem
};

// 1D operators of one type, compact, in shared memory
template <int PO, int P, typename T>
struct Ops1D {
  T Lm[PO * P];   // SIPG rows (patch columns only)
  // mass rows, block diagonal by cell and, with the GLL mass, diagonal plus
  // rank one per cell: row r (patch node a) = mw[r] e_a + mu[r] (ma on a's cell)
  T mw[PO], mu[PO], ma[P / 2];
  T hlo[PO], hhi[PO];
  T S[PO * PO];   // S[j][i]: row j, column i (column i = eigenvector i)
  T lam[PO];
  int first, last;  // rows of V_j are [first, last] (patch-node numbering minus OFF)
  // FP32: the same operators as pairs of consecutive rows (outputs), for the
  // packed two-lane FMA of sm_100+: one instruction computes two outputs
  static constexpr int NP = sizeof(T) == 4 ? 1 : 0;
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  T2 S2[NP ? PO * PO / 2 : 1];   // S2[j][q] = (S[j][2q], S[j][2q+1])      (S^T rows)
  T2 St2[NP ? PO * PO / 2 : 1];  // St2[q][j] = (S[2q][j], S[2q+1][j])     (S rows)
  T2 L2[NP ? PO * P / 2 : 1];    // L2[q][c] = (Lm[2q][c], Lm[2q+1][c])
  T2 mw2[NP ? PO / 2 : 1], mu2[NP ? PO / 2 : 1];
};

template <int DIM, int NN, bool BND, typename T>
constexpr int smooth_prefix_bytes() {
  using C = SC<DIM, NN, BND, T>;
  // boundary kernel: the four 1D operator sets; interior kernel: the table of
  // inverse eigenvalue sums 1 / (lambda_i + lambda_j (+ lambda_k))
  constexpr int dinv = DIM == 3 ? C::PO * C::PO * C::PO : C::PO * C::PO;
  constexpr int bytes = BND ? C::NT * (int)sizeof(Ops1D<C::PO, C::P, T>) : dinv * (int)sizeof(T);
  return (bytes + 15) / 16 * 16;
}

// Same rows with the mass as diagonal plus rank one per cell: one dot
// product per patch cell, then two FMAs per row
template <int PO, int P, int NN, int OFF, typename T>
__device__ __forceinline__ void mass_rows1(const Ops1D<PO, P, T>& op, const T (&v)[P], T (&o)[PO]) {
  T s[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T a = op.ma[0] * v[c * NN];
#pragma unroll
    for (int j = 1; j < NN; ++j) a = fma(op.ma[j], v[c * NN + j], a);
    s[c] = a;
  }
#pragma unroll
  for (int r = 0; r < PO; ++r) o[r] = fma(op.mu[r], s[(r + OFF) / NN], op.mw[r] * v[r + OFF]);
}

template <int PO, int P, int NN, int OFF, typename T>
__device__ __forceinline__ void mass_rows1_acc(const Ops1D<PO, P, T>& op, const T (&v)[P], T (&o)[PO]) {
  T s[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T a = op.ma[0] * v[c * NN];
#pragma unroll
    for (int j = 1; j < NN; ++j) a = fma(op.ma[j], v[c * NN + j], a);
    s[c] = a;
  }
#pragma unroll
  for (int r = 0; r < PO; ++r) o[r] = fma(op.mu[r], s[(r + OFF) / NN], fma(op.mw[r], v[r + OFF], o[r]));
}


// Structural nonzeros of the 1D patch SIPG matrix (rows/columns = patch
// nodes a, c): the own cell is dense; the coupling to the other patch cell is
// rank two (Sec. 2.2 face terms with GLL nodes): the vertex node's row couples
// to the whole other cell, every other row only to the other cell's node next
// to the vertex.  The low halo node couples to rows of the first cell, the
// high halo node to rows of the second.
template <int NN>
__host__ __device__ constexpr bool lr_nz(int a, int c) {
  return (a / NN == c / NN) || (a < NN ? (a == NN - 1 || c == NN) : (a == NN || c == NN - 1));
}

// out[r] = sum_c Lm[r][c] v[c] + hlo[r] h0 + hhi[r] h1 (structural zeros skipped)
template <int PO, int P, int NN, int OFF, typename T>
__device__ __forceinline__ void sipg_rows(const Ops1D<PO, P, T>& op, const T (&v)[P], T h0, T h1, T (&o)[PO]) {
#pragma unroll
  for (int r = 0; r < PO; ++r) {
    const int a = r + OFF;
    T s = (a < NN) ? op.hlo[r] * h0 : op.hhi[r] * h1;
#pragma unroll
    for (int c = 0; c < P; ++c)
      if (lr_nz<NN>(a, c)) s = fma(op.Lm[r * P + c], v[c], s);
    o[r] = s;
  }
}

// out[i] = sum_j S[j][i] v[j]   (S^T v)
template <int PO, typename T>
__device__ __forceinline__ void st_rows(const T* __restrict__ S, const T (&v)[PO], T (&o)[PO]) {
#pragma unroll
  for (int i = 0; i < PO; ++i) {
    T s = S[i] * v[0];
#pragma unroll
    for (int j = 1; j < PO; ++j) s = fma(S[j * PO + i], v[j], s);
    o[i] = s;
  }
}

// out[i] = sum_j S[i][j] v[j]   (S v)
template <int PO, typename T>
__device__ __forceinline__ void s_rows(const T* __restrict__ S, const T (&v)[PO], T (&o)[PO]) {
#pragma unroll
  for (int i = 0; i < PO; ++i) {
    T s = S[i * PO] * v[0];
#pragma unroll
    for (int j = 1; j < PO; ++j) s = fma(S[i * PO + j], v[j], s);
    o[i] = s;
  }
}

// Packed FP32 (two outputs per FMA instruction) versions of the line
// contractions; same products and summation order per output as the scalar
// ones, so the results are bitwise equal.
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

template <int PO>
__device__ __forceinline__ void st_rows2(const float2* __restrict__ S2, const float (&v)[PO], float (&o)[PO]) {
#pragma unroll
  for (int q = 0; q < PO / 2; ++q) {
    float2 s = __fmul2_rn(S2[q], bc2(v[0]));
#pragma unroll
    for (int j = 1; j < PO; ++j) s = __ffma2_rn(S2[j * (PO / 2) + q], bc2(v[j]), s);
    o[2 * q] = s.x;
    o[2 * q + 1] = s.y;
  }
}

template <int PO>
__device__ __forceinline__ void s_rows2(const float2* __restrict__ St2, const float (&v)[PO], float (&o)[PO]) {
#pragma unroll
  for (int q = 0; q < PO / 2; ++q) {
    float2 s = __fmul2_rn(St2[q * PO], bc2(v[0]));
#pragma unroll
    for (int j = 1; j < PO; ++j) s = __ffma2_rn(St2[q * PO + j], bc2(v[j]), s);
    o[2 * q] = s.x;
    o[2 * q + 1] = s.y;
  }
}

// rows 2q, 2q+1 of the SIPG rows over the union of their structural nonzeros
// (a column that is a structural zero of one row carries an exact 0 there)
template <int PO, int P, int NN, int OFF>
__device__ __forceinline__ void sipg_rows2(const Ops1D<PO, P, float>& op, const float (&v)[P], float h0, float h1,
                                           float (&o)[PO]) {
#pragma unroll
  for (int q = 0; q < PO / 2; ++q) {
    const int a0 = 2 * q + OFF, a1 = a0 + 1;
    float2 s = make_float2((a0 < NN) ? op.hlo[2 * q] * h0 : op.hhi[2 * q] * h1,
                           (a1 < NN) ? op.hlo[2 * q + 1] * h0 : op.hhi[2 * q + 1] * h1);
#pragma unroll
    for (int c = 0; c < P; ++c)
      if (lr_nz<NN>(a0, c) || lr_nz<NN>(a1, c)) s = __ffma2_rn(op.L2[q * P + c], bc2(v[c]), s);
    o[2 * q] = s.x;
    o[2 * q + 1] = s.y;
  }
}

template <int PO, int P, int NN, int OFF, bool ACC>
__device__ __forceinline__ void mass_rows2(const Ops1D<PO, P, float>& op, const float (&v)[P], float (&o)[PO]) {
  float sc[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    float a = op.ma[0] * v[c * NN];
#pragma unroll
    for (int j = 1; j < NN; ++j) a = fmaf(op.ma[j], v[c * NN + j], a);
    sc[c] = a;
  }
#pragma unroll
  for (int q = 0; q < PO / 2; ++q) {
    const int a0 = 2 * q + OFF, a1 = a0 + 1;
    const float2 vv = make_float2(v[a0], v[a1]);
    const float2 ss = make_float2(sc[a0 / NN], sc[a1 / NN]);
    float2 t;
    if (ACC)
      t = __ffma2_rn(op.mw2[q], vv, make_float2(o[2 * q], o[2 * q + 1]));
    else
      t = __fmul2_rn(op.mw2[q], vv);
    t = __ffma2_rn(op.mu2[q], ss, t);
    o[2 * q] = t.x;
    o[2 * q + 1] = t.y;
  }
}

template <int L, typename T>
__device__ __forceinline__ void ld(const T* p, int stride, T (&v)[L]) {
#pragma unroll
  for (int j = 0; j < L; ++j) v[j] = p[j * stride];
}
template <int L, typename T>
__device__ __forceinline__ void st(T* p, int stride, const T (&v)[L]) {
#pragma unroll
  for (int j = 0; j < L; ++j) p[j * stride] = v[j];
}

// Asynchronous element copy global -> shared (cp.async, no register staging);
// with valid == false the destination is zero-filled and nothing is read.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gmem_src, bool valid) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  const int src_size = valid ? (int)sizeof(T) : 0;
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem_src), "r"(src_size) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem_src), "r"(src_size) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int NTASK, int TPP, typename F>
__device__ __forceinline__ void for_lines(int lane, F&& f) {
#pragma unroll 1
  for (int rr = 0; rr < (NTASK + TPP - 1) / TPP; ++rr) {
    const int t = lane + rr * TPP;
    if (t < NTASK) f(t);
  }
}

template <int PO, int P, typename T, int NT>
struct SmoothOps {
  Ops1D<PO, P, T> t[NT];
};

// Host: the 1D operators of type t from the level constants.  Interior
// kernel: rows = V_j of type 0 (p = 2k).  Boundary kernel: rows = all P patch
// nodes; rows outside V_j get zero operators, S is padded by the identity and
// Lambda by 1.
template <int PO, int P, bool BND, typename T>
void make_ops(const LevelConst<T>& lc, int t, Ops1D<PO, P, T>& op) {
  const int first = lc.first[t], p = lc.p[t];
  const int off = BND ? first : 0;  // row r of the padded set <-> row r - off of V_j
  for (int r = 0; r < PO; ++r) {
    const int rv = r - off;
    const bool in = BND ? (rv >= 0 && rv < p) : true;
    for (int c = 0; c < P; ++c) {
      op.Lm[r * P + c] = in ? lc.Lr[t][rv][1 + c] : T(0);
    }
    op.hlo[r] = in ? lc.Lr[t][rv][0] : T(0);
    op.hhi[r] = in ? lc.Lr[t][rv][P + 1] : T(0);
    op.lam[r] = in ? lc.lam[t][rv] : T(1);
    const int node = (r + (BND ? 0 : 1)) % (P / 2);  // local node of row r in its cell
    op.mw[r] = in ? lc.Mw[node] : T(0);
    op.mu[r] = in ? lc.Mu[node] : T(0);
  }
  for (int j = 0; j < P / 2; ++j) op.ma[j] = lc.Ma[j];
  for (int j = 0; j < PO; ++j)
    for (int i = 0; i < PO; ++i) {
      const int jv = j - off, iv = i - off;
      const bool in = BND ? (jv >= 0 && jv < p && iv >= 0 && iv < p) : true;
      op.S[j * PO + i] = in ? lc.S[t][jv][iv] : (BND && j == i ? T(1) : T(0));
    }
  op.first = BND ? first : 0;
  op.last = BND ? first + p - 1 : PO - 1;
  if constexpr (sizeof(T) == 4) {
    for (int q = 0; q < PO / 2; ++q) {
      for (int j = 0; j < PO; ++j) {
        op.S2[j * (PO / 2) + q] = make_float2(op.S[j * PO + 2 * q], op.S[j * PO + 2 * q + 1]);
        op.St2[q * PO + j] = make_float2(op.S[2 * q * PO + j], op.S[(2 * q + 1) * PO + j]);
      }
      for (int c = 0; c < P; ++c) op.L2[q * P + c] = make_float2(op.Lm[2 * q * P + c], op.Lm[(2 * q + 1) * P + c]);
      op.mw2[q] = make_float2(op.mw[2 * q], op.mw[2 * q + 1]);
      op.mu2[q] = make_float2(op.mu[2 * q], op.mu[2 * q + 1]);
    }
  }
}

// patch enumeration of colour c: per direction m in [0, cnt), v = 2m+1 (odd
// parity) or 2m+2 (even); interior box [lo, hi) in m.
struct PatchGrid {
  int cnt[3], lo[3], hi[3];
  // the interior-box widths w = hi - lo as divisions by multiplication
  // (Granlund and Montgomery, "Division by invariant integers using
  // multiplication", 1994, Thm. 4.2 with N = 31): q / w = umulhi(q, dmul) >>
  // dshift for 0 <= q < 2^31; dmul = 0 marks w <= 1 (q / 1 = q)
  unsigned int dmul[3];
  int dshift[3];
  long long n_int, n_bnd;
};

__device__ __forceinline__ int div_width(int q, unsigned int dmul, int dshift) {
  return dmul ? (int)(__umulhi((unsigned int)q, dmul) >> dshift) : q;
}

__device__ __forceinline__ int outside_map(int q, int lo, int hi) { return q < lo ? q : q - lo + hi; }

template <int DIM, bool BND>
__device__ __forceinline__ void patch_index(const PatchGrid& g, long long idx, int (&m)[3]) {
  if (!BND) {
    // interior indices stay below 2^31: a colour with 2^31 interior patches
    // would need more than 2^34 DoFs, beyond any device memory
    int q = (int)idx;
    for (int e = 0; e < DIM; ++e) {
      const int w = g.hi[e] - g.lo[e];
      const int qn = div_width(q, g.dmul[e], g.dshift[e]);
      m[e] = g.lo[e] + (q - qn * w);
      q = qn;
    }
    return;
  }
  // shell of the box: slabs outside in the slowest direction first
  long long q = idx;
  if (DIM == 3) {
    const int I0 = g.hi[0] - g.lo[0], I1 = g.hi[1] - g.lo[1], I2 = g.hi[2] - g.lo[2];
    const long long cA = (long long)(g.cnt[2] - I2) * g.cnt[1] * g.cnt[0];
    const long long cB = (long long)I2 * (g.cnt[1] - I1) * g.cnt[0];
    if (q < cA) {
      m[0] = (int)(q % g.cnt[0]);
      q /= g.cnt[0];
      m[1] = (int)(q % g.cnt[1]);
      m[2] = outside_map((int)(q / g.cnt[1]), g.lo[2], g.hi[2]);
    } else if ((q -= cA) < cB) {
      m[0] = (int)(q % g.cnt[0]);
      q /= g.cnt[0];
      m[1] = outside_map((int)(q % (g.cnt[1] - I1)), g.lo[1], g.hi[1]);
      m[2] = g.lo[2] + (int)(q / (g.cnt[1] - I1));
    } else {
      q -= cB;
      const int w0 = g.cnt[0] - I0;
      m[0] = outside_map((int)(q % w0), g.lo[0], g.hi[0]);
      q /= w0;
      m[1] = g.lo[1] + (int)(q % I1);
      m[2] = g.lo[2] + (int)(q / I1);
    }
  } else {
    const int I0 = g.hi[0] - g.lo[0], I1 = g.hi[1] - g.lo[1];
    const long long cA = (long long)(g.cnt[1] - I1) * g.cnt[0];
    if (q < cA) {
      m[0] = (int)(q % g.cnt[0]);
      m[1] = outside_map((int)(q / g.cnt[0]), g.lo[1], g.hi[1]);
    } else {
      q -= cA;
      const int w0 = g.cnt[0] - I0;
      m[0] = outside_map((int)(q % w0), g.lo[0], g.hi[0]);
      m[1] = g.lo[1] + (int)(q / w0);
    }
    m[2] = 0;
  }
}

template <int DIM, int NN>
__device__ __forceinline__ long long gidx(int N, int c0, int c1, int c2, int i0, int i1, int i2) {
  constexpr int ND = DIM == 3 ? NN * NN * NN : NN * NN;
  long long c = c0 + (long long)N * (c1 + (DIM == 3 ? (long long)N * c2 : 0));
  return c * ND + i0 + NN * (i1 + (DIM == 3 ? NN * i2 : 0));
}

template <int TPP>
__device__ __forceinline__ void group_sync() {
  if (TPP <= 32 && 32 % TPP == 0) __syncwarp();  // patch groups never straddle warps
  else __syncthreads();
}

// Operator sets and shared tables of one CTA: the interior path reads the
// kernel parameters directly (compile-time offsets: constant-bank operands),
// the boundary path reads its four padded sets from shared memory (runtime
// type index).
template <int DIM, int NN, bool BND, typename T>
__device__ __forceinline__ void smooth_prefix_setup(
    const SmoothOps<SC<DIM, NN, BND, T>::PO, SC<DIM, NN, BND, T>::P, T, SC<DIM, NN, BND, T>::NT>& ops,
    unsigned char* prefix) {
  using C = SC<DIM, NN, BND, T>;
  constexpr int PO = C::PO;
  using Ops = Ops1D<PO, C::P, T>;
  if (BND) {
    const int* src = reinterpret_cast<const int*>(&ops);
    int* dst = reinterpret_cast<int*>(prefix);
    for (int e = threadIdx.x; e < (int)(sizeof(Ops) * C::NT / sizeof(int)); e += blockDim.x) dst[e] = src[e];
  } else {
    T* dinv = reinterpret_cast<T*>(prefix);
    constexpr int ND3 = DIM == 3 ? PO * PO * PO : PO * PO;
    for (int e = threadIdx.x; e < ND3; e += blockDim.x) {
      const int r0 = e % PO, r1 = (e / PO) % PO, r2 = e / (PO * PO);
      T ls = ops.t[0].lam[r0] + ops.t[0].lam[r1];
      if (DIM == 3) ls += ops.t[0].lam[r2];
      dinv[e] = T(1) / ls;
    }
  }
}

// Process patches pbase + slot (slot < PPC) of colour `colour`.  Every thread
// of the CTA must call this (it contains CTA or warp barriers); threads whose
// slot is >= PPC, or whose patch is past the end, only take part in barriers.
template <int DIM, int NN, bool BND, typename T, int PPC, bool WIDE = (sizeof(T) == 4)>
__device__ __forceinline__ void smooth_chunk(
    const SmoothOps<SC<DIM, NN, BND, T>::PO, SC<DIM, NN, BND, T>::P, T, SC<DIM, NN, BND, T>::NT>& ops,
    const unsigned char* prefix, T* base, long long pbase, int colour, const T* __restrict__ b, T* x, int N,
    int consistent, const PatchGrid& grid) {
  using C = SC<DIM, NN, BND, T, WIDE>;
  constexpr int P = C::P, PO = C::PO, OFF = C::OFF, SX = C::SX, SO = C::SO, TPP = C::TPP;
  using Ops = Ops1D<PO, P, T>;
  const Ops* sops = reinterpret_cast<const Ops*>(prefix);
  const T* dinv = reinterpret_cast<const T*>(prefix);
  const int tid = threadIdx.x;
  const int lane = tid % TPP;
  const int pl = tid / TPP;  // patch slot in the CTA

  const long long npatch = BND ? grid.n_bnd : grid.n_int;
  const long long pidx = pbase + pl;
  const bool valid = pl < PPC && pidx < npatch;
  int m[3] = {0, 0, 0};
  if (valid) patch_index<DIM, BND>(grid, pidx, m);
  int v[3] = {1, 1, 1}, ty[3] = {0, 0, 0};
  for (int e = 0; e < DIM; ++e) {
    const int par = (colour >> e) & 1;
    v[e] = par ? 2 * m[e] + 1 : 2 * m[e] + 2;
    ty[e] = BND ? ((v[e] == 1 ? 1 : 0) | (v[e] == N - 1 ? 2 : 0)) : 0;
  }
  T* sm = base + (size_t)(pl < PPC ? pl : 0) * C::PER_PATCH;
  T* R1 = sm;                 // tile + halos, later C/D, later FD ping
  T* R2 = sm + C::RA_SZ;      // A/B, later residual and FD pong
  T* R3 = R1;                 // C/D alias the tile (dead after S1)
  T* Bv = R2 + C::RB_SZ;
  // R1 layout: X | Hx (lo, hi) | Hy/Hz faces as x-lines
  T* X = R1;
  T* Hx = X + C::X_SZ;
  T* Hyz = Hx + C::HX_SZ;

  // ---------------------------------------------------------------- load
  // strides of the cell grid and of the nodes inside a cell
  const long long cstr[3] = {1, (long long)N, (long long)N * N};
  constexpr int nstr[3] = {1, NN, NN * NN};
  constexpr int ND = DIM == 3 ? NN * NN * NN : NN * NN;
  const long long cbase = (v[0] - 1) + cstr[1] * (v[1] - 1) + (DIM == 3 ? cstr[2] * (v[2] - 1) : 0);
  if (valid) {
    constexpr int NC = DIM == 3 ? 8 : 4;
    constexpr int QR = (ND + TPP - 1) / TPP;  // rounds per cell
    int li[QR], xoff[QR], ri[QR][3];
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      const int i = lane + q * TPP;
      const int i0 = i % NN, i1 = (i / NN) % NN, i2 = DIM == 3 ? i / (NN * NN) : 0;
      li[q] = i;
      xoff[q] = (DIM == 3 ? i2 * P + i1 : i1) * SX + i0;
      ri[q][0] = i0;
      ri[q][1] = i1;
      ri[q][2] = i2;
    }
    // patch cells (x) and b on V_j, coalesced per cell
#pragma unroll
    for (int o = 0; o < NC; ++o) {
      const int oc[3] = {o & 1, (o >> 1) & 1, o >> 2};
      const long long cell = cbase + oc[0] + cstr[1] * oc[1] + (DIM == 3 ? cstr[2] * oc[2] : 0);
      const T* xp = x + cell * ND;
      const T* bp = b + cell * ND;
      const int tile = (DIM == 3 ? (oc[2] * NN * P + oc[1] * NN) : oc[1] * NN) * SX + oc[0] * NN;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        if (ND % TPP != 0 && li[q] >= ND) continue;
        cp_async_elem(&X[tile + xoff[q]], &xp[li[q]], true);
        int r[3] = {0, 0, 0};
        bool in = true;
#pragma unroll
        for (int e = 0; e < DIM; ++e) {
          r[e] = oc[e] * NN + ri[q][e] - OFF;
          const int lo = BND ? sops[ty[e]].first : 0;
          const int hi = BND ? sops[ty[e]].last : PO - 1;
          in = in && r[e] >= lo && r[e] <= hi;
        }
        if (in) cp_async_elem(&Bv[(DIM == 3 ? r[2] * PO * PO : 0) + r[1] * PO + r[0]], &bp[li[q]], true);
      }
    }
    // halo faces: face-node layer of the cells across each patch face (zero
    // when that cell is outside the domain, or for the paper's kernel)
    constexpr int FACE = DIM == 3 ? P * P : P;
    constexpr int QF = (FACE + TPP - 1) / TPP;
#pragma unroll
    for (int dir = 0; dir < DIM; ++dir) {
      const int d1 = dir == 0 ? 1 : 0;               // first tangential direction
      const int d2 = dir == 2 ? 1 : 2;               // second (3D only)
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int nb = side ? v[dir] + 1 : v[dir] - 2;
        const bool exists = consistent && nb >= 0 && nb < N;
        const long long fcell = cbase + cstr[dir] * (nb - (v[dir] - 1));
        const int nnode = (side ? 0 : NN - 1) * nstr[dir];
#pragma unroll
        for (int q = 0; q < QF; ++q) {
          const int f = lane + q * TPP;
          if (FACE % TPP != 0 && f >= FACE) continue;
          const int s0 = f % P, s1 = DIM == 3 ? f / P : 0;
          const T* src = x;  // any valid address when the halo is zero-filled
          if (exists) {
            long long cell = fcell + cstr[d1] * (s0 / NN);
            int node = nnode + nstr[d1] * (s0 % NN);
            if (DIM == 3) {
              cell += cstr[d2] * (s1 / NN);
              node += nstr[d2] * (s1 % NN);
            }
            src = x + cell * ND + node;
          }
          T* dst = (dir == 0) ? &Hx[side * FACE + f]
                              : &Hyz[(((dir - 1) * 2 + side) * (DIM == 3 ? P : 1) + s1) * SX + s0];
          cp_async_elem(dst, src, exists);
        }
      }
    }
  }
  cp_async_wait_all();
  group_sync<TPP>();

  const Ops& ox = BND ? sops[ty[0]] : ops.t[0];
  const Ops& oy = BND ? sops[ty[1]] : ops.t[0];
  const Ops& oz = BND ? sops[DIM == 3 ? ty[2] : 0] : ops.t[0];

  if constexpr (DIM == 3) {
    T* A = R2;
    T* Bm = A + C::AB_SZ;
    T* AH = Bm + C::AB_SZ;  // [slot(ylo,yhi,zlo,zhi)][P lines][SO]
    // ---------------------------------------------------- S1: along x
    if (valid) {
      for_lines<P * P + 4 * P, TPP>(lane, [&](const int t) {
        if (t < P * P) {
          const int a1 = t % P, a2 = t / P;
          T vin[P], oa[PO], ob[PO];
          ld<P>(X + (a2 * P + a1) * SX, 1, vin);
          mass_rows1<PO, P, NN, OFF>(ox, vin, oa);
          sipg_rows<PO, P, NN, OFF>(ox, vin, Hx[a2 * P + a1], Hx[P * P + a2 * P + a1], ob);
          st<PO>(A + (a2 * P + a1) * SO, 1, oa);
          st<PO>(Bm + (a2 * P + a1) * SO, 1, ob);
        } else {
          const int h = t - P * P;  // slot * P + line
          T vin[P], oa[PO];
          ld<P>(Hyz + h * SX, 1, vin);
          mass_rows1<PO, P, NN, OFF>(ox, vin, oa);
          st<PO>(AH + h * SO, 1, oa);
        }
      });
    }
    group_sync<TPP>();
    // ---------------------------------------------------- S2: along y
    T* Cc = R3;                   // [a2][r1][r0]
    T* Dd = Cc + C::CD_SZ;        // [a2][r1][r0]
    T* Cz = Dd + C::CD_SZ;        // [side][r1][r0]
    if (valid) {
      for_lines<PO * P + 2 * PO, TPP>(lane, [&](const int t) {
        if (t < PO * P) {
          const int r0 = t % PO, a2 = t / PO;
          T va[P], vb[P], oc[PO], od[PO];
          ld<P>(A + a2 * P * SO + r0, SO, va);
          ld<P>(Bm + a2 * P * SO + r0, SO, vb);
          mass_rows1<PO, P, NN, OFF>(oy, va, oc);
          // y-halo faces with M_x applied: AH slots 0 (lo), 1 (hi), line a2
          sipg_rows<PO, P, NN, OFF>(oy, va, AH[(0 * P + a2) * SO + r0], AH[(1 * P + a2) * SO + r0], od);
          mass_rows1_acc<PO, P, NN, OFF>(oy, vb, od);
          st<PO>(Cc + a2 * PO * PO + r0, PO, oc);
          st<PO>(Dd + a2 * PO * PO + r0, PO, od);
        } else {
          const int q = t - PO * P, side = q / PO, r0 = q % PO;
          T va[P], oc[PO];
          ld<P>(AH + (2 + side) * P * SO + r0, SO, va);  // z faces, lines indexed by a1
          mass_rows1<PO, P, NN, OFF>(oy, va, oc);
          st<PO>(Cz + side * PO * PO + r0, PO, oc);
        }
      });
    }
    group_sync<TPP>();
    // ---------------------------------------------------- S3: along z, residual
    T* Rr = R2;  // [r2][r1][r0], x-lines padded to SO
    if (valid) {
      for_lines<PO * PO, TPP>(lane, [&](const int t) {
        const int r0 = t % PO, r1 = t / PO;
        T vc[P], vd[P], o[PO];
        ld<P>(Cc + r1 * PO + r0, PO * PO, vc);
        ld<P>(Dd + r1 * PO + r0, PO * PO, vd);
        sipg_rows<PO, P, NN, OFF>(oz, vc, Cz[r1 * PO + r0], Cz[PO * PO + r1 * PO + r0], o);
        mass_rows1_acc<PO, P, NN, OFF>(oz, vd, o);
        const bool inxy = !BND || (r0 >= ox.first && r0 <= ox.last && r1 >= oy.first && r1 <= oy.last);
#pragma unroll
        for (int r2 = 0; r2 < PO; ++r2) {
          const bool in = inxy && (!BND || (r2 >= oz.first && r2 <= oz.last));
          Rr[(r2 * PO + r1) * SO + r0] = in ? Bv[(r2 * PO + r1) * PO + r0] - o[r2] : T(0);
        }
      });
    }
    group_sync<TPP>();
    // ---------------------------------------------------- fast diagonalisation
    T* T1 = R1;
    if (valid) {  // F1: S_x^T along x
      for_lines<PO * PO, TPP>(lane, [&](const int t) {
        T vin[PO], o[PO];
        ld<PO>(Rr + t * SO, 1, vin);
        st_rows<PO>(ox.S, vin, o);
        st<PO>(T1 + t * SO, 1, o);
      });
    }
    group_sync<TPP>();
    T* T2 = R2;
    if (valid) {  // F2: S_y^T along y; lines (r0, r2)
      for_lines<PO * PO, TPP>(lane, [&](const int t) {
        const int r0 = t % PO, r2 = t / PO;
        T vin[PO], o[PO];
        ld<PO>(T1 + r2 * PO * SO + r0, SO, vin);
        st_rows<PO>(oy.S, vin, o);
        st<PO>(T2 + r2 * PO * SO + r0, SO, o);
      });
    }
    group_sync<TPP>();
    if (valid) {  // F3: S_z^T, divide by the eigenvalue sums, S_z; lines (r0, r1)
      for_lines<PO * PO, TPP>(lane, [&](const int t) {
        const int r0 = t % PO, r1 = t / PO;
        T vin[PO], o[PO];
        ld<PO>(T2 + r1 * SO + r0, PO * SO, vin);
        st_rows<PO>(oz.S, vin, o);
        if (BND) {
          const T lxy = ox.lam[r0] + oy.lam[r1];
#pragma unroll
          for (int r2 = 0; r2 < PO; ++r2) o[r2] = o[r2] / (lxy + oz.lam[r2]);
        } else {
#pragma unroll
          for (int r2 = 0; r2 < PO; ++r2) o[r2] *= dinv[(r2 * PO + r1) * PO + r0];
        }
        s_rows<PO>(oz.S, o, vin);
        st<PO>(T1 + r1 * SO + r0, PO * SO, vin);
      });
    }
    group_sync<TPP>();
    if (valid) {  // G2: S_y along y
      for_lines<PO * PO, TPP>(lane, [&](const int t) {
        const int r0 = t % PO, r2 = t / PO;
        T vin[PO], o[PO];
        ld<PO>(T1 + r2 * PO * SO + r0, SO, vin);
        s_rows<PO>(oy.S, vin, o);
        st<PO>(T2 + r2 * PO * SO + r0, SO, o);
      });
    }
    group_sync<TPP>();
    if (valid) {  // G1: S_x along x, x[V_j] += u
      for_lines<PO * PO, TPP>(lane, [&](const int t) {
        const int r1 = t % PO, r2 = t / PO;
        const bool in12 = !BND || (r1 >= oy.first && r1 <= oy.last && r2 >= oz.first && r2 <= oz.last);
        T vin[PO], o[PO];
        ld<PO>(T2 + t * SO, 1, vin);
        s_rows<PO>(ox.S, vin, o);
        if (in12) {
          const int a1 = r1 + OFF, a2 = r2 + OFF;
          const long long c0 = cbase + cstr[1] * (a1 / NN) + cstr[2] * (a2 / NN);
          T* xl = x + c0 * ND + NN * (a1 % NN) + NN * NN * (a2 % NN);  // cell o0 = 0 of this line
#pragma unroll
          for (int r0 = 0; r0 < PO; ++r0) {
            if (BND && (r0 < ox.first || r0 > ox.last)) continue;
            const int a0 = r0 + OFF;
            xl[(a0 / NN) * ND + a0 % NN] += o[r0];
          }
        }
      });
    }
  } else {
    // ================================================================ 2D
    T* A = R2;
    T* Bm = A + C::AB_SZ;
    T* AH = Bm + C::AB_SZ;  // y faces with M_x applied: [side][SO]
    if (valid) {
      for_lines<P + 2, TPP>(lane, [&](const int t) {
        if (t < P) {
          T vin[P], oa[PO], ob[PO];
          ld<P>(X + t * SX, 1, vin);
          mass_rows1<PO, P, NN, OFF>(ox, vin, oa);
          sipg_rows<PO, P, NN, OFF>(ox, vin, Hx[t], Hx[P + t], ob);
          st<PO>(A + t * SO, 1, oa);
          st<PO>(Bm + t * SO, 1, ob);
        } else {
          const int side = t - P;
          T vin[P], oa[PO];
          ld<P>(Hyz + side * SX, 1, vin);
          mass_rows1<PO, P, NN, OFF>(ox, vin, oa);
          st<PO>(AH + side * SO, 1, oa);
        }
      });
    }
    group_sync<TPP>();
    T* Rr = R1;  // [r1][r0] padded
    if (valid) {
      for_lines<PO, TPP>(lane, [&](const int t) {
        const int r0 = t;
        T va[P], vb[P], o[PO];
        ld<P>(A + r0, SO, va);
        ld<P>(Bm + r0, SO, vb);
        sipg_rows<PO, P, NN, OFF>(oy, va, AH[r0], AH[SO + r0], o);
        mass_rows1_acc<PO, P, NN, OFF>(oy, vb, o);
        const bool in0 = !BND || (r0 >= ox.first && r0 <= ox.last);
#pragma unroll
        for (int r1 = 0; r1 < PO; ++r1) {
          const bool in = in0 && (!BND || (r1 >= oy.first && r1 <= oy.last));
          Rr[r1 * SO + r0] = in ? Bv[r1 * PO + r0] - o[r1] : T(0);
        }
      });
    }
    group_sync<TPP>();
    T* T1 = R2;
    if (valid) {  // S_x^T along x
      for_lines<PO, TPP>(lane, [&](const int t) {
        T vin[PO], o[PO];
        ld<PO>(Rr + t * SO, 1, vin);
        st_rows<PO>(ox.S, vin, o);
        st<PO>(T1 + t * SO, 1, o);
      });
    }
    group_sync<TPP>();
    if (valid) {  // S_y^T, scale, S_y along y
      for_lines<PO, TPP>(lane, [&](const int t) {
        const int r0 = t;
        T vin[PO], o[PO];
        ld<PO>(T1 + r0, SO, vin);
        st_rows<PO>(oy.S, vin, o);
        if (BND) {
#pragma unroll
          for (int r1 = 0; r1 < PO; ++r1) o[r1] = o[r1] / (ox.lam[r0] + oy.lam[r1]);
        } else {
#pragma unroll
          for (int r1 = 0; r1 < PO; ++r1) o[r1] *= dinv[r1 * PO + r0];
        }
        s_rows<PO>(oy.S, o, vin);
        st<PO>(Rr + r0, SO, vin);
      });
    }
    group_sync<TPP>();
    if (valid) {  // S_x along x, x += u
      for_lines<PO, TPP>(lane, [&](const int t) {
        const int r1 = t;
        const bool in1 = !BND || (r1 >= oy.first && r1 <= oy.last);
        T vin[PO], o[PO];
        ld<PO>(Rr + r1 * SO, 1, vin);
        s_rows<PO>(ox.S, vin, o);
        if (in1) {
          const int a1 = r1 + OFF;
          T* xl = x + (cbase + cstr[1] * (a1 / NN)) * ND + NN * (a1 % NN);
#pragma unroll
          for (int r0 = 0; r0 < PO; ++r0) {
            if (BND && (r0 < ox.first || r0 > ox.last)) continue;
            const int a0 = r0 + OFF;
            xl[(a0 / NN) * ND + a0 % NN] += o[r0];
          }
        }
      });
    }
  }
}

// One colour pass over the interior (BND = false) or boundary patches.
template <int DIM, int NN, bool BND, typename T, int PPC>
__global__ void __launch_bounds__(SC<DIM, NN, BND, T>::TPP * PPC)
    smooth_fast_kernel(const __grid_constant__ SmoothOps<SC<DIM, NN, BND, T>::PO, SC<DIM, NN, BND, T>::P, T,
                                                         SC<DIM, NN, BND, T>::NT> ops,
                       int colour, const T* __restrict__ b, T* x, int N, int consistent, long long ndofs,
                       PatchGrid grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  smooth_prefix_setup<DIM, NN, BND, T>(ops, smem_raw);
  __syncthreads();
  T* base = reinterpret_cast<T*>(smem_raw + smooth_prefix_bytes<DIM, NN, BND, T>());
  const long long col = (long long)blockIdx.y * ndofs;
  smooth_chunk<DIM, NN, BND, T, PPC>(ops, smem_raw, base, (long long)blockIdx.x * PPC, colour, b + col, x + col,
                                     N, consistent, grid);
}

// patches per CTA: as many as fit 112 KB of shared memory and 512 threads,
// preferring a whole number of warps
template <int DIM, int NN, bool BND, typename T>
constexpr int smooth_ppc() {
  using C = SC<DIM, NN, BND, T>;
  constexpr int per = C::PER_PATCH * (int)sizeof(T);
  constexpr int budget = 112 * 1024 - smooth_prefix_bytes<DIM, NN, BND, T>();
  int k = budget / per;
  if (k > 512 / C::TPP) k = 512 / C::TPP;
  if (k < 1) k = 1;
  for (int p = k; p >= 1; --p)
    if ((C::TPP * p) % 32 == 0) return p;
  return k;
}

template <int DIM, int NN, bool BND, typename T>
size_t smooth_smem_bytes() {
  using C = SC<DIM, NN, BND, T>;
  constexpr int PPC = smooth_ppc<DIM, NN, BND, T>();
  return (size_t)smooth_prefix_bytes<DIM, NN, BND, T>() + (size_t)PPC * C::PER_PATCH * sizeof(T);
}

template <int DIM, int NN, bool BND, typename T>
cudaError_t launch_part(const sipg_handle* h, int level, int colour, const T* b, T* x, const PatchGrid& g,
                        cudaStream_t s) {
  const long long np = BND ? g.n_bnd : g.n_int;
  if (np <= 0) return cudaSuccess;
  constexpr int PPC = smooth_ppc<DIM, NN, BND, T>();
  using C = SC<DIM, NN, BND, T>;
  const size_t smem = smooth_smem_bytes<DIM, NN, BND, T>();
  cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(smooth_fast_kernel<DIM, NN, BND, T, PPC>), (int)smem);
  if (e != cudaSuccess) return e;
  SmoothOps<C::PO, C::P, T, C::NT> ops;
  for (int t = 0; t < C::NT; ++t) make_ops<C::PO, C::P, BND, T>(h->hcst<T>(level), t, ops.t[t]);
  dim3 grid((unsigned)((np + PPC - 1) / PPC), h->prm.nrhs);
  smooth_fast_kernel<DIM, NN, BND, T, PPC><<<grid, C::TPP * PPC, smem, s>>>(
      ops, colour, b, x, h->lv[level].N, h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0,
      (long long)h->lv[level].ndofs, g);
  return cudaGetLastError();
}

PatchGrid make_grid(int dim, int N, int colour);

// ------------------------------------------------------------------ fused step
// All 2^d colours of one smoothing step in one cooperative launch, for levels
// whose colour passes are latency bound (one wave of CTAs).  Colours are
// separated by a grid barrier; every wait is bounded: after ~0.5 s the CTA
// sets *status and returns (the host reports SIPG_ETIMEOUT), so the GPU never
// hangs.  Loads of x after a barrier see the other CTAs' writes: the waiting
// thread fences (gpu scope) after the release is observed, then the CTA
// synchronises.
struct StepGrids {
  PatchGrid g[8];
};

__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* status, unsigned int expected) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    volatile int* vstatus = status;
    int good = 1;
    if (*vstatus != 0) {
      // an earlier wait gave up: the arrival count is no longer aligned, so
      // leave at once instead of spending another full wait
      good = 0;
    } else {
      const unsigned int gen = *vgen;
      __threadfence();
      const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
      if (arrived == expected) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        long long it = 0;
        while (*vgen == gen) {
          if (*vstatus != 0) {  // another CTA gave up
            good = 0;
            break;
          }
          if (++it > (1LL << 23)) {
            good = 0;
            atomicExch(status, 1);
            break;
          }
          __nanosleep(40);
        }
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

#include "smooth_int3.cuh"
#include "smooth_int2.cuh"
#include "smooth_w3.cuh"

template <int DIM, int NN, bool BND, typename T>
cudaError_t launch_patches(const sipg_handle* h, int level, int colour, const T* b, T* x, const PatchGrid& g,
                           cudaStream_t s) {
  if constexpr (DIM == 2 && sizeof(T) == 4) {
    if (g.n_int < (1LL << 31) && (reinterpret_cast<uintptr_t>(b) % 16) == 0 &&
        (reinterpret_cast<uintptr_t>(x) % 16) == 0)
      return launch_int2<NN, T, BND>(h, level, colour, b, x, g, s);
  }
  if constexpr (DIM == 3 && sizeof(T) == 4 && !BND) {
    if (h->tf32) {
      const cudaError_t e = launch_tc3(h, level, colour, reinterpret_cast<const float*>(b),
                                       reinterpret_cast<float*>(x), s);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  if constexpr (DIM == 3 && sizeof(T) == 4) {
    if (use_int3<DIM, T>(g, b, x)) {
      if constexpr (!BND)
        switch (h->tuned_tile(1, level)) {
          case 1: return launch_int3<NN, T, BND, 1>(h, level, colour, b, x, g, s);
          case 2: return launch_int3<NN, T, BND, 2>(h, level, colour, b, x, g, s);
          case 3: return launch_int3<NN, T, BND, 3>(h, level, colour, b, x, g, s);
          case 4: return launch_int3<NN, T, BND, 4>(h, level, colour, b, x, g, s);
          default: break;
        }
      return launch_int3<NN, T, BND, 0>(h, level, colour, b, x, g, s);
    }
  }
  return launch_part<DIM, NN, BND, T>(h, level, colour, b, x, g, s);
}

template <typename T, int DIM, int NN>
cudaError_t smooth_dispatch2(const sipg_handle* h, int level, int colour, const T* b, T* x, cudaStream_t s) {
  const PatchGrid g = make_grid(DIM, h->lv[level].N, colour);
  if (g.n_int + g.n_bnd <= 0) return cudaSuccess;  // no patch of this colour (N = 2)
  cudaError_t e;
  if (g.n_int > 0 && g.n_bnd > 0 && h->side) {
    // the boundary-patch kernel runs beside the interior one (patches of one
    // colour write disjoint nodes and read none that another one writes);
    // the boundary kernel is launched first and at the device's greatest
    // priority, so the block scheduler hands out its few long CTAs (rows
    // padded to 2n) first and the many short interior CTAs make the tail of
    // the pass (measured at Q3 64^3: 501 us per FP32 step against 514 us with
    // the interior kernel first)
    if ((e = cudaEventRecord(h->ev_fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->side, h->ev_fork, 0)) != cudaSuccess) return e;
    if (h->bnd_first) {
      if ((e = launch_patches<DIM, NN, true, T>(h, level, colour, b, x, g, h->side)) != cudaSuccess) return e;
      if ((e = launch_patches<DIM, NN, false, T>(h, level, colour, b, x, g, s)) != cudaSuccess) return e;
    } else {
      if ((e = launch_patches<DIM, NN, false, T>(h, level, colour, b, x, g, s)) != cudaSuccess) return e;
      if ((e = launch_patches<DIM, NN, true, T>(h, level, colour, b, x, g, h->side)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(h->ev_join, h->side)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(s, h->ev_join, 0);
  }
  e = launch_patches<DIM, NN, false, T>(h, level, colour, b, x, g, s);
  if (e != cudaSuccess) return e;
  return launch_patches<DIM, NN, true, T>(h, level, colour, b, x, g, s);
}

template <int DIM, int NN, typename T>
struct StepCfg {
  using CI = SC<DIM, NN, false, T, true>;
  using CB = SC<DIM, NN, true, T, true>;
  // one patch per CTA: small levels then spread over every SM (an SM's FP64
  // pipe, and its latency chain, serve one patch instead of a pack)
  static constexpr int PPC_I = 1;
  static constexpr int THREADS = CI::TPP > CB::TPP ? CI::TPP : CB::TPP;
  static constexpr int PPC_B = 1;
  static constexpr int PRE_I = smooth_prefix_bytes<DIM, NN, false, T>();
  static constexpr int PRE_B = smooth_prefix_bytes<DIM, NN, true, T>();
  static constexpr size_t SLOTS_I = (size_t)PPC_I * CI::PER_PATCH * sizeof(T);
  static constexpr size_t SLOTS_B = (size_t)PPC_B * CB::PER_PATCH * sizeof(T);
  static constexpr size_t SMEM = PRE_I + PRE_B + (SLOTS_I > SLOTS_B ? SLOTS_I : SLOTS_B);
};

template <int DIM, int NN, typename T>
__global__ void __launch_bounds__(StepCfg<DIM, NN, T>::THREADS)
    smooth_step_kernel(const __grid_constant__ SmoothOps<SC<DIM, NN, false, T>::PO, SC<DIM, NN, false, T>::P, T, 1> opsi,
                       const __grid_constant__ SmoothOps<SC<DIM, NN, true, T>::PO, SC<DIM, NN, true, T>::P, T, 4> opsb,
                       int reverse, const T* __restrict__ b, T* x, int N, int consistent, long long ndofs, int nrhs,
                       StepGrids grids, unsigned int* bar, int* status) {
  using Cfg = StepCfg<DIM, NN, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* pre_i = smem_raw;
  unsigned char* pre_b = smem_raw + Cfg::PRE_I;
  T* base = reinterpret_cast<T*>(smem_raw + Cfg::PRE_I + Cfg::PRE_B);
  smooth_prefix_setup<DIM, NN, false, T>(opsi, pre_i);
  smooth_prefix_setup<DIM, NN, true, T>(opsb, pre_b);
  __syncthreads();
  constexpr int nc = 1 << DIM;
  for (int ci = 0; ci < nc; ++ci) {
    const int c = reverse ? nc - 1 - ci : ci;
    const PatchGrid& g = grids.g[c];
    // interior and boundary chunks form one index range, so that with enough
    // CTAs every CTA handles a single patch per colour
    const long long chi = (g.n_int + Cfg::PPC_I - 1) / Cfg::PPC_I;
    const long long chb = (g.n_bnd + Cfg::PPC_B - 1) / Cfg::PPC_B;
    for (long long q = blockIdx.x; q < (chi + chb) * nrhs; q += gridDim.x) {
      const long long r = q / (chi + chb), ch = q % (chi + chb);
      if (ch < chi)
        smooth_chunk<DIM, NN, false, T, Cfg::PPC_I, true>(opsi, pre_i, base, ch * Cfg::PPC_I, c, b + r * ndofs,
                                                          x + r * ndofs, N, consistent, g);
      else
        smooth_chunk<DIM, NN, true, T, Cfg::PPC_B, true>(opsb, pre_b, base, (ch - chi) * Cfg::PPC_B, c,
                                                         b + r * ndofs, x + r * ndofs, N, consistent, g);
      __syncthreads();  // the next chunk reuses (and re-lays out) the slots
    }
    if (ci + 1 < nc && !grid_barrier(bar, status, gridDim.x)) return;
  }
}

// Self test of the bounded wait: a barrier expecting `extra` more CTAs than
// were launched can never open, so every CTA must give up and set *status.
__global__ void barrier_selftest_kernel(unsigned int* bar, int* status, int extra) {
  grid_barrier(bar, status, gridDim.x + (unsigned int)extra);
}

PatchGrid make_grid(int dim, int N, int colour) {
  PatchGrid g;
  long long tot = 1, inner = 1;
  for (int e = 0; e < 3; ++e) {
    if (e < dim) {
      const int par = (colour >> e) & 1;
      g.cnt[e] = par ? N / 2 : N / 2 - 1;
      g.lo[e] = par ? 1 : 0;
      g.hi[e] = N / 2 - 1;
      if (g.hi[e] < g.lo[e]) g.hi[e] = g.lo[e];
    } else {
      g.cnt[e] = 1;
      g.lo[e] = 0;
      g.hi[e] = 1;
    }
    tot *= g.cnt[e] > 0 ? g.cnt[e] : 0;
    inner *= (g.hi[e] - g.lo[e]);
    // multiplier ceil(2^(31 + l) / w) with 2^l >= w > 2^(l-1): exact for
    // every dividend below 2^31 and below 2^32 itself
    const long long w = g.hi[e] - g.lo[e];
    int l = 0;
    while ((1LL << l) < w) ++l;
    g.dmul[e] = w > 1 ? (unsigned int)(((1ULL << (31 + l)) + (unsigned long long)w - 1) / (unsigned long long)w) : 0u;
    g.dshift[e] = w > 1 ? l - 1 : 0;
  }
  if (tot <= 0) {
    g.n_int = g.n_bnd = 0;
  } else {
    g.n_int = inner;
    g.n_bnd = tot - inner;
  }
  return g;
}

// Returns cudaErrorNotSupported when the fused path does not apply (the caller
// then launches the colours one by one).
template <typename T, int DIM, int NN>
cudaError_t step_dispatch2(const sipg_handle* h, int level, int reverse, const T* b, T* x, cudaStream_t s) {
  if constexpr (DIM == 3) {
    // the smallest levels (at most 64 patches per colour): one patch per
    // CTA, every stage spread over the CTA (latency, not throughput, bounds a
    // colour pass there); measured on GB300, Q3: 60 / 59 us per FP32 step at
    // N = 8 / 4 against 69 / 65 for the line kernels, 178 against 328 in FP64.
    // At N = 16 (512 patches per colour) the line kernels stay ahead.
    const int N = h->lv[level].N;
    if (N <= 8) return stepw3_dispatch<NN, T>(h, level, reverse, b, x, s);
  }
  using Cfg = StepCfg<DIM, NN, T>;
  if (Cfg::SMEM > 227 * 1024 || h->num_sms <= 0) return cudaErrorNotSupported;
  int max_active = 0;
  cudaError_t e0 = smem_opt_in_occupancy(reinterpret_cast<const void*>(smooth_step_kernel<DIM, NN, T>),
                                         Cfg::THREADS, (int)Cfg::SMEM, &max_active);
  if (e0 != cudaSuccess) return e0;
  if (max_active <= 0) return cudaErrorNotSupported;
  const int N = h->lv[level].N;
  StepGrids sg;
  long long most = 0;
  for (int c = 0; c < (1 << DIM); ++c) {
    sg.g[c] = make_grid(DIM, N, c);
    long long ch = (sg.g[c].n_int + Cfg::PPC_I - 1) / Cfg::PPC_I;
    long long cb = (sg.g[c].n_bnd + Cfg::PPC_B - 1) / Cfg::PPC_B;
    most = std::max(most, (ch + cb) * (long long)h->prm.nrhs);
  }
  const long long resident = (long long)max_active * h->num_sms;
  if (most > resident) return cudaErrorNotSupported;  // several waves: per-colour launches
  SmoothOps<SC<DIM, NN, false, T>::PO, SC<DIM, NN, false, T>::P, T, 1> opsi;
  SmoothOps<SC<DIM, NN, true, T>::PO, SC<DIM, NN, true, T>::P, T, 4> opsb;
  make_ops<SC<DIM, NN, false, T>::PO, SC<DIM, NN, false, T>::P, false, T>(h->hcst<T>(level), 0, opsi.t[0]);
  for (int t = 0; t < 4; ++t)
    make_ops<SC<DIM, NN, true, T>::PO, SC<DIM, NN, true, T>::P, true, T>(h->hcst<T>(level), t, opsb.t[t]);
  const unsigned grid = (unsigned)std::max<long long>(1, most);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(Cfg::THREADS);
  cfg.dynamicSmemBytes = Cfg::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  unsigned int* bar = reinterpret_cast<unsigned int*>(h->ws + h->off_sync);
  int* status = reinterpret_cast<int*>(h->ws + h->off_sync + 2 * sizeof(unsigned int));
  return cudaLaunchKernelEx(&cfg, smooth_step_kernel<DIM, NN, T>, opsi, opsb, reverse, b, x, N,
                            h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0, (long long)h->lv[level].ndofs,
                            h->prm.nrhs, sg, bar, status);
}

}  // namespace

// One colour pass / one fused smoothing step for a compile-time (d, T, n);
// explicitly instantiated in the smooth_i_*.cu translation units.
template <int DIM, typename T, int NN>
cudaError_t smooth_colour_n(const sipg_handle* h, int level, int colour, const T* b, T* x, cudaStream_t s) {
  return smooth_dispatch2<T, DIM, NN>(h, level, colour, b, x, s);
}
template <int DIM, typename T, int NN>
cudaError_t smooth_step_n(const sipg_handle* h, int level, int reverse, const T* b, T* x, cudaStream_t s) {
  return step_dispatch2<T, DIM, NN>(h, level, reverse, b, x, s);
}
// One fused clamped-kernel colour pass (3D FP32): cudaErrorNotSupported where
// the register-direct kernel does not apply (alignment, patch count).
template <int NN>
cudaError_t clamped_colour3_n(const sipg_handle* h, int level, int colour, const float* b, float* x,
                              cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(b) % 16) != 0 || (reinterpret_cast<uintptr_t>(x) % 16) != 0)
    return cudaErrorNotSupported;
  return launch_int3_clamped<NN, float>(h, level, colour, b, x, s);
}
#define SIPG_CLAMPED_INST(NN)                                                                                 \
  template cudaError_t clamped_colour3_n<NN>(const sipg_handle*, int, int, const float*, float*, cudaStream_t);

// The full kernel's patch solves of one colour (3D FP32) from the level's
// residual r (the caller computes it).
template <int NN>
cudaError_t full3_colour_n(const sipg_handle* h, int level, int colour, const float* r, float* x, cudaStream_t s) {
  return launch_full3<NN>(h, level, colour, r, x, s);
}
#define SIPG_FULL3_INST(NN)                                                                                   \
  template cudaError_t full3_colour_n<NN>(const sipg_handle*, int, int, const float*, float*, cudaStream_t);

#define SIPG_SMOOTH_INST(DIM, T, NN)                                                                         \
  template cudaError_t smooth_colour_n<DIM, T, NN>(const sipg_handle*, int, int, const T*, T*, cudaStream_t); \
  template cudaError_t smooth_step_n<DIM, T, NN>(const sipg_handle*, int, int, const T*, T*, cudaStream_t);
