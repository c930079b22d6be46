// 3D interior colour pass (Algorithm 1) whose fast-diagonalisation local
// solve (Eq. inverse3d, u = (S_z x S_y x S_x) Lambda^{-1} (S_z x S_y x S_x)^T
// r) runs on the fifth-generation tensor cores: TF32 operands in shared
// memory, FP32 accumulation in tensor memory (tcgen05.mma, one elected
// thread per CTA, completion through an mbarrier).  The local residual r on
// V_j is computed first by the same sum-factorised FP32 sweeps as the
// register-direct kernel (x, y, z sweeps of the 1D patch mass and SIPG rows,
// face-node halos of the consistent residual), then the six p x p
// eigenvector sweeps are six small GEMMs:
//     out[line][n] = sum_k in[line][k] Bmat[k][n],
// with the lines of one patch as rows (p^2 of them, padded to a 16 x 16
// grid: 256 rows = two M = 128 tiles), K = N = 16 (p <= 14 padded by
// zeros), Bmat = S or S^T (rounded to TF32 once per CTA).  Between two
// sweeps the 16 outputs of a row are written back as the next sweep's
// operand: the new index becomes a row index and the old row index the
// contraction index.  Row <-> line map: thread t reads tensor-memory lane t
// (tile t / 128), and owns the line (a, b) = phi(t) with
//     a = (t % 8) + 8 ((t / 32) % 2),   b = (t % 32) / 8 + 4 (t / 64),
// so that a warp covers 8 values of a and 4 of b; with the operand strides
// below every scattered store of a warp hits 32 distinct banks.
//
// One patch per CTA iteration, 256 threads, a persistent loop over the
// colour's patches; every mbarrier wait is bounded (a wait that runs out
// sets the status word, the CTA leaves the loop, frees its tensor memory
// and returns).  TF32 rounding (unit 2^-11) of the local solve's operands
// is the only difference from the FP32 kernel; the outer FP64 Krylov
// iteration absorbs it (Sec. 5.2's mixed-precision argument).
#include "smoother_impl.cuh"
#include "tcgen05.cuh"

namespace {

template <int NN>
struct TC3 {
  static constexpr int P = 2 * NN, PO = 2 * NN - 2, OFF = 1, ND = NN * NN * NN;
  static constexpr int NT = 256;  // threads: one per operand row
  static_assert(PO <= 16, "patch rows must fit the 16-wide operand tiles");
  // residual-sweep tiles (floats), laid out as in the register-direct kernel
  static constexpr int SA1 = i3_pad32(P * PO, 16);
  static constexpr int SC = i3_pad32(PO * PO, PO);
  static constexpr int CZS = i3_pad32(PO * PO, 16);
  // operand A: 256 rows x 16 (TF32), K-major; core-matrix strides in bytes
  // along K and between 8-row groups (16 x 292 and 16 x 9: odd multiples
  // that spread a warp's scattered stores over all banks)
  static constexpr int AK = 4672, AR = 144;
  static constexpr int ABYTES = 3 * AK + 32 * AR;
  // operand B: 16 x 16, K-major, dense core matrices
  static constexpr int BK = 128, BR = 512, BBYTES = 2048;
  // shared memory (bytes): [RA / operand A][RB][B_st][B_s][mbar, tmem slot]
  static constexpr int RA_BYTES = i3_max((2 * P + 4) * SA1 * 4, ABYTES);
  static constexpr int RB_BYTES = (2 * P * SC + 2 * CZS) * 4;
  static constexpr int OFF_RB = (RA_BYTES + 127) / 128 * 128;
  static constexpr int OFF_BST = (OFF_RB + RB_BYTES + 127) / 128 * 128;
  static constexpr int OFF_BS = OFF_BST + BBYTES;
  static constexpr int OFF_MISC = OFF_BS + BBYTES;
  static constexpr int SMEM = OFF_MISC + 128;
};

__device__ __forceinline__ int phi_a(int t) { return (t & 7) + 8 * ((t >> 5) & 1); }
__device__ __forceinline__ int phi_b(int t) { return ((t & 31) >> 3) + 4 * (t >> 6); }
__device__ __forceinline__ int phi_row(int a, int b) { return 32 * (2 * (b >> 2) + (a >> 3)) + (a & 7) + 8 * (b & 3); }

// byte offset of element (row, k) of operand A
template <int NN>
__device__ __forceinline__ int a_off(int row, int k) {
  return (k & 3) * 4 + (row & 7) * 16 + (k >> 2) * TC3<NN>::AK + (row >> 3) * TC3<NN>::AR;
}

// B operands: Bst(n, k) = S[k][n] (sweeps by S^T), Bs(n, k) = S[n][k] (by S);
// zero outside p x p.  S[j][i] = op.S[j * PO + i] (column i = eigenvector i).
template <int PO>
__device__ void tc3_fill_b(const float* S, unsigned char* bst, unsigned char* bs) {
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int n = e >> 4, k = e & 15;
    const int off = (k & 3) * 4 + (n & 7) * 16 + (k >> 2) * 128 + (n >> 3) * 512;
    const bool in = n < PO && k < PO;
    *reinterpret_cast<float*>(bst + off) = in ? tc::to_tf32(S[k * PO + n]) : 0.f;
    *reinterpret_cast<float*>(bs + off) = in ? tc::to_tf32(S[n * PO + k]) : 0.f;
  }
}

// Issue D[tile] = A[tile] x B for both 128-row tiles (K = 16: two MMAs
// each) and commit to the mbarrier; called by one thread.
template <int NN>
__device__ __forceinline__ void tc3_issue(uint32_t tmem, uint32_t a_s, uint32_t b_s, uint64_t* mbar) {
  using C = TC3<NN>;
  constexpr uint32_t idesc = tc::idesc_tf32(128, 16);
  tc::fence_after_sync();
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
      tc::mma_tf32(tmem + 16 * t, tc::smem_desc(a_s + 16 * t * C::AR + 2 * ks * C::AK, C::AK, C::AR),
                   tc::smem_desc(b_s + 2 * ks * C::BK, C::BK, C::BR), idesc, ks > 0);
  tc::mma_commit(mbar);
}

// Everything this thread wrote to operand A is visible to the tensor core,
// every tensor-memory load of the previous sweep has completed, then one
// thread issues the sweep; all wait for its completion (bounded) and read
// their row.  Returns false when the wait ran out.
template <int NN>
__device__ __forceinline__ bool tc3_sweep(uint32_t tmem, uint32_t a_s, uint32_t b_s, uint64_t* mbar,
                                          uint32_t& parity, float (&v)[16]) {
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) tc3_issue<NN>(tmem, a_s, b_s, mbar);
  bool ok = tc::mbar_wait(mbar, parity);
  if (!ok) tc::mbar_wait(mbar, parity);  // a late completion still lands before we leave
  ok = __syncthreads_and(ok) != 0;      // one decision for the whole CTA
  parity ^= 1u;
  tc::fence_after_sync();
  if (!ok) return false;
  const int w = threadIdx.x >> 5;
  tc::tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + 16 * (w >> 2), v);
  return true;
}

// Scattered store of the 16 outputs of line (a, b): value j goes to row
// phi_row(a, j) (SLOW = true: j is the new slow index) or phi_row(j, b), at
// contraction index k; zeros for padded lines and for j >= PO.
template <int NN, bool SLOW>
__device__ __forceinline__ void tc3_scatter(unsigned char* A, const float (&v)[16], int a, int b, int k,
                                            bool valid) {
  constexpr int PO = TC3<NN>::PO;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int row = SLOW ? phi_row(a, j) : phi_row(j, b);
    *reinterpret_cast<float*>(A + a_off<NN>(row, k)) = (valid && j < PO) ? tc::to_tf32(v[j]) : 0.f;
  }
}

// own row: 16 values at contraction indices 0..15 (four 16-byte stores)
template <int NN>
__device__ __forceinline__ void tc3_store_row(unsigned char* A, int row, const float (&v)[16], bool valid) {
  constexpr int PO = TC3<NN>::PO;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    float4 w;
    w.x = (valid && 4 * g + 0 < PO) ? tc::to_tf32(v[4 * g + 0]) : 0.f;
    w.y = (valid && 4 * g + 1 < PO) ? tc::to_tf32(v[4 * g + 1]) : 0.f;
    w.z = (valid && 4 * g + 2 < PO) ? tc::to_tf32(v[4 * g + 2]) : 0.f;
    w.w = (valid && 4 * g + 3 < PO) ? tc::to_tf32(v[4 * g + 3]) : 0.f;
    *reinterpret_cast<float4*>(A + a_off<NN>(row, 4 * g)) = w;
  }
}

template <int NN>
__global__ void __launch_bounds__(256, 3)
    smooth_tc3_kernel(const __grid_constant__ SmoothOps<2 * NN - 2, 2 * NN, float, 1> ops, int colour,
                      const float* __restrict__ bvec, float* xvec, int N, int consistent, long long ndofs,
                      PatchGrid grid, int* status) {
  using C = TC3<NN>;
  using Ops = Ops1D<C::PO, C::P, float>;
  constexpr int P = C::P, PO = C::PO, OFF = C::OFF, ND = C::ND, NT = C::NT;
  constexpr int SA1 = C::SA1, SC = C::SC, CZS = C::CZS;
  constexpr int VW = run_vw<NN, float>();
  extern __shared__ __align__(1024) unsigned char sm[];
  float* RA = reinterpret_cast<float*>(sm);
  unsigned char* Aop = sm;  // operand A, aliased on RA once the y sweep has read it
  float* RB = reinterpret_cast<float*>(sm + C::OFF_RB);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + C::OFF_MISC);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + C::OFF_MISC + 8);
  const Ops& op = ops.t[0];
  const int tid = threadIdx.x;

  // ---- per-CTA set-up: B operands, mbarrier, tensor memory (32 columns:
  // two 128 x 16 FP32 tiles)
  tc3_fill_b<PO>(op.S, sm + C::OFF_BST, sm + C::OFF_BS);
  if (tid == 0) tc::mbar_init(mbar, 1);
  if (tid < 32) tc::tmem_alloc(tslot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t a_s = tc::smem_u32(Aop);
  const uint32_t bst_s = tc::smem_u32(sm + C::OFF_BST), bs_s = tc::smem_u32(sm + C::OFF_BS);
  uint32_t parity = 0;

  const float* b = bvec + (long long)blockIdx.y * ndofs;
  float* x = xvec + (long long)blockIdx.y * ndofs;
  const int a = phi_a(tid), bb = phi_b(tid);
  const bool own = a < PO && bb < PO;  // this thread's line is a real patch line

  for (long long pidx = blockIdx.x; pidx < grid.n_int; pidx += gridDim.x) {
    int v[3];
    {
      int q = (int)pidx;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int w = grid.hi[e] - grid.lo[e];
        const int qn = div_width(q, grid.dmul[e], grid.dshift[e]);
        const int m = grid.lo[e] + (q - qn * w);
        q = qn;
        v[e] = ((colour >> e) & 1) ? 2 * m + 1 : 2 * m + 2;
      }
    }
    const float* xb = x + ((long long)(v[0] - 1) + (long long)N * ((v[1] - 1) + (long long)N * (v[2] - 1))) * ND;
    const int cs1 = N * ND, cs2 = N * N * ND;

    // ---------------------------------------------------------- x sweep
    // lines t < P^2: (a1, a2) = (t / P, t % P); then 4P halo lines (slot, j):
    // slot 0/1 = y faces below/above (j = a2), 2/3 = z faces (j = a1).  All
    // of a thread's loads are issued before any line is contracted.
    {
      constexpr int L1 = P * P + 4 * P;
      constexpr int R1 = (L1 + NT - 1) / NT;
      float vin[R1][P], hl[R1][2];
#pragma unroll
      for (int q = 0; q < R1; ++q) {
        const int t = tid + q * NT;
        int off = 0;
        const bool act = t < L1, main = t < P * P;
        bool ld = main;
        if (main) {
          const int a2 = t % P, a1 = t / P;
          off = (a1 / NN) * cs1 + (a2 / NN) * cs2 + (a1 % NN) * NN + (a2 % NN) * NN * NN;
        } else if (act) {
          const int hh = t - P * P, slot = hh / P, j = hh % P;
          if (slot < 2) {
            off = (slot ? 2 : -1) * cs1 + (slot ? 0 : (NN - 1) * NN) + (j / NN) * cs2 + (j % NN) * NN * NN;
          } else {
            off = (slot == 3 ? 2 : -1) * cs2 + (slot == 3 ? 0 : (NN - 1) * NN * NN) + (j / NN) * cs1 + (j % NN) * NN;
          }
          ld = consistent != 0;
        }
        if (ld) {
          i3_ldrun<NN, VW, float, true>(xb + off, &vin[q][0]);
          i3_ldrun<NN, VW, float, true>(xb + off + ND, &vin[q][NN]);
        } else {
#pragma unroll
          for (int c = 0; c < P; ++c) vin[q][c] = 0.f;
        }
        hl[q][0] = (main && consistent) ? __ldg(xb + off - ND + (NN - 1)) : 0.f;
        hl[q][1] = (main && consistent) ? __ldg(xb + off + 2 * ND) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < R1; ++q) {
        const int t = tid + q * NT;
        if (t >= L1) continue;
        const bool main = t < P * P;
        const int dst = main ? SA1 * (t / P) + PO * (t % P) : (2 * P + (t - P * P) / P) * SA1 + PO * ((t - P * P) % P);
        float oa[PO];
        mass_rows2<PO, P, NN, OFF, false>(op, vin[q], oa);
        i3_st_pairs<PO>(RA + dst, oa);
        if (main) {
          float ob[PO];
          sipg_rows2<PO, P, NN, OFF>(op, vin[q], hl[q][0], hl[q][1], ob);
          i3_st_pairs<PO>(RA + P * SA1 + dst, ob);
        }
      }
    }
    __syncthreads();

    // ---------------------------------------------------------- y sweep
    float* Cc = RB;
    float* Dd = RB + P * SC;
    float* CZ = RB + 2 * P * SC;
    {
      constexpr int L2 = PO * P + 2 * PO;
      constexpr int R2 = (L2 + NT - 1) / NT;
#pragma unroll
      for (int q = 0; q < R2; ++q) {
        const int t = tid + q * NT;
        if (t >= L2) continue;
        if (t < PO * P) {
          const int r0 = t % PO, a2 = t / PO;
          float va[P], vb[P], oc[PO], od[PO];
#pragma unroll
          for (int a1 = 0; a1 < P; ++a1) {
            va[a1] = RA[SA1 * a1 + t];
            vb[a1] = RA[P * SA1 + SA1 * a1 + t];
          }
          const float hy0 = RA[2 * P * SA1 + t], hy1 = RA[(2 * P + 1) * SA1 + t];
          mass_rows2<PO, P, NN, OFF, false>(op, va, oc);
          sipg_rows2<PO, P, NN, OFF>(op, va, hy0, hy1, od);
          mass_rows2<PO, P, NN, OFF, true>(op, vb, od);
#pragma unroll
          for (int r1 = 0; r1 < PO; ++r1) {
            Cc[SC * a2 + PO * r1 + r0] = oc[r1];
            Dd[SC * a2 + PO * r1 + r0] = od[r1];
          }
        } else {
          const int hh = t - PO * P, r0 = hh % PO, side = hh / PO;
          float vz[P], oc[PO];
#pragma unroll
          for (int a1 = 0; a1 < P; ++a1) vz[a1] = RA[(2 * P + 2 + side) * SA1 + PO * a1 + r0];
          mass_rows2<PO, P, NN, OFF, false>(op, vz, oc);
#pragma unroll
          for (int r1 = 0; r1 < PO; ++r1) CZ[side * CZS + PO * r1 + r0] = oc[r1];
        }
      }
    }
    __syncthreads();

    // ------------------------------------------ z sweep: residual line (a, bb)
    // = (r0, r1) into operand row tid (= phi_row(a, bb)), contraction index r2
    const int goff = ((a + OFF) / NN) * ND + ((bb + OFF) / NN) * cs1 + ((a + OFF) % NN) + ((bb + OFF) % NN) * NN;
    {
      float res[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) res[j] = 0.f;
      if (own) {
        const int zl = a + PO * bb;
        const float* gb = b + (xb - x) + goff;
        float bv[PO], vc[P], vd[P], o[PO];
#pragma unroll
        for (int r2 = 0; r2 < PO; ++r2) bv[r2] = __ldg(gb + ((r2 + OFF) / NN) * cs2 + ((r2 + OFF) % NN) * NN * NN);
#pragma unroll
        for (int a2 = 0; a2 < P; ++a2) {
          vc[a2] = Cc[SC * a2 + zl];
          vd[a2] = Dd[SC * a2 + zl];
        }
        sipg_rows2<PO, P, NN, OFF>(op, vc, CZ[zl], CZ[CZS + zl], o);
        mass_rows2<PO, P, NN, OFF, true>(op, vd, o);
#pragma unroll
        for (int r2 = 0; r2 < PO; ++r2) res[r2] = bv[r2] - o[r2];
      }
      tc3_store_row<NN>(Aop, tid, res, own);
    }

    // -------------------------------- fast diagonalisation on the tensor cores
    // x on the line's V_j rows, read now so that the loads overlap the
    // tensor-core sweeps
    float* gx = x + (xb - x) + goff;
    float xo[PO];
#pragma unroll
    for (int r2 = 0; r2 < PO; ++r2) xo[r2] = own ? gx[((r2 + OFF) / NN) * cs2 + ((r2 + OFF) % NN) * NN * NN] : 0.f;
    // (each sweep's MMA has completed before its outputs are read, so the
    // operand can be rewritten at once; ok is the same in every thread)
    float w[16];
    bool ok = tc3_sweep<NN>(tmem, a_s, bst_s, mbar, parity, w);  // S_z^T: line (r0, r1) -> k2
    if (ok) {
      tc3_scatter<NN, true>(Aop, w, a, bb, bb, own);  // row (r0, k2), index r1
      ok = tc3_sweep<NN>(tmem, a_s, bst_s, mbar, parity, w);  // S_y^T: (r0, k2) -> k1
    }
    if (ok) {
      tc3_scatter<NN, false>(Aop, w, a, bb, a, own);  // row (k1, k2), index r0
      ok = tc3_sweep<NN>(tmem, a_s, bst_s, mbar, parity, w);  // S_x^T: (k1, k2) -> k0
    }
    if (ok) {
      // Lambda^{-1}: line (k1, k2) = (a, bb), k0 = j
      // (approximate reciprocal, 2 ulp: far below the TF32 rounding of the
      // operands this scaling feeds)
      const float lyz = own ? op.lam[a] + op.lam[bb] : 1.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) w[j] = (own && j < PO) ? __fdividef(w[j], op.lam[j < PO ? j : 0] + lyz) : 0.f;
      tc3_store_row<NN>(Aop, tid, w, own);  // row (k1, k2), index k0
      ok = tc3_sweep<NN>(tmem, a_s, bs_s, mbar, parity, w);  // S_x: (k1, k2) -> r0
    }
    if (ok) {
      tc3_scatter<NN, false>(Aop, w, a, bb, a, own);  // row (r0, k2), index k1
      ok = tc3_sweep<NN>(tmem, a_s, bs_s, mbar, parity, w);  // S_y: (r0, k2) -> r1
    }
    if (ok) {
      tc3_scatter<NN, true>(Aop, w, a, bb, bb, own);  // row (r0, r1), index k2
      ok = tc3_sweep<NN>(tmem, a_s, bs_s, mbar, parity, w);  // S_z: (r0, r1) -> r2
    }
    if (!ok) {
      if (tid == 0) atomicExch(status, 2);
      break;
    }
    // x[V_j] += u on line (r0, r1)
    if (own) {
#pragma unroll
      for (int r2 = 0; r2 < PO; ++r2) gx[((r2 + OFF) / NN) * cs2 + ((r2 + OFF) % NN) * NN * NN] = xo[r2] + w[r2];
    }
    __syncthreads();  // RA / operand A and RB are rewritten by the next patch
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_free(tmem, 32);
}

// One CTA: D = A x B^T for A 256 x 16 and B 16 x 16 (row-major FP32 in
// global memory, rounded to TF32), through the same operand layouts, MMA
// issue, mbarrier completion and tensor-memory loads as the colour pass.
// The operand region sits at the start of a 96 KB shared allocation.
__global__ void __launch_bounds__(256, 1)
    tc_selftest_kernel(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ D,
                       int* status) {
  using C = TC3<8>;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Aop = sm;
  unsigned char* Bop = sm + 65536;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 65536 + 4096);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 65536 + 4096 + 8);
  const int tid = threadIdx.x;
  for (int e = tid; e < 256; e += 256) {
    const int n = e >> 4, k = e & 15;
    *reinterpret_cast<float*>(Bop + (k & 3) * 4 + (n & 7) * 16 + (k >> 2) * 128 + (n >> 3) * 512) =
        tc::to_tf32(B[n * 16 + k]);
  }
  for (int e = tid; e < 256 * 16; e += 256) {
    const int m = e >> 4, k = e & 15;
    *reinterpret_cast<float*>(Aop + a_off<8>(m, k)) = tc::to_tf32(A[m * 16 + k]);
  }
  if (tid == 0) tc::mbar_init(mbar, 1);
  if (tid < 32) tc::tmem_alloc(tslot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  uint32_t parity = 0;
  float v[16];
  const bool ok = tc3_sweep<8>(tmem, tc::smem_u32(Aop), tc::smem_u32(Bop), mbar, parity, v);
  if (ok) {
#pragma unroll
    for (int j = 0; j < 16; ++j) D[tid * 16 + j] = v[j];
  } else if (tid == 0) {
    atomicExch(status, 2);
  }
  // the operand region holds either reading of the two descriptor strides:
  // up to 2 * AK + AR * 16 + AK * 15 + AR + 128 bytes from its start
  static_assert(2 * C::AK + 16 * C::AR + 15 * C::AK + C::AR + 128 <= 96 * 1024, "operand region");
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_free(tmem, 32);
}

template <int NN>
cudaError_t launch_tc3_impl(const sipg_handle* h, int level, int colour, const float* b, float* x,
                            const PatchGrid& g, cudaStream_t s) {
  using C = TC3<NN>;
  if (g.n_int <= 0) return cudaSuccess;
  cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(smooth_tc3_kernel<NN>), C::SMEM);
  if (e != cudaSuccess) return e;
  if (h->num_sms <= 0) return cudaErrorNotSupported;
  SmoothOps<C::PO, C::P, float, 1> ops;
  make_ops<C::PO, C::P, false, float>(h->hcst<float>(level), 0, ops.t[0]);
  // A non-cooperative persistent loop: up to six CTAs per SM (three are
  // resident at a time by shared memory and registers; the others start as
  // slots free up), each taking every gridDim.x-th patch.  (The occupancy
  // query is not used here: it reported one CTA per SM for this kernel.)
  const long long cap = (long long)h->num_sms * 6;
  const unsigned gx = (unsigned)(g.n_int < cap ? g.n_int : cap);
  int* status = reinterpret_cast<int*>(h->ws + h->off_sync + 2 * sizeof(unsigned int));
  smooth_tc3_kernel<NN><<<dim3(gx, h->prm.nrhs), C::NT, C::SMEM, s>>>(
      ops, colour, b, x, h->lv[level].N, h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0,
      (long long)h->lv[level].ndofs, g, status);
  return cudaGetLastError();
}

}  // namespace

// Interior patches of one 3D FP32 colour pass with the tensor-core local
// solves; cudaErrorNotSupported where this kernel does not apply (degree,
// alignment, patch count), so the caller falls back to the FP32 kernel.
cudaError_t launch_tc3(const sipg_handle* h, int level, int colour, const float* b, float* x, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(b) % 16) != 0 || (reinterpret_cast<uintptr_t>(x) % 16) != 0)
    return cudaErrorNotSupported;
  const PatchGrid g = make_grid(3, h->lv[level].N, colour);
  if (g.n_int >= (1LL << 31)) return cudaErrorNotSupported;
  // degree 7 only: with p = 2k < 14 the 16-wide operand tiles are mostly
  // padding, and the FP32 kernel is faster (GB300, 32^3 colour 0: k = 5
  // 60.8 against 39.4 us, k = 6 77.5 against 66.8 us; k = 7 97.3 against 109)
  switch (h->n) {
    case 8: return launch_tc3_impl<8>(h, level, colour, b, x, g, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_tc_selftest(const sipg_handle* h, const float* A, const float* B, float* D, cudaStream_t s) {
  const int smem = 96 * 1024;
  cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(tc_selftest_kernel), smem);
  if (e != cudaSuccess) return e;
  int* status = reinterpret_cast<int*>(h->ws + h->off_sync + 2 * sizeof(unsigned int));
  tc_selftest_kernel<<<1, 256, smem, s>>>(A, B, D, status);
  return cudaGetLastError();
}
