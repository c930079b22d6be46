// Interior vertex patches in 3D, register-direct variant of the colour pass
// (Algorithm 1 with the fast-diagonalisation local solve of Eq. inverse3d).
// Included by smoother.cu after its line-contraction helpers.
//
// Same arithmetic as the generic colour pass: the patch residual on V_j by
// three sum-factorised sweeps (x, y, z) of the rows V_j of the 1D patch mass
// and SIPG matrices, then u = (S x S x S) Lambda^{-1} (S x S x S)^T r and
// x[V_j] += u.  What differs is the data movement, designed for the FP32 path
// on GB300 where the generic kernel was bound by shared-memory wavefronts and
// instruction issue rather than by HBM or the FMA pipe:
//   * the x sweep reads its lines straight from global memory into registers
//     (each cell's x-line of n nodes is contiguous: vector loads), including
//     the face-node halos, so the patch tile is never staged in shared memory;
//   * the z sweep keeps its residual line in registers and applies S_z^T in
//     place; the x-direction forward transform, the scaling by the inverse
//     eigenvalue sums and the x-direction backward transform share one line;
//     the last backward transform (z) adds to x straight from registers;
//   * every shared-memory exchange between sweeps uses a layout in which the
//     32 lanes of a warp touch 32 distinct banks (strides chosen modulo 32;
//     the patch stride is congruent to the threads per patch, so warps that
//     straddle two patches stay conflict-free), and the x sweep stores pairs;
//   * TPP = p^2 threads per patch (one line each in the z sweep and in every
//     transform), several patches per CTA, six CTA barriers per colour pass.

constexpr int i3_pad32(int m, int r) {
  int s = m;
  while (((s % 32) + 32) % 32 != ((r % 32) + 32) % 32) ++s;
  return s;
}
constexpr int i3_max(int a, int b) { return a > b ? a : b; }

template <int NN, typename T>
struct I3 {
  static constexpr int P = 2 * NN;       // patch nodes per direction
  static constexpr int PO = 2 * NN - 2;  // V_j rows per direction (interior)
  static constexpr int TPP = PO * PO;
  static constexpr int W = (int)(sizeof(T) / 4);  // 32-bit words per element
  // strides in elements; the bank rules are stated for 4-byte words and hold
  // for 8-byte elements accessed by half-warps
  static constexpr int SA1 = i3_pad32(P * PO, 16);   // A/B/halo rows (per a1 or halo slot)
  static constexpr int SC = i3_pad32(PO * PO, PO);   // C/D planes (per a2)
  static constexpr int CZS = i3_pad32(PO * PO, 16);  // z halo faces after the y sweep
  static constexpr int ST = i3_pad32(PO * PO, PO);   // T1/T4 planes
  static constexpr int SQ = i3_pad32(PO * PO, 1);    // T2/T3 planes
  static constexpr int RA = i3_max((2 * P + 4) * SA1, i3_max(PO * ST, PO * SQ));
  static constexpr int RB = i3_max(2 * P * SC + 2 * CZS, i3_max(PO * SQ, PO * ST));
  static constexpr int PS = i3_pad32(RA + RB, TPP);  // patch stride (elements)
  static constexpr int DINV = PO * PO * PO;
  static constexpr int PREFIX = (DINV * (int)sizeof(T) + 15) / 16 * 16;
  // patches per CTA: fill about 54 KB of shared memory (four CTAs per SM) with
  // at most 512 threads
  static constexpr int ppc() {
    int k = (54 * 1024 - PREFIX) / (PS * (int)sizeof(T));
    if (k > 512 / TPP) k = 512 / TPP;
    return k < 1 ? 1 : k;
  }
  static constexpr int PPC = ppc();
  static constexpr int THREADS = TPP * PPC;
  static constexpr size_t SMEM = (size_t)PREFIX + (size_t)PPC * PS * sizeof(T);
  static constexpr int minblocks() {
    int by_smem = (int)((228 * 1024) / (SMEM + 1024));
    int by_thr = 2048 / THREADS;
    int m = by_smem < by_thr ? by_smem : by_thr;
    return m < 1 ? 1 : (m > 4 ? 4 : m);
  }
  static constexpr int MINB = minblocks();
  // vector width (elements) of a contiguous run of NN nodes: 16-byte loads
  // when the run is 16-byte aligned, else 8-byte, else scalar
  static constexpr int VW = (NN * (int)sizeof(T)) % 16 == 0 ? 16 / (int)sizeof(T)
                            : ((NN * (int)sizeof(T)) % 8 == 0 ? 8 / (int)sizeof(T) : 1);
};

template <typename T, int V>
struct i3_vec;
template <> struct i3_vec<float, 4> { using t = float4; };
template <> struct i3_vec<float, 2> { using t = float2; };
template <> struct i3_vec<float, 1> { using t = float; };
template <> struct i3_vec<double, 2> { using t = double2; };
template <> struct i3_vec<double, 1> { using t = double; };

// v[0..NN) = p[0..NN) through the read-only path (vector loads of width VW)
template <int NN, int VW, typename T>
__device__ __forceinline__ void i3_ldrun(const T* __restrict__ p, T* v) {
  using V = typename i3_vec<T, VW>::t;
  const V* q = reinterpret_cast<const V*>(p);
#pragma unroll
  for (int j = 0; j < NN / VW; ++j) {
    const V w = __ldg(q + j);
    const T* e = reinterpret_cast<const T*>(&w);
#pragma unroll
    for (int c = 0; c < VW; ++c) v[j * VW + c] = e[c];
  }
}

// store PO consecutive values as pairs (PO is even)
template <int PO, typename T>
__device__ __forceinline__ void i3_st_pairs(T* p, const T (&o)[PO]) {
  using V2 = typename i3_vec<T, 2>::t;
#pragma unroll
  for (int r = 0; r < PO; r += 2) {
    V2 w;
    w.x = o[r];
    w.y = o[r + 1];
    *reinterpret_cast<V2*>(p + r) = w;
  }
}

template <int NN, typename T>
__global__ void __launch_bounds__(I3<NN, T>::THREADS, I3<NN, T>::MINB)
    smooth_int3_kernel(const __grid_constant__ SmoothOps<2 * NN - 2, 2 * NN, T, 1> ops, int colour,
                       const T* __restrict__ b, T* x, int N, int consistent, long long ndofs, PatchGrid grid) {
  using C = I3<NN, T>;
  constexpr int P = C::P, PO = C::PO, TPP = C::TPP, PPC = C::PPC, ND = NN * NN * NN;
  constexpr int SA1 = C::SA1, SC = C::SC, CZS = C::CZS, ST = C::ST, SQ = C::SQ;
  const auto& op = ops.t[0];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* dinv = reinterpret_cast<T*>(smem_raw);  // [k0][k2][k1]
  for (int e = threadIdx.x; e < C::DINV; e += blockDim.x) {
    const int k1 = e % PO, k2 = (e / PO) % PO, k0 = e / (PO * PO);
    dinv[e] = T(1) / (op.lam[k0] + op.lam[k1] + op.lam[k2]);
  }
  const int tid = threadIdx.x;
  const int lane = tid % TPP;
  const int pl = tid / TPP;
  T* RA = reinterpret_cast<T*>(smem_raw + C::PREFIX) + (size_t)pl * C::PS;
  T* RB = RA + C::RA;

  const long long col = (long long)blockIdx.y * ndofs;
  b += col;
  x += col;
  const int pidx = blockIdx.x * PPC + pl;
  const bool valid = pidx < (int)grid.n_int;
  int v[3];
  {
    int q = valid ? pidx : 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int w = grid.hi[e] - grid.lo[e];
      const int m = grid.lo[e] + q % w;
      q /= w;
      v[e] = ((colour >> e) & 1) ? 2 * m + 1 : 2 * m + 2;
    }
  }
  // cell (v0-1, v1-1, v2-1), node 0: all patch offsets below are relative to it
  const T* xb = x + ((long long)(v[0] - 1) + (long long)N * ((v[1] - 1) + (long long)N * (v[2] - 1))) * ND;
  const int cs1 = N * ND, cs2 = N * N * ND;  // cell strides in y and z (elements)

  // ------------------------------------------------------------------ x sweep
  // lines t < P^2: (a1, a2) = (t / P, t % P); then 4P halo lines (slot, j):
  // slot 0/1 = y faces below/above (j = a2), 2/3 = z faces (j = a1), M_x only
  constexpr int L1 = P * P + 4 * P;
  constexpr int R1 = (L1 + TPP - 1) / TPP;
  if (valid) {
    T vin[R1][P], hl[R1][2];
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      const int t = lane + q * TPP;
      int off = 0;
      bool act = t < L1, main = t < P * P;
      if (main) {
        const int a2 = t % P, a1 = t / P;
        off = (a1 / NN) * cs1 + (a2 / NN) * cs2 + (a1 % NN) * NN + (a2 % NN) * NN * NN;
      } else if (act) {
        const int h = t - P * P, slot = h / P, j = h % P;
        if (slot < 2) {  // y face: cell row v1-2 (node layer n-1) or v1+1 (layer 0); j = a2
          off = (slot ? 2 : -1) * cs1 + (slot ? 0 : (NN - 1) * NN) + (j / NN) * cs2 + (j % NN) * NN * NN;
        } else {         // z face: cell layer v2-2 or v2+1; j = a1
          off = (slot == 3 ? 2 : -1) * cs2 + (slot == 3 ? 0 : (NN - 1) * NN * NN) + (j / NN) * cs1 + (j % NN) * NN;
        }
      }
      if (act && (main || consistent)) {
        i3_ldrun<NN, C::VW>(xb + off, &vin[q][0]);
        i3_ldrun<NN, C::VW>(xb + off + ND, &vin[q][NN]);
      } else {
#pragma unroll
        for (int c = 0; c < P; ++c) vin[q][c] = T(0);
      }
      // x halos of a main line: node n-1 of cell v0-2, node 0 of cell v0+1
      hl[q][0] = (main && consistent) ? __ldg(xb + off - ND + (NN - 1)) : T(0);
      hl[q][1] = (main && consistent) ? __ldg(xb + off + 2 * ND) : T(0);
    }
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      const int t = lane + q * TPP;
      if (t >= L1) continue;
      // destination row: A/B[a1][a2][.] for main lines, halo[slot][j][.]
      const int dst = t < P * P ? SA1 * (t / P) + PO * (t % P)
                                : (2 * P + (t - P * P) / P) * SA1 + PO * ((t - P * P) % P);
      T oa[PO];
      T(&vq)[P] = vin[q];
      mass_rows<PO, P, NN, 1>(op.Mm, vq, oa);
      i3_st_pairs<PO>(RA + dst, oa);
      if (t < P * P) {
        T ob[PO];
        sipg_rows<PO, P, NN, 1>(op, vq, hl[q][0], hl[q][1], ob);
        i3_st_pairs<PO>(RA + P * SA1 + dst, ob);
      }
    }
  }
  __syncthreads();

  // ------------------------------------------------------------------ y sweep
  // lines t < PO P: (r0, a2) = (t % PO, t / PO):
  //   C = M_y A,  D = L_y [A with the y halos] + M_y B;
  // then 2 PO lines (r0, side): CZ = M_y (z halo face after M_x)
  constexpr int L2 = PO * P + 2 * PO;
  constexpr int R2 = (L2 + TPP - 1) / TPP;
  T* Cc = RB;
  T* Dd = RB + P * SC;
  T* CZ = RB + 2 * P * SC;
  if (valid) {
#pragma unroll
    for (int q = 0; q < R2; ++q) {
      const int t = lane + q * TPP;
      if (t >= L2) continue;
      if (t < PO * P) {
        const int r0 = t % PO, a2 = t / PO;
        T va[P], vb[P], oc[PO], od[PO];
#pragma unroll
        for (int a1 = 0; a1 < P; ++a1) {
          va[a1] = RA[SA1 * a1 + t];
          vb[a1] = RA[P * SA1 + SA1 * a1 + t];
        }
        const T h0 = RA[2 * P * SA1 + t], h1 = RA[(2 * P + 1) * SA1 + t];
        mass_rows<PO, P, NN, 1>(op.Mm, va, oc);
        sipg_rows<PO, P, NN, 1>(op, va, h0, h1, od);
        mass_rows_acc<PO, P, NN, 1>(op.Mm, vb, od);
#pragma unroll
        for (int r1 = 0; r1 < PO; ++r1) {
          Cc[SC * a2 + PO * r1 + r0] = oc[r1];
          Dd[SC * a2 + PO * r1 + r0] = od[r1];
        }
      } else {
        const int h = t - PO * P, r0 = h % PO, side = h / PO;
        T vz[P], oc[PO];
#pragma unroll
        for (int a1 = 0; a1 < P; ++a1) vz[a1] = RA[(2 * P + 2 + side) * SA1 + PO * a1 + r0];
        mass_rows<PO, P, NN, 1>(op.Mm, vz, oc);
#pragma unroll
        for (int r1 = 0; r1 < PO; ++r1) CZ[side * CZS + PO * r1 + r0] = oc[r1];
      }
    }
  }
  __syncthreads();

  // ------------------------------------------------ z sweep, residual, S_z^T
  // line (r0, r1) = (lane % PO, lane / PO); node (r0+1, r1+1, r2+1)
  const int r0 = lane % PO, r1 = lane / PO;
  const int goff = ((r0 + 1) / NN) * ND + ((r1 + 1) / NN) * cs1 + ((r0 + 1) % NN) + ((r1 + 1) % NN) * NN;
  T* gx = const_cast<T*>(xb) + goff;
  const T* gb = b + (xb - x) + goff;
  if (valid) {
    T bv[PO], vc[P], vd[P], o[PO], t1[PO];
#pragma unroll
    for (int r2 = 0; r2 < PO; ++r2)
      bv[r2] = __ldg(gb + ((r2 + 1) / NN) * cs2 + ((r2 + 1) % NN) * NN * NN);
#pragma unroll
    for (int a2 = 0; a2 < P; ++a2) {
      vc[a2] = Cc[SC * a2 + lane];
      vd[a2] = Dd[SC * a2 + lane];
    }
    sipg_rows<PO, P, NN, 1>(op, vc, CZ[lane], CZ[CZS + lane], o);
    mass_rows_acc<PO, P, NN, 1>(op.Mm, vd, o);
#pragma unroll
    for (int r2 = 0; r2 < PO; ++r2) o[r2] = bv[r2] - o[r2];
    st_rows<PO>(op.S, o, t1);
#pragma unroll
    for (int k2 = 0; k2 < PO; ++k2) RA[ST * r1 + PO * k2 + r0] = t1[k2];
  }
  __syncthreads();

  // ------------------------------------------------------------- S_y^T
  // line (r0, k2) = (lane % PO, lane / PO)
  if (valid) {
    T w[PO], o[PO];
#pragma unroll
    for (int j = 0; j < PO; ++j) w[j] = RA[ST * j + lane];
    st_rows<PO>(op.S, w, o);
#pragma unroll
    for (int k1 = 0; k1 < PO; ++k1) RB[SQ * r0 + PO * r1 + k1] = o[k1];  // r1 here = k2
  }
  __syncthreads();

  // ------------------------------------ S_x^T, Lambda^{-1}, S_x  (line (k1, k2))
  if (valid) {
    T w[PO], o[PO];
#pragma unroll
    for (int j = 0; j < PO; ++j) w[j] = RB[SQ * j + lane];
    st_rows<PO>(op.S, w, o);
#pragma unroll
    for (int k0 = 0; k0 < PO; ++k0) o[k0] *= dinv[k0 * PO * PO + lane];
    s_rows<PO>(op.S, o, w);
#pragma unroll
    for (int j = 0; j < PO; ++j) RA[SQ * r0 + PO * r1 + j] = w[j];  // (k1, k2) = (r0, r1)
  }
  __syncthreads();

  // ------------------------------------------------------------- S_y  (line (r0, k2))
  if (valid) {
    T w[PO], o[PO];
#pragma unroll
    for (int j = 0; j < PO; ++j) w[j] = RA[SQ * j + lane];
    s_rows<PO>(op.S, w, o);
#pragma unroll
    for (int j = 0; j < PO; ++j) RB[ST * j + lane] = o[j];
  }
  __syncthreads();

  // ------------------------------------------------- S_z, x += u  (line (r0, r1))
  if (valid) {
    T w[PO], o[PO], xo[PO];
#pragma unroll
    for (int r2 = 0; r2 < PO; ++r2) xo[r2] = gx[((r2 + 1) / NN) * cs2 + ((r2 + 1) % NN) * NN * NN];
#pragma unroll
    for (int k2 = 0; k2 < PO; ++k2) w[k2] = RB[ST * r1 + PO * k2 + r0];
    s_rows<PO>(op.S, w, o);
#pragma unroll
    for (int r2 = 0; r2 < PO; ++r2) gx[((r2 + 1) / NN) * cs2 + ((r2 + 1) % NN) * NN * NN] = xo[r2] + o[r2];
  }
}

template <int NN, typename T>
cudaError_t launch_int3(const sipg_handle* h, int level, int colour, const T* b, T* x, const PatchGrid& g,
                        cudaStream_t s) {
  using C = I3<NN, T>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(smooth_int3_kernel<NN, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  SmoothOps<C::PO, C::P, T, 1> ops;
  make_ops<C::PO, C::P, false, T>(h->hcst<T>(level), 0, ops.t[0]);
  dim3 grid((unsigned)((g.n_int + C::PPC - 1) / C::PPC), h->prm.nrhs);
  smooth_int3_kernel<NN, T><<<grid, C::THREADS, C::SMEM, s>>>(
      ops, colour, b, x, h->lv[level].N, h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0,
      (long long)h->lv[level].ndofs, g);
  return cudaGetLastError();
}

// The register-direct kernel takes the interior patches of 3D FP32 colour
// passes: its vector loads need 16-byte aligned vectors, and patch indices
// are 32-bit.
template <int DIM, typename T>
bool use_int3(const PatchGrid& g, const void* b, const void* x) {
  return DIM == 3 && sizeof(T) == 4 && g.n_int > 0 && g.n_int < (1LL << 31) &&
         (reinterpret_cast<uintptr_t>(b) % 16) == 0 && (reinterpret_cast<uintptr_t>(x) % 16) == 0;
}
