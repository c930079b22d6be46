// 3D vertex patches, register-direct variant of the colour pass (Algorithm 1
// with the fast-diagonalisation local solve of Eq. inverse3d).  Included by
// smoother.cu after its line-contraction helpers.
//
// Same arithmetic as the generic colour pass: the patch residual on V_j by
// three sum-factorised sweeps (x, y, z) of the rows V_j of the 1D patch mass
// and SIPG matrices, then u = (S_z x S_y x S_x) Lambda^{-1} (...)^T r and
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
// Interior patches (BND = false) run with p = 2k rows per direction and the
// operators as kernel parameters (constant-bank operands).  Patches touching
// the domain boundary (BND = true) run with p = 2n rows: per direction one of
// four operator sets (interior, low end, high end, both) read from shared
// memory, rows outside V_j with zero operators, S padded by the identity, the
// residual zeroed outside V_j and halos outside the domain read as zero.

template <int NN, typename T, bool BND, int TILE = 0>
struct I3 {
  static constexpr int P = 2 * NN;                      // patch nodes per direction
  static constexpr int PO = BND ? 2 * NN : 2 * NN - 2;  // rows per direction
  static constexpr int OFF = BND ? 0 : 1;               // patch node of row 0
  static constexpr int TPP = PO * PO;
  static constexpr int NT = BND ? 4 : 1;                // operator sets
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
  // CTA prefix (interior): the table 1 / (lambda_k0 + lambda_k1 + lambda_k2)
  static constexpr int DINV = BND ? 0 : PO * PO * PO;
  static constexpr int PREFIX = (DINV * (int)sizeof(T) + 15) / 16 * 16;
  // patches per CTA: fill about 54 KB of shared memory (four CTAs per SM) with
  // at most 512 threads
  // (TILE = 1: half as many, for the autotuner; TILE = 2, 3: the default
  // tile with b and x on V_j loaded ahead of the sweeps that use them, at
  // four and three CTAs per SM; TILE = 4: tile 3 with the x and y sweeps on
  // whole warps)
  static constexpr int ppc() {
    int k = (54 * 1024 - PREFIX) / (PS * (int)sizeof(T));
    if (k > 512 / TPP) k = 512 / TPP;
    if (TILE == 1) k /= 2;
    return k < 1 ? 1 : k;
  }
  static constexpr int PPC = ppc();
  static constexpr int THREADS = TPP * PPC;
  static constexpr size_t SMEM = (size_t)PREFIX + (size_t)PPC * PS * sizeof(T);
  static constexpr int minblocks() {
    int by_smem = (int)((228 * 1024) / (SMEM + 1024));
    int by_thr = 2048 / THREADS;
    int m = by_smem < by_thr ? by_smem : by_thr;
    // boundary patches: longer lines need more registers; they run beside
    // the interior kernel
    const int cap = BND ? 2 : (TILE == 1 ? 8 : (TILE >= 3 ? 3 : 4));
    return m < 1 ? 1 : (m > cap ? cap : m);
  }
  static constexpr int MINB = minblocks();
  static constexpr bool PF = !BND && TILE >= 2;  // loads of b and x on V_j issued early
  // TILE = 4: the x and y sweeps run on whole warps, WPP warps per patch, so
  // that their rounds of lines do not straddle two patches in one warp
  static constexpr int WPP = (THREADS / 32) / PPC;
  static constexpr bool WP = !BND && TILE == 4 && WPP >= 1;
  static constexpr int TPA = WP ? 32 * WPP : TPP;  // threads per patch in the x and y sweeps
  static constexpr int VW = run_vw<NN, T>();
};

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

// Calls f(std::integral_constant<int, TY>) for the patch's operator type of
// one direction, so that the body reads that operator set from the kernel
// parameters at compile-time offsets (constant-bank operands).  The boundary
// kernel has p^2 = 4n^2 threads per patch, a multiple of 32: the branch is
// uniform within each warp.
template <bool BND, class F>
__device__ __forceinline__ void i3_with_type(int ty, F&& f) {
  if constexpr (!BND) {
    f(std::integral_constant<int, 0>{});
  } else {
    switch (ty) {
      case 0: f(std::integral_constant<int, 0>{}); break;
      case 1: f(std::integral_constant<int, 1>{}); break;
      case 2: f(std::integral_constant<int, 2>{}); break;
      default: f(std::integral_constant<int, 3>{}); break;
    }
  }
}

// Interior table 1 / (lambda_k0 + lambda_k1 + lambda_k2), layout [k0][k2][k1].
template <int NN, typename T>
__device__ __forceinline__ void int3_dinv(const Ops1D<2 * NN - 2, 2 * NN, T>& o0, T* dinv) {
  constexpr int PO = 2 * NN - 2;
  for (int e = threadIdx.x; e < PO * PO * PO; e += blockDim.x) {
    const int k1 = e % PO, k2 = (e / PO) % PO, k0 = e / (PO * PO);
    dinv[e] = T(1) / (o0.lam[k0] + o0.lam[k1] + o0.lam[k2]);
  }
}

// Patches pbase + slot (slot < PPC, TPP threads each) of one colour.  Every
// thread of the CTA calls this (it holds CTA barriers); b and x point at the
// right-hand side's column; buf holds PPC patch buffers of I3::PS elements;
// dinv (interior) as written by int3_dinv.  NC: x is read through the
// read-only (non-coherent) path, valid when no other CTA writes what this
// launch reads (one colour per launch); the fused step, whose later colours
// read what other CTAs wrote, uses coherent loads.
// FULL (with BND): the full kernel's local solve (Sec. 3.1, Table 1) on all
// P = 2n patch nodes per direction: the patch residual is read from the
// global residual vector passed as b (no residual sweeps), then the same
// transforms with the whole-patch eigenpairs in ops; FINT: the patches are
// the colour's interior ones (interior decode) in this all-rows layout,
// otherwise the shell of patches touching the domain boundary.
template <int NN, typename T, bool BND, int PPC, bool NC, bool PF = false, int TILE = 0, bool FULL = false,
          bool FINT = false>
__device__ __forceinline__ void int3_body(const SmoothOps<I3<NN, T, BND>::PO, 2 * NN, T, I3<NN, T, BND>::NT>& ops,
                                          const T* dinv, T* buf, long long pbase, int colour,
                                          const T* __restrict__ b, T* x, int N, int consistent,
                                          const PatchGrid& grid) {
  using C = I3<NN, T, BND>;
  using Ops = Ops1D<C::PO, 2 * NN, T>;
  constexpr int P = C::P, PO = C::PO, OFF = C::OFF, TPP = C::TPP, ND = NN * NN * NN;
  constexpr int SA1 = C::SA1, SC = C::SC, CZS = C::CZS, ST = C::ST, SQ = C::SQ;
  const int tid = threadIdx.x;
  const int lane = tid % TPP;
  const int pl = tid / TPP;
  T* RA = buf + (size_t)(pl < PPC ? pl : 0) * C::PS;
  T* RB = RA + C::RA;

  static_assert(!FULL || BND, "the full kernel's pass uses the all-rows layout");
  const long long npatch = (BND && !FINT) ? grid.n_bnd : grid.n_int;
  const long long pidx = pbase + pl;
  const bool valid = pl < PPC && pidx < npatch;
  int v[3], ty[3] = {0, 0, 0};
  if (BND && !FINT) {
    int m[3] = {0, 0, 0};
    patch_index<3, true>(grid, valid ? pidx : 0, m);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      v[e] = ((colour >> e) & 1) ? 2 * m[e] + 1 : 2 * m[e] + 2;
      ty[e] = (v[e] == 1 ? 1 : 0) | (v[e] == N - 1 ? 2 : 0);
    }
  } else {
    int q = valid ? (int)pidx : 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int w = grid.hi[e] - grid.lo[e];
      const int qn = div_width(q, grid.dmul[e], grid.dshift[e]);
      const int m = grid.lo[e] + (q - qn * w);
      q = qn;
      v[e] = ((colour >> e) & 1) ? 2 * m + 1 : 2 * m + 2;
    }
  }
  // face-node halos: the cells across each patch face, when inside the domain
  bool exlo[3], exhi[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    exlo[e] = consistent && (!BND || v[e] >= 2);
    exhi[e] = consistent && (!BND || v[e] + 1 <= N - 1);
  }

  // cell (v0-1, v1-1, v2-1), node 0: all patch offsets below are relative to it
  const T* xb = x + ((long long)(v[0] - 1) + (long long)N * ((v[1] - 1) + (long long)N * (v[2] - 1))) * ND;
  const int cs1 = N * ND, cs2 = N * N * ND;  // cell strides in y and z (elements)

  // the x and y sweeps' view: this thread's patch and line index there (the
  // same as above unless the sweeps run on whole warps, WP)
  using CT = I3<NN, T, BND, TILE>;
  constexpr bool WP = CT::WP;
  constexpr int TPA = CT::TPA;
  int lA = lane;
  bool vA = valid;
  const T* xA = xb;
  T* RAA = RA;
  if constexpr (WP) {
    const int wid = tid / 32;
    const int pa = wid / CT::WPP;
    lA = (wid % CT::WPP) * 32 + (tid % 32);
    vA = pa < PPC && pbase + pa < npatch;
    int q = vA ? (int)(pbase + pa) : 0;
    int va[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int w = grid.hi[e] - grid.lo[e];
      const int qn = div_width(q, grid.dmul[e], grid.dshift[e]);
      const int m = grid.lo[e] + (q - qn * w);
      q = qn;
      va[e] = ((colour >> e) & 1) ? 2 * m + 1 : 2 * m + 2;
    }
    xA = x + ((long long)(va[0] - 1) + (long long)N * ((va[1] - 1) + (long long)N * (va[2] - 1))) * ND;
    RAA = buf + (size_t)(pa < PPC ? pa : 0) * C::PS;
  }
  T* RBA = RAA + C::RA;

  // ------------------------------------------------------------------ x sweep
  // lines t < P^2: (a1, a2) = (t / P, t % P); then 4P halo lines (slot, j):
  // slot 0/1 = y faces below/above (j = a2), 2/3 = z faces (j = a1), M_x only
  constexpr int L1 = P * P + 4 * P;
  constexpr int R1 = (L1 + TPA - 1) / TPA;
  if (!FULL && vA) {
    T vin[R1][P], hl[R1][2];
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      const int t = lA + q * TPA;
      int off = 0;
      const bool act = t < L1, main = t < P * P;
      bool ld = main;
      if (main) {
        const int a2 = t % P, a1 = t / P;
        off = (a1 / NN) * cs1 + (a2 / NN) * cs2 + (a1 % NN) * NN + (a2 % NN) * NN * NN;
      } else if (act) {
        const int h = t - P * P, slot = h / P, j = h % P;
        if (slot < 2) {  // y face: cell row v1-2 (node layer n-1) or v1+1 (layer 0); j = a2
          off = (slot ? 2 : -1) * cs1 + (slot ? 0 : (NN - 1) * NN) + (j / NN) * cs2 + (j % NN) * NN * NN;
          ld = slot ? exhi[1] : exlo[1];
        } else {         // z face: cell layer v2-2 or v2+1; j = a1
          off = (slot == 3 ? 2 : -1) * cs2 + (slot == 3 ? 0 : (NN - 1) * NN * NN) + (j / NN) * cs1 + (j % NN) * NN;
          ld = slot == 3 ? exhi[2] : exlo[2];
        }
      }
      if (ld) {
        i3_ldrun<NN, C::VW, T, NC>(xA + off, &vin[q][0]);
        i3_ldrun<NN, C::VW, T, NC>(xA + off + ND, &vin[q][NN]);
      } else {
#pragma unroll
        for (int c = 0; c < P; ++c) vin[q][c] = T(0);
      }
      // x halos of a main line: node n-1 of cell v0-2, node 0 of cell v0+1
      hl[q][0] = (main && exlo[0]) ? ld_elem<NC>(xA + off - ND + (NN - 1)) : T(0);
      hl[q][1] = (main && exhi[0]) ? ld_elem<NC>(xA + off + 2 * ND) : T(0);
    }
    i3_with_type<BND>(ty[0], [&](auto tc) {
      const Ops& ox = ops.t[decltype(tc)::value];
#pragma unroll
      for (int q = 0; q < R1; ++q) {
        const int t = lA + q * TPA;
        if (t >= L1) continue;
        // destination row: A/B[a1][a2][.] for main lines, halo[slot][j][.]
        const int dst = t < P * P ? SA1 * (t / P) + PO * (t % P)
                                  : (2 * P + (t - P * P) / P) * SA1 + PO * ((t - P * P) % P);
        T oa[PO];
        T(&vq)[P] = vin[q];
        mass_rows2<PO, P, NN, OFF, false>(ox, vq, oa);
        i3_st_pairs<PO>(RAA + dst, oa);
        if (t < P * P) {
          T ob[PO];
          sipg_rows2<PO, P, NN, OFF>(ox, vq, hl[q][0], hl[q][1], ob);
          i3_st_pairs<PO>(RAA + P * SA1 + dst, ob);
        }
      }
    });
  }
  // PF: b on this thread's z line of V_j, loaded now so that the loads
  // overlap the y sweep (interior patches: every row is in V_j)
  T bvp[PO], xop[PO];
  if constexpr (PF) {
    if (valid) {
      const int q0 = lane % PO, q1 = lane / PO;
      const T* gbp = b + ((v[0] - 1) + (long long)N * ((v[1] - 1) + (long long)N * (v[2] - 1))) * ND +
                     ((q0 + OFF) / NN) * ND + ((q1 + OFF) / NN) * cs1 + ((q0 + OFF) % NN) + ((q1 + OFF) % NN) * NN;
#pragma unroll
      for (int r2 = 0; r2 < PO; ++r2) bvp[r2] = __ldg(gbp + ((r2 + OFF) / NN) * cs2 + ((r2 + OFF) % NN) * NN * NN);
    }
  }
  if constexpr (!FULL) __syncthreads();

  // ------------------------------------------------------------------ y sweep
  // lines t < PO P: (r0, a2) = (t % PO, t / PO):
  //   C = M_y A,  D = L_y [A with the y halos] + M_y B;
  // then 2 PO lines (r0, side): CZ = M_y (z halo face after M_x)
  constexpr int L2 = PO * P + 2 * PO;
  constexpr int R2 = (L2 + TPA - 1) / TPA;
  T* Cc = RB;
  T* Dd = RB + P * SC;
  T* CZ = RB + 2 * P * SC;
  T* CcA = RBA;  // the sweep's patch (WP: the warp's)
  T* DdA = RBA + P * SC;
  T* CZA = RBA + 2 * P * SC;
  if (!FULL && vA) {
    i3_with_type<BND>(ty[1], [&](auto tc) {
      const Ops& oy = ops.t[decltype(tc)::value];
#pragma unroll
      for (int q = 0; q < R2; ++q) {
        const int t = lA + q * TPA;
        if (t >= L2) continue;
        if (t < PO * P) {
          const int r0 = t % PO, a2 = t / PO;
          T va[P], vb[P], oc[PO], od[PO];
#pragma unroll
          for (int a1 = 0; a1 < P; ++a1) {
            va[a1] = RAA[SA1 * a1 + t];
            vb[a1] = RAA[P * SA1 + SA1 * a1 + t];
          }
          const T h0 = RAA[2 * P * SA1 + t], h1 = RAA[(2 * P + 1) * SA1 + t];
          mass_rows2<PO, P, NN, OFF, false>(oy, va, oc);
          sipg_rows2<PO, P, NN, OFF>(oy, va, h0, h1, od);
          mass_rows2<PO, P, NN, OFF, true>(oy, vb, od);
#pragma unroll
          for (int r1 = 0; r1 < PO; ++r1) {
            CcA[SC * a2 + PO * r1 + r0] = oc[r1];
            DdA[SC * a2 + PO * r1 + r0] = od[r1];
          }
        } else {
          const int h = t - PO * P, r0 = h % PO, side = h / PO;
          T vz[P], oc[PO];
#pragma unroll
          for (int a1 = 0; a1 < P; ++a1) vz[a1] = RAA[(2 * P + 2 + side) * SA1 + PO * a1 + r0];
          mass_rows2<PO, P, NN, OFF, false>(oy, vz, oc);
#pragma unroll
          for (int r1 = 0; r1 < PO; ++r1) CZA[side * CZS + PO * r1 + r0] = oc[r1];
        }
      }
    });
  }
  if constexpr (!FULL) __syncthreads();

  // ------------------------------------------------ z sweep, residual, S_z^T
  // line (r0, r1) = (lane % PO, lane / PO); patch node (r0, r1, r2) + OFF
  const int r0 = lane % PO, r1 = lane / PO;
  const int goff = ((r0 + OFF) / NN) * ND + ((r1 + OFF) / NN) * cs1 + ((r0 + OFF) % NN) + ((r1 + OFF) % NN) * NN;
  T* gx = const_cast<T*>(xb) + goff;
  const T* gb = b + (xb - x) + goff;
  // rows of V_j (all rows for interior patches): [first, last] per direction
  int zlo = 0, zhi = PO - 1;
  bool inxy = true;
  if (BND) {
    const Ops& fx = ops.t[ty[0]];
    const Ops& fy = ops.t[ty[1]];
    const Ops& fz = ops.t[ty[2]];
    inxy = r0 >= fx.first && r0 <= fx.last && r1 >= fy.first && r1 <= fy.last;
    zlo = fz.first;
    zhi = fz.last;
  }
  if (valid) {
    i3_with_type<BND>(ty[2], [&](auto tc) {
      const Ops& oz = ops.t[decltype(tc)::value];
      T bv[PO], vc[P], vd[P], o[PO], t1[PO];
#pragma unroll
      for (int r2 = 0; r2 < PO; ++r2) {
        const bool in = inxy && r2 >= zlo && r2 <= zhi;
        if constexpr (PF)
          bv[r2] = bvp[r2];
        else
          bv[r2] = in ? __ldg(gb + ((r2 + OFF) / NN) * cs2 + ((r2 + OFF) % NN) * NN * NN) : T(0);
      }
      if constexpr (FULL) {
#pragma unroll
        for (int r2 = 0; r2 < PO; ++r2) {
          const bool in = inxy && r2 >= zlo && r2 <= zhi;
          o[r2] = in ? bv[r2] : T(0);  // the global residual on the patch
        }
      } else {
#pragma unroll
        for (int a2 = 0; a2 < P; ++a2) {
          vc[a2] = Cc[SC * a2 + lane];
          vd[a2] = Dd[SC * a2 + lane];
        }
        sipg_rows2<PO, P, NN, OFF>(oz, vc, CZ[lane], CZ[CZS + lane], o);
        mass_rows2<PO, P, NN, OFF, true>(oz, vd, o);
#pragma unroll
        for (int r2 = 0; r2 < PO; ++r2) {
          const bool in = inxy && r2 >= zlo && r2 <= zhi;
          o[r2] = in ? bv[r2] - o[r2] : T(0);
        }
      }
      st_rows2<PO>(oz.S2, o, t1);
#pragma unroll
      for (int k2 = 0; k2 < PO; ++k2) RA[ST * r1 + PO * k2 + r0] = t1[k2];
      // PF: x on the same line, for the final update (only this patch
      // writes it), loaded now so that the loads overlap the transforms
      if constexpr (PF) {
#pragma unroll
        for (int r2 = 0; r2 < PO; ++r2) xop[r2] = ld_elem<NC>(gx + ((r2 + OFF) / NN) * cs2 + ((r2 + OFF) % NN) * NN * NN);
      }
    });
  }
  __syncthreads();

  // ------------------------------------------------------------- S_y^T
  // line (r0, k2) = (lane % PO, lane / PO)
  if (valid) {
    i3_with_type<BND>(ty[1], [&](auto tc) {
      const Ops& oy = ops.t[decltype(tc)::value];
      T w[PO], o[PO];
#pragma unroll
      for (int j = 0; j < PO; ++j) w[j] = RA[ST * j + lane];
      st_rows2<PO>(oy.S2, w, o);
#pragma unroll
      for (int k1 = 0; k1 < PO; ++k1) RB[SQ * r0 + PO * r1 + k1] = o[k1];  // r1 here = k2
    });
  }
  __syncthreads();

  // ------------------------------------ S_x^T, Lambda^{-1}, S_x  (line (k1, k2))
  if (valid) {
    // lambda_y(k1) + lambda_z(k2), (k1, k2) = (r0, r1)
    const T lyz = BND ? ops.t[ty[1]].lam[r0] + ops.t[ty[2]].lam[r1] : T(0);
    i3_with_type<BND>(ty[0], [&](auto tc) {
      const Ops& ox = ops.t[decltype(tc)::value];
      T w[PO], o[PO];
#pragma unroll
      for (int j = 0; j < PO; ++j) w[j] = RB[SQ * j + lane];
      st_rows2<PO>(ox.S2, w, o);
      if (BND) {
#pragma unroll
        for (int k0 = 0; k0 < PO; ++k0) o[k0] = o[k0] / (ox.lam[k0] + lyz);
      } else {
#pragma unroll
        for (int k0 = 0; k0 < PO; ++k0) o[k0] *= dinv[k0 * PO * PO + lane];
      }
      s_rows2<PO>(ox.St2, o, w);
#pragma unroll
      for (int j = 0; j < PO; ++j) RA[SQ * r0 + PO * r1 + j] = w[j];
    });
  }
  __syncthreads();

  // ------------------------------------------------------------- S_y  (line (r0, k2))
  if (valid) {
    i3_with_type<BND>(ty[1], [&](auto tc) {
      const Ops& oy = ops.t[decltype(tc)::value];
      T w[PO], o[PO];
#pragma unroll
      for (int j = 0; j < PO; ++j) w[j] = RA[SQ * j + lane];
      s_rows2<PO>(oy.St2, w, o);
#pragma unroll
      for (int j = 0; j < PO; ++j) RB[ST * j + lane] = o[j];
    });
  }
  __syncthreads();

  // ------------------------------------------------- S_z, x += u  (line (r0, r1))
  if (valid) {
    i3_with_type<BND>(ty[2], [&](auto tc) {
      const Ops& oz = ops.t[decltype(tc)::value];
      T w[PO], o[PO], xo[PO];
#pragma unroll
      for (int r2 = 0; r2 < PO; ++r2) {
        const bool in = inxy && r2 >= zlo && r2 <= zhi;
        if constexpr (PF)
          xo[r2] = xop[r2];
        else
          xo[r2] = in ? gx[((r2 + OFF) / NN) * cs2 + ((r2 + OFF) % NN) * NN * NN] : T(0);
      }
#pragma unroll
      for (int k2 = 0; k2 < PO; ++k2) w[k2] = RB[ST * r1 + PO * k2 + r0];
      s_rows2<PO>(oz.St2, w, o);
#pragma unroll
      for (int r2 = 0; r2 < PO; ++r2) {
        const bool in = inxy && r2 >= zlo && r2 <= zhi;
        if (in) gx[((r2 + OFF) / NN) * cs2 + ((r2 + OFF) % NN) * NN * NN] = xo[r2] + o[r2];
      }
    });
  }
}

template <int NN, typename T, bool BND, int TILE>
__global__ void __launch_bounds__(I3<NN, T, BND, TILE>::THREADS, I3<NN, T, BND, TILE>::MINB)
    smooth_int3_kernel(const __grid_constant__ SmoothOps<I3<NN, T, BND>::PO, 2 * NN, T, I3<NN, T, BND>::NT> ops,
                       int colour, const T* __restrict__ b, T* x, int N, int consistent, long long ndofs,
                       PatchGrid grid) {
  using C = I3<NN, T, BND, TILE>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* dinv = reinterpret_cast<T*>(smem_raw);
  if constexpr (!BND) int3_dinv<NN, T>(ops.t[0], dinv);  // read after the first CTA barrier of the body
  const long long col = (long long)blockIdx.y * ndofs;
  int3_body<NN, T, BND, C::PPC, true, C::PF, TILE>(ops, dinv, reinterpret_cast<T*>(smem_raw + C::PREFIX), (long long)blockIdx.x * C::PPC,
                                colour, b + col, x + col, N, consistent, grid);
}

template <int NN, typename T, bool BND, int TILE>
cudaError_t launch_int3(const sipg_handle* h, int level, int colour, const T* b, T* x, const PatchGrid& g,
                        cudaStream_t s) {
  using C = I3<NN, T, BND, TILE>;
  const long long np = BND ? g.n_bnd : g.n_int;
  if (np <= 0) return cudaSuccess;
  cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(smooth_int3_kernel<NN, T, BND, TILE>), (int)C::SMEM);
  if (e != cudaSuccess) return e;
  SmoothOps<C::PO, C::P, T, C::NT> ops;
  for (int t = 0; t < C::NT; ++t) make_ops<C::PO, C::P, BND, T>(h->hcst<T>(level), t, ops.t[t]);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((np + C::PPC - 1) / C::PPC), h->prm.nrhs);
  cfg.blockDim = dim3(C::THREADS);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute la[1];
  la[0].id = cudaLaunchAttributePriority;
  la[0].val.priority = h->prio_hi;
  cfg.attrs = la;
  cfg.numAttrs = (BND == h->bnd_first) ? 1 : 0;  // the patch set launched first (see the colour-pass dispatch)
  return cudaLaunchKernelEx(&cfg, smooth_int3_kernel<NN, T, BND, TILE>, ops, colour, b, x, h->lv[level].N,
                            h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0, (long long)h->lv[level].ndofs, g);
}

// The register-direct kernels take the 3D FP32 colour passes: their vector
// loads need 16-byte aligned vectors, and interior patch indices are 32-bit.
template <int DIM, typename T>
bool use_int3(const PatchGrid& g, const void* b, const void* x) {
  return DIM == 3 && sizeof(T) == 4 && g.n_int < (1LL << 31) && (reinterpret_cast<uintptr_t>(b) % 16) == 0 &&
         (reinterpret_cast<uintptr_t>(x) % 16) == 0;
}

// A launch with the device's greatest stream priority when `prio` (the
// patch set of a colour pass that goes first, see the colour-pass dispatch).
template <typename... KArgs, typename... Args>
cudaError_t launch_prio(void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t s, bool prio,
                        int prio_value, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute la[1];
  la[0].id = cudaLaunchAttributePriority;
  la[0].val.priority = prio_value;
  cfg.attrs = la;
  cfg.numAttrs = prio ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------- clamped
// The clamped kernel (Sec. 3.1): V_j = patch functions with v = d_n v = 0 on
// the patch boundary inside the domain.  Every face term of the patch
// boundary vanishes for such test functions, so the local residual
// B^T R_D (b - A x) equals B^T (R_D b - A_D R_D x) with A_D the principal
// block of A on the 2^d patch cells: no halo, no coupling to other patches.
// One fused pass per colour therefore runs the register-direct kernel in its
// boundary layout (all P = 2n patch nodes per direction as rows) over every
// patch of the colour, with per direction type t the operators
//   rows of A_D: the full 2n x 2n patch block of the 1D SIPG matrix (own cell
//   blocks with their face terms, rank-two couplings across the vertex),
//   rows of M: the block-diagonal cell mass (diagonal plus rank one),
//   S = B S_m (P x m, zero columns beyond m), Lambda (1 beyond m): the
//   eigenpairs of the projected 1D patch matrices B^T L_D B, B^T M_D B,
// so that u = (S (x) S (x) S) Lambda^{-1} (S (x) S (x) S)^T r_D is
// B (B^T A_D B)^{-1} B^T r_D, added to x on the patch cells (zero on the
// patch-end nodes).  Same-colour patches tile disjoint cells and read no
// other patch's cells: the pass is race-free and equals the sequential one.
template <int NN, typename T>
void make_ops_clamped(const LevelConst<T>& lc, int t, Ops1D<2 * NN, 2 * NN, T>& op) {
  constexpr int P = 2 * NN, k = NN - 1;
  const int tl = (t & 1) ? 1 : 0, tr = (t & 2) ? 2 : 0;
  for (int a = 0; a < P; ++a) {
    const int oa = a / NN, ia = a % NN;
    for (int c = 0; c < P; ++c) {
      const int ob = c / NN, ib = c % NN;
      T v;
      if (oa == ob) v = lc.Lself[oa ? tr : tl][ia][ib];
      else if (oa == 0) v = (ia == k ? lc.ahi[ib] : T(0)) + (ib == 0 ? lc.ghi[ia] : T(0));  // test low cell, trial high
      else v = (ia == 0 ? lc.alo[ib] : T(0)) + (ib == k ? lc.glo[ia] : T(0));             // test high cell, trial low
      op.Lm[a * P + c] = v;
    }
    op.hlo[a] = op.hhi[a] = T(0);
    op.lam[a] = lc.lamf[t][a];
    op.mw[a] = lc.Mw[ia];
    op.mu[a] = lc.Mu[ia];
  }
  for (int j = 0; j < NN; ++j) op.ma[j] = lc.Ma[j];
  for (int j = 0; j < P; ++j)
    for (int i = 0; i < P; ++i) op.S[j * P + i] = lc.Sf[t][j][i];
  op.first = 0;
  op.last = P - 1;
  if constexpr (sizeof(T) == 4) {
    for (int q = 0; q < P / 2; ++q) {
      for (int j = 0; j < P; ++j) {
        op.S2[j * (P / 2) + q] = make_float2(op.S[j * P + 2 * q], op.S[j * P + 2 * q + 1]);
        op.St2[q * P + j] = make_float2(op.S[2 * q * P + j], op.S[(2 * q + 1) * P + j]);
      }
      for (int c = 0; c < P; ++c) op.L2[q * P + c] = make_float2(op.Lm[2 * q * P + c], op.Lm[(2 * q + 1) * P + c]);
      op.mw2[q] = make_float2(op.mw[2 * q], op.mw[2 * q + 1]);
      op.mu2[q] = make_float2(op.mu[2 * q], op.mu[2 * q + 1]);
    }
  }
}

// Interior patches (no end on the domain boundary): the clamped basis B
// vanishes on the two patch-end nodes of each direction, so B^T r_D needs
// the residual only on the other p = 2k rows and the correction lives there:
// the pass is the interior (Dirichlet-row) layout of the kernel with the rows
// 1..2n-2 of A_D (no halo: consistent = 0), of B S_m (zero columns beyond m)
// and Lambda.
template <int NN, typename T>
void make_ops_clamped_interior(const LevelConst<T>& lc, Ops1D<2 * NN - 2, 2 * NN, T>& op) {
  constexpr int P = 2 * NN, PO = 2 * NN - 2;
  Ops1D<P, P, T> full;
  make_ops_clamped<NN, T>(lc, 0, full);
  for (int r = 0; r < PO; ++r) {
    for (int c = 0; c < P; ++c) op.Lm[r * P + c] = full.Lm[(r + 1) * P + c];
    op.hlo[r] = op.hhi[r] = T(0);
    op.lam[r] = full.lam[r];
    op.mw[r] = full.mw[r + 1];
    op.mu[r] = full.mu[r + 1];
  }
  for (int j = 0; j < NN; ++j) op.ma[j] = lc.Ma[j];
  for (int j = 0; j < PO; ++j)
    for (int i = 0; i < PO; ++i) op.S[j * PO + i] = full.S[(j + 1) * P + i];
  op.first = 0;
  op.last = PO - 1;
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

// One clamped colour pass (3D FP32): interior patches in the interior layout
// on the calling stream, patches touching the domain boundary in the
// boundary layout (all 2n rows) beside them on the second stream (the two
// sets tile disjoint cells and read only their own cells).
template <int NN, typename T>
cudaError_t launch_int3_clamped(const sipg_handle* h, int level, int colour, const T* b, T* x, cudaStream_t s) {
  using CI = I3<NN, T, false, 0>;
  using CB = I3<NN, T, true, 0>;
  const PatchGrid g = make_grid(3, h->lv[level].N, colour);
  if (g.n_int + g.n_bnd <= 0) return cudaSuccess;
  const int N = h->lv[level].N;
  const long long nd = (long long)h->lv[level].ndofs;
  cudaError_t e;
  const bool fork = g.n_int > 0 && g.n_bnd > 0 && h->side;
  cudaStream_t sb = fork ? h->side : s;
  if (fork) {
    if ((e = cudaEventRecord(h->ev_fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->side, h->ev_fork, 0)) != cudaSuccess) return e;
  }
  // the boundary patches first at the greatest priority (as for the
  // Dirichlet kernel), unless the handle says otherwise
  auto run_int = [&]() -> cudaError_t {
    if (g.n_int <= 0) return cudaSuccess;
    cudaError_t ee = smem_opt_in(reinterpret_cast<const void*>(smooth_int3_kernel<NN, T, false, 0>), (int)CI::SMEM);
    if (ee != cudaSuccess) return ee;
    SmoothOps<CI::PO, CI::P, T, 1> ops;
    make_ops_clamped_interior<NN, T>(h->hcst<T>(level), ops.t[0]);
    dim3 grid((unsigned)((g.n_int + CI::PPC - 1) / CI::PPC), h->prm.nrhs);
    return launch_prio(smooth_int3_kernel<NN, T, false, 0>, grid, CI::THREADS, CI::SMEM, s, !h->bnd_first,
                       h->prio_hi, ops, colour, b, x, N, 0, nd, g);
  };
  auto run_bnd = [&]() -> cudaError_t {
    if (g.n_bnd <= 0) return cudaSuccess;
    cudaError_t ee = smem_opt_in(reinterpret_cast<const void*>(smooth_int3_kernel<NN, T, true, 0>), (int)CB::SMEM);
    if (ee != cudaSuccess) return ee;
    SmoothOps<CB::PO, CB::P, T, CB::NT> ops;
    for (int t = 0; t < CB::NT; ++t) make_ops_clamped<NN, T>(h->hcst<T>(level), t, ops.t[t]);
    dim3 grid((unsigned)((g.n_bnd + CB::PPC - 1) / CB::PPC), h->prm.nrhs);
    return launch_prio(smooth_int3_kernel<NN, T, true, 0>, grid, CB::THREADS, CB::SMEM, sb, h->bnd_first,
                       h->prio_hi, ops, colour, b, x, N, 0, nd, g);
  };
  if ((e = h->bnd_first ? run_bnd() : run_int()) != cudaSuccess) return e;
  if ((e = h->bnd_first ? run_int() : run_bnd()) != cudaSuccess) return e;
  if (fork) {
    if ((e = cudaEventRecord(h->ev_join, h->side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, h->ev_join, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ full
// The full kernel's patch solves (Sec. 3.1, Table 1) in the register-direct
// all-rows layout: after the whole-level residual r = b - A x of the colour,
// every patch of the colour adds A_j^{-1} R_j r, A_j^{-1} = (S (x) S (x) S)
// Lambda^{-1} (...)^T with the whole-patch eigenpairs of the patch's 1D
// types.  Interior and boundary patches run as two launches (two streams);
// same-colour patches write disjoint nodes and read only r.
template <int NN, bool FINT>
__global__ void __launch_bounds__(I3<NN, float, true>::THREADS, I3<NN, float, true>::MINB)
    smooth_full3_kernel(const __grid_constant__ SmoothOps<2 * NN, 2 * NN, float, 4> ops, int colour,
                        const float* __restrict__ r, float* x, int N, long long ndofs, PatchGrid grid) {
  using C = I3<NN, float, true>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long col = (long long)blockIdx.y * ndofs;
  int3_body<NN, float, true, C::PPC, true, false, 0, true, FINT>(ops, nullptr,
                                                               reinterpret_cast<float*>(smem_raw + C::PREFIX),
                                                               (long long)blockIdx.x * C::PPC, colour, r + col,
                                                               x + col, N, 0, grid);
}

template <int NN>
cudaError_t launch_full3(const sipg_handle* h, int level, int colour, const float* r, float* x, cudaStream_t s) {
  using C = I3<NN, float, true>;
  const PatchGrid g = make_grid(3, h->lv[level].N, colour);
  if (g.n_int + g.n_bnd <= 0) return cudaSuccess;
  const int N = h->lv[level].N;
  const long long nd = (long long)h->lv[level].ndofs;
  SmoothOps<2 * NN, 2 * NN, float, 4> ops;
  for (int t = 0; t < 4; ++t) make_ops_clamped<NN, float>(h->hcst<float>(level), t, ops.t[t]);
  cudaError_t e;
  const bool fork = g.n_int > 0 && g.n_bnd > 0 && h->side;
  cudaStream_t sb = fork ? h->side : s;
  if (fork) {
    if ((e = cudaEventRecord(h->ev_fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->side, h->ev_fork, 0)) != cudaSuccess) return e;
  }
  auto run_int = [&]() -> cudaError_t {
    if (g.n_int <= 0) return cudaSuccess;
    cudaError_t ee = smem_opt_in(reinterpret_cast<const void*>(smooth_full3_kernel<NN, true>), (int)C::SMEM);
    if (ee != cudaSuccess) return ee;
    dim3 grid((unsigned)((g.n_int + C::PPC - 1) / C::PPC), h->prm.nrhs);
    return launch_prio(smooth_full3_kernel<NN, true>, grid, C::THREADS, C::SMEM, s, !h->bnd_first, h->prio_hi, ops,
                       colour, r, x, N, nd, g);
  };
  auto run_bnd = [&]() -> cudaError_t {
    if (g.n_bnd <= 0) return cudaSuccess;
    cudaError_t ee = smem_opt_in(reinterpret_cast<const void*>(smooth_full3_kernel<NN, false>), (int)C::SMEM);
    if (ee != cudaSuccess) return ee;
    dim3 grid((unsigned)((g.n_bnd + C::PPC - 1) / C::PPC), h->prm.nrhs);
    return launch_prio(smooth_full3_kernel<NN, false>, grid, C::THREADS, C::SMEM, sb, h->bnd_first, h->prio_hi, ops,
                       colour, r, x, N, nd, g);
  };
  if ((e = h->bnd_first ? run_bnd() : run_int()) != cudaSuccess) return e;
  if ((e = h->bnd_first ? run_int() : run_bnd()) != cudaSuccess) return e;
  if (fork) {
    if ((e = cudaEventRecord(h->ev_join, h->side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, h->ev_join, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
