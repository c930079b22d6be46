// 2D vertex patches, register-direct colour pass (Algorithm 1 with the
// fast-diagonalisation local solve of Eq. inverse2d).  Included by
// smoother_impl.cuh after smooth_int3.cuh.
//
// Same arithmetic as the generic colour pass: the patch residual on V_j by
// two sum-factorised sweeps of the rows V_j of the 1D patch mass and SIPG
// matrices, then u = (S_y x S_x) (Lambda_x + Lambda_y)^{-1} (S_y x S_x)^T r
// and x[V_j] += u.  Data movement as in the 3D kernel: the x sweep reads its
// lines straight from global memory into registers (vector loads of each
// cell's contiguous x-lines, face-node halos included); the y sweep keeps its
// residual column in registers and applies S_y^T in place; the x-direction
// forward transform, the scaling and the backward transform share one line;
// the last transform (y) adds to x from registers.  p threads per patch (one
// line each), many patches per CTA, three CTA barriers per pass; packed
// two-lane FP32 FMAs.  Interior patches (p = 2k) read their operators as
// kernel parameters; boundary patches (p = 2n, padded) read one of four
// operator sets per direction from shared memory.

template <int NN, typename T, bool BND>
struct I2 {
  static constexpr int P = 2 * NN;
  static constexpr int PO = BND ? 2 * NN : 2 * NN - 2;
  static constexpr int OFF = BND ? 0 : 1;
  static constexpr int TPP = PO;
  static constexpr int NT = BND ? 4 : 1;
  static constexpr int SA = PO + 1;               // odd row stride of every exchange array
  static constexpr int RA = (2 * P + 2) * SA;     // A, B (P rows each), y halos (2 rows); later T2
  static constexpr int RB = PO * SA;              // T1
  static constexpr int PS = RA + RB;
  static constexpr int PREFIX = BND ? ((NT * (int)sizeof(Ops1D<PO, P, T>) + 15) / 16 * 16) : 0;
  static constexpr int ppc() {
    int k = 256 / TPP;
    const int by_smem = (48 * 1024 - PREFIX) / (PS * (int)sizeof(T));
    if (k > by_smem) k = by_smem;
    return k < 1 ? 1 : k;
  }
  static constexpr int PPC = ppc();
  static constexpr int THREADS = TPP * PPC;
  static constexpr size_t SMEM = (size_t)PREFIX + (size_t)PPC * PS * sizeof(T);
  static constexpr int VW = run_vw<NN, T>();
};

// Patches pbase + slot (slot < PPC, TPP threads each) of one colour; every
// thread of the CTA calls this (it holds CTA barriers), threads past the PPC
// slots only take part in the barriers.  smem_raw: the kernel's dynamic
// shared memory (the boundary operator sets are copied there).  NC: x is read
// through the read-only path, valid when no other CTA writes what this launch
// reads (one colour per launch); launches that run several colours with grid
// barriers between them use coherent loads.
template <int NN, typename T, bool BND, bool NC>
__device__ __forceinline__ void int2_body(const SmoothOps<I2<NN, T, BND>::PO, 2 * NN, T, I2<NN, T, BND>::NT>& ops,
                                          unsigned char* smem_raw, long long pbase, int colour,
                                          const T* __restrict__ b, T* x, int N, int consistent,
                                          const PatchGrid& grid) {
  using C = I2<NN, T, BND>;
  using Ops = Ops1D<C::PO, 2 * NN, T>;
  constexpr int P = C::P, PO = C::PO, OFF = C::OFF, TPP = C::TPP, PPC = C::PPC, SA = C::SA, ND = NN * NN;
  const Ops* sops = reinterpret_cast<const Ops*>(smem_raw);
  if (BND) {
    const int* src = reinterpret_cast<const int*>(&ops);
    int* dst = reinterpret_cast<int*>(smem_raw);
    for (int e = threadIdx.x; e < (int)(sizeof(Ops) * C::NT / sizeof(int)); e += blockDim.x) dst[e] = src[e];
  }
  const int tid = threadIdx.x;
  const int lane = tid % TPP;
  const int pl = tid / TPP;
  T* RA = reinterpret_cast<T*>(smem_raw + C::PREFIX) + (size_t)(pl < PPC ? pl : 0) * C::PS;
  T* RB = RA + C::RA;
  const long long npatch = BND ? grid.n_bnd : grid.n_int;
  const long long pidx = pbase + pl;
  const bool valid = pl < PPC && pidx < npatch;
  int m[3] = {0, 0, 0};
  patch_index<2, BND>(grid, valid ? pidx : 0, m);
  int v[2], ty[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    v[e] = ((colour >> e) & 1) ? 2 * m[e] + 1 : 2 * m[e] + 2;
    ty[e] = BND ? ((v[e] == 1 ? 1 : 0) | (v[e] == N - 1 ? 2 : 0)) : 0;
  }
  bool exlo[2], exhi[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    exlo[e] = consistent && (!BND || v[e] >= 2);
    exhi[e] = consistent && (!BND || v[e] + 1 <= N - 1);
  }
  if (BND) __syncthreads();  // operator sets in shared memory
  const Ops& ox = BND ? sops[ty[0]] : ops.t[0];
  const Ops& oy = BND ? sops[ty[1]] : ops.t[0];
  // cell (v0-1, v1-1), node 0
  const T* xb = x + ((long long)(v[0] - 1) + (long long)N * (v[1] - 1)) * ND;
  const int cs1 = N * ND;  // cell stride in y

  // ------------------------------------------------------------------ x sweep
  // lines t < P: row a1 = t (A = M_x, B = L_x with the x halos); t = P, P+1:
  // the y-halo rows below / above (M_x only)
  constexpr int L1 = P + 2;
  constexpr int R1 = (L1 + TPP - 1) / TPP;
  if (valid) {
    T vin[R1][P], hl[R1][2];
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      const int t = lane + q * TPP;
      const bool main = t < P;
      int off = 0;
      bool ld = main;
      if (main) {
        off = (t / NN) * cs1 + (t % NN) * NN;
      } else if (t < L1) {
        const int side = t - P;
        off = side ? 2 * cs1 : -cs1 + (NN - 1) * NN;
        ld = side ? exhi[1] : exlo[1];
      }
      if (ld) {
        i3_ldrun<NN, C::VW, T, NC>(xb + off, &vin[q][0]);
        i3_ldrun<NN, C::VW, T, NC>(xb + off + ND, &vin[q][NN]);
      } else {
#pragma unroll
        for (int c = 0; c < P; ++c) vin[q][c] = T(0);
      }
      hl[q][0] = (main && exlo[0]) ? ld_elem<NC>(xb + off - ND + (NN - 1)) : T(0);
      hl[q][1] = (main && exhi[0]) ? ld_elem<NC>(xb + off + 2 * ND) : T(0);
    }
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      const int t = lane + q * TPP;
      if (t >= L1) continue;
      T oa[PO];
      mass_rows2<PO, P, NN, OFF, false>(ox, vin[q], oa);
      if (t < P) {
        T ob[PO];
        sipg_rows2<PO, P, NN, OFF>(ox, vin[q], hl[q][0], hl[q][1], ob);
#pragma unroll
        for (int r = 0; r < PO; ++r) {
          RA[t * SA + r] = oa[r];
          RA[(P + t) * SA + r] = ob[r];
        }
      } else {
#pragma unroll
        for (int r = 0; r < PO; ++r) RA[(2 * P + (t - P)) * SA + r] = oa[r];
      }
    }
  }
  __syncthreads();

  // ------------------------------------------- y sweep, residual, S_y^T (column r0)
  const int r0 = lane;
  const int goff = ((r0 + OFF) / NN) * ND + ((r0 + OFF) % NN);
  T* gx = const_cast<T*>(xb) + goff;
  const T* gb = b + (xb - x) + goff;
  const bool inx = !BND || (r0 >= ox.first && r0 <= ox.last);
  const int ylo = BND ? oy.first : 0, yhi = BND ? oy.last : PO - 1;
  if (valid) {
    T bv[PO], va[P], vb[P], o[PO], t1[PO];
#pragma unroll
    for (int r1 = 0; r1 < PO; ++r1) {
      const bool in = inx && r1 >= ylo && r1 <= yhi;
      bv[r1] = in ? __ldg(gb + ((r1 + OFF) / NN) * cs1 + ((r1 + OFF) % NN) * NN) : T(0);
    }
#pragma unroll
    for (int a1 = 0; a1 < P; ++a1) {
      va[a1] = RA[a1 * SA + r0];
      vb[a1] = RA[(P + a1) * SA + r0];
    }
    sipg_rows2<PO, P, NN, OFF>(oy, va, RA[2 * P * SA + r0], RA[(2 * P + 1) * SA + r0], o);
    mass_rows2<PO, P, NN, OFF, true>(oy, vb, o);
#pragma unroll
    for (int r1 = 0; r1 < PO; ++r1) {
      const bool in = inx && r1 >= ylo && r1 <= yhi;
      o[r1] = in ? bv[r1] - o[r1] : T(0);
    }
    st_rows2<PO>(oy.S2, o, t1);
#pragma unroll
    for (int k1 = 0; k1 < PO; ++k1) RB[k1 * SA + r0] = t1[k1];
  }
  __syncthreads();

  // ------------------------------------- S_x^T, (Lambda_x + Lambda_y)^{-1}, S_x (row k1)
  if (valid) {
    const int k1 = lane;
    T w[PO], o[PO];
#pragma unroll
    for (int j = 0; j < PO; ++j) w[j] = RB[k1 * SA + j];
    st_rows2<PO>(ox.S2, w, o);
    const T ly = oy.lam[k1];
#pragma unroll
    for (int k0 = 0; k0 < PO; ++k0) o[k0] = o[k0] / (ox.lam[k0] + ly);
    s_rows2<PO>(ox.St2, o, w);
#pragma unroll
    for (int j = 0; j < PO; ++j) RA[k1 * SA + j] = w[j];
  }
  __syncthreads();

  // -------------------------------------------------- S_y, x += u (column r0)
  if (valid) {
    T w[PO], u[PO], xo[PO];
#pragma unroll
    for (int r1 = 0; r1 < PO; ++r1) {
      const bool in = inx && r1 >= ylo && r1 <= yhi;
      xo[r1] = in ? gx[((r1 + OFF) / NN) * cs1 + ((r1 + OFF) % NN) * NN] : T(0);
    }
#pragma unroll
    for (int k1 = 0; k1 < PO; ++k1) w[k1] = RA[k1 * SA + r0];
    s_rows2<PO>(oy.St2, w, u);
#pragma unroll
    for (int r1 = 0; r1 < PO; ++r1) {
      const bool in = inx && r1 >= ylo && r1 <= yhi;
      if (in) gx[((r1 + OFF) / NN) * cs1 + ((r1 + OFF) % NN) * NN] = xo[r1] + u[r1];
    }
  }
}

template <int NN, typename T, bool BND>
__global__ void __launch_bounds__(I2<NN, T, BND>::THREADS)
    smooth_int2_kernel(const __grid_constant__ SmoothOps<I2<NN, T, BND>::PO, 2 * NN, T, I2<NN, T, BND>::NT> ops,
                       int colour, const T* __restrict__ b, T* x, int N, int consistent, long long ndofs,
                       PatchGrid grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long col = (long long)blockIdx.y * ndofs;
  int2_body<NN, T, BND, true>(ops, smem_raw, (long long)blockIdx.x * I2<NN, T, BND>::PPC, colour, b + col, x + col,
                              N, consistent, grid);
}

template <int NN, typename T, bool BND>
cudaError_t launch_int2(const sipg_handle* h, int level, int colour, const T* b, T* x, const PatchGrid& g,
                        cudaStream_t s) {
  using C = I2<NN, T, BND>;
  const long long np = BND ? g.n_bnd : g.n_int;
  if (np <= 0) return cudaSuccess;
  cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(smooth_int2_kernel<NN, T, BND>), (int)C::SMEM);
  if (e != cudaSuccess) return e;
  SmoothOps<C::PO, C::P, T, C::NT> ops;
  for (int t = 0; t < C::NT; ++t) make_ops<C::PO, C::P, BND, T>(h->hcst<T>(level), t, ops.t[t]);
  dim3 grid((unsigned)((np + C::PPC - 1) / C::PPC), h->prm.nrhs);
  smooth_int2_kernel<NN, T, BND><<<grid, C::THREADS, C::SMEM, s>>>(
      ops, colour, b, x, h->lv[level].N, h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0,
      (long long)h->lv[level].ndofs, g);
  return cudaGetLastError();
}
