// 3D vertex-patch local solve spread over many threads: the latency-bound
// variant of the colour pass for small levels (Algorithm 1 with the
// fast-diagonalisation local solve of Eq. inverse3d).  Included by
// smoother_impl.cuh after smooth_int3.cuh.
//
// On the coarse levels of the V-cycle a colour holds few patches, so the
// time of a colour pass is the latency of one patch, not throughput.  Here a
// patch owns a whole CTA and every stage hands out single outputs (one
// element of one 1D contraction) to the threads, so a thread's chain per
// stage is one dot product of length <= 2n:
//   load   patch tile + six halo faces into shared memory; each thread also
//          prefetches b and x of the V_j entries it will update
//   S1     A = M_x X, B = L_x [X with x halos], M_x on the y and z halo faces
//   S2     C = M_y A, D = L_y [A with y halos] + M_y B, M_y on the z faces
//   S3     r = b - (L_z [C with z halos] + M_z D)     (zero outside V_j)
//   F1-F3  S_z^T, S_y^T, S_x^T and the scaling by 1 / (lambda + lambda + lambda)
//   G3-G1  S_x, S_y, S_z; x[V_j] += u
// The arithmetic per output equals that of the line kernels (same 1D rows,
// same summation order within each dot product, structural zeros included).
// Interior patches use p = 2k rows per direction, patches on the boundary
// p = 2n with padded operators (zero rows outside V_j, S padded by the
// identity), as in the other colour-pass kernels.

template <int NN, typename T, bool BND>
struct W3 {
  static constexpr int P = 2 * NN;
  static constexpr int PO = BND ? 2 * NN : 2 * NN - 2;
  static constexpr int OFF = BND ? 0 : 1;
  static constexpr int NT = BND ? 4 : 1;
  static constexpr int LP = P + 1;   // padded row length of the 1D operators in shared memory
  static constexpr int SP = PO + 1;  // padded row length of S
  // threads per patch: one per V_j entry when that fits 1024 threads
  static constexpr int RS = PO * PO * PO <= 1024 ? PO : 1024 / (PO * PO);
  static constexpr int TPP = PO * PO * RS;
  static constexpr int ITEMS = (PO * PO * PO + TPP - 1) / TPP;  // V_j entries per thread
  // shared-memory regions (elements)
  static constexpr int R1 = i3_max(P * P * P + 6 * P * P, PO * PO * PO);
  static constexpr int R2 = i3_max(2 * P * P * PO + 4 * P * PO, PO * PO * PO);
  static constexpr int R3 = i3_max(2 * P * PO * PO + 2 * PO * PO, PO * PO * PO);
  // operator sets: Lm (PO x LP), mw, mu (PO), ma (n), hlo, hhi, lam (PO),
  // S (PO x SP), first, last; the mass rows are diagonal plus rank one per cell
  static constexpr int OPS = PO * LP + 2 * PO + NN + 3 * PO + PO * SP + 2;
  static constexpr size_t SMEM = sizeof(T) * ((size_t)NT * OPS + R1 + R2 + R3);
};

// copy the operator sets of the kernel parameters into padded rows
template <int PO, int P, typename T, int NT>
__device__ __forceinline__ void w3_ops_setup(const SmoothOps<PO, P, T, NT>& ops, T* dst) {
  constexpr int NN = P / 2, LP = P + 1, SP = PO + 1, OPS = PO * LP + 2 * PO + NN + 3 * PO + PO * SP + 2;
  constexpr int MW = PO * LP, MU = MW + PO, MA = MU + PO, HL = MA + NN, HH = HL + PO, LA = HH + PO, SS = LA + PO;
  for (int t = 0; t < NT; ++t) {
    const Ops1D<PO, P, T>& o = ops.t[t];
    T* d = dst + t * OPS;
    for (int e = threadIdx.x; e < PO * P; e += blockDim.x) d[(e / P) * LP + e % P] = o.Lm[e];
    for (int e = threadIdx.x; e < PO; e += blockDim.x) {
      d[MW + e] = o.mw[e];
      d[MU + e] = o.mu[e];
      d[HL + e] = o.hlo[e];
      d[HH + e] = o.hhi[e];
      d[LA + e] = o.lam[e];
    }
    for (int e = threadIdx.x; e < NN; e += blockDim.x) d[MA + e] = o.ma[e];
    for (int e = threadIdx.x; e < PO * PO; e += blockDim.x) d[SS + (e / PO) * SP + e % PO] = o.S[e];
    if (threadIdx.x == 0) {
      d[OPS - 2] = T(o.first);
      d[OPS - 1] = T(o.last);
    }
  }
}

// Views of one operator set laid out by w3_ops_setup (offsets are constants,
// so a view costs one pointer).
template <int NN, typename T, bool BND>
struct W3View {
  using C = W3<NN, T, BND>;
  const T* base;
  static constexpr int MW = C::PO * C::LP, MU = MW + C::PO, MA = MU + C::PO, HL = MA + NN, HH = HL + C::PO,
                       LA = HH + C::PO, SS = LA + C::PO;
  __device__ const T* Lm() const { return base; }
  __device__ const T* mw() const { return base + MW; }
  __device__ const T* mu() const { return base + MU; }
  __device__ const T* ma() const { return base + MA; }
  __device__ const T* hlo() const { return base + HL; }
  __device__ const T* hhi() const { return base + HH; }
  __device__ const T* lam() const { return base + LA; }
  __device__ const T* S() const { return base + SS; }
  // acc + (mass row r) . in: diagonal plus rank one over the cell of row r,
  // in(c) = element c of the input line
  template <int OFF, class F>
  __device__ T mass(int r, F in, T acc) const {
    const int c0 = ((r + OFF) / NN) * NN;
    T d = ma()[0] * in(c0);
#pragma unroll
    for (int j = 1; j < NN; ++j) d = fma(ma()[j], in(c0 + j), d);
    return fma(mu()[r], d, fma(mw()[r], in(r + OFF), acc));
  }
  __device__ int first() const { return (int)base[C::OPS - 2]; }
  __device__ int last() const { return (int)base[C::OPS - 1]; }
};

// One patch on this CTA (every thread calls; the patch index is CTA-uniform).
// sops: NT operator sets laid out by w3_ops_setup; buf: R1 + R2 + R3 elements.
template <int NN, typename T, bool BND>
__device__ __forceinline__ void w3_patch(const T* sops, T* buf, long long pidx, int colour, const T* __restrict__ b,
                                         T* x, int N, int consistent, const PatchGrid& grid) {
  using C = W3<NN, T, BND>;
  constexpr int P = C::P, PO = C::PO, OFF = C::OFF, LP = C::LP, SP = C::SP, TPP = C::TPP;
  constexpr int ND = NN * NN * NN, P2 = P * P, PO2 = PO * PO, PO3 = PO * PO * PO;
  // threads past TPP take part in the barriers only (their item loops are empty)
  const int tid = threadIdx.x < TPP ? (int)threadIdx.x : (1 << 28);
  int v[3], ty[3] = {0, 0, 0};
  if (BND) {
    int m[3] = {0, 0, 0};
    patch_index<3, true>(grid, pidx, m);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      v[e] = ((colour >> e) & 1) ? 2 * m[e] + 1 : 2 * m[e] + 2;
      ty[e] = (v[e] == 1 ? 1 : 0) | (v[e] == N - 1 ? 2 : 0);
    }
  } else {
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
  const W3View<NN, T, BND> ox{sops + ty[0] * C::OPS}, oy{sops + ty[1] * C::OPS}, oz{sops + ty[2] * C::OPS};
  const long long cb = ((long long)(v[0] - 1) + (long long)N * ((v[1] - 1) + (long long)N * (v[2] - 1))) * ND;
  T* xb = x + cb;
  const T* bb = b + cb;
  const int cs1 = N * ND, cs2 = N * N * ND;
  // global offset (from xb) of patch node (a0, a1, a2), a in [-1, P]
  auto goff = [&](int a0, int a1, int a2) {
    const int o0 = a0 < 0 ? -1 : a0 / NN, o1 = a1 < 0 ? -1 : a1 / NN, o2 = a2 < 0 ? -1 : a2 / NN;
    const int i0 = a0 - o0 * NN, i1 = a1 - o1 * NN, i2 = a2 - o2 * NN;
    return o0 * ND + o1 * cs1 + o2 * cs2 + i0 + NN * i1 + NN * NN * i2;
  };
  const bool exlo[3] = {consistent && (!BND || v[0] >= 2), consistent && (!BND || v[1] >= 2),
                        consistent && (!BND || v[2] >= 2)};
  const bool exhi[3] = {consistent && (!BND || v[0] + 1 <= N - 1), consistent && (!BND || v[1] + 1 <= N - 1),
                        consistent && (!BND || v[2] + 1 <= N - 1)};
  auto inside = [&](int r0, int r1, int r2) {
    return !BND || (r0 >= ox.first() && r0 <= ox.last() && r1 >= oy.first() && r1 <= oy.last() &&
                    r2 >= oz.first() && r2 <= oz.last());
  };

  T* R1 = buf;
  T* R2 = R1 + C::R1;
  T* R3 = R2 + C::R2;
  // R1: X[a2][a1][a0] | HX[s][a2][a1] | HY[s][a2][a0] | HZ[s][a1][a0]
  T* X = R1;
  T* HX = X + P * P2;
  T* HY = HX + 2 * P2;
  T* HZ = HY + 2 * P2;

  // ------------------------------------------------------------------ load
  T bv[C::ITEMS], xo[C::ITEMS];
#pragma unroll
  for (int k = 0; k < C::ITEMS; ++k) {
    const int e = tid + k * TPP;
    bv[k] = T(0);
    xo[k] = T(0);
    if (e < PO3) {
      const int r0 = e % PO, r1 = (e / PO) % PO, r2 = e / PO2;
      if (inside(r0, r1, r2)) {
        const int g = goff(r0 + OFF, r1 + OFF, r2 + OFF);
        bv[k] = __ldg(bb + g);
        xo[k] = xb[g];
      }
    }
  }
  for (int e = tid; e < P * P2 + 6 * P2; e += TPP) {
    T val = T(0);
    if (e < P * P2) {
      const int a0 = e % P, a1 = (e / P) % P, a2 = e / P2;
      val = xb[goff(a0, a1, a2)];
      X[e] = val;
    } else {
      const int h = e - P * P2, face = h / P2, s = face & 1, dir = face >> 1, f = h % P2;
      const int u = f % P, w = f / P;  // x faces: (a1, a2) = (u, w); y: (a0, a2); z: (a0, a1)
      const bool ex = s ? exhi[dir] : exlo[dir];
      if (ex) {
        const int an = s ? P : -1;
        const int g = dir == 0 ? goff(an, u, w) : (dir == 1 ? goff(u, an, w) : goff(u, w, an));
        val = xb[g];
      }
      (dir == 0 ? HX : (dir == 1 ? HY : HZ))[s * P2 + f] = val;
    }
  }
  __syncthreads();

  // ------------------------------------------------------------------ S1 (x)
  // R2: A[a2][a1][r0] | B[a2][a1][r0] | AHy[s][a2][r0] | AHz[s][a1][r0]
  T* A = R2;
  T* B = A + P2 * PO;
  T* AHy = B + P2 * PO;
  T* AHz = AHy + 2 * P * PO;
  for (int e = tid; e < 2 * P2 * PO + 4 * P * PO; e += TPP) {
    if (e < P2 * PO) {  // A
      const int r0 = e % PO, line = e / PO;
      const T* in = X + line * P;
      A[e] = ox.template mass<OFF>(r0, [&](int c) { return in[c]; }, T(0));
    } else if (e < 2 * P2 * PO) {  // B
      const int f = e - P2 * PO, r0 = f % PO, line = f / PO;
      const T* in = X + line * P;
      T s = ox.hlo()[r0] * HX[line] + ox.hhi()[r0] * HX[P2 + line];
#pragma unroll
      for (int c = 0; c < P; ++c) s = fma(ox.Lm()[r0 * LP + c], in[c], s);
      B[f] = s;
    } else {  // M_x on the y faces (lines (s, a2)) and z faces (lines (s, a1))
      const int f = e - 2 * P2 * PO, r0 = f % PO, line = f / PO;  // line in [0, 4P)
      const T* in = (line < 2 * P ? HY : HZ) + (line % (2 * P)) * P;
      AHy[f] = ox.template mass<OFF>(r0, [&](int c) { return in[c]; }, T(0));  // AHy and AHz are contiguous
    }
  }
  __syncthreads();

  // ------------------------------------------------------------------ S2 (y)
  // R3: Cc[a2][r1][r0] | Dd[a2][r1][r0] | CZ[s][r1][r0]
  T* Cc = R3;
  T* Dd = Cc + P * PO2;
  T* CZ = Dd + P * PO2;
  for (int e = tid; e < 2 * P * PO2 + 2 * PO2; e += TPP) {
    if (e < 2 * P * PO2) {
      const bool isD = e >= P * PO2;
      const int f = isD ? e - P * PO2 : e;
      const int r0 = f % PO, r1 = (f / PO) % PO, a2 = f / PO2;
      const T* a = A + a2 * P * PO + r0;  // A[a2][c][r0] at a[c * PO]
      if (!isD) {
        Cc[f] = oy.template mass<OFF>(r1, [&](int c) { return a[c * PO]; }, T(0));
      } else {
        const T* bm = B + a2 * P * PO + r0;
        T s = oy.hlo()[r1] * AHy[a2 * PO + r0] + oy.hhi()[r1] * AHy[P * PO + a2 * PO + r0];
#pragma unroll
        for (int c = 0; c < P; ++c) s = fma(oy.Lm()[r1 * LP + c], a[c * PO], s);
        Dd[f] = oy.template mass<OFF>(r1, [&](int c) { return bm[c * PO]; }, s);
      }
    } else {
      const int f = e - 2 * P * PO2, r0 = f % PO, r1 = (f / PO) % PO, s = f / PO2;
      const T* a = AHz + s * P * PO + r0;
      CZ[f] = oy.template mass<OFF>(r1, [&](int c) { return a[c * PO]; }, T(0));
    }
  }
  __syncthreads();

  // ------------------------------------------------------------------ S3 (z), residual
  T* Rr = R1;  // [r2][r1][r0]
#pragma unroll
  for (int k = 0; k < C::ITEMS; ++k) {
    const int e = tid + k * TPP;
    if (e < PO3) {
      const int r0 = e % PO, r1 = (e / PO) % PO, r2 = e / PO2;
      const int col = r1 * PO + r0;
      T s = oz.hlo()[r2] * CZ[col] + oz.hhi()[r2] * CZ[PO2 + col];
#pragma unroll
      for (int c = 0; c < P; ++c) s = fma(oz.Lm()[r2 * LP + c], Cc[c * PO2 + col], s);
      s = oz.template mass<OFF>(r2, [&](int c) { return Dd[c * PO2 + col]; }, s);
      Rr[e] = inside(r0, r1, r2) ? bv[k] - s : T(0);
    }
  }
  __syncthreads();

  // ------------------------------------------------------------------ fast diagonalisation
  // F1: T1[k2][r1][r0] = sum_j Sz[j][k2] R[j][r1][r0]
  T* T1 = R2;
  for (int e = tid; e < PO3; e += TPP) {
    const int col = e % PO2, k2 = e / PO2;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < PO; ++j) s = fma(oz.S()[j * SP + k2], Rr[j * PO2 + col], s);
    T1[e] = s;
  }
  __syncthreads();
  // F2: T2[k2][k1][r0] = sum_j Sy[j][k1] T1[k2][j][r0]
  T* T2 = R3;
  for (int e = tid; e < PO3; e += TPP) {
    const int r0 = e % PO, k1 = (e / PO) % PO, k2 = e / PO2;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < PO; ++j) s = fma(oy.S()[j * SP + k1], T1[k2 * PO2 + j * PO + r0], s);
    T2[e] = s;
  }
  __syncthreads();
  // F3: T3[k2][k1][k0] = (sum_j Sx[j][k0] T2[k2][k1][j]) / (lx + ly + lz)
  T* T3 = R1;
  for (int e = tid; e < PO3; e += TPP) {
    const int k0 = e % PO, k1 = (e / PO) % PO, k2 = e / PO2;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < PO; ++j) s = fma(ox.S()[j * SP + k0], T2[k2 * PO2 + k1 * PO + j], s);
    T3[e] = s / (ox.lam()[k0] + oy.lam()[k1] + oz.lam()[k2]);
  }
  __syncthreads();
  // G3: U3[k2][k1][r0] = sum_j Sx[r0][j] T3[k2][k1][j]
  T* U3 = R2;
  for (int e = tid; e < PO3; e += TPP) {
    const int r0 = e % PO, rest = e / PO;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < PO; ++j) s = fma(ox.S()[r0 * SP + j], T3[rest * PO + j], s);
    U3[e] = s;
  }
  __syncthreads();
  // G2: U2[k2][r1][r0] = sum_j Sy[r1][j] U3[k2][j][r0]
  T* U2 = R3;
  for (int e = tid; e < PO3; e += TPP) {
    const int r0 = e % PO, r1 = (e / PO) % PO, k2 = e / PO2;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < PO; ++j) s = fma(oy.S()[r1 * SP + j], U3[k2 * PO2 + j * PO + r0], s);
    U2[e] = s;
  }
  __syncthreads();
  // G1: u[r2][r1][r0] = sum_j Sz[r2][j] U2[j][r1][r0];  x += u on V_j
#pragma unroll
  for (int k = 0; k < C::ITEMS; ++k) {
    const int e = tid + k * TPP;
    if (e < PO3) {
      const int r0 = e % PO, r1 = (e / PO) % PO, r2 = e / PO2;
      T s = T(0);
#pragma unroll
      for (int j = 0; j < PO; ++j) s = fma(oz.S()[r2 * SP + j], U2[j * PO2 + r1 * PO + r0], s);
      if (inside(r0, r1, r2)) xb[goff(r0 + OFF, r1 + OFF, r2 + OFF)] = xo[k] + s;
    }
  }
}

// All 8 colours of one smoothing step in one cooperative launch, one patch
// per CTA at a time; a bounded grid barrier separates the colours.
template <int NN, typename T>
struct FW3 {
  using CI = W3<NN, T, false>;
  using CB = W3<NN, T, true>;
  static constexpr int THREADS = CI::TPP > CB::TPP ? CI::TPP : CB::TPP;
  static constexpr size_t BUF = (size_t)i3_max(CI::R1 + CI::R2 + CI::R3, CB::R1 + CB::R2 + CB::R3);
  static constexpr size_t SMEM = sizeof(T) * ((size_t)CI::OPS + 4 * CB::OPS + BUF);
};

template <int NN, typename T>
__global__ void __launch_bounds__(FW3<NN, T>::THREADS, FW3<NN, T>::THREADS <= 512 ? 2 : 1)
    stepw3_kernel(const __grid_constant__ SmoothOps<2 * NN - 2, 2 * NN, T, 1> opsi,
                  const __grid_constant__ SmoothOps<2 * NN, 2 * NN, T, 4> opsb, int reverse, const T* __restrict__ b,
                  T* x, int N, int consistent, long long ndofs, int nrhs, StepGrids grids, unsigned int* bar,
                  int* status) {
  using F = FW3<NN, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* si = reinterpret_cast<T*>(smem_raw);
  T* sb = si + F::CI::OPS;
  T* buf = sb + 4 * F::CB::OPS;
  w3_ops_setup(opsi, si);
  w3_ops_setup(opsb, sb);
  __syncthreads();
  for (int ci = 0; ci < 8; ++ci) {
    const int c = reverse ? 7 - ci : ci;
    const PatchGrid& g = grids.g[c];
    const long long tot = g.n_int + g.n_bnd;
    for (long long q = blockIdx.x; q < tot * nrhs; q += gridDim.x) {
      const long long r = q / tot, ch = q % tot;
      if (ch < g.n_int)
        w3_patch<NN, T, false>(si, buf, ch, c, b + r * ndofs, x + r * ndofs, N, consistent, g);
      else
        w3_patch<NN, T, true>(sb, buf, ch - g.n_int, c, b + r * ndofs, x + r * ndofs, N, consistent, g);
      __syncthreads();  // the next patch reuses the buffers
    }
    if (ci + 1 < 8 && !grid_barrier(bar, status, gridDim.x)) return;
  }
}

// Fused smoothing step with the wide patch kernel (3D); as many CTAs as are
// resident (each loops over the patches of a colour), cudaErrorNotSupported
// if the kernel does not fit.
template <int NN, typename T>
cudaError_t stepw3_dispatch(const sipg_handle* h, int level, int reverse, const T* b, T* x, cudaStream_t s) {
  using F = FW3<NN, T>;
  if (F::SMEM > 227 * 1024 || h->num_sms <= 0) return cudaErrorNotSupported;
  int max_active = 0;
  cudaError_t e0 = smem_opt_in_occupancy(reinterpret_cast<const void*>(stepw3_kernel<NN, T>), F::THREADS,
                                         (int)F::SMEM, &max_active);
  if (e0 != cudaSuccess) return e0;
  if (max_active <= 0) return cudaErrorNotSupported;
  const int N = h->lv[level].N;
  StepGrids sg;
  long long most = 0;
  for (int c = 0; c < 8; ++c) {
    sg.g[c] = make_grid(3, N, c);
    most = std::max(most, (sg.g[c].n_int + sg.g[c].n_bnd) * (long long)h->prm.nrhs);
  }
  const long long resident = (long long)max_active * h->num_sms;
  SmoothOps<2 * NN - 2, 2 * NN, T, 1> opsi;
  SmoothOps<2 * NN, 2 * NN, T, 4> opsb;
  make_ops<2 * NN - 2, 2 * NN, false, T>(h->hcst<T>(level), 0, opsi.t[0]);
  for (int t = 0; t < 4; ++t) make_ops<2 * NN, 2 * NN, true, T>(h->hcst<T>(level), t, opsb.t[t]);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::max<long long>(1, std::min(most, resident)));
  cfg.blockDim = dim3(F::THREADS);
  cfg.dynamicSmemBytes = F::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  unsigned int* bar = reinterpret_cast<unsigned int*>(h->ws + h->off_sync);
  int* status = reinterpret_cast<int*>(h->ws + h->off_sync + 2 * sizeof(unsigned int));
  return cudaLaunchKernelEx(&cfg, stepw3_kernel<NN, T>, opsi, opsb, reverse, b, x, N,
                            h->prm.smoother == SIPG_SMOOTHER_CONSISTENT ? 1 : 0, (long long)h->lv[level].ndofs,
                            h->prm.nrhs, sg, bar, status);
}
