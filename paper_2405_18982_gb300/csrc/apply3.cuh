// 3D operator apply organised by coarse cells, with the residual restriction
// fused in (Sec. 2.2 operator; Sec. 3 restriction = transpose of the
// canonical embedding).  Included by apply.cu.
//
// Same arithmetic as apply_kernel: per cell
//   (A x)_c = M_z M_y Z_0 + M_z M_x Z_1 + M_y M_x Z_2,
//   Z_e = Lself[type_e] x_c + (rank-two couplings to the two neighbours along e),
// evaluated as Z_e (three normal sweeps), then
//   B1 (x-lines)  U = M_x Z_1,  V = M_x Z_2
//   B2 (y-lines)  T = M_y Z_0 + U,  W = M_y V
//   B3 (z-lines)  A x = M_z T + W.
// Layout for GB300: a CTA owns G groups of the 2 x 2 x 2 fine cells below a
// coarse cell, n^2 threads per cell (one line per direction); the cell tiles
// are staged once in shared memory with odd line strides (conflict-free line
// reads in all three directions); the 1D operators are kernel parameters
// (constant-bank operands, the boundary type picked by a branch that only
// diverges in warps holding a boundary cell); of the six neighbour lines
// of a cell three belong to sibling cells of the group (read from shared
// memory), the others are read from global memory.  With MODE_RESTRICT the
// residual b - A x stays in shared memory and the group restricts it to its
// coarse cell (x, y, z sweeps of Pc^T), so the fine residual is never written.

enum { A3_APPLY = 0, A3_RESIDUAL = 1, A3_RESTRICT = 2 };

template <int NN, typename T>
struct A3Ops {
  T Ls[3][NN * NN];  // Lself of types 0 (interior), 1 (low face on boundary), 2 (high)
  T alo[NN], glo[NN], ahi[NN], ghi[NN];
  T Mw[NN], Ma[NN], Mu[NN];  // mass = diag(Mw) + Mu Ma^T (GLL: diagonal plus rank one)
  T PcT[2][NN * NN];  // PcT[o][j * NN + i] = Pc[o][i][j]
};

// o = M v for the mass as diagonal plus rank one (3n FMAs instead of n^2)
template <int NN, typename T>
__device__ __forceinline__ void a3_mass(const A3Ops<NN, T>& op, const T (&v)[NN], T (&o)[NN]) {
  T s = op.Ma[0] * v[0];
#pragma unroll
  for (int j = 1; j < NN; ++j) s = fma(op.Ma[j], v[j], s);
#pragma unroll
  for (int i = 0; i < NN; ++i) o[i] = fma(op.Mu[i], s, op.Mw[i] * v[i]);
}

template <int NN, typename T>
struct A3 {
  static constexpr int XS = NN | 1;       // odd stride of x-lines
  static constexpr int PZ = NN * XS;      // stride of z-planes
  static constexpr int CSZ = i3_pad32(NN * PZ, 16);  // cell tile stride
  static constexpr int G = NN <= 4 ? 2 : 1;          // coarse-cell groups per CTA
  static constexpr int CELLS = 8 * G;
  static constexpr int NL = NN * NN;                 // lines per direction
  static constexpr int THREADS = CELLS * NL;
  static constexpr size_t SMEM = (size_t)4 * CELLS * CSZ * sizeof(T);  // X, Z0, Z1, Z2
};

template <int NN, typename T>
__device__ __forceinline__ int a3_off(int i0, int i1, int i2) {
  return A3<NN, T>::PZ * i2 + A3<NN, T>::XS * i1 + i0;
}

// o = Ls[ty] v for the boundary type of the line's cell
template <int NN, typename T>
__device__ __forceinline__ void a3_self(const A3Ops<NN, T>& op, int ty, const T (&v)[NN], T (&o)[NN]) {
  if (ty == 0)
    matvec_line<NN>(op.Ls[0], v, o);
  else if (ty == 1)
    matvec_line<NN>(op.Ls[1], v, o);
  else
    matvec_line<NN>(op.Ls[2], v, o);
}

template <int NN, typename T, int MODE>
__global__ void __launch_bounds__(A3<NN, T>::THREADS)
    apply3_kernel(const __grid_constant__ A3Ops<NN, T> op, const T* __restrict__ bvec, const T* __restrict__ x,
                  T* y, int N, long long ndofs, long long ndofs_out) {
  using C = A3<NN, T>;
  constexpr int ND = NN * NN * NN, NL = C::NL, CSZ = C::CSZ, G = C::G, CELLS = C::CELLS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Xs = reinterpret_cast<T*>(smem_raw);
  T* Z0 = Xs + CELLS * CSZ;
  T* Z1 = Z0 + CELLS * CSZ;
  T* Z2 = Z1 + CELLS * CSZ;

  const long long col = (long long)blockIdx.y;
  x += col * ndofs;
  if (MODE != A3_APPLY) bvec += col * ndofs;
  y += col * ndofs_out;
  const int Nc = N / 2, rowb = Nc / G;  // CTAs per row of coarse cells
  const int bx = blockIdx.x;
  const int C0 = (bx % rowb) * G, C1 = (bx / rowb) % Nc, C2 = bx / (rowb * Nc);
  const int tid = threadIdx.x;
  const int l = tid % NL, q = tid / NL;
  const int l0 = l % NN, l1 = l / NN;
  const int g = q / 8, o = q % 8;
  const int f[3] = {2 * (C0 + g) + (o & 1), 2 * C1 + ((o >> 1) & 1), 2 * C2 + (o >> 2)};
  const long long cell = (long long)f[0] + (long long)N * (f[1] + (long long)N * f[2]);
  const long long cstr[3] = {1, (long long)N, (long long)N * N};
  T* Xq = Xs + q * CSZ;

  // ---------------------------------------------- stage the CTA's cells (x-lines)
  for (int e = tid; e < CELLS * NL; e += C::THREADS) {
    const int qq = e / NL, ll = e % NL, oo = qq % 8, gg = qq / 8;
    const long long cc = (long long)(2 * (C0 + gg) + (oo & 1)) +
                         (long long)N * ((2 * C1 + ((oo >> 1) & 1)) + (long long)N * (2 * C2 + (oo >> 2)));
    T v[NN];
    i3_ldrun<NN, run_vw<NN, T>()>(x + cc * ND + ll * NN, v);
    T* d = Xs + qq * CSZ + a3_off<NN, T>(0, ll % NN, ll / NN);
#pragma unroll
    for (int i = 0; i < NN; ++i) d[i] = v[i];
  }
  __syncthreads();

  // ---------------------------------------------- normal sweeps Z_e
  // line of this thread along e: e = 0 (i1, i2) = (l0, l1); e = 1 (i0, i2);
  // e = 2 (i0, i1).  Element j of the line sits at base + j * step in a tile
  // and at gbase + j * gstep in a cell of the global vector.
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    int base, step, gbase, gstep;
    if (e == 0) { base = a3_off<NN, T>(0, l0, l1); step = 1; gbase = NN * l0 + NN * NN * l1; gstep = 1; }
    else if (e == 1) { base = a3_off<NN, T>(l0, 0, l1); step = C::XS; gbase = l0 + NN * NN * l1; gstep = NN; }
    else { base = a3_off<NN, T>(l0, l1, 0); step = C::PZ; gbase = l0 + NN * l1; gstep = NN * NN; }
    T v[NN], z[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) v[j] = Xq[base + j * step];
    const int fe = f[e], oe = (o >> e) & 1;
    const int ty = fe == 0 ? 1 : (fe == N - 1 ? 2 : 0);
    a3_self<NN, T>(op, ty, v, z);
    // neighbour below along e: node n-1 value and the dot with alo
    if (fe > 0) {
      T w[NN];
      if (oe == 1) {  // sibling in the group
        const T* s = Xs + (q ^ (1 << e)) * CSZ + base;
#pragma unroll
        for (int j = 0; j < NN; ++j) w[j] = s[j * step];
      } else {
        const T* s = x + (cell - cstr[e]) * ND + gbase;
        if (e == 0) {
          i3_ldrun<NN, run_vw<NN, T>()>(s, w);
        } else {
#pragma unroll
          for (int j = 0; j < NN; ++j) w[j] = __ldg(s + j * gstep);
        }
      }
      T sdot = T(0);
#pragma unroll
      for (int j = 0; j < NN; ++j) sdot = fma(op.alo[j], w[j], sdot);
      z[0] += sdot;
#pragma unroll
      for (int i = 0; i < NN; ++i) z[i] = fma(op.glo[i], w[NN - 1], z[i]);
    }
    if (fe < N - 1) {
      T w[NN];
      if (oe == 0) {
        const T* s = Xs + (q ^ (1 << e)) * CSZ + base;
#pragma unroll
        for (int j = 0; j < NN; ++j) w[j] = s[j * step];
      } else {
        const T* s = x + (cell + cstr[e]) * ND + gbase;
        if (e == 0) {
          i3_ldrun<NN, run_vw<NN, T>()>(s, w);
        } else {
#pragma unroll
          for (int j = 0; j < NN; ++j) w[j] = __ldg(s + j * gstep);
        }
      }
      T sdot = T(0);
#pragma unroll
      for (int j = 0; j < NN; ++j) sdot = fma(op.ahi[j], w[j], sdot);
      z[NN - 1] += sdot;
#pragma unroll
      for (int i = 0; i < NN; ++i) z[i] = fma(op.ghi[i], w[0], z[i]);
    }
    T* Zq = (e == 0 ? Z0 : (e == 1 ? Z1 : Z2)) + q * CSZ + base;
#pragma unroll
    for (int j = 0; j < NN; ++j) Zq[j * step] = z[j];
  }
  __syncthreads();

  // ---------------------------------------------- B1: x-lines  U = M Z1 (into X), V = M Z2
  {
    const int base = a3_off<NN, T>(0, l0, l1);
    T v[NN], u[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) v[j] = Z1[q * CSZ + base + j];
    a3_mass<NN, T>(op, v, u);
#pragma unroll
    for (int j = 0; j < NN; ++j) Xq[base + j] = u[j];
#pragma unroll
    for (int j = 0; j < NN; ++j) v[j] = Z2[q * CSZ + base + j];
    a3_mass<NN, T>(op, v, u);
#pragma unroll
    for (int j = 0; j < NN; ++j) Z2[q * CSZ + base + j] = u[j];
  }
  __syncthreads();
  // ---------------------------------------------- B2: y-lines  T = M Z0 + U (into Z0), W = M V (into Z1)
  {
    const int base = a3_off<NN, T>(l0, 0, l1);
    constexpr int st = C::XS;
    T v[NN], t[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) v[j] = Z0[q * CSZ + base + j * st];
    a3_mass<NN, T>(op, v, t);
#pragma unroll
    for (int j = 0; j < NN; ++j) Z0[q * CSZ + base + j * st] = t[j] + Xq[base + j * st];
#pragma unroll
    for (int j = 0; j < NN; ++j) v[j] = Z2[q * CSZ + base + j * st];
    a3_mass<NN, T>(op, v, t);
#pragma unroll
    for (int j = 0; j < NN; ++j) Z1[q * CSZ + base + j * st] = t[j];
  }
  __syncthreads();
  // ---------------------------------------------- B3: z-lines  A x = M T + W
  {
    const int base = a3_off<NN, T>(l0, l1, 0);
    constexpr int st = C::PZ;
    T v[NN], r[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) v[j] = Z0[q * CSZ + base + j * st];
    a3_mass<NN, T>(op, v, r);
#pragma unroll
    for (int j = 0; j < NN; ++j) r[j] += Z1[q * CSZ + base + j * st];
    const long long gb = cell * ND + l0 + NN * l1;
    if (MODE == A3_APPLY) {
#pragma unroll
      for (int j = 0; j < NN; ++j) y[gb + j * NN * NN] = r[j];
    } else {
#pragma unroll
      for (int j = 0; j < NN; ++j) r[j] = __ldg(bvec + gb + j * NN * NN) - r[j];
      if (MODE == A3_RESIDUAL) {
#pragma unroll
        for (int j = 0; j < NN; ++j) y[gb + j * NN * NN] = r[j];
      } else {
#pragma unroll
        for (int j = 0; j < NN; ++j) Xq[base + j * st] = r[j];
      }
    }
  }
  if (MODE != A3_RESTRICT) return;
  __syncthreads();

  // ---------------------------------------------- restriction of the group's residual
  // R1 (x): U'[g][o12] = sum_o0 Pc[o0]^T r_(o0, o12)   (4 NL lines per group)
  const int tg = tid % (8 * NL);  // thread within its group
  {
    const int oo = tg / NL;  // o12 = oo for oo < 4
    if (oo < 4) {
      const int base = a3_off<NN, T>(0, l0, l1);
      T acc[NN];
#pragma unroll
      for (int i = 0; i < NN; ++i) acc[i] = T(0);
#pragma unroll
      for (int o0 = 0; o0 < 2; ++o0) {
        const T* src = Xs + (8 * g + o0 + 2 * oo) * CSZ + base;
        T v[NN];
#pragma unroll
        for (int j = 0; j < NN; ++j) v[j] = src[j];
#pragma unroll
        for (int i = 0; i < NN; ++i)
#pragma unroll
          for (int j = 0; j < NN; ++j) acc[i] = fma(op.PcT[o0][i * NN + j], v[j], acc[i]);
      }
      T* dst = Z2 + (8 * g + oo) * CSZ + base;
#pragma unroll
      for (int i = 0; i < NN; ++i) dst[i] = acc[i];
    }
  }
  __syncthreads();
  // R2 (y): V'[g][o2] = sum_o1 Pc[o1]^T U'[o1 + 2 o2]   (2 NL lines per group)
  {
    const int oo = tg / NL;  // o2 for oo < 2
    if (oo < 2) {
      const int base = a3_off<NN, T>(l0, 0, l1);
      constexpr int st = C::XS;
      T acc[NN];
#pragma unroll
      for (int i = 0; i < NN; ++i) acc[i] = T(0);
#pragma unroll
      for (int o1 = 0; o1 < 2; ++o1) {
        const T* src = Z2 + (8 * g + o1 + 2 * oo) * CSZ + base;
        T v[NN];
#pragma unroll
        for (int j = 0; j < NN; ++j) v[j] = src[j * st];
#pragma unroll
        for (int i = 0; i < NN; ++i)
#pragma unroll
          for (int j = 0; j < NN; ++j) acc[i] = fma(op.PcT[o1][i * NN + j], v[j], acc[i]);
      }
      T* dst = Z1 + (8 * g + oo) * CSZ + base;
#pragma unroll
      for (int i = 0; i < NN; ++i) dst[i * st] = acc[i];
    }
  }
  __syncthreads();
  // R3 (z): r_coarse = sum_o2 Pc[o2]^T V'[o2]   (NL lines per group)
  if (tg < NL) {
    const int base = a3_off<NN, T>(l0, l1, 0);
    constexpr int st = C::PZ;
    T acc[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) acc[i] = T(0);
#pragma unroll
    for (int o2 = 0; o2 < 2; ++o2) {
      const T* src = Z1 + (8 * g + o2) * CSZ + base;
      T v[NN];
#pragma unroll
      for (int j = 0; j < NN; ++j) v[j] = src[j * st];
#pragma unroll
      for (int i = 0; i < NN; ++i)
#pragma unroll
        for (int j = 0; j < NN; ++j) acc[i] = fma(op.PcT[o2][i * NN + j], v[j], acc[i]);
    }
    const long long cc = (long long)(C0 + g) + (long long)Nc * (C1 + (long long)Nc * C2);
    T* dst = y + cc * ND + l0 + NN * l1;
#pragma unroll
    for (int i = 0; i < NN; ++i) dst[i * NN * NN] = acc[i];
  }
}

template <int NN, typename T>
A3Ops<NN, T> a3_ops(const LevelConst<T>& lc) {
  A3Ops<NN, T> op;
  for (int t = 0; t < 3; ++t)
    for (int i = 0; i < NN; ++i)
      for (int j = 0; j < NN; ++j) op.Ls[t][i * NN + j] = lc.Lself[t][i][j];
  for (int i = 0; i < NN; ++i) {
    op.alo[i] = lc.alo[i];
    op.glo[i] = lc.glo[i];
    op.ahi[i] = lc.ahi[i];
    op.ghi[i] = lc.ghi[i];
    op.Mw[i] = lc.Mw[i];
    op.Ma[i] = lc.Ma[i];
    op.Mu[i] = lc.Mu[i];
    for (int j = 0; j < NN; ++j) {
      op.PcT[0][i * NN + j] = lc.Pc[0][j][i];
      op.PcT[1][i * NN + j] = lc.Pc[1][j][i];
    }
  }
  return op;
}

// 3D apply / residual / restricted residual on `level` (N even); out is the
// fine vector, or the coarse vector of level - 1 for A3_RESTRICT.
template <int NN, typename T>
cudaError_t launch_apply3(const sipg_handle* h, int level, int mode, const T* b, const T* x, T* out,
                          cudaStream_t s) {
  using C = A3<NN, T>;
  const LevelInfo& li = h->lv[level];
  const int N = li.N;
  if (N % 2 != 0 || (N / 2) % C::G != 0) return cudaErrorNotSupported;
  const A3Ops<NN, T> op = a3_ops<NN, T>(h->hcst<T>(level));
  const long long nblk = (long long)(N / 2 / C::G) * (N / 2) * (N / 2);
  dim3 grid((unsigned)nblk, h->prm.nrhs);
  const long long nout = mode == A3_RESTRICT ? (long long)h->lv[level - 1].ndofs : (long long)li.ndofs;
  cudaError_t e = cudaSuccess;
  auto go = [&](auto kern, int) {
    e = smem_opt_in(reinterpret_cast<const void*>(kern), (int)C::SMEM);
    if (e != cudaSuccess) return;
    kern<<<grid, C::THREADS, C::SMEM, s>>>(op, b, x, out, N, (long long)li.ndofs, nout);
    e = cudaGetLastError();
  };
  if (mode == A3_APPLY) go(apply3_kernel<NN, T, A3_APPLY>, 0);
  else if (mode == A3_RESIDUAL) go(apply3_kernel<NN, T, A3_RESIDUAL>, 1);
  else go(apply3_kernel<NN, T, A3_RESTRICT>, 2);
  return e;
}
