// Device-side FP64 level setup: 1D Q_k Lagrange basis on Gauss-Lobatto points
// (Appendix A), 1D SIPG operator blocks (Sec. 2.1-2.2), vertex-patch 1D
// matrices and their generalised eigenpairs L S = M S Lambda (Sec. 3.2, Eq.
// fast_inverse), the coarsest level's global 1D eigenpairs and the transfer
// matrices of the canonical embedding (Sec. 3).  One CTA per level; the
// eigenproblems are small (<= 16 for patches, <= 64 for the coarse level) and
// are solved by Cholesky reduction to a standard problem and cyclic Jacobi
// rotations (Golub & Van Loan, Matrix Computations, Sec. 8.5).
#include <math.h>

#include "sipg_internal.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

// P_m(x) and P_{m-1}(x) by the three-term recurrence (m >= 1).
__device__ void legendre_pair(int m, double x, double& p, double& pm1) {
  double a = 1.0, b = x;
  for (int j = 2; j <= m; ++j) {
    double c = ((2.0 * j - 1.0) * x * b - (j - 1.0) * a) / j;
    a = b;
    b = c;
  }
  p = b;
  pm1 = a;
}

// Gauss-Lobatto points on [0,1]: +-1 and the roots of P_k', found by Newton
// steps on q(x) = (1-x^2) P_k'(x) = k (P_{k-1} - x P_k), q' = -k(k+1) P_k.
__device__ void gauss_lobatto_nodes(int k, double* xi) {
  for (int i = 0; i <= k; ++i) {
    double x = -cos(kPi * i / k);
    if (i > 0 && i < k) {
      for (int it = 0; it < 100; ++it) {
        double p, pm1;
        legendre_pair(k, x, p, pm1);
        double dx = (x * p - pm1) / ((k + 1.0) * p);
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
    }
    xi[i] = 0.5 * (x + 1.0);
  }
  xi[0] = 0.0;
  xi[k] = 1.0;
}

// m-point Gauss-Legendre rule on [0,1]: Newton on P_m, weights
// 2 / ((1 - x^2) P_m'(x)^2) on [-1,1].
__device__ void gauss_rule(int m, double* x, double* w) {
  for (int i = 0; i < m; ++i) {
    double t = cos(kPi * (i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p, pm1;
      legendre_pair(m, t, p, pm1);
      dp = m * (t * p - pm1) / (t * t - 1.0);
      double dt = p / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double p, pm1;
    legendre_pair(m, t, p, pm1);
    dp = m * (t * p - pm1) / (t * t - 1.0);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // half of the [-1,1] weight
  }
}

// Lagrange basis on `xi` (n points) at x: phi_j(x) = prod_{m!=j} (x-xi_m)/(xi_j-xi_m).
__device__ void lagrange_at(int n, const double* xi, double x, double* phi) {
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) v *= (x - xi[m]) / (xi[j] - xi[m]);
    phi[j] = v;
  }
}

// Cholesky B = C C^T (lower, row-major, leading dimension ld).
__device__ bool cholesky(int m, const double* B, double* C, int ld) {
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < m; ++i) C[i * ld + j] = 0.0;
  }
  for (int j = 0; j < m; ++j) {
    double s = B[j * ld + j];
    for (int p = 0; p < j; ++p) s -= C[j * ld + p] * C[j * ld + p];
    if (!(s > 0.0)) return false;
    double d = sqrt(s);
    C[j * ld + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double t = B[i * ld + j];
      for (int p = 0; p < j; ++p) t -= C[i * ld + p] * C[j * ld + p];
      C[i * ld + j] = t / d;
    }
  }
  return true;
}

// Generalised symmetric-definite eigenproblem A S = B S Lambda, S^T B S = I.
// Work arrays W1, W2 of m x m (ld).  Returns false if B is not SPD.
__device__ bool generalised_eigen(int m, const double* A, const double* B, int ld, double* S,
                                  double* lam, double* W1, double* W2) {
  double* C = W1;
  if (!cholesky(m, B, C, ld)) return false;
  // Y = C^{-1} A
  double* Y = W2;
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < m; ++i) {
      double t = A[i * ld + c];
      for (int p = 0; p < i; ++p) t -= C[i * ld + p] * Y[p * ld + c];
      Y[i * ld + c] = t / C[i * ld + i];
    }
  // Z = C^{-1} Y^T = C^{-1} A C^{-T}
  double* Z = S;
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < m; ++i) {
      double t = Y[c * ld + i];
      for (int p = 0; p < i; ++p) t -= C[i * ld + p] * Z[p * ld + c];
      Z[i * ld + c] = t / C[i * ld + i];
    }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      double a = 0.5 * (Z[i * ld + j] + Z[j * ld + i]);
      Z[i * ld + j] = a;
      Z[j * ld + i] = a;
    }
  // cyclic Jacobi: Z <- J^T Z J, Q <- Q J
  double* Q = W2;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Q[i * ld + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double z2 = Z[i * ld + j] * Z[i * ld + j];
        tot += z2;
        if (i != j) off += z2;
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        double apq = Z[p * ld + q];
        if (apq == 0.0) continue;
        double tau = (Z[q * ld + q] - Z[p * ld + p]) / (2.0 * apq);
        double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        for (int r = 0; r < m; ++r) {
          double zp = Z[r * ld + p], zq = Z[r * ld + q];
          Z[r * ld + p] = c * zp - s * zq;
          Z[r * ld + q] = s * zp + c * zq;
        }
        for (int r = 0; r < m; ++r) {
          double zp = Z[p * ld + r], zq = Z[q * ld + r];
          Z[p * ld + r] = c * zp - s * zq;
          Z[q * ld + r] = s * zp + c * zq;
        }
        for (int r = 0; r < m; ++r) {
          double qp = Q[r * ld + p], qq = Q[r * ld + q];
          Q[r * ld + p] = c * qp - s * qq;
          Q[r * ld + q] = s * qp + c * qq;
        }
      }
  }
  for (int i = 0; i < m; ++i) lam[i] = Z[i * ld + i];
  // S = C^{-T} Q (back substitution with C^T)
  for (int c = 0; c < m; ++c)
    for (int i = m - 1; i >= 0; --i) {
      double t = Q[i * ld + c];
      for (int p = i + 1; p < m; ++p) t -= C[p * ld + i] * S[p * ld + c];
      S[i * ld + c] = t / C[i * ld + i];
    }
  return true;
}

struct Basis1D {
  double xi[SIPG_MAXN];
  double lead[SIPG_MAXN];          // leading coefficient of phi_j: 1 / prod_{m != j} (xi_j - xi_m)
  double D[SIPG_MAXN][SIPG_MAXN];  // D[i][j] = phi_j'(xi_i) (reference)
  double Mhat[SIPG_MAXN][SIPG_MAXN];
  double Khat[SIPG_MAXN][SIPG_MAXN];
  double Pc[2][SIPG_MAXN][SIPG_MAXN];
};

__device__ void build_basis(int k, Basis1D& B) {
  const int n = k + 1;
  gauss_lobatto_nodes(k, B.xi);
  // barycentric weights and the differentiation matrix on the nodes
  double bw[SIPG_MAXN];
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) p *= (B.xi[j] - B.xi[m]);
    bw[j] = 1.0 / p;
    B.lead[j] = bw[j];
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      double v = (bw[j] / bw[i]) / (B.xi[i] - B.xi[j]);
      B.D[i][j] = v;
      diag -= v;
    }
    B.D[i][i] = diag;
  }
  // exact mass and stiffness with the (k+1)-point Gauss rule
  double gx[SIPG_MAXN], gw[SIPG_MAXN];
  gauss_rule(n, gx, gw);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) B.Mhat[i][j] = B.Khat[i][j] = 0.0;
  for (int q = 0; q < n; ++q) {
    double phi[SIPG_MAXN], dphi[SIPG_MAXN];
    lagrange_at(n, B.xi, gx[q], phi);
    // phi_j' has degree k-1 <= k: interpolate it on the nodes
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += phi[i] * B.D[i][j];
      dphi[j] = s;
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        B.Mhat[i][j] += gw[q] * phi[i] * phi[j];
        B.Khat[i][j] += gw[q] * dphi[i] * dphi[j];
      }
  }
  // canonical embedding: fine node i of child o sits at (o + xi_i)/2 of the parent
  for (int o = 0; o < 2; ++o)
    for (int i = 0; i < n; ++i) {
      double phi[SIPG_MAXN];
      lagrange_at(n, B.xi, 0.5 * (o + B.xi[i]), phi);
      for (int j = 0; j < n; ++j) B.Pc[o][i][j] = phi[j];
    }
}

// 1D blocks of kappa * a_h on a uniform mesh with cell size h (Sec. 2.1 in 1D):
// interior face between c-1 (minus) and c (plus), [[u]] = u^- - u^+,
// {u'} = (u'^- + u'^+)/2; boundary faces [[u]] = u n, {u'} = u'.
__device__ void level_blocks(const Basis1D& B, int k, double h, double gamma, double kappa,
                             bool penalty_only, double self[3][SIPG_MAXN][SIPG_MAXN],
                             double* alo, double* glo, double* ahi, double* ghi) {
  const int n = k + 1;
  const double c1 = penalty_only ? 0.0 : 1.0;   // switches the flux terms off
  const double g = penalty_only ? 1.0 : gamma;
  const double kst = penalty_only ? 0.0 : 1.0;
  double d0[SIPG_MAXN], d1[SIPG_MAXN];           // reference phi_j'(0), phi_j'(1)
  for (int j = 0; j < n; ++j) {
    d0[j] = B.D[0][j];
    d1[j] = B.D[k][j];
  }
  const double ih = 1.0 / h;
  for (int t = 0; t < 3; ++t)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = kst * B.Khat[i][j] * ih;
        // low face (xi = 0): interior for t != 1, boundary for t == 1
        double fl = (t == 1) ? 1.0 : 0.5;      // weight of the mean (1 on the boundary)
        v += g * (i == 0) * (j == 0) + c1 * fl * ih * (d0[j] * (i == 0) + d0[i] * (j == 0));
        // high face (xi = 1): interior for t != 2, boundary for t == 2
        double fh = (t == 2) ? 1.0 : 0.5;
        v += g * (i == k) * (j == k) - c1 * fh * ih * (d1[j] * (i == k) + d1[i] * (j == k));
        self[t][i][j] = kappa * v;
      }
  // neighbours: l_lo[i][j] = delta_{i0} alo[j] + delta_{jk} glo[i]
  //             l_hi[i][j] = delta_{ik} ahi[j] + delta_{j0} ghi[i]
  for (int j = 0; j < n; ++j) {
    alo[j] = kappa * (-g * (j == k) + c1 * 0.5 * ih * d1[j]);
    glo[j] = kappa * (-c1 * 0.5 * ih * d0[j]);
    ahi[j] = kappa * (-g * (j == 0) - c1 * 0.5 * ih * d0[j]);
    ghi[j] = kappa * (c1 * 0.5 * ih * d1[j]);
  }
}

__device__ double l_lo_entry(const LevelConst<double>& c, int k, int i, int j) {
  return (i == 0 ? c.alo[j] : 0.0) + (j == k ? c.glo[i] : 0.0);
}
__device__ double l_hi_entry(const LevelConst<double>& c, int k, int i, int j) {
  return (i == k ? c.ahi[j] : 0.0) + (j == 0 ? c.ghi[i] : 0.0);
}

__global__ void setup_levels_kernel(LevelConst<double>* out, int k, int N_finest, int n_levels,
                                    double kappa, double eta, int smoother, double* scratch,
                                    int* status) {
  const bool paper_residual = smoother == SIPG_SMOOTHER_PAPER;
  const int l = blockIdx.x;
  const int L = n_levels - 1;
  const int n = k + 1;
  const int N = N_finest >> (L - l);
  LevelConst<double>& c = out[l];
  __shared__ Basis1D B;
  if (threadIdx.x == 0) {
    build_basis(k, B);
    const double h = 1.0 / N;
    const double gamma = eta * k * (k + 1.0) * (2.0 / h);
    c.N = N;
    c.n = n;
    c.m0 = (l == 0) ? N * n : 0;
    c.pad_ = 0;
    c.h = h;
    c.gamma = gamma;
    level_blocks(B, k, h, gamma, kappa, false, c.Lself, c.alo, c.glo, c.ahi, c.ghi);
    level_blocks(B, k, h, gamma, kappa, true, c.Pself, c.palo, c.pglo, c.pahi, c.pghi);
    for (int i = 0; i < n; ++i) {
      c.nodes[i] = B.xi[i];
      for (int j = 0; j < n; ++j) {
        c.M[i][j] = h * B.Mhat[i][j];
        c.Pc[0][i][j] = B.Pc[0][i][j];
        c.Pc[1][i][j] = B.Pc[1][i][j];
      }
    }
    // rank-one part e a a^T of Mhat from its first and last nodes' coupling
    // (the largest |a_0 a_k|), then the diagonal remainder (the GLL weights)
    const double e = B.Mhat[0][n - 1] / (B.lead[0] * B.lead[n - 1]);
    for (int i = 0; i < n; ++i) {
      c.Ma[i] = B.lead[i];
      c.Mu[i] = h * e * B.lead[i];
      c.Mw[i] = h * (B.Mhat[i][i] - e * B.lead[i] * B.lead[i]);
    }
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < 4) {
    // 1D patch around an interior vertex: cells (v-1, v); type bit 0: v-1 is
    // the first cell (low end on the boundary), bit 1: v is the last cell.
    const int P = 2 * n;
    const int tl = (t & 1) ? 1 : 0;
    const int tr = (t & 2) ? 2 : 0;
    double Lp[SIPG_MAXP][SIPG_MAXP], Mp[SIPG_MAXP][SIPG_MAXP];
    for (int a = 0; a < P; ++a)
      for (int b = 0; b < P; ++b) {
        int oa = a / n, ia = a % n, ob = b / n, ib = b % n;
        double lv, mv = 0.0;
        if (oa == 0 && ob == 0) lv = c.Lself[tl][ia][ib];
        else if (oa == 1 && ob == 1) lv = c.Lself[tr][ia][ib];
        else if (oa == 0) lv = l_hi_entry(c, k, ia, ib);    // test left cell, trial right
        else lv = l_lo_entry(c, k, ia, ib);                 // test right cell, trial left
        if (oa == ob) mv = c.M[ia][ib];
        Lp[a][b] = lv;
        Mp[a][b] = mv;
      }
    const int first = (t & 1) ? 0 : 1;
    const int last = (t & 2) ? P - 1 : P - 2;
    const int p = last - first + 1;
    c.p[t] = p;
    c.first[t] = first;
    for (int r = 0; r < SIPG_MAXP; ++r)
      for (int s = 0; s < SIPG_MAXPE; ++s) {
        c.Lr[t][r][s] = 0.0;
        c.Mr[t][r][s] = 0.0;
      }
    for (int r = 0; r < p; ++r) {
      const int a = first + r;
      for (int b = 0; b < P; ++b) {
        c.Lr[t][r][1 + b] = Lp[a][b];
        c.Mr[t][r][1 + b] = Mp[a][b];
      }
      // halo: face node k of cell v-2 (low) and node 0 of cell v+1 (high)
      double hlo = (!(t & 1) && a < n) ? l_lo_entry(c, k, a, k) : 0.0;
      double hhi = (!(t & 2) && a >= n) ? l_hi_entry(c, k, a - n, 0) : 0.0;
      if (paper_residual) {
        // Dirichlet kernel (Sec. 3.1): the last face term -[[u]].{grad v} of
        // a patch-boundary face inside the domain is left out.  For rows in
        // V_j it couples only the two face nodes, with opposite coefficients
        // (the jump of a constant vanishes), so leaving it out adds the halo
        // coefficient to the patch end node's column and drops the halo.
        c.Lr[t][r][1] += hlo;
        c.Lr[t][r][P] += hhi;
        hlo = hhi = 0.0;
      }
      c.Lr[t][r][0] = hlo;
      c.Lr[t][r][P + 1] = hhi;
    }
    double As[SIPG_MAXP * SIPG_MAXP], Bs[SIPG_MAXP * SIPG_MAXP];
    double Ss[SIPG_MAXP * SIPG_MAXP], W1[SIPG_MAXP * SIPG_MAXP], W2[SIPG_MAXP * SIPG_MAXP];
    double lam[SIPG_MAXP];
    for (int r = 0; r < p; ++r)
      for (int s = 0; s < p; ++s) {
        As[r * SIPG_MAXP + s] = Lp[first + r][first + s];
        Bs[r * SIPG_MAXP + s] = Mp[first + r][first + s];
      }
    bool ok = generalised_eigen(p, As, Bs, SIPG_MAXP, Ss, lam, W1, W2);
    if (!ok) atomicExch(status, 1);
    for (int r = 0; r < SIPG_MAXP; ++r) {
      c.lam[t][r] = (r < p) ? lam[r] : 0.0;
      for (int s = 0; s < SIPG_MAXP; ++s) c.S[t][r][s] = (r < p && s < p) ? Ss[r * SIPG_MAXP + s] : 0.0;
    }
    // Full kernel: the same eigenproblem on all P patch nodes.  Clamped
    // kernel: on the subspace of patch functions with v = v' = 0 at each
    // patch end inside the domain, spanned by the columns of Bc: one column
    // per free coefficient f, with the two end coefficients of that end
    // eliminated (v = 0 fixes the end node; v' = 0 then fixes its
    // neighbour: sum_j phi_j'(end) c_j = 0).  Sf = Bc S (P x m, zero columns
    // beyond m) and lamf = 1 beyond m, so the full-kernel patch kernel
    // applies (Bc S) Lambda^{-1} (Bc S)^T = Bc (Bc^T A_D Bc)^{-1} Bc^T.
    const bool clamped = smoother == SIPG_SMOOTHER_CLAMPED;
    double Bc[SIPG_MAXP][SIPG_MAXP];
    int mc = 0;
    if (clamped) {
      const bool lo = !(t & 1), hi = !(t & 2);
      for (int f = 0; f < P; ++f) {
        if (lo && f < 2) continue;
        if (hi && f >= P - 2) continue;
        for (int r = 0; r < P; ++r) Bc[r][mc] = (r == f) ? 1.0 : 0.0;
        if (lo && f < n) Bc[1][mc] = -B.D[0][f] / B.D[0][1];
        if (hi && f >= n) Bc[P - 2][mc] = -B.D[n - 1][f - n] / B.D[n - 1][n - 2];
        ++mc;
      }
      for (int r = 0; r < mc; ++r)
        for (int s = 0; s < mc; ++s) {
          double a = 0.0, m = 0.0;
          for (int i = 0; i < P; ++i)
            for (int j = 0; j < P; ++j) {
              a += Bc[i][r] * Lp[i][j] * Bc[j][s];
              m += Bc[i][r] * Mp[i][j] * Bc[j][s];
            }
          As[r * SIPG_MAXP + s] = a;
          Bs[r * SIPG_MAXP + s] = m;
        }
    } else {
      mc = P;
      for (int r = 0; r < P; ++r)
        for (int s = 0; s < P; ++s) {
          As[r * SIPG_MAXP + s] = Lp[r][s];
          Bs[r * SIPG_MAXP + s] = Mp[r][s];
        }
    }
    ok = mc > 0 && generalised_eigen(mc, As, Bs, SIPG_MAXP, Ss, lam, W1, W2);
    if (!ok) atomicExch(status, 1);
    for (int r = 0; r < SIPG_MAXP; ++r) {
      c.lamf[t][r] = (r < mc) ? lam[r] : 1.0;
      for (int s = 0; s < SIPG_MAXP; ++s) {
        double v = 0.0;
        if (r < P && s < mc) {
          if (clamped)
            for (int q = 0; q < mc; ++q) v += Bc[r][q] * Ss[q * SIPG_MAXP + s];
          else
            v = Ss[r * SIPG_MAXP + s];
        }
        c.Sf[t][r][s] = v;
      }
    }
  } else if (t == 4 && l == 0) {
    // coarsest level: global 1D SIPG matrix and mass, N n x N n
    const int m = N * n;
    const int ld = SIPG_MAXM0;
    double* A = scratch;
    double* Bm = A + ld * ld;
    double* S = Bm + ld * ld;
    double* W1 = S + ld * ld;
    double* W2 = W1 + ld * ld;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        int ci = i / n, ii = i % n, cj = j / n, ij = j % n;
        double lv = 0.0, mv = 0.0;
        int ty = (ci == 0) ? 1 : ((ci == N - 1) ? 2 : 0);
        if (ci == cj) {
          lv = c.Lself[ty][ii][ij];
          mv = c.M[ii][ij];
        } else if (cj == ci - 1) {
          lv = l_lo_entry(c, k, ii, ij);
        } else if (cj == ci + 1) {
          lv = l_hi_entry(c, k, ii, ij);
        }
        A[i * ld + j] = lv;
        Bm[i * ld + j] = mv;
      }
    double lam[SIPG_MAXM0];
    bool ok = generalised_eigen(m, A, Bm, ld, S, lam, W1, W2);
    if (!ok) atomicExch(status, 2);
    for (int i = 0; i < SIPG_MAXM0; ++i) {
      c.lam0[i] = (i < m) ? lam[i] : 0.0;
      for (int j = 0; j < SIPG_MAXM0; ++j) c.S0[i][j] = (i < m && j < m) ? S[i * ld + j] : 0.0;
    }
  }
}

// FP32 twin of the FP64 constants, element by element.
__global__ void constants_to_float_kernel(const LevelConst<double>* in, LevelConst<float>* out) {
  const LevelConst<double>& a = in[blockIdx.x];
  LevelConst<float>& b = out[blockIdx.x];
  if (threadIdx.x == 0) {
    b.N = a.N;
    b.n = a.n;
    b.m0 = a.m0;
    b.pad_ = 0;
    b.h = (float)a.h;
    b.gamma = (float)a.gamma;
    for (int t = 0; t < 4; ++t) {
      b.p[t] = a.p[t];
      b.first[t] = a.first[t];
    }
  }
#define SIPG_CONVERT(field)                                                        \
  {                                                                                \
    const double* src = reinterpret_cast<const double*>(&a.field);                 \
    float* dst = reinterpret_cast<float*>(&b.field);                               \
    const int cnt = sizeof(a.field) / sizeof(double);                              \
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) dst[i] = (float)src[i];    \
  }
  SIPG_CONVERT(Mw)
  SIPG_CONVERT(Ma)
  SIPG_CONVERT(Mu)
  SIPG_CONVERT(Lself)
  SIPG_CONVERT(alo)
  SIPG_CONVERT(glo)
  SIPG_CONVERT(ahi)
  SIPG_CONVERT(ghi)
  SIPG_CONVERT(Pself)
  SIPG_CONVERT(palo)
  SIPG_CONVERT(pglo)
  SIPG_CONVERT(pahi)
  SIPG_CONVERT(pghi)
  SIPG_CONVERT(M)
  SIPG_CONVERT(Lr)
  SIPG_CONVERT(Mr)
  SIPG_CONVERT(S)
  SIPG_CONVERT(lam)
  SIPG_CONVERT(Sf)
  SIPG_CONVERT(lamf)
  SIPG_CONVERT(Pc)
  SIPG_CONVERT(nodes)
  SIPG_CONVERT(S0)
  SIPG_CONVERT(lam0)
#undef SIPG_CONVERT
}

}  // namespace

cudaError_t launch_setup(sipg_handle* h, cudaStream_t s) {
  const int nl = h->prm.n_levels;
  int* status = reinterpret_cast<int*>(h->ws + h->off_scratch_setup);
  double* scratch = reinterpret_cast<double*>(h->ws + h->off_scratch_setup + 256);
  cudaMemsetAsync(status, 0, sizeof(int), s);
  setup_levels_kernel<<<nl, 32, 0, s>>>(h->c64(0), h->prm.degree, 1 << h->prm.log2_cells, nl,
                                        h->prm.kappa, h->prm.penalty_factor, h->prm.smoother, scratch,
                                        status);
  constants_to_float_kernel<<<nl, 256, 0, s>>>(h->c64(0), h->c32(0));
  h->launches += 2;
  return cudaGetLastError();
}
