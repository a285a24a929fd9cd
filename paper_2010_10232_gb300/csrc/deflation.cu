// Adapted deflation preconditioner (Section 3: Eq. adef1, P = I - A Q,
// Q = Z E^{-1} Z^T, E = Z^T A Z, with the quadratic rational-Bezier stencil
// for Z and its epsilon-weighted variant).
//
// Index convention: 1-based interior indices, coarse dof J sits at fine dof
// 2J; m_x = floor(n_x / 2); stencil terms outside the index ranges are
// dropped.  Z^T row = (1, 4, 6 - eps, 4, 1)/8 on fine 2J-2 .. 2J+2 (the
// paper's printed row repeats an index; it is read as the transpose of Z).
// 2D: Z = Z_y (x) Z_x.
//
// E^{-1} for constant k by fast diagonalisation: E = Mc (x) Kc + Kc (x) Mc
// - k^2 Mc (x) Mc with the 1D Galerkin matrices Kc = Z^T K Z, Mc = Z^T M Z.
// The generalised eigenvectors V (V^T Mc V = I, V^T Kc V = diag(lambda))
// give E^{-1} = (V (x) V) diag(1 / (lambda_i + lambda_j - k^2)) (V (x) V)^T,
// applied as four real-by-complex GEMMs on the m_x x m_x coarse grid.
#include "common.cuh"
#include <cmath>


// ------------------------------------------------------------------ Z, Z^T
__device__ __forceinline__ double zt_w(int a, double eps) {   // a in -2..2
  const double w[5] = {1.0 / 8.0, 4.0 / 8.0, 0.0, 4.0 / 8.0, 1.0 / 8.0};
  return a == 0 ? (6.0 - eps) / 8.0 : w[a + 2];
}

// c = Z^T x
__global__ void k_zt(int nx, int ny, int mx, int my, double eps, const double2* x, double2* c, float2* cf) {
  size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (j >= (size_t)mx * my) return;
  int jy = (int)(j / mx), jx = (int)(j - (size_t)jy * mx);
  int fx = 2 * jx + 1, fy = 2 * jy + 1;   // 0-based fine index of coarse centre (1-based 2J)
  double2 acc = make_double2(0.0, 0.0);
  if (ny == 1) {
    for (int a = -2; a <= 2; ++a) {
      int ix = fx + a;
      if (ix >= 0 && ix < nx) acc = cfma(zt_w(a, eps), x[ix], acc);
    }
  } else {
    for (int b = -2; b <= 2; ++b) {
      int iy = fy + b;
      if (iy < 0 || iy >= ny) continue;
      double2 row = make_double2(0.0, 0.0);
      for (int a = -2; a <= 2; ++a) {
        int ix = fx + a;
        if (ix >= 0 && ix < nx) row = cfma(zt_w(a, eps), x[(size_t)iy * nx + ix], row);
      }
      acc = cfma(zt_w(b, eps), row, acc);
    }
  }
  c[j] = acc;
  if (cf) cf[j] = tof(acc);     // FP32 copy for the coarse solve's first transform
}

// 1D Z row for fine (0-based) i: up to 3 (coarse index, weight) pairs
__device__ __forceinline__ int z_row(int i, int m, double eps, int* idx, double* w) {
  int I = i + 1, cnt = 0;
  if ((I & 1) == 0) {
    int J = I / 2;
    int js[3] = {J - 1, J, J + 1};
    double ws[3] = {1.0 / 8.0, (6.0 - eps) / 8.0, 1.0 / 8.0};
    for (int t = 0; t < 3; ++t)
      if (js[t] >= 1 && js[t] <= m) { idx[cnt] = js[t] - 1; w[cnt] = ws[t]; ++cnt; }
  } else {
    int js[2] = {(I - 1) / 2, (I + 1) / 2};
    for (int t = 0; t < 2; ++t)
      if (js[t] >= 1 && js[t] <= m) { idx[cnt] = js[t] - 1; w[cnt] = 0.5; ++cnt; }
  }
  return cnt;
}

// x = Z c
__global__ void k_z(int nx, int ny, int mx, int my, double eps, const double2* c, double2* x) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nx * ny) return;
  int iy = (int)(i / nx), ix = (int)(i - (size_t)iy * nx);
  int cxi[3], cyi[3];
  double wx[3], wy[3];
  int nxc = z_row(ix, mx, eps, cxi, wx);
  double2 acc = make_double2(0.0, 0.0);
  if (ny == 1) {
    for (int a = 0; a < nxc; ++a) acc = cfma(wx[a], c[cxi[a]], acc);
  } else {
    int nyc = z_row(iy, my, eps, cyi, wy);
    for (int b = 0; b < nyc; ++b) {
      double2 row = make_double2(0.0, 0.0);
      for (int a = 0; a < nxc; ++a) row = cfma(wx[a], c[(size_t)cyi[b] * mx + cxi[a]], row);
      acc = cfma(wy[b], row, acc);
    }
  }
  x[i] = acc;
}

// Dense 1D coarse matrices Kc = Z^T K Z, Mc = Z^T M Z (thread per entry)
__global__ void k_coarse_1d(int nx, int mx, int p, double eps, const double* K, const double* M, double* Kc,
                            double* Mc) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mx * mx) return;
  int I = idx / mx, J = idx - I * mx;
  int W = 2 * p + 1;
  double kv = 0.0, mv = 0.0;
  if (abs(I - J) <= (p + 4) / 2 + 1) {
    int fi = 2 * I + 1, fj = 2 * J + 1;
    for (int a = -2; a <= 2; ++a) {
      int r = fi + a;
      if (r < 0 || r >= nx) continue;
      for (int b = -2; b <= 2; ++b) {
        int c = fj + b;
        if (c < 0 || c >= nx) continue;
        int d = c - r;
        if (d < -p || d > p) continue;
        double w = zt_w(a, eps) * zt_w(b, eps);
        kv += w * K[(size_t)r * W + d + p];
        mv += w * M[(size_t)r * W + d + p];
      }
    }
  }
  Kc[idx] = kv;
  Mc[idx] = mv;
}

// ------------------------------------------------------------------ dense helpers (setup)
// In-place Cholesky A = L L^T of a dense SPD matrix (one block, right-looking).
__global__ void k_cholesky(double* A, int n, int* info) {
  __shared__ double piv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double d = A[(size_t)k * n + k];
      if (!(d > 0.0)) { *info = 2; d = 1.0; }
      piv = sqrt(d);
      A[(size_t)k * n + k] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + k] /= piv;
    __syncthreads();
    int m = n - k - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j <= i) A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
    }
    __syncthreads();
  }
}

// X = L^{-1} B  (L lower triangular in the lower part of Lm), thread per column.
__global__ void k_trsm_lower(const double* Lm, const double* B, double* X, int n) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < n; ++i) {
    double s = B[(size_t)i * n + c];
    for (int k = 0; k < i; ++k) s -= Lm[(size_t)i * n + k] * X[(size_t)k * n + c];
    X[(size_t)i * n + c] = s / Lm[(size_t)i * n + i];
  }
}
// X = L^{-T} B, thread per column
__global__ void k_trsm_lower_t(const double* Lm, const double* B, double* X, int n) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = n - 1; i >= 0; --i) {
    double s = B[(size_t)i * n + c];
    for (int k = i + 1; k < n; ++k) s -= Lm[(size_t)k * n + i] * X[(size_t)k * n + c];
    X[(size_t)i * n + c] = s / Lm[(size_t)i * n + i];
  }
}
__global__ void k_transpose(const double* A, double* B, int n) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n * n) { int i = idx / n, j = idx - i * n; B[(size_t)j * n + i] = A[idx]; }
}
// pad an n x n symmetric matrix to np x np (np = n or n+1), symmetrised
__global__ void k_pad_sym(const double* A, double* P, int n, int np) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= np * np) return;
  int i = idx / np, j = idx - i * np;
  P[idx] = (i < n && j < n) ? 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]) : 0.0;
}
__global__ void k_eye_d(double* V, int n) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n * n) V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

// ------------------------------------------------------------------ parallel cyclic Jacobi
// Round r of the round-robin ordering pairs index positions (k, np-1-k).
__device__ __forceinline__ int rr_index(int k, int r, int np) { return k == 0 ? 0 : 1 + (k - 1 + r) % (np - 1); }

// Rotation (c, s) annihilating A[p][q]: G = [[c, s], [-s, c]], G^T A_pq G diagonal
// (the symmetric 2x2 Schur decomposition).
__global__ void k_jac_angles(const double* A, int np, int r, double* cs) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np / 2) return;
  int i1 = rr_index(k, r, np), i2 = rr_index(np - 1 - k, r, np);
  int p = min(i1, i2), q = max(i1, i2);
  double app = A[(size_t)p * np + p], aqq = A[(size_t)q * np + q], apq = A[(size_t)p * np + q];
  double c = 1.0, s = 0.0;
  if (apq != 0.0) {
    double tau = (aqq - app) / (2.0 * apq);
    double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
  }
  cs[4 * k + 0] = c;
  cs[4 * k + 1] = s;
  cs[4 * k + 2] = p;
  cs[4 * k + 3] = q;
}

// A_new = J^T A J over all 2x2 blocks of the pairing; V <- V J.
__global__ void k_jac_apply(const double* A, double* An, double* V, int np, const double* cs) {
  int h = np / 2;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < h * h) {
    int k1 = idx / h, k2 = idx - k1 * h;
    double c1 = cs[4 * k1], s1 = cs[4 * k1 + 1], c2 = cs[4 * k2], s2 = cs[4 * k2 + 1];
    int p1 = (int)cs[4 * k1 + 2], q1 = (int)cs[4 * k1 + 3], p2 = (int)cs[4 * k2 + 2], q2 = (int)cs[4 * k2 + 3];
    double b00 = A[(size_t)p1 * np + p2], b01 = A[(size_t)p1 * np + q2];
    double b10 = A[(size_t)q1 * np + p2], b11 = A[(size_t)q1 * np + q2];
    // G1^T B
    double t00 = c1 * b00 - s1 * b10, t01 = c1 * b01 - s1 * b11;
    double t10 = s1 * b00 + c1 * b10, t11 = s1 * b01 + c1 * b11;
    // (G1^T B) G2
    An[(size_t)p1 * np + p2] = t00 * c2 - t01 * s2;
    An[(size_t)p1 * np + q2] = t00 * s2 + t01 * c2;
    An[(size_t)q1 * np + p2] = t10 * c2 - t11 * s2;
    An[(size_t)q1 * np + q2] = t10 * s2 + t11 * c2;
  }
  int v = idx - h * h;
  if (v >= 0 && v < np * h) {
    int row = v / h, k = v - row * h;
    double c = cs[4 * k], s = cs[4 * k + 1];
    int p = (int)cs[4 * k + 2], q = (int)cs[4 * k + 3];
    double vp = V[(size_t)row * np + p], vq = V[(size_t)row * np + q];
    V[(size_t)row * np + p] = c * vp - s * vq;
    V[(size_t)row * np + q] = s * vp + c * vq;
  }
}

// off-diagonal and total squared Frobenius norm (one block)
__global__ void k_offnorm(const double* A, int np, double* out) {
  __shared__ double so[256], st[256];
  double o = 0.0, t = 0.0;
  for (int idx = threadIdx.x; idx < np * np; idx += blockDim.x) {
    double v = A[idx];
    t += v * v;
    if (idx / np != idx % np) o += v * v;
  }
  so[threadIdx.x] = o;
  st[threadIdx.x] = t;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) { so[threadIdx.x] += so[threadIdx.x + s]; st[threadIdx.x] += st[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = so[0]; out[1] = st[0]; }
}

__global__ void k_diag_extract(const double* A, int np, int n, double* lam) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lam[i] = A[(size_t)i * np + i];
}
// W (np x np) -> n x n top-left block
__global__ void k_crop(const double* W, int np, int n, double* out) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n * n) { int i = idx / n, j = idx - i * n; out[idx] = W[(size_t)i * np + j]; }
}

// ------------------------------------------------------------------ accuracy fixes
// Rayleigh quotients lambda_k = v_k^T Kc v_k / v_k^T Mc v_k with the original
// (banded) coarse matrices: the eigenvalue error becomes quadratic in the
// eigenvector error, which matters when lambda_i + lambda_j - k^2 nearly cancels.
__global__ void k_rayleigh(const double* V, const double* Kc, const double* Mc, int n, int bw, double* lam) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double num = 0.0, den = 0.0;
  for (int i = 0; i < n; ++i) {
    double vi = V[(size_t)i * n + k];
    double sk = 0.0, sm = 0.0;
    for (int j = max(0, i - bw); j <= min(n - 1, i + bw); ++j) {
      double vj = V[(size_t)j * n + k];
      sk += Kc[(size_t)i * n + j] * vj;
      sm += Mc[(size_t)i * n + j] * vj;
    }
    num += vi * sk;
    den += vi * sm;
  }
  lam[k] = num / den;
}


// FP32 variant of the FDM transform for the refined coarse solve: X is double2
// (first pass) or float2, the output float2 or double2, V in FP32, products
// accumulated in FP32; the eigenvalue denominators stay FP64.
__device__ __forceinline__ float2 ld_f2(const double2* p) { return tof(*p); }
__device__ __forceinline__ float2 ld_f2(const float2* p) { return *p; }
__device__ __forceinline__ void st_c(double2* p, float2 v) { *p = tod(v); }
__device__ __forceinline__ void st_c(float2* p, float2 v) { *p = v; }

// out = R X (LEFT) or X R (RIGHT) with R a row-major m x m FP32 matrix (V or
// V^T, both stored), so every operand tile is read with unit stride.  The
// K extent of both operand panels is staged in shared memory in stages of TK
// (the whole K for short panels: one round of loads).  ACC: out (FP64) += result.
constexpr int FDM_TY = 8, FDM_TX = 16, FDM_TK = 192;
__host__ __device__ inline size_t fdm_gemm_smem(int tk) {
  return sizeof(float2) * ((size_t)FDM_TY * (tk + 1) + (size_t)tk * (FDM_TX + 1));
}

// stage n elements of a panel into shared memory, issuing FDM_LPT independent
// loads per thread before any store (one round of L2 latency per batch)
constexpr int FDM_LPT = 16;
template <int LPT, typename D, typename F>
__device__ __forceinline__ void stage_panel(int total, D* dst, F src_at) {
  for (int base = 0; base < total; base += 128 * LPT) {
    D v[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      const int t = base + q * 128 + (int)threadIdx.x;
      v[q] = t < total ? src_at(t) : D{};
    }
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      const int t = base + q * 128 + (int)threadIdx.x;
      if (t < total) dst[t] = v[q];
    }
  }
}

template <bool LEFT, bool DIVIDE, bool ACC, typename XT, typename OT, int LPT>
__global__ void __launch_bounds__(128) k_fdm_gemm32(const float* R, const XT* X, OT* out, int rows, int cols,
                                                   const float2* dinv, int TK) {
  constexpr int TY = FDM_TY, TX = FDM_TX;
  extern __shared__ __align__(16) unsigned char fsm[];
  // LEFT: Rs[TY][TK+1] and Xs[TK][TX+1]; RIGHT: Xs[TY][TK+1] and Rs[TK][TX+1]
  float2* Xsm = reinterpret_cast<float2*>(fsm);
  float* Rsm = reinterpret_cast<float*>(Xsm + (LEFT ? (size_t)TK * (TX + 1) : (size_t)TY * (TK + 1)));
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int i = blockIdx.y * TY + ty, j = blockIdx.x * TX + tx;
  const int row0 = blockIdx.y * TY, col0 = blockIdx.x * TX;
  int K = LEFT ? rows : cols;
  float2 acc = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += TK) {
    const int kc = min(TK, K - k0);
    if (LEFT) {
      // Rs[r][kk] = R[row0 + r][k0 + kk]; Xs[kk][c] = X[k0 + kk][col0 + c]  (coalesced)
      stage_panel<LPT, float>(TY * kc, Rsm, [&](int t) {
        int r = t / kc, kk = t - r * kc;
        return row0 + r < rows ? R[(size_t)(row0 + r) * rows + k0 + kk] : 0.f;
      });
      stage_panel<LPT, float2>(kc * TX, Xsm, [&](int t) {
        int kk = t / TX, c = t - kk * TX;
        return col0 + c < cols ? ld_f2(X + (size_t)(k0 + kk) * cols + col0 + c) : make_float2(0.f, 0.f);
      });
      __syncthreads();
      {   // four independent accumulators: a quarter of the dependent FMA chain
        float2 a4[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        int kk = 0;
#pragma unroll 2
        for (; kk + 4 <= kc; kk += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) a4[u] = cfma(Rsm[ty * kc + kk + u], Xsm[(kk + u) * TX + tx], a4[u]);
        }
        for (; kk < kc; ++kk) a4[0] = cfma(Rsm[ty * kc + kk], Xsm[kk * TX + tx], a4[0]);
        acc = acc + ((a4[0] + a4[1]) + (a4[2] + a4[3]));
      }
    } else {
      stage_panel<LPT, float2>(TY * kc, Xsm, [&](int t) {
        int r = t / kc, kk = t - r * kc;
        return row0 + r < rows ? ld_f2(X + (size_t)(row0 + r) * cols + k0 + kk) : make_float2(0.f, 0.f);
      });
      // Rs[kk][c] = R[k0 + kk][col0 + c]  (c fastest: coalesced)
      stage_panel<LPT, float>(kc * TX, Rsm, [&](int t) {
        int kk = t / TX, c = t - kk * TX;
        return col0 + c < cols ? R[(size_t)(k0 + kk) * cols + col0 + c] : 0.f;
      });
      __syncthreads();
      {
        float2 a4[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        int kk = 0;
#pragma unroll 2
        for (; kk + 4 <= kc; kk += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) a4[u] = cfma(Rsm[(kk + u) * TX + tx], Xsm[ty * kc + kk + u], a4[u]);
        }
        for (; kk < kc; ++kk) a4[0] = cfma(Rsm[kk * TX + tx], Xsm[ty * kc + kk], a4[0]);
        acc = acc + ((a4[0] + a4[1]) + (a4[2] + a4[3]));
      }
    }
    __syncthreads();
  }
  if (i < rows && j < cols) {
    if (DIVIDE) acc = cmul(dinv[(size_t)i * cols + j], acc);
    if constexpr (ACC) {
      OT* o = out + (size_t)i * cols + j;
      *o = *o + tod(acc);
    } else {
      st_c(out + (size_t)i * cols + j, acc);
    }
  }
}

// Long panels (m_x > FDM_TK): register-blocked form.  A block computes a
// 32 x 32 tile of out with 64 threads, each 4 rows x 4 columns (16 complex
// accumulators); K runs in chunks of 16 through two shared-memory buffers,
// the next chunk's global loads held in registers while the current one is
// used.  The real operand R and the complex operand X are staged so that a
// thread reads its four rows (columns) with one or two 16-byte loads.
// LEFT: out = R X (R rows x rows, X rows x cols); RIGHT: out = X R (R cols x
// cols).  Same epilogue as k_fdm_gemm32.
constexpr int FRB_T = 32, FRB_K = 16, FRB_RS = 36, FRB_XS = 34;   // padded rows, 16-byte aligned
template <bool LEFT, bool DIVIDE, bool ACC, typename XT, typename OT>
__global__ void __launch_bounds__(64) k_fdm_gemm_rb(const float* __restrict__ R, const XT* __restrict__ X,
                                                    OT* out, int rows, int cols, const float2* __restrict__ dinv) {
  __shared__ __align__(16) float Rs[2][FRB_K][FRB_RS];    // LEFT: R^T chunk [k][i]; RIGHT: R chunk [k][j]
  __shared__ __align__(16) float2 Xs[2][FRB_K][FRB_XS];   // LEFT: X chunk [k][j];  RIGHT: X^T chunk [k][i]
  const int t = threadIdx.x, ty = t >> 3, tx = t & 7;
  const int i0 = blockIdx.y * FRB_T, j0 = blockIdx.x * FRB_T;
  const int K = LEFT ? rows : cols;
  // this thread's share of a chunk: elements e = 64 q + t, q = 0..7, of the
  // 32 x 16 panel read along its contiguous index (16 K entries of a row, or
  // 32 entries of a K row), so consecutive lanes load consecutive addresses
  float rv[8];
  float2 xv[8];
  auto load_chunk = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = 64 * q + t;
      const int a = e >> 4, kk = e & 15;     // row a of a 32 x 16 [row][k] panel
      const int kr = e >> 5, c = e & 31;     // k row kr of a 16 x 32 [k][column] panel
      if (LEFT) {
        rv[q] = (i0 + a < rows && k0 + kk < K) ? R[(size_t)(i0 + a) * K + k0 + kk] : 0.f;
        xv[q] = (k0 + kr < K && j0 + c < cols) ? ld_f2(X + (size_t)(k0 + kr) * cols + j0 + c) : make_float2(0.f, 0.f);
      } else {
        xv[q] = (i0 + a < rows && k0 + kk < K) ? ld_f2(X + (size_t)(i0 + a) * cols + k0 + kk) : make_float2(0.f, 0.f);
        rv[q] = (k0 + kr < K && j0 + c < cols) ? R[(size_t)(k0 + kr) * cols + j0 + c] : 0.f;
      }
    }
  };
  auto store_chunk = [&](int b) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = 64 * q + t;
      const int a = e >> 4, kk = e & 15, kr = e >> 5, c = e & 31;
      if (LEFT) {
        Rs[b][kk][a] = rv[q];
        Xs[b][kr][c] = xv[q];
      } else {
        Xs[b][kk][a] = xv[q];
        Rs[b][kr][c] = rv[q];
      }
    }
  };
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
  const int nch = (K + FRB_K - 1) / FRB_K;
  load_chunk(0);
  store_chunk(0);
  __syncthreads();
  for (int ch = 0; ch < nch; ++ch) {
    const int b = ch & 1;
    if (ch + 1 < nch) load_chunk((ch + 1) * FRB_K);
#pragma unroll
    for (int k = 0; k < FRB_K; ++k) {
      if (LEFT) {
        const float4 a = *reinterpret_cast<const float4*>(&Rs[b][k][4 * ty]);
        const float4 x01 = *reinterpret_cast<const float4*>(&Xs[b][k][4 * tx]);
        const float4 x23 = *reinterpret_cast<const float4*>(&Xs[b][k][4 * tx + 2]);
        const float ar[4] = {a.x, a.y, a.z, a.w};
        const float2 xc[4] = {make_float2(x01.x, x01.y), make_float2(x01.z, x01.w), make_float2(x23.x, x23.y),
                              make_float2(x23.z, x23.w)};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = cfma(ar[r], xc[c], acc[r][c]);
      } else {
        const float4 x01 = *reinterpret_cast<const float4*>(&Xs[b][k][4 * ty]);
        const float4 x23 = *reinterpret_cast<const float4*>(&Xs[b][k][4 * ty + 2]);
        const float4 a = *reinterpret_cast<const float4*>(&Rs[b][k][4 * tx]);
        const float ar[4] = {a.x, a.y, a.z, a.w};
        const float2 xc[4] = {make_float2(x01.x, x01.y), make_float2(x01.z, x01.w), make_float2(x23.x, x23.y),
                              make_float2(x23.z, x23.w)};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = cfma(ar[c], xc[r], acc[r][c]);
      }
    }
    if (ch + 1 < nch) store_chunk(b ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + 4 * ty + r;
    if (i >= rows) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + 4 * tx + c;
      if (j >= cols) continue;
      float2 v = acc[r][c];
      if (DIVIDE) v = cmul(dinv[(size_t)i * cols + j], v);
      if constexpr (ACC) {
        OT* o = out + (size_t)i * cols + j;
        *o = *o + tod(v);
      } else {
        st_c(out + (size_t)i * cols + j, v);
      }
    }
  }
}

template <bool LEFT, bool DIVIDE, bool ACC, typename XT, typename OT>
static void launch_fdm_gemm(iga_ctx* ctx, const float* R, const XT* X, OT* out, int rows, int cols,
                            const float2* dinv) {
  // up to FDM_TK the whole K extent in one stage, 16 loads in flight per
  // thread; longer panels by the register-blocked kernel
  const int K = LEFT ? rows : cols;
  dim3 g(cdiv(cols, FDM_TX), cdiv(rows, FDM_TY));
  if (K <= FDM_TK) {
    k_fdm_gemm32<LEFT, DIVIDE, ACC, XT, OT, 16><<<g, 128, fdm_gemm_smem(K), ctx->st>>>(R, X, out, rows, cols, dinv, K);
  } else {
    dim3 gb(cdiv(cols, FRB_T), cdiv(rows, FRB_T));
    k_fdm_gemm_rb<LEFT, DIVIDE, ACC, XT, OT><<<gb, 64, 0, ctx->st>>>(R, X, out, rows, cols, dinv);
  }
  iga_count_launch();
}

// one-time: allow the whole-K panels above 48 KB of shared memory
static iga_status fdm_gemm_attrs(iga_ctx* ctx) {
  const int sm = (int)fdm_gemm_smem(FDM_TK);
  CK(cudaFuncSetAttribute(k_fdm_gemm32<false, true, false, double2, float2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fdm_gemm32<false, false, false, float2, double2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fdm_gemm32<false, false, true, float2, double2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fdm_gemm32<true, false, false, double2, float2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fdm_gemm32<false, true, false, float2, float2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fdm_gemm32<true, false, false, float2, float2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  return IGA_OK;
}

// dinv[i][j] = 1 / (lambda_i + lambda_j + c) (2D) or 1 / (lambda_j + c) (1D),
// c = -k^2 for E, -(beta1 - i beta2) k^2 for the CSLP matrix: the sum is formed
// in FP64 (for E it nearly cancels for modes close to k^2), the reciprocal is
// rounded once to FP32 (imaginary part exactly 0 when c is real).
__global__ void k_fdm_dinv(const double* lam, int n, int dim, double2 c, float2* dinv) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t tot = dim == 2 ? (size_t)n * n : (size_t)n;
  if (idx >= tot) return;
  int i = (int)(idx / n), j = (int)(idx - (size_t)i * n);
  double2 d = make_double2((dim == 2 ? lam[i] : 0.0) + lam[j] + c.x, c.y);
  if (d.y == 0.0) dinv[idx] = make_float2((float)(1.0 / d.x), 0.0f);
  else dinv[idx] = tof(cinv(d));
}

__global__ void k_transpose_f(const float* A, float* B, int n) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n * n) { int i = idx / n, j = idx - i * n; B[(size_t)j * n + i] = A[idx]; }
}

// band extraction of a dense (banded) matrix: B[i][d + bw] = A[i][i + d]
__global__ void k_dense_to_band(const double* A, int n, int bw, double* B) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int W = 2 * bw + 1;
  if (idx >= n * W) return;
  int i = idx / W, d = idx - i * W - bw, j = i + d;
  B[idx] = (j >= 0 && j < n) ? A[(size_t)i * n + j] : 0.0;
}
__global__ void k_d2f_vec(const double* a, float* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ------------------------------------------------------------------ host
// dense [n][n] from a band [n][2bw+1] (Mat[i][i+d] at B[i][d+bw])
__global__ void k_band_to_dense(const double* B, int n, int bw, double* A) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  int i = (int)(idx / n), j = (int)(idx - (size_t)i * n), d = j - i;
  A[idx] = (d >= -bw && d <= bw) ? B[(size_t)i * (2 * bw + 1) + d + bw] : 0.0;
}

// Generalised eigenpairs of the dense SPD pencil (Kd, Md) of size n (both with
// half bandwidth bw): Cholesky Md = L L^T, parallel cyclic Jacobi on
// L^{-1} Kd L^{-T}, V = L^{-T} W, eigenvalues recomputed as Rayleigh quotients;
// then the FP32 copies of V, V^T and the denominators 1 / (lam_i + lam_j + c).
static iga_status fdm_build(iga_ctx* ctx, FdmData& F, int n, const double* Kd, const double* Md, int bw, double2 c) {
  const int np = n + (n & 1);
  cudaStream_t st = ctx->st;
  F.n = n;
  double* Lm = dalloc<double>(ctx, (size_t)n * n);
  double* Y = dalloc<double>(ctx, (size_t)n * n);
  double* Yt = dalloc<double>(ctx, (size_t)n * n);
  double* Cm = dalloc<double>(ctx, (size_t)n * n);
  double* A0 = dalloc<double>(ctx, (size_t)np * np);
  double* A1 = dalloc<double>(ctx, (size_t)np * np);
  double* Vj = dalloc<double>(ctx, (size_t)np * np);
  double* W = dalloc<double>(ctx, (size_t)n * n);
  double* cs = dalloc<double>(ctx, (size_t)4 * (np / 2 + 1));
  double* nrm = dalloc<double>(ctx, 2);
  int* info = dalloc<int>(ctx, 1);
  F.V = dalloc<double>(ctx, (size_t)n * n);
  F.lam = dalloc<double>(ctx, n);
  if (!Lm || !Y || !Yt || !Cm || !A0 || !A1 || !Vj || !W || !cs || !nrm || !info || !F.V || !F.lam)
    return set_err(ctx, IGA_E_OOM, "fdm alloc");
  CK(cudaMemsetAsync(info, 0, sizeof(int), st));
  CK(cudaMemcpyAsync(Lm, Md, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
  k_cholesky<<<1, 512, 0, st>>>(Lm, n, info); iga_count_launch();
  CKL();
  // C = L^{-1} Kd L^{-T} = L^{-1} (L^{-1} Kd)^T
  k_trsm_lower<<<cdiv(n, 64), 64, 0, st>>>(Lm, Kd, Y, n); iga_count_launch();
  k_transpose<<<cdiv((size_t)n * n, 256), 256, 0, st>>>(Y, Yt, n); iga_count_launch();
  k_trsm_lower<<<cdiv(n, 64), 64, 0, st>>>(Lm, Yt, Cm, n); iga_count_launch();
  k_pad_sym<<<cdiv((size_t)np * np, 256), 256, 0, st>>>(Cm, A0, n, np); iga_count_launch();
  k_eye_d<<<cdiv((size_t)np * np, 256), 256, 0, st>>>(Vj, np); iga_count_launch();
  CKL();
  double hn[2] = {0, 0};
  double* cur = A0;
  double* nxt = A1;
  bool conv = false;
  int extra = -1;                    // one more sweep after the threshold is met
  const int h = np / 2;
  for (int sweep = 0; sweep < 40 && !conv; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      k_jac_angles<<<cdiv(h, 128), 128, 0, st>>>(cur, np, r, cs); iga_count_launch();
      k_jac_apply<<<cdiv((size_t)h * h + (size_t)np * h, 256), 256, 0, st>>>(cur, nxt, Vj, np, cs); iga_count_launch();
      std::swap(cur, nxt);
    }
    CKL();
    k_offnorm<<<1, 256, 0, st>>>(cur, np, nrm); iga_count_launch();
    CK(cudaMemcpyAsync(hn, nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (extra >= 0) conv = true;
    else if (hn[0] <= 1e-26 * hn[1] || hn[0] == 0.0) extra = sweep;
  }
  if (!conv) return set_err(ctx, IGA_E_INVALID, "Jacobi eigen-solver did not converge (off %.3e)", hn[0]);
  k_diag_extract<<<cdiv(n, 128), 128, 0, st>>>(cur, np, n, F.lam); iga_count_launch();
  k_crop<<<cdiv((size_t)n * n, 256), 256, 0, st>>>(Vj, np, n, W); iga_count_launch();
  // generalised eigenvectors V = L^{-T} W
  k_trsm_lower_t<<<cdiv(n, 64), 64, 0, st>>>(Lm, W, F.V, n); iga_count_launch();
  k_rayleigh<<<cdiv(n, 64), 64, 0, st>>>(F.V, Kd, Md, n, bw, F.lam); iga_count_launch();
  const size_t mm = ctx->dim == 2 ? (size_t)n * n : (size_t)n;
  F.Vf = dalloc<float>(ctx, (size_t)n * n);
  F.Vtf = dalloc<float>(ctx, (size_t)n * n);
  F.w1 = dalloc<float2>(ctx, mm);
  F.w2 = dalloc<float2>(ctx, mm);
  F.dinv = dalloc<float2>(ctx, mm);
  if (!F.Vf || !F.Vtf || !F.w1 || !F.w2 || !F.dinv) return set_err(ctx, IGA_E_OOM, "fdm32 alloc");
  k_fdm_dinv<<<cdiv(mm, 256), 256, 0, st>>>(F.lam, n, ctx->dim, c, F.dinv); iga_count_launch();
  TRY(fdm_gemm_attrs(ctx));
  k_d2f_vec<<<cdiv((size_t)n * n, 256), 256, 0, st>>>(F.V, F.Vf, (size_t)n * n); iga_count_launch();
  k_transpose_f<<<cdiv((size_t)n * n, 256), 256, 0, st>>>(F.Vf, F.Vtf, n); iga_count_launch();
  CKL();
  int hinfo = 0;
  CK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hinfo) return set_err(ctx, IGA_E_INVALID, "mass matrix of the fast diagonalisation not positive definite");
  return IGA_OK;
}

static iga_status fdm_setup(iga_ctx* ctx) {
  const int n = ctx->mx;
  const int bw = (ctx->p + 4) / 2;
  TRY(fdm_build(ctx, ctx->fdmE, n, ctx->kc, ctx->mc, bw + 1, make_double2(-ctx->k2const, 0.0)));
  ctx->kcb = dalloc<double>(ctx, (size_t)n * (2 * bw + 1));
  ctx->mcb = dalloc<double>(ctx, (size_t)n * (2 * bw + 1));
  if (!ctx->kcb || !ctx->mcb) return set_err(ctx, IGA_E_OOM, "E bands");
  k_dense_to_band<<<cdiv((size_t)n * (2 * bw + 1), 128), 128, 0, ctx->st>>>(ctx->kc, n, bw, ctx->kcb); iga_count_launch();
  k_dense_to_band<<<cdiv((size_t)n * (2 * bw + 1), 128), 128, 0, ctx->st>>>(ctx->mc, n, bw, ctx->mcb); iga_count_launch();
  CKL();
  return IGA_OK;
}

// 1D: E = Z^T A Z is a band matrix of half bandwidth (p + 4) / 2 (a Z column
// covers at most five fine functions, A has half bandwidth p), whatever k(x)
// and the boundary terms; its band is probed with 2 (p + 4) / 2 + 1
// applications of Z^T A Z and factorised by the band solver.
static iga_status setup_banded_E(iga_ctx* ctx) {
  const int m = (int)ctx->m, bw = (ctx->p + 4) / 2;
  double2* Ab = dalloc<double2>(ctx, (size_t)m * (2 * bw + 1));
  if (!Ab) return set_err(ctx, IGA_E_OOM, "E band");
  auto apply = [ctx](const double2* c, double2* e) -> iga_status {
    TRY(defl_z(ctx, c, ctx->w0));
    TRY(op_apply<double>(ctx, 0, OP_A, ctx->w0, ctx->w1, nullptr, EPI_Y, nullptr, 0.0));
    return defl_zt(ctx, ctx->w1, e, nullptr);
  };
  TRY(band_probe(ctx, m, bw, apply, ctx->cs, ctx->cw, Ab));
  return band_setup(ctx, ctx->bandE, Ab, m, bw);
}

iga_status setup_deflation(iga_ctx* ctx) {
  LevelData& L = ctx->lv[0];
  ctx->mx = L.nx / 2;
  ctx->m = ctx->dim == 2 ? (size_t)ctx->mx * ctx->mx : (size_t)ctx->mx;
  if (ctx->mx < 1) return set_err(ctx, IGA_E_INVALID, "mesh too small for deflation");
  ctx->ct = dalloc<double2>(ctx, ctx->m);
  ctx->cs = dalloc<double2>(ctx, ctx->m);
  ctx->cw = dalloc<double2>(ctx, ctx->m);
  ctx->ce1 = dalloc<double2>(ctx, ctx->m);
  ctx->ce2 = dalloc<double2>(ctx, ctx->m);
  ctx->ctf = dalloc<float2>(ctx, ctx->m);
  ctx->cef = dalloc<float2>(ctx, ctx->m);
  if (!ctx->ce1 || !ctx->ce2 || !ctx->ctf || !ctx->cef) return set_err(ctx, IGA_E_OOM, "deflation alloc");
  // 1D: the band solver, except for small constant-k problems without a
  // Sommerfeld end, where the dense fast diagonalisation (a few tiny GEMVs)
  // beats a sequential band recurrence
  if (ctx->dim == 1 && (ctx->vark || ctx->robin_k != 0.0 || ctx->mx > FDM_TK)) return setup_banded_E(ctx);
  ctx->kc = dalloc<double>(ctx, (size_t)ctx->mx * ctx->mx);
  ctx->mc = dalloc<double>(ctx, (size_t)ctx->mx * ctx->mx);
  if (!ctx->ct || !ctx->cs || !ctx->cw || !ctx->kc || !ctx->mc) return set_err(ctx, IGA_E_OOM, "deflation alloc");
  k_coarse_1d<<<cdiv((size_t)ctx->mx * ctx->mx, 128), 128, 0, ctx->st>>>(L.nx, ctx->mx, ctx->p, ctx->prm.eps, L.K, L.M,
                                                                       ctx->kc, ctx->mc); iga_count_launch();
  CKL();
  if (ctx->vark) return setup_block_E(ctx);
  return fdm_setup(ctx);
}

iga_status defl_zt(iga_ctx* ctx, const double2* x, double2* c, float2* cf) {
  const LevelData& L = ctx->lv[0];
  int my = ctx->dim == 2 ? ctx->mx : 1;
  k_zt<<<cdiv(ctx->m, 256), 256, 0, ctx->st>>>(L.nx, L.ny, ctx->mx, my, ctx->prm.eps, x, c, cf); iga_count_launch();
  CKL();
  return IGA_OK;
}

iga_status defl_z(iga_ctx* ctx, const double2* c, double2* x) {
  const LevelData& L = ctx->lv[0];
  int my = ctx->dim == 2 ? ctx->mx : 1;
  k_z<<<cdiv(L.n, 256), 256, 0, ctx->st>>>(L.nx, L.ny, ctx->mx, my, ctx->prm.eps, c, x); iga_count_launch();
  CKL();
  return IGA_OK;
}

// s ~ Op^{-1} t by fast diagonalisation with FP32 transforms (the FP32
// intermediates live in F.w1, F.w2).  tf (optional): the same right-hand side
// already rounded to FP32 (saves every block of the first transform
// converting its FP64 panel).  accumulate: s += result.
static iga_status fdm_solve32(iga_ctx* ctx, const FdmData& F, const double2* t, double2* s, bool accumulate = false,
                              const float2* tf = nullptr) {
  const int mx = F.n;
  const float* V = F.Vf;
  const float* Vt = F.Vtf;
  if (ctx->dim == 1) {
    // s^T = ((t^T V) / d) V^T with t as a 1 x m row
    launch_fdm_gemm<false, true, false>(ctx, V, t, F.w1, 1, mx, F.dinv);
    if (accumulate) launch_fdm_gemm<false, false, true>(ctx, Vt, F.w1, s, 1, mx, nullptr);
    else launch_fdm_gemm<false, false, false>(ctx, Vt, F.w1, s, 1, mx, nullptr);
  } else {
    // T1 = V^T T; T2 = T1 V / D; T3 = V T2; S = T3 V^T (or s += S)
    if (tf) launch_fdm_gemm<true, false, false>(ctx, Vt, tf, F.w1, mx, mx, nullptr);
    else launch_fdm_gemm<true, false, false>(ctx, Vt, t, F.w1, mx, mx, nullptr);
    launch_fdm_gemm<false, true, false>(ctx, V, F.w1, F.w2, mx, mx, F.dinv);
    launch_fdm_gemm<true, false, false>(ctx, V, F.w2, F.w1, mx, mx, nullptr);
    if (accumulate) launch_fdm_gemm<false, false, true>(ctx, Vt, F.w1, s, mx, mx, nullptr);
    else launch_fdm_gemm<false, false, false>(ctx, Vt, F.w1, s, mx, mx, nullptr);
  }
  CKL();
  return IGA_OK;
}

// s = E0^{-1} t for the Kronecker-structured part E0 = Z^T (S - k^2 M) Z:
// fast diagonalisation with FP32 transforms and FP64 eigenvalue denominators,
// followed by fdmE.refine steps of iterative refinement s += FDM(t - E0 s) with
// the residual in FP64 (E0 applied by the banded tensor-product kernel on the
// coarse grid).  Two steps bring the solve to ~1e-11 of a sparse LU even where
// lambda_i + lambda_j ~ k^2 nearly cancels.
static iga_status e0_solve(iga_ctx* ctx, const double2* t, double2* s, const float2* tf) {
  TRY(fdm_solve32(ctx, ctx->fdmE, t, s, false, tf));
  const int bw = (ctx->p + 4) / 2;
  const int my = ctx->dim == 2 ? ctx->mx : 1;
  float2* rf = ctx->dim == 2 ? ctx->cef : nullptr;
  for (int it = 0; it < ctx->fdmE.refine; ++it) {
    TRY(op_apply_bands(ctx, bw, ctx->mx, my, ctx->kcb, ctx->mcb, make_double2(-ctx->k2const, 0.0), s, ctx->ce1, t,
                       EPI_ZMINUS, rf));
    TRY(fdm_solve32(ctx, ctx->fdmE, ctx->ce1, s, true, rf));   // s += FDM(r)
  }
  CKL();
  return IGA_OK;
}

// s = E^{-1} t.  Constant k by fast diagonalisation (e0_solve), 2D variable k
// by block LU, 1D otherwise (and above m_x = FDM_TK) by the band solver.
iga_status defl_esolve(iga_ctx* ctx, const double2* t, double2* s, const float2* tf) {
  if (ctx->dim == 1 && ctx->bandE.n > 0) return band_solve(ctx, ctx->bandE, t, s);
  if (ctx->vark) return block_E_solve(ctx, t, s);
  return e0_solve(ctx, t, s, tf);
}

// y = Q x = Z E^{-1} Z^T x
iga_status defl_q(iga_ctx* ctx, const double2* x, double2* y) {
  float2* ctf = (!ctx->vark && ctx->dim == 2) ? ctx->ctf : nullptr;
  TRY(defl_zt(ctx, x, ctx->ct, ctf));
  TRY(defl_esolve(ctx, ctx->ct, ctx->cs, ctf));
  return defl_z(ctx, ctx->cs, y);
}

// y = P x = x - A Z E^{-1} Z^T x  (the final A apply fuses the subtraction)
iga_status defl_apply(iga_ctx* ctx, const double2* x, double2* y) {
  TRY(defl_q(ctx, x, ctx->w3));
  return op_apply<double>(ctx, 0, OP_A, ctx->w3, y, x, EPI_ZMINUS, nullptr, 0.0);
}

__global__ void k_sub(const double2* a, const double2* b, double2* out, size_t n) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < n) out[e] = a[e] - b[e];
}

// y = P^T x = x - Q A x (A and Q complex symmetric, so P^T = I - Q A)
iga_status defl_apply_T(iga_ctx* ctx, const double2* x, double2* y, double2* tmp1, double2* tmp2) {
  const size_t n = ctx->lv[0].n;
  TRY(op_apply<double>(ctx, 0, OP_A, x, tmp1, nullptr, EPI_Y, nullptr, 0.0));
  TRY(defl_q(ctx, tmp1, tmp2));
  k_sub<<<cdiv(n, 256), 256, 0, ctx->st>>>(x, tmp2, y, n); iga_count_launch();
  CKL();
  return IGA_OK;
}

// ------------------------------------------------------------------ exact CSLP (C_ex)
// 1D: the band solver.  2D: the finest-level CSLP matrix
// M_beta = K (x) M + M (x) K - sigma k^2 M (x) M (constant k) is a
// tensor-product operator like E, so it is inverted by the
// same fast diagonalisation: the 1D pencil of the fine band matrices, complex
// denominators 1 / (lam_i + lam_j - sigma k^2), FP32 transforms and FP64
// iterative refinement whose residual r = t - M_beta s is the FP64 operator
// kernel of the finest level.
constexpr int EXACT_CSLP_MAX_N = 2048;

iga_status setup_exact_cslp(iga_ctx* ctx) {
  const LevelData& L = ctx->lv[0];
  if (ctx->dim == 1) {
    // 1D: M_beta (any k(x), with the Sommerfeld term where present) is a band
    // matrix of half bandwidth p; probed and factorised by the band solver
    double2* Ab = dalloc<double2>(ctx, (size_t)L.n * (2 * ctx->p + 1));
    if (!Ab) return set_err(ctx, IGA_E_OOM, "exact CSLP band");
    auto apply = [ctx](const double2* x, double2* y) -> iga_status {
      return op_apply<double>(ctx, 0, OP_MB, x, y, nullptr, EPI_Y, nullptr, 0.0);
    };
    TRY(band_probe(ctx, L.n, ctx->p, apply, ctx->w0, ctx->w1, Ab));
    return band_setup(ctx, ctx->bandX, Ab, L.n, ctx->p);
  }
  if (ctx->vark) return set_err(ctx, IGA_E_UNSUPPORTED, "exact CSLP in 2D: constant k only");
  const int n = L.nx, p = ctx->p;
  if (n > EXACT_CSLP_MAX_N)
    return set_err(ctx, IGA_E_UNSUPPORTED, "exact CSLP: n_x = %d above %d (dense 1D eigenvectors)", n, EXACT_CSLP_MAX_N);
  double* Kd = dalloc<double>(ctx, (size_t)n * n);
  double* Md = dalloc<double>(ctx, (size_t)n * n);
  ctx->cxr = dalloc<double2>(ctx, L.n);
  if (!Kd || !Md || !ctx->cxr) return set_err(ctx, IGA_E_OOM, "exact CSLP alloc");
  k_band_to_dense<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(L.K, n, p, Kd); iga_count_launch();
  k_band_to_dense<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(L.M, n, p, Md); iga_count_launch();
  CKL();
  const double2 c = make_double2(-ctx->sig.x * ctx->k2const, -ctx->sig.y * ctx->k2const);   // -sigma k^2
  TRY(fdm_build(ctx, ctx->fdmC, n, Kd, Md, p, c));
  ctx->fdmC.refine = 2;
  return IGA_OK;
}

// z = M_beta^{-1} r (finest level) to FP64 accuracy
iga_status cslp_exact_solve(iga_ctx* ctx, const double2* r, double2* z) {
  if (ctx->dim == 1) return band_solve(ctx, ctx->bandX, r, z);
  TRY(fdm_solve32(ctx, ctx->fdmC, r, z, false, nullptr));
  for (int it = 0; it < ctx->fdmC.refine; ++it) {
    TRY(op_apply<double>(ctx, 0, OP_MB, z, ctx->cxr, r, EPI_ZMINUS, nullptr, 0.0));
    TRY(fdm_solve32(ctx, ctx->fdmC, ctx->cxr, z, true, nullptr));
  }
  return IGA_OK;
}
