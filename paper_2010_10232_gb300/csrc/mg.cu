// Geometric multigrid V-cycle for the CSLP (Section 3: damped Jacobi,
// omega = 0.6; Section 4.2: V-cycle with coarse correction between nested
// spline spaces).  Transfers are knot insertion (B-spline refinement), whose
// p = 1 case is the paper's linear interpolation; restriction is its
// transpose.  The coarsest level is solved with a dense inverse built at setup.
#include "common.cuh"

// ------------------------------------------------------------------ kernels
// First Jacobi sweep from x = 0:  x = omega D^{-1} b.
template <typename T>
__global__ void k_jacobi0(int nx, int ny, int p, const T* K, const T* M, typename cplx<T>::t c,
                          const typename cplx<T>::t* dinv, const typename cplx<T>::t* b,
                          typename cplx<T>::t* x, T omega) {
  using C = typename cplx<T>::t;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nx * ny) return;
  C di;
  if (dinv) {
    di = dinv[i];
  } else {
    int W = 2 * p + 1;
    int iy = (int)(i / nx), ix = (int)(i - (size_t)iy * nx);
    T kx = K[(size_t)ix * W + p], mx = M[(size_t)ix * W + p];
    C d;
    if (ny == 1) {
      d = mkc(kx, (T)0) + mx * c;
    } else {
      T ky = K[(size_t)iy * W + p], my = M[(size_t)iy * W + p];
      d = my * (mkc(kx, (T)0) + mx * c) + mkc(ky * mx, (T)0);
    }
    di = cinv(d);
  }
  x[i] = omega * cmul(di, b[i]);
}

// coarse = P^T fine  (2D: tensor product of the 1D restriction rows)
// With xc != nullptr the same kernel also performs the coarse level's first
// damped Jacobi sweep from zero, xc = omega D_c^{-1} c (D_c from the coarse 1D
// band diagonals, or dinv for variable k).
template <typename T>
__global__ void k_restrict(int nxf, int nyf, int nxc, int nyc, int wR, const T* Rw, const int* Rlo,
                           const typename cplx<T>::t* f, typename cplx<T>::t* c, typename cplx<T>::t* xc, int p,
                           const T* Kc, const T* Mc, typename cplx<T>::t cm, const typename cplx<T>::t* dinv,
                           T omega) {
  using C = typename cplx<T>::t;
  size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (j >= (size_t)nxc * nyc) return;
  int jy = (int)(j / nxc), jx = (int)(j - (size_t)jy * nxc);
  C acc = czero<C>();
  int lx = Rlo[jx];
  if (nyc == 1) {
    for (int kx = 0; kx < wR; ++kx) {
      int ix = lx + kx;
      T w = Rw[(size_t)jx * wR + kx];
      if (w != (T)0 && ix >= 0 && ix < nxf) acc = cfma(w, f[ix], acc);
    }
  } else {
    int ly = Rlo[jy];
    for (int ky = 0; ky < wR; ++ky) {
      int iy = ly + ky;
      T wy = Rw[(size_t)jy * wR + ky];
      if (wy == (T)0 || iy < 0 || iy >= nyf) continue;
      C row = czero<C>();
      for (int kx = 0; kx < wR; ++kx) {
        int ix = lx + kx;
        T w = Rw[(size_t)jx * wR + kx];
        if (w != (T)0 && ix >= 0 && ix < nxf) row = cfma(w, f[(size_t)iy * nxf + ix], row);
      }
      acc = cfma(wy, row, acc);
    }
  }
  c[j] = acc;
  if (xc) {
    C di;
    if (dinv) {
      di = dinv[j];
    } else {
      int W = 2 * p + 1;
      T kx = Kc[(size_t)jx * W + p], mx = Mc[(size_t)jx * W + p];
      C d;
      if (nyc == 1) {
        d = mkc(kx, (T)0) + mx * cm;
      } else {
        T ky = Kc[(size_t)jy * W + p], my = Mc[(size_t)jy * W + p];
        d = my * (mkc(kx, (T)0) + mx * cm) + mkc(ky * mx, (T)0);
      }
      di = cinv(d);
    }
    xc[j] = omega * cmul(di, acc);
  }
}

// fine += P coarse
template <typename T>
__global__ void k_prolong_add(int nxf, int nyf, int nxc, int nyc, int wP, const T* Pw, const int* Plo,
                              const typename cplx<T>::t* c, typename cplx<T>::t* f) {
  using C = typename cplx<T>::t;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nxf * nyf) return;
  int iy = (int)(i / nxf), ix = (int)(i - (size_t)iy * nxf);
  C acc = czero<C>();
  int lx = Plo[ix];
  if (nyf == 1) {
    for (int kx = 0; kx < wP; ++kx) {
      int jx = lx + kx;
      T w = Pw[(size_t)ix * wP + kx];
      if (w != (T)0 && jx >= 0 && jx < nxc) acc = cfma(w, c[jx], acc);
    }
  } else {
    int ly = Plo[iy];
    for (int ky = 0; ky < wP; ++ky) {
      int jy = ly + ky;
      T wy = Pw[(size_t)iy * wP + ky];
      if (wy == (T)0 || jy < 0 || jy >= nyc) continue;
      C row = czero<C>();
      for (int kx = 0; kx < wP; ++kx) {
        int jx = lx + kx;
        T w = Pw[(size_t)ix * wP + kx];
        if (w != (T)0 && jx >= 0 && jx < nxc) row = cfma(w, c[(size_t)jy * nxc + jx], row);
      }
      acc = cfma(wy, row, acc);
    }
  }
  f[i] = f[i] + acc;
}

// x = Minv b, one block, dense
template <typename C>
__global__ void k_dense_mv(int n, const C* Minv, const C* b, C* x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    C acc = czero<C>();
    for (int j = 0; j < n; ++j) acc = acc + cmul(Minv[(size_t)i * n + j], b[j]);
    x[i] = acc;
  }
}

// Gauss-Jordan inversion with partial pivoting (one block): A (n x n, row
// major, destroyed), Inv starts as the identity.
__global__ void k_gauss_jordan(double2* A, double2* Inv, int n, int* info) {
  extern __shared__ double2 fcol[];
  __shared__ int piv;
  __shared__ double2 pinv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int best = k;
      double bv = -1.0;
      for (int i = k; i < n; ++i) {
        double2 v = A[(size_t)i * n + k];
        double m = v.x * v.x + v.y * v.y;
        if (m > bv) { bv = m; best = i; }
      }
      piv = best;
      if (!(bv > 0.0)) *info = 1;
    }
    __syncthreads();
    if (piv != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double2 t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)piv * n + j]; A[(size_t)piv * n + j] = t;
        t = Inv[(size_t)k * n + j]; Inv[(size_t)k * n + j] = Inv[(size_t)piv * n + j]; Inv[(size_t)piv * n + j] = t;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) pinv = cinv(A[(size_t)k * n + k]);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      A[(size_t)k * n + j] = cmul(pinv, A[(size_t)k * n + j]);
      Inv[(size_t)k * n + j] = cmul(pinv, Inv[(size_t)k * n + j]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = A[(size_t)i * n + k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      int i = idx / n, j = idx - i * n;
      if (i == k) continue;
      double2 f = fcol[i];
      A[(size_t)i * n + j] = A[(size_t)i * n + j] - cmul(f, A[(size_t)k * n + j]);
      Inv[(size_t)i * n + j] = Inv[(size_t)i * n + j] - cmul(f, Inv[(size_t)k * n + j]);
    }
    __syncthreads();
  }
}

__global__ void k_unit(double2* e, int n, int j) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) e[i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}
__global__ void k_eye(double2* e, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * n) e[i] = make_double2((i / n) == (i % n) ? 1.0 : 0.0, 0.0);
}
// columns (stored as rows of colsT) -> row-major matrix
__global__ void k_transpose_c(const double2* colsT, double2* A, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * n) { int r = i / n, c = i % n; A[(size_t)r * n + c] = colsT[(size_t)c * n + r]; }
}
__global__ void k_c2f(const double2* a, float2* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = tof(a[i]);
}
__global__ void k_f2d(const float2* a, double2* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = tod(a[i]);
}
template <typename C>
__global__ void k_axpy1(C* y, const C* x, size_t n) {   // y += x
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = y[i] + x[i];
}

void launch_convert_d2f(const double2* a, float2* b, size_t n, cudaStream_t st) {
  k_c2f<<<cdiv(n, 256), 256, 0, st>>>(a, b, n); iga_count_launch();
}
void launch_convert_f2d(const float2* a, double2* b, size_t n, cudaStream_t st) {
  k_f2d<<<cdiv(n, 256), 256, 0, st>>>(a, b, n); iga_count_launch();
}

// ------------------------------------------------------------------ host
iga_status setup_coarse_inverse(iga_ctx* ctx) {
  int l = ctx->L - 1;
  LevelData& L = ctx->lv[l];
  int n = L.n;
  ctx->nc = n;
  // one block inverts the coarsest matrix (a row of it in shared memory)
  if (n > IGA_MAX_COARSEST)
    return set_err(ctx, IGA_E_INVALID,
                   "coarsest level has %d dofs (> %d): n_el must halve to a coarsest mesh of at most ~%d "
                   "elements per direction", n, IGA_MAX_COARSEST, 40);
  double2* cols = dalloc<double2>(ctx, (size_t)n * n);   // row j = M_beta e_j
  double2* A = dalloc<double2>(ctx, (size_t)n * n);
  double2* e = dalloc<double2>(ctx, n);
  ctx->cinv = dalloc<double2>(ctx, (size_t)n * n);
  ctx->cinvf = dalloc<float2>(ctx, (size_t)n * n);
  int* info = dalloc<int>(ctx, 1);
  if (!cols || !A || !e || !ctx->cinv || !ctx->cinvf || !info) return set_err(ctx, IGA_E_OOM, "coarse alloc");
  for (int j = 0; j < n; ++j) {
    k_unit<<<cdiv(n, 128), 128, 0, ctx->st>>>(e, n, j); iga_count_launch();
    TRY(op_apply<double>(ctx, l, OP_MB, e, cols + (size_t)j * n, nullptr, EPI_Y, nullptr, 0.0));
  }
  k_transpose_c<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(cols, A, n); iga_count_launch();
  k_eye<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(ctx->cinv, n); iga_count_launch();
  CK(cudaMemsetAsync(info, 0, sizeof(int), ctx->st));
  k_gauss_jordan<<<1, 256, n * sizeof(double2), ctx->st>>>(A, ctx->cinv, n, info); iga_count_launch();
  CKL();
  k_c2f<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(ctx->cinv, ctx->cinvf, (size_t)n * n); iga_count_launch();
  int hinfo = 0;
  CK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (hinfo) return set_err(ctx, IGA_E_INVALID, "coarsest CSLP matrix is singular");
  return IGA_OK;
}

template <typename T> struct LvBuf;
template <> struct LvBuf<double> {
  static double2* b(LevelData& L) { return L.vb; }
  static double2* x(LevelData& L) { return L.vx; }
  static double2* y(LevelData& L) { return L.vy; }
  static double2* r(LevelData& L) { return L.vr; }
  static const double* K(LevelData& L) { return L.K; }
  static const double* M(LevelData& L) { return L.M; }
  static const double2* dinv(LevelData& L) { return L.dinv; }
  static const double* Pw(LevelData& L) { return L.Pw; }
  static const double* Rw(LevelData& L) { return L.Rw; }
  static const double2* cinv(iga_ctx* c) { return c->cinv; }
};
template <> struct LvBuf<float> {
  static float2* b(LevelData& L) { return L.fb; }
  static float2* x(LevelData& L) { return L.fx; }
  static float2* y(LevelData& L) { return L.fy; }
  static float2* r(LevelData& L) { return L.fr; }
  static const float* K(LevelData& L) { return L.Kf; }
  static const float* M(LevelData& L) { return L.Mf; }
  static const float2* dinv(LevelData& L) { return L.dinvf; }
  static const float* Pw(LevelData& L) { return L.Pwf; }
  static const float* Rw(LevelData& L) { return L.Rwf; }
  static const float2* cinv(iga_ctx* c) { return c->cinvf; }
};

// D^{-1} for the Jacobi sweeps where it is kept in memory: every 2D FP64 level
// (FP64 division is slow), FP32 only with variable k; else formed on the fly
template <typename T>
static const typename cplx<T>::t* jac_dinv(iga_ctx* ctx, LevelData& L) {
  if (ctx->dim != 2) return nullptr;
  if (sizeof(T) == 8 || ctx->vark) return LvBuf<T>::dinv(L);
  return nullptr;
}

template <typename T>
iga_status mg_jacobi0(iga_ctx* ctx, int l, const typename cplx<T>::t* b, typename cplx<T>::t* x) {
  using C = typename cplx<T>::t;
  LevelData& L = ctx->lv[l];
  double2 cm = make_double2(-ctx->sig.x, -ctx->sig.y);
  if (!ctx->vark) cm = ctx->k2const * cm;
  const C* dinv = jac_dinv<T>(ctx, L);
  k_jacobi0<T><<<cdiv(L.n, 256), 256, 0, ctx->st>>>(L.nx, L.ny, ctx->p, LvBuf<T>::K(L), LvBuf<T>::M(L),
                                                    cconv<C>(cm), dinv, b, x, (T)ctx->prm.omega); iga_count_launch();
  CKL();
  return IGA_OK;
}

template <typename T>
iga_status mg_restrict(iga_ctx* ctx, int l, const typename cplx<T>::t* f, typename cplx<T>::t* c) {
  LevelData& F = ctx->lv[l];
  LevelData& Cc = ctx->lv[l + 1];
  k_restrict<T><<<cdiv(Cc.n, 256), 256, 0, ctx->st>>>(F.nx, F.ny, Cc.nx, Cc.ny, F.wR, LvBuf<T>::Rw(F), F.Rlo, f, c,
                                                     nullptr, 0, nullptr, nullptr, czero<typename cplx<T>::t>(),
                                                     nullptr, (T)0); iga_count_launch();
  CKL();
  return IGA_OK;
}

// c = P^T f and xc = omega D_c^{-1} c (the coarse level's first Jacobi sweep)
template <typename T>
static iga_status mg_restrict_j0(iga_ctx* ctx, int l, const typename cplx<T>::t* f, typename cplx<T>::t* c,
                                 typename cplx<T>::t* xc) {
  using C = typename cplx<T>::t;
  LevelData& F = ctx->lv[l];
  LevelData& Cc = ctx->lv[l + 1];
  double2 cm = make_double2(-ctx->sig.x, -ctx->sig.y);
  if (!ctx->vark) cm = ctx->k2const * cm;
  const C* dinv = jac_dinv<T>(ctx, Cc);
  k_restrict<T><<<cdiv(Cc.n, 256), 256, 0, ctx->st>>>(F.nx, F.ny, Cc.nx, Cc.ny, F.wR, LvBuf<T>::Rw(F), F.Rlo, f, c, xc,
                                                     ctx->p, LvBuf<T>::K(Cc), LvBuf<T>::M(Cc), cconv<C>(cm), dinv,
                                                     (T)ctx->prm.omega); iga_count_launch();
  CKL();
  return IGA_OK;
}

template <typename T>
iga_status mg_prolong_add(iga_ctx* ctx, int l, const typename cplx<T>::t* c, typename cplx<T>::t* f) {
  LevelData& F = ctx->lv[l];
  LevelData& Cc = ctx->lv[l + 1];
  k_prolong_add<T><<<cdiv(F.n, 256), 256, 0, ctx->st>>>(F.nx, F.ny, Cc.nx, Cc.ny, F.wP, LvBuf<T>::Pw(F), F.Plo, c, f); iga_count_launch();
  CKL();
  return IGA_OK;
}

template <typename T>
iga_status mg_coarse(iga_ctx* ctx, const typename cplx<T>::t* b, typename cplx<T>::t* x) {
  using C = typename cplx<T>::t;
  k_dense_mv<C><<<1, 256, 0, ctx->st>>>(ctx->nc, LvBuf<T>::cinv(ctx), b, x); iga_count_launch();
  CKL();
  return IGA_OK;
}

// One V-cycle on level l for M_beta x = b from x = 0.  The result is written to
// `out`; `alt` is a second level-sized buffer used for Jacobi ping-pong.
// Buffer (out or alt) in which level l's pre-smoothing starts, so that the
// last post-sweep lands in `out`.
static int start_buffer(iga_ctx* ctx) {
  const int nu1 = ctx->prm.nu_pre, nu2 = ctx->prm.nu_post;
  const int before_post = nu2 & 1;
  return (nu1 >= 1) ? (before_post ^ ((nu1 - 1) & 1)) : before_post;
}

// pre_done: the first Jacobi sweep (from zero) was already written into the
// start buffer by the parent's fused restriction.
template <typename T>
static iga_status vcycle_level(iga_ctx* ctx, int l, const typename cplx<T>::t* b, typename cplx<T>::t* out,
                               typename cplx<T>::t* alt, bool pre_done = false) {
  using C = typename cplx<T>::t;
  LevelData& L = ctx->lv[l];
  if (l == ctx->L - 1) return mg_coarse<T>(ctx, b, out);
  const int nu1 = ctx->prm.nu_pre, nu2 = ctx->prm.nu_post;
  const double om = ctx->prm.omega;
  // Choose the buffer the pre-smoother starts in so that, after the nu2
  // post-sweeps (each flips the buffer), the result lands in `out`.
  C* bufs[2] = {out, alt};
  int cur = start_buffer(ctx);
  if (nu1 >= 1) {
    if (!pre_done) TRY(mg_jacobi0<T>(ctx, l, b, bufs[cur]));
    for (int s = 1; s < nu1; ++s) {
      TRY(op_apply<T>(ctx, l, OP_MB, bufs[cur], bufs[cur ^ 1], nullptr, EPI_JACOBI, b, om));
      cur ^= 1;
    }
  } else {
    CK(cudaMemsetAsync(bufs[cur], 0, sizeof(C) * L.n, ctx->st));
  }
  C* r = LvBuf<T>::r(L);
  if (nu1 >= 1) {
    TRY(op_apply<T>(ctx, l, OP_MB, bufs[cur], r, b, EPI_ZMINUS, nullptr, 0.0));
  } else {
    CK(cudaMemcpyAsync(r, b, sizeof(C) * L.n, cudaMemcpyDeviceToDevice, ctx->st));
  }
  LevelData& Cl = ctx->lv[l + 1];
  if (nu1 >= 1 && l + 1 < ctx->L - 1) {
    C* cstart = start_buffer(ctx) ? LvBuf<T>::y(Cl) : LvBuf<T>::x(Cl);
    TRY(mg_restrict_j0<T>(ctx, l, r, LvBuf<T>::b(Cl), cstart));
    TRY(vcycle_level<T>(ctx, l + 1, LvBuf<T>::b(Cl), LvBuf<T>::x(Cl), LvBuf<T>::y(Cl), true));
  } else {
    TRY(mg_restrict<T>(ctx, l, r, LvBuf<T>::b(Cl)));
    TRY(vcycle_level<T>(ctx, l + 1, LvBuf<T>::b(Cl), LvBuf<T>::x(Cl), LvBuf<T>::y(Cl)));
  }
  TRY(mg_prolong_add<T>(ctx, l, LvBuf<T>::x(Cl), bufs[cur]));
  for (int s = 0; s < nu2; ++s) {
    TRY(op_apply<T>(ctx, l, OP_MB, bufs[cur], bufs[cur ^ 1], nullptr, EPI_JACOBI, b, om));
    cur ^= 1;
  }
  if (cur != 0) CK(cudaMemcpyAsync(out, bufs[cur], sizeof(C) * L.n, cudaMemcpyDeviceToDevice, ctx->st));
  return IGA_OK;
}

// z = n_vcycles V-cycles applied to r on the finest level (stationary
// iteration z <- z + V(r - M_beta z) from z = 0).
// one V-cycle from zero on the finest level: the fused level kernels where they
// apply (2D, constant k, one pre- and one post-sweep, FP32), else operation by
// operation
// (in FP64 the halo recomputation costs more FP64 work than the saved
// launches are worth)
template <typename T>
static iga_status vcycle0(iga_ctx* ctx, const typename cplx<T>::t* b, typename cplx<T>::t* out) {
  if (ctx->vc_fused && sizeof(T) == 4) return mg_vcycle_fused<T>(ctx, b, out);
  return vcycle_level<T>(ctx, 0, b, out, LvBuf<T>::y(ctx->lv[0]));
}

template <typename T>
iga_status mg_vcycle(iga_ctx* ctx, const typename cplx<T>::t* r, typename cplx<T>::t* z) {
  using C = typename cplx<T>::t;
  LevelData& L = ctx->lv[0];
  TRY(vcycle0<T>(ctx, r, z));
  for (int c = 1; c < ctx->prm.n_vcycles; ++c) {
    C* res = LvBuf<T>::b(L);
    C* e = LvBuf<T>::x(L);
    TRY(op_apply<T>(ctx, 0, OP_MB, z, res, r, EPI_ZMINUS, nullptr, 0.0));
    TRY(vcycle0<T>(ctx, res, e));
    k_axpy1<C><<<cdiv(L.n, 256), 256, 0, ctx->st>>>(z, e, L.n); iga_count_launch();
    CKL();
  }
  return IGA_OK;
}

template iga_status mg_vcycle<double>(iga_ctx*, const double2*, double2*);
template iga_status mg_vcycle<float>(iga_ctx*, const float2*, float2*);
template iga_status mg_restrict<double>(iga_ctx*, int, const double2*, double2*);
template iga_status mg_prolong_add<double>(iga_ctx*, int, const double2*, double2*);
template iga_status mg_coarse<double>(iga_ctx*, const double2*, double2*);
template iga_status mg_coarse<float>(iga_ctx*, const float2*, float2*);
template iga_status mg_jacobi0<double>(iga_ctx*, int, const double2*, double2*);
