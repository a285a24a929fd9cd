// Setup kernels: knot vectors, Gauss tables, B-spline tables, 1D band matrices
// and knot-insertion transfer operators for every multigrid level.
//
// Everything here runs once per context; all of it is computed on the device.
// Paper: Section 2.3.1 (knots, Cox-de Boor), Section 2.3 (Galerkin matrices),
// Section 4.2 (transfer between nested spaces; linear interpolation at p = 1).
#include "common.cuh"
#include "bspline.cuh"
#include <cstdarg>
#include <cmath>

iga_status set_err(iga_ctx* c, iga_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

// Open uniform knot vector: p+1 zeros, i/n_el for i = 1..n_el-1 (one IEEE
// division each, never accumulated), p+1 ones.
__global__ void k_knots(double* t, int n_el, int p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int len = n_el + 2 * p + 1;
  if (i >= len) return;
  double v;
  if (i <= p) v = 0.0;
  else if (i >= n_el + p) v = 1.0;
  else v = (double)(i - p) / (double)n_el;
  t[i] = v;
}

// Per element e and Gauss point q: point, weight, values and derivatives of
// the p+1 active functions.  Point x = a + (b - a) * ((1 + g) / 2) and weight
// (w * (b - a)) / 2 are formed without contraction.
__global__ void k_tables(const double* t, int n_el, int p, double* xq, double* wq, double* B, double* D) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int Q = p + 1;
  if (idx >= n_el * Q) return;
  int e = idx / Q, q = idx % Q;
  double g, w;
  gauss_node(Q, q, &g, &w);
  int s = e + p;
  double a = t[s], b = t[s + 1];
  double h = __dadd_rn(b, -a);
  double x = __dadd_rn(a, __dmul_rn(h, __dadd_rn(1.0, g) / 2.0));
  xq[idx] = x;
  wq[idx] = __dmul_rn(w, h) / 2.0;
  double v[IGA_MAXP + 1], d[IGA_MAXP + 1];
  active_basis(t, p, s, x, v, d);
  for (int c = 0; c <= p; ++c) {
    B[(size_t)idx * (p + 1) + c] = v[c];
    D[(size_t)idx * (p + 1) + c] = d[c];
  }
}

// Interior 1D stiffness and mass bands: thread per (row i, offset d).
__global__ void k_bands(int n_el, int p, int nx, const double* wq, const double* B, const double* D,
                        double* K, double* M) {
  int W = 2 * p + 1;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nx * W) return;
  int i = idx / W, d = idx % W - p;
  int j = i + d;
  double kv = 0.0, mv = 0.0;
  if (j >= 0 && j < nx) {
    int bi = i + 1, bj = j + 1, Q = p + 1;
    int elo = max(max(bi, bj) - p, 0), ehi = min(min(bi, bj), n_el - 1);
    for (int e = elo; e <= ehi; ++e) {
      int a = bi - e, c = bj - e;
      double ks = 0.0, ms = 0.0;
      for (int q = 0; q < Q; ++q) {
        size_t o = ((size_t)e * Q + q) * (p + 1);
        double w = wq[e * Q + q];
        ks += w * D[o + a] * D[o + c];
        ms += w * B[o + a] * B[o + c];
      }
      kv += ks;
      mv += ms;
    }
  }
  K[idx] = kv;
  M[idx] = mv;
}

// Discrete B-spline (Oslo algorithm): coefficient of fine function i in the
// expansion of coarse function j, for nested knot vectors tau (coarse) and t
// (fine):  alpha_{j,0}(i) = [tau_j <= t_i < tau_{j+1}],
// alpha_{j,q}(i) = (t_{i+q} - tau_j)/(tau_{j+q} - tau_j) alpha_{j,q-1}(i)
//                + (tau_{j+q+1} - t_{i+q})/(tau_{j+q+1} - tau_{j+1}) alpha_{j+1,q-1}(i).
__device__ double oslo_alpha(const double* tau, const double* t, int p, int j, int i) {
  double a[IGA_MAXP + 1];
  for (int r = 0; r <= p; ++r) {
    int jj = j + r;
    a[r] = (tau[jj] <= t[i] && t[i] < tau[jj + 1]) ? 1.0 : 0.0;
  }
  for (int q = 1; q <= p; ++q)
    for (int r = 0; r <= p - q; ++r) {
      int jj = j + r;
      double v = 0.0;
      double d1 = tau[jj + q] - tau[jj];
      if (d1 != 0.0) v += (t[i + q] - tau[jj]) / d1 * a[r];
      double d2 = tau[jj + q + 1] - tau[jj + 1];
      if (d2 != 0.0) v += (tau[jj + q + 1] - t[i + q]) / d2 * a[r + 1];
      a[r] = v;
    }
  return a[0];
}

// Transfer rows are computed over a wide candidate window, then compacted to a
// tight window starting at the first non-zero; *err is set if a non-zero would
// be dropped.
#define IGA_TWIDE 16

// Prolongation rows: fine interior i -> coarse interior columns Plo[i] + k.
// keep_last = 1 (a Sommerfeld end at x = 1): the last function of both
// spaces is an unknown too.
__global__ void k_prolong_rows(const double* tc, const double* tf, int p, int nbc, int nbf, int wP,
                               double* Pw, int* Plo, int* err, int keep_last) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int nxf = nbf - 2 + keep_last;
  if (i >= nxf) return;
  int bi = i + 1;
  int lo = max(0, (bi - 1) / 2 - 4);
  double a[IGA_TWIDE];
  int k0 = -1;
  for (int k = 0; k < IGA_TWIDE; ++k) {
    int bj = lo + k;
    a[k] = (bj >= 1 && bj <= nbc - 2 + keep_last) ? oslo_alpha(tc, tf, p, bj, bi) : 0.0;
    if (a[k] != 0.0 && k0 < 0) k0 = k;
  }
  if (k0 < 0) k0 = 0;
  Plo[i] = lo + k0 - 1;
  for (int k = 0; k < wP; ++k) Pw[(size_t)i * wP + k] = (k0 + k < IGA_TWIDE) ? a[k0 + k] : 0.0;
  for (int k = k0 + wP; k < IGA_TWIDE; ++k)
    if (a[k] != 0.0) atomicExch(err, 1);
}

// Restriction rows: coarse interior j -> fine interior rows Rlo[j] + k.
__global__ void k_restrict_rows(const double* tc, const double* tf, int p, int nbc, int nbf, int wR,
                                double* Rw, int* Rlo, int* err, int keep_last) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int nxc = nbc - 2 + keep_last;
  if (j >= nxc) return;
  int bj = j + 1;
  int lo = max(0, 2 * bj - p - 4);
  double a[IGA_TWIDE];
  int k0 = -1;
  for (int k = 0; k < IGA_TWIDE; ++k) {
    int bi = lo + k;
    a[k] = (bi >= 1 && bi <= nbf - 2 + keep_last) ? oslo_alpha(tc, tf, p, bj, bi) : 0.0;
    if (a[k] != 0.0 && k0 < 0) k0 = k;
  }
  if (k0 < 0) k0 = 0;
  Rlo[j] = lo + k0 - 1;
  for (int k = 0; k < wR; ++k) Rw[(size_t)j * wR + k] = (k0 + k < IGA_TWIDE) ? a[k0 + k] : 0.0;
  for (int k = k0 + wR; k < IGA_TWIDE; ++k)
    if (a[k] != 0.0) atomicExch(err, 1);
}

__global__ void k_d2f(const double* a, float* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

static iga_status to_float(iga_ctx* ctx, const double* a, float** out, size_t n) {
  *out = dalloc<float>(ctx, n);
  if (!*out) return set_err(ctx, IGA_E_OOM, "alloc");
  k_d2f<<<cdiv(n, 256), 256, 0, ctx->st>>>(a, *out, n); iga_count_launch();
  CKL();
  return IGA_OK;
}

iga_status setup_levels(iga_ctx* ctx) {
  const int p = ctx->p, Q = p + 1, W = 2 * p + 1;
  int ne = ctx->prm.n_el;
  ctx->L = 0;
  while (true) {
    LevelData& L = ctx->lv[ctx->L];
    L.n_el = ne;
    L.nx = ne + p - 2 + (ctx->prm.robin ? 1 : 0);   // a Sommerfeld end keeps the last function
    L.ny = ctx->dim == 2 ? L.nx : 1;
    L.n = L.nx * L.ny;
    ctx->L++;
    if (!(ne % 2 == 0 && ne >= 8) || ctx->L == IGA_MAX_LEVELS) break;
    ne /= 2;
  }
  for (int l = 0; l < ctx->L; ++l) {
    LevelData& L = ctx->lv[l];
    int tl = L.n_el + 2 * p + 1;
    L.knots = dalloc<double>(ctx, tl);
    L.xq = dalloc<double>(ctx, (size_t)L.n_el * Q);
    L.wq = dalloc<double>(ctx, (size_t)L.n_el * Q);
    L.B = dalloc<double>(ctx, (size_t)L.n_el * Q * Q);
    L.D = dalloc<double>(ctx, (size_t)L.n_el * Q * Q);
    L.K = dalloc<double>(ctx, (size_t)L.nx * W);
    L.M = dalloc<double>(ctx, (size_t)L.nx * W);
    if (!L.knots || !L.xq || !L.wq || !L.B || !L.D || !L.K || !L.M) return set_err(ctx, IGA_E_OOM, "level alloc");
    k_knots<<<cdiv(tl, 128), 128, 0, ctx->st>>>(L.knots, L.n_el, p); iga_count_launch();
    CKL();
    k_tables<<<cdiv(L.n_el * Q, 128), 128, 0, ctx->st>>>(L.knots, L.n_el, p, L.xq, L.wq, L.B, L.D); iga_count_launch();
    CKL();
    k_bands<<<cdiv(L.nx * W, 128), 128, 0, ctx->st>>>(L.n_el, p, L.nx, L.wq, L.B, L.D, L.K, L.M); iga_count_launch();
    CKL();
    TRY(to_float(ctx, L.K, &L.Kf, (size_t)L.nx * W));
    TRY(to_float(ctx, L.M, &L.Mf, (size_t)L.nx * W));
    if (L.nx > 4 * p + 1) {   // the interior stencil (every row >= 2p from the ends), FP32, on the host
      const size_t ci = (size_t)(L.nx / 2) * W;
      CK(cudaMemcpyAsync(L.sK, L.Kf + ci, sizeof(float) * W, cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaMemcpyAsync(L.sM, L.Mf + ci, sizeof(float) * W, cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
      L.has_stencil = true;
    }
    TRY(to_float(ctx, L.B, &L.Bf, (size_t)L.n_el * Q * Q));
    TRY(to_float(ctx, L.wq, &L.wqf, (size_t)L.n_el * Q));
  }
  int* err = dalloc<int>(ctx, 1);
  if (!err) return set_err(ctx, IGA_E_OOM, "alloc");
  CK(cudaMemsetAsync(err, 0, sizeof(int), ctx->st));
  for (int l = 0; l + 1 < ctx->L; ++l) {
    LevelData& F = ctx->lv[l];
    LevelData& C = ctx->lv[l + 1];
    int nbf = F.n_el + p, nbc = C.n_el + p;
    F.wP = p / 2 + 3;
    F.wR = p + 3;
    F.Pw = dalloc<double>(ctx, (size_t)F.nx * F.wP);
    F.Plo = dalloc<int>(ctx, F.nx);
    F.Rw = dalloc<double>(ctx, (size_t)C.nx * F.wR);
    F.Rlo = dalloc<int>(ctx, C.nx);
    if (!F.Pw || !F.Plo || !F.Rw || !F.Rlo) return set_err(ctx, IGA_E_OOM, "transfer alloc");
    const int keep = ctx->prm.robin ? 1 : 0;
    k_prolong_rows<<<cdiv(F.nx, 128), 128, 0, ctx->st>>>(C.knots, F.knots, p, nbc, nbf, F.wP, F.Pw, F.Plo, err,
                                                          keep); iga_count_launch();
    CKL();
    k_restrict_rows<<<cdiv(C.nx, 128), 128, 0, ctx->st>>>(C.knots, F.knots, p, nbc, nbf, F.wR, F.Rw, F.Rlo, err,
                                                           keep); iga_count_launch();
    CKL();
    TRY(to_float(ctx, F.Pw, &F.Pwf, (size_t)F.nx * F.wP));
    TRY(to_float(ctx, F.Rw, &F.Rwf, (size_t)C.nx * F.wR));
  }
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (herr) return set_err(ctx, IGA_E_INVALID, "knot-insertion transfer wider than its window");
  return IGA_OK;
}
