// C ABI of the IgA Helmholtz library (declared in include/iga_helmholtz.h).
// Argument checking, context construction and dispatch to the kernels.
#include "common.cuh"
#include "bspline.cuh"
#include <cmath>
#include <new>
#include <type_traits>

#include <atomic>

static bool aligned16(const void* p) { return p && (((uintptr_t)p) & 15u) == 0; }
static std::atomic<unsigned long long> g_launches{0};
void iga_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void iga_add_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

extern "C" {

void iga_default_params(iga_params* prm) {
  if (!prm) return;
  iga_params d{};
  d.dim = 2;
  d.p = 3;
  d.n_el = 32;
  d.n_lines = 0;
  d.k_values[0] = 10.0;
  d.beta1 = 1.0;
  d.beta2 = 0.5;
  d.eps = 0.0;
  d.nu_pre = 1;
  d.nu_post = 1;
  d.omega = 0.6;
  d.n_vcycles = 1;
  d.precision = 0;
  d.flexible = 0;
  d.skip_deflation = 0;
  d.host_loop = 0;
  d.arnoldi = 1;
  d.fused_vcycle = 0;
  d.stream = nullptr;
  d.precond = 0;
  d.deflation = 1;
  d.robin = 0;
  *prm = d;
}

const char* iga_status_str(iga_status s) {
  switch (s) {
    case IGA_OK: return "IGA_OK";
    case IGA_NOT_CONVERGED: return "IGA_NOT_CONVERGED";
    case IGA_E_INVALID: return "IGA_E_INVALID";
    case IGA_E_CUDA: return "IGA_E_CUDA";
    case IGA_E_OOM: return "IGA_E_OOM";
    case IGA_E_BREAKDOWN: return "IGA_E_BREAKDOWN";
    case IGA_E_NONFINITE: return "IGA_E_NONFINITE";
    case IGA_E_TIMEOUT: return "IGA_E_TIMEOUT";
    case IGA_E_UNSUPPORTED: return "IGA_E_UNSUPPORTED";
  }
  return "unknown";
}

const char* iga_last_error(const iga_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

unsigned long long iga_launch_count(void) { return g_launches.load(); }

static iga_status alloc_level_vectors(iga_ctx* ctx) {
  for (int l = 0; l < ctx->L; ++l) {
    LevelData& L = ctx->lv[l];
    L.vb = dalloc<double2>(ctx, L.n);
    L.vx = dalloc<double2>(ctx, L.n);
    L.vy = dalloc<double2>(ctx, L.n);
    L.vr = dalloc<double2>(ctx, L.n);
    L.fb = dalloc<float2>(ctx, L.n);
    L.fx = dalloc<float2>(ctx, L.n);
    L.fy = dalloc<float2>(ctx, L.n);
    L.fr = dalloc<float2>(ctx, L.n);
    if (!L.vb || !L.vx || !L.vy || !L.vr || !L.fb || !L.fx || !L.fy || !L.fr)
      return set_err(ctx, IGA_E_OOM, "level vectors");
  }
  return IGA_OK;
}

iga_status iga_setup(const iga_params* prm, iga_ctx** out) {
  if (!prm || !out) return IGA_E_INVALID;
  *out = nullptr;
  const iga_params& P = *prm;
  if (P.dim != 1 && P.dim != 2) return IGA_E_INVALID;
  if (P.p < 1 || P.p > IGA_MAXP) return IGA_E_INVALID;
  if (P.n_el < 2 || P.n_el + P.p - 2 < 2) return IGA_E_INVALID;
  if (P.n_lines < 0 || P.n_lines > IGA_MAX_LINES || (P.n_lines > 0 && P.dim != 2)) return IGA_E_INVALID;
  if (!(P.omega > 0.0) || P.nu_pre < 0 || P.nu_post < 0 || P.n_vcycles < 0) return IGA_E_INVALID;
  if (P.precond < 0 || P.precond > 1 || P.deflation < 0 || P.deflation > 2) return IGA_E_INVALID;
  if (P.precond == 0 && P.n_vcycles < 1 && P.deflation == 0) return IGA_E_INVALID;   // nothing left to solve with
  if (P.deflation == 2 && (P.precision != 0 || P.flexible != 0)) return IGA_E_INVALID;
  if (P.precond == 1 && P.n_lines > 0) return IGA_E_UNSUPPORTED;
  if (P.robin < 0 || P.robin > 1) return IGA_E_INVALID;
  if (P.robin && (P.dim != 1 || P.n_lines > 0)) return IGA_E_UNSUPPORTED;     // 1D, constant k
  if (P.precision < 0 || P.precision > 1) return IGA_E_INVALID;
  if (P.arnoldi < 0 || P.arnoldi > 1) return IGA_E_INVALID;
  if (P.fused_vcycle < 0 || P.fused_vcycle > 1) return IGA_E_INVALID;
  for (int l = 0; l <= P.n_lines; ++l)
    if (!std::isfinite(P.k_values[l]) || P.k_values[l] < 0.0) return IGA_E_INVALID;
  iga_ctx* ctx = new (std::nothrow) iga_ctx();
  if (!ctx) return IGA_E_OOM;
  ctx->prm = P;
  ctx->dim = P.dim;
  ctx->p = P.p;
  ctx->Q = P.p + 1;
  ctx->st = (cudaStream_t)P.stream;
  ctx->vark = P.n_lines > 0;
  ctx->kf.n_lines = P.n_lines;
  for (int l = 0; l < IGA_MAX_LINES; ++l)
    for (int c = 0; c < 3; ++c) ctx->kf.lines[l][c] = l < P.n_lines ? P.lines[l][c] : 0.0;
  for (int l = 0; l <= IGA_MAX_LINES; ++l) ctx->kf.k2[l] = l <= P.n_lines ? P.k_values[l] * P.k_values[l] : 0.0;
  ctx->k2const = P.k_values[0] * P.k_values[0];
  ctx->robin_k = P.robin ? P.k_values[0] : 0.0;     // 1D: k at x = 1
  ctx->sig = make_double2(P.beta1, -P.beta2);
  ctx->use_graph = P.host_loop == 0;
  ctx->arnoldi_cgs = P.arnoldi == 1;
  for (int l = 0; l < IGA_MAX_LEVELS; ++l) ctx->tile[l][0] = ctx->tile[l][1] = -1;
  iga_status s = IGA_OK;
  do {
    if (cudaGetDevice(&ctx->device) != cudaSuccess) { s = set_err(ctx, IGA_E_CUDA, "no CUDA device"); break; }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if ((s = setup_levels(ctx)) != IGA_OK) break;
    if (ctx->vark && ctx->dim == 2)
      for (int l = 0; l < ctx->L && s == IGA_OK; ++l) s = setup_vark_diag(ctx, l);
    if (s != IGA_OK) break;
    if ((s = setup_const_dinv(ctx)) != IGA_OK) break;
    if ((s = setup_robin_dinv(ctx)) != IGA_OK) break;
    if ((s = setup_tiled_transfers(ctx)) != IGA_OK) break;
    if ((s = alloc_level_vectors(ctx)) != IGA_OK) break;
    if ((s = autotune_tiles(ctx)) != IGA_OK) break;
    if ((s = setup_coarse_inverse(ctx)) != IGA_OK) break;
    if ((s = setup_fused_vcycle(ctx)) != IGA_OK) break;
    size_t n = ctx->lv[0].n;
    ctx->w0 = dalloc<double2>(ctx, n);
    ctx->w1 = dalloc<double2>(ctx, n);
    ctx->w2 = dalloc<double2>(ctx, n);
    ctx->w3 = dalloc<double2>(ctx, n);
    ctx->fin = dalloc<float2>(ctx, n);
    ctx->fout = dalloc<float2>(ctx, n);
    ctx->partials = dalloc<double>(ctx, 4 * (size_t)(2 * ctx->num_sms) + 16);
    if (!ctx->w0 || !ctx->w1 || !ctx->w2 || !ctx->w3 || !ctx->fin || !ctx->fout || !ctx->partials) {
      s = set_err(ctx, IGA_E_OOM, "work vectors");
      break;
    }
    if (!P.skip_deflation && P.deflation != 0 && (s = setup_deflation(ctx)) != IGA_OK) break;
    if (P.precond == 1 && (s = setup_exact_cslp(ctx)) != IGA_OK) break;
    cudaError_t e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) { s = set_err(ctx, IGA_E_CUDA, "setup: %s", cudaGetErrorString(e)); break; }
  } while (0);
  if (s != IGA_OK) {
    fprintf(stderr, "iga_setup: %s: %s\n", iga_status_str(s), ctx->err.c_str());
    delete ctx;
    return s;
  }
  *out = ctx;
  return IGA_OK;
}

}  // extern "C"

// A context for the same problem that shares every setup table, factor and
// tuned tile shape of `parent` and owns fresh copies of everything a solve
// writes (level vectors, work vectors, deflation and band-solve scratch; the
// Krylov workspace is allocated by its first solve), so that it can solve at
// the same time as the parent.  Owned by the parent (iga_destroy).  Not for a
// context with a network attached (the network's buffers are not copied).
iga_ctx* clone_workspace(iga_ctx* parent) {
  iga_ctx* c = new (std::nothrow) iga_ctx(*parent);
  if (!c) return nullptr;
  c->bufs.ptrs.clear();            // the parent's allocations stay the parent's
  c->clones.clear();
  c->err.clear();
  c->graph = nullptr; c->gexec = nullptr; c->cap_stream = nullptr; c->gcond = 0;
  c->graph_flex = false; c->graph_maxit = 0; c->body_kernels = 0;
  c->maxit_alloc = -1;
  c->Vb = c->Zb = c->H = c->gsn = c->gg = c->gy = nullptr;
  c->gstate = nullptr; c->gflag = nullptr; c->hflag = nullptr;
  c->kvec = nullptr; c->kint = nullptr; c->kbar = nullptr;
  c->cgs_part = nullptr; c->cgs_h = nullptr; c->cgs_ticket = nullptr;
  c->hf = c->hu = nullptr; c->brec = nullptr; c->brec_cap = 0; c->hres = nullptr;
  c->net = nullptr; c->net_rms = nullptr; c->net_bad = nullptr;
  bool ok = alloc_level_vectors(c) == IGA_OK;
  const size_t n = c->lv[0].n;
  auto fresh = [&](auto*& ptr, size_t count) {
    using E = std::remove_reference_t<decltype(*ptr)>;
    if (!ptr) return;
    ptr = dalloc<E>(c, count);
    ok = ok && ptr != nullptr;
  };
  fresh(c->w0, n); fresh(c->w1, n); fresh(c->w2, n); fresh(c->w3, n);
  fresh(c->fin, n); fresh(c->fout, n);
  fresh(c->partials, 4 * (size_t)(2 * c->num_sms) + 16);
  fresh(c->ct, c->m); fresh(c->cs, c->m); fresh(c->cw, c->m); fresh(c->ce1, c->m); fresh(c->ce2, c->m);
  fresh(c->ctf, c->m); fresh(c->cef, c->m);
  const size_t mmE = c->fdmE.n ? (c->dim == 2 ? (size_t)c->fdmE.n * c->fdmE.n : (size_t)c->fdmE.n) : 0;
  fresh(c->fdmE.w1, mmE); fresh(c->fdmE.w2, mmE);
  const size_t mmC = c->fdmC.n ? (c->dim == 2 ? (size_t)c->fdmC.n * c->fdmC.n : (size_t)c->fdmC.n) : 0;
  fresh(c->fdmC.w1, mmC); fresh(c->fdmC.w2, mmC);
  fresh(c->cxr, n);
  fresh(c->ep_t, (size_t)c->enb * c->eblk); fresh(c->ep_g, (size_t)c->enb * c->eblk); fresh(c->ep_v, (size_t)c->eblk);
  fresh(c->cband_t, (size_t)c->nc); fresh(c->cband_x, (size_t)c->nc);
  ok = ok && band_clone_scratch(c, c->bandE) == IGA_OK && band_clone_scratch(c, c->bandC) == IGA_OK &&
       band_clone_scratch(c, c->bandX) == IGA_OK;
  if (!ok) {
    delete c;
    return nullptr;
  }
  return c;
}

extern "C" {

static void destroy_one(iga_ctx* ctx) {
  cudaStreamSynchronize(ctx->st);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

void iga_destroy(iga_ctx* ctx) {
  if (!ctx) return;
  for (iga_ctx* c : ctx->clones) destroy_one(c);
  ctx->clones.clear();
  cudaStreamSynchronize(ctx->st);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

size_t iga_ndof(const iga_ctx* ctx) { return ctx ? (size_t)ctx->lv[0].n : 0; }
size_t iga_coarse_ndof(const iga_ctx* ctx) { return ctx ? ctx->m : 0; }
int iga_num_levels(const iga_ctx* ctx) { return ctx ? ctx->L : 0; }
int iga_level_nx(const iga_ctx* ctx, int level) {
  return (ctx && level >= 0 && level < ctx->L) ? ctx->lv[level].nx : -1;
}
int iga_level_nel(const iga_ctx* ctx, int level) {
  return (ctx && level >= 0 && level < ctx->L) ? ctx->lv[level].n_el : -1;
}

iga_status iga_get_knots(iga_ctx* ctx, int level, double* out, int cap) {
  if (!ctx || !out || level < 0 || level >= ctx->L) return IGA_E_INVALID;
  int len = ctx->lv[level].n_el + 2 * ctx->p + 1;
  if (cap < len) return set_err(ctx, IGA_E_INVALID, "capacity %d < %d", cap, len);
  CK(cudaMemcpyAsync(out, ctx->lv[level].knots, sizeof(double) * len, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return IGA_OK;
}

iga_status iga_get_band(iga_ctx* ctx, int level, int which, double* out, size_t cap) {
  if (!ctx || !out || level < 0 || level >= ctx->L || which < 0 || which > 1) return IGA_E_INVALID;
  size_t len = (size_t)ctx->lv[level].nx * (2 * ctx->p + 1);
  if (cap < len) return set_err(ctx, IGA_E_INVALID, "capacity");
  CK(cudaMemcpyAsync(out, which == 0 ? ctx->lv[level].K : ctx->lv[level].M, sizeof(double) * len,
                     cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return IGA_OK;
}

iga_status iga_get_prolongation(iga_ctx* ctx, int level, double* out, size_t cap) {
  if (!ctx || !out || level < 0 || level + 1 >= ctx->L) return IGA_E_INVALID;
  const LevelData& F = ctx->lv[level];
  const LevelData& C = ctx->lv[level + 1];
  if (cap < (size_t)F.nx * C.nx) return set_err(ctx, IGA_E_INVALID, "capacity");
  std::vector<double> pw((size_t)F.nx * F.wP);
  std::vector<int> plo(F.nx);
  CK(cudaMemcpyAsync(pw.data(), F.Pw, sizeof(double) * pw.size(), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(plo.data(), F.Plo, sizeof(int) * plo.size(), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (size_t i = 0; i < (size_t)F.nx * C.nx; ++i) out[i] = 0.0;
  for (int i = 0; i < F.nx; ++i)
    for (int k = 0; k < F.wP; ++k) {
      int j = plo[i] + k;
      if (j >= 0 && j < C.nx) out[(size_t)i * C.nx + j] = pw[(size_t)i * F.wP + k];
    }
  return IGA_OK;
}

#define CHECK_CTX() do { if (!ctx) return IGA_E_INVALID; } while (0)
#define CHECK_DEFL() do { if (ctx->prm.skip_deflation || ctx->prm.deflation == 0) return set_err(ctx, IGA_E_INVALID, "context built without deflation"); } while (0)
#define CHECK_SOLVE() do { if (ctx->prm.skip_deflation) return set_err(ctx, IGA_E_INVALID, "context built for operators only"); } while (0)
#define CHECK_PTR(p) do { if (!aligned16(p)) return set_err(ctx, IGA_E_INVALID, "pointer %s NULL or not 16-byte aligned", #p); } while (0)

iga_status iga_apply_A(iga_ctx* ctx, const iga_c128* x, iga_c128* y) {
  CHECK_CTX(); CHECK_PTR(x); CHECK_PTR(y);
  if ((const void*)x == (const void*)y) return set_err(ctx, IGA_E_INVALID, "x and y alias");
  return op_apply<double>(ctx, 0, OP_A, (const double2*)x, (double2*)y, nullptr, EPI_Y, nullptr, 0.0);
}

iga_status iga_apply_Mshift(iga_ctx* ctx, int level, const iga_c128* x, iga_c128* y) {
  CHECK_CTX(); CHECK_PTR(x); CHECK_PTR(y);
  if (level < 0 || level >= ctx->L) return set_err(ctx, IGA_E_INVALID, "level");
  return op_apply<double>(ctx, level, OP_MB, (const double2*)x, (double2*)y, nullptr, EPI_Y, nullptr, 0.0);
}

iga_status iga_jacobi(iga_ctx* ctx, int level, const iga_c128* b, iga_c128* x_in, iga_c128* x_out, int sweeps) {
  CHECK_CTX(); CHECK_PTR(b); CHECK_PTR(x_in); CHECK_PTR(x_out);
  if (level < 0 || level >= ctx->L || sweeps < 1) return set_err(ctx, IGA_E_INVALID, "level/sweeps");
  double2* a = (double2*)x_in;
  double2* c = (double2*)x_out;
  // ping-pong so that the last sweep writes x_out
  double2* src = (sweeps & 1) ? a : c;
  double2* dst = (sweeps & 1) ? c : a;
  if (src != a) CK(cudaMemcpyAsync(src, a, sizeof(double2) * ctx->lv[level].n, cudaMemcpyDeviceToDevice, ctx->st));
  for (int s = 0; s < sweeps; ++s) {
    TRY(op_apply<double>(ctx, level, OP_MB, src, dst, nullptr, EPI_JACOBI, (const double2*)b, ctx->prm.omega));
    std::swap(src, dst);
  }
  return IGA_OK;
}

static bool aligned8(const void* p) { return p && (((uintptr_t)p) & 7u) == 0; }

iga_status iga_apply_Mshift32(iga_ctx* ctx, int level, const iga_c64* x, iga_c64* y) {
  CHECK_CTX();
  if (!aligned8(x) || !aligned8(y)) return set_err(ctx, IGA_E_INVALID, "x / y NULL or not 8-byte aligned");
  if (level < 0 || level >= ctx->L) return set_err(ctx, IGA_E_INVALID, "level");
  if ((const void*)x == (const void*)y) return set_err(ctx, IGA_E_INVALID, "x and y alias");
  return op_apply<float>(ctx, level, OP_MB, (const float2*)x, (float2*)y, nullptr, EPI_Y, nullptr, 0.0);
}

iga_status iga_jacobi32(iga_ctx* ctx, int level, const iga_c64* b, const iga_c64* x_in, iga_c64* x_out) {
  CHECK_CTX();
  if (!aligned8(b) || !aligned8(x_in) || !aligned8(x_out)) return set_err(ctx, IGA_E_INVALID, "NULL or not 8-byte aligned");
  if (level < 0 || level >= ctx->L) return set_err(ctx, IGA_E_INVALID, "level");
  if ((const void*)x_in == (const void*)x_out) return set_err(ctx, IGA_E_INVALID, "x_in and x_out alias");
  return op_apply<float>(ctx, level, OP_MB, (const float2*)x_in, (float2*)x_out, nullptr, EPI_JACOBI,
                         (const float2*)b, ctx->prm.omega);
}

iga_status iga_restrict(iga_ctx* ctx, int level, const iga_c128* fine, iga_c128* coarse) {
  CHECK_CTX(); CHECK_PTR(fine); CHECK_PTR(coarse);
  if (level < 0 || level + 1 >= ctx->L) return set_err(ctx, IGA_E_INVALID, "level");
  return mg_restrict<double>(ctx, level, (const double2*)fine, (double2*)coarse);
}

iga_status iga_prolong_add(iga_ctx* ctx, int level, const iga_c128* coarse, iga_c128* fine) {
  CHECK_CTX(); CHECK_PTR(fine); CHECK_PTR(coarse);
  if (level < 0 || level + 1 >= ctx->L) return set_err(ctx, IGA_E_INVALID, "level");
  return mg_prolong_add<double>(ctx, level, (const double2*)coarse, (double2*)fine);
}

iga_status iga_coarse_solve(iga_ctx* ctx, const iga_c128* b, iga_c128* x) {
  CHECK_CTX(); CHECK_PTR(b); CHECK_PTR(x);
  return mg_coarse<double>(ctx, (const double2*)b, (double2*)x);
}

iga_status iga_vcycle_cslp(iga_ctx* ctx, const iga_c128* r, iga_c128* z) {
  CHECK_CTX(); CHECK_PTR(r); CHECK_PTR(z);
  if (ctx->prm.n_vcycles < 1) return set_err(ctx, IGA_E_INVALID, "context built with n_vcycles = 0");
  if ((const void*)r == (const void*)z) return set_err(ctx, IGA_E_INVALID, "r and z alias");
  if (ctx->prm.precision == 0) return mg_vcycle<double>(ctx, (const double2*)r, (double2*)z);
  if (!ctx->net) return mg_vcycle32_c128(ctx, (const double2*)r, (double2*)z);
  size_t n = ctx->lv[0].n;
  launch_convert_d2f((const double2*)r, ctx->fin, n, ctx->st);
  TRY(mg_vcycle<float>(ctx, ctx->fin, ctx->fout));
  if (ctx->net) TRY(net_correct(ctx, ctx->fin, ctx->fout));
  launch_convert_f2d(ctx->fout, (double2*)z, n, ctx->st);
  CKL();
  return IGA_OK;
}

iga_status iga_precond(iga_ctx* ctx, const iga_c128* r, iga_c128* z) {
  CHECK_CTX(); CHECK_PTR(r); CHECK_PTR(z);
  if ((const void*)r == (const void*)z) return set_err(ctx, IGA_E_INVALID, "r and z alias");
  return kry_precond(ctx, (const double2*)r, (double2*)z);
}

iga_status iga_zt(iga_ctx* ctx, const iga_c128* x, iga_c128* c) {
  CHECK_CTX(); CHECK_DEFL(); CHECK_PTR(x); CHECK_PTR(c);
  return defl_zt(ctx, (const double2*)x, (double2*)c);
}
iga_status iga_z(iga_ctx* ctx, const iga_c128* c, iga_c128* x) {
  CHECK_CTX(); CHECK_DEFL(); CHECK_PTR(x); CHECK_PTR(c);
  return defl_z(ctx, (const double2*)c, (double2*)x);
}
iga_status iga_esolve(iga_ctx* ctx, const iga_c128* t, iga_c128* s) {
  CHECK_CTX(); CHECK_DEFL(); CHECK_PTR(t); CHECK_PTR(s);
  if ((const void*)t == (const void*)s) return set_err(ctx, IGA_E_INVALID, "t and s alias");
  return defl_esolve(ctx, (const double2*)t, (double2*)s);
}
iga_status iga_deflate(iga_ctx* ctx, const iga_c128* x, iga_c128* y) {
  CHECK_CTX(); CHECK_DEFL(); CHECK_PTR(x); CHECK_PTR(y);
  if ((const void*)x == (const void*)y) return set_err(ctx, IGA_E_INVALID, "x and y alias");
  return defl_apply(ctx, (const double2*)x, (double2*)y);
}

__global__ void k_point_source(const double* t, int n_el, int p, int nx, int dim, double x0, double y0,
                               double2* f);

// f_i = -g A[i][first function] for the unknowns i = 0 .. p-1 (full index i + 1;
// only element 0 couples them to function 0): stiffness and k^2-mass entries
// from the element-0 Gauss tables.
__global__ void k_dirichlet_lift(int p, int nx, const double* wq, const double* B, const double* D, double k2,
                                 double2 g, double2* f) {
  const int i = threadIdx.x;
  if (i >= p || i >= nx) return;
  const int a = i + 1, Q = p + 1;
  double ks = 0.0, ms = 0.0;
  for (int q = 0; q < Q; ++q) {
    const size_t o = (size_t)q * (p + 1);
    ks += wq[q] * D[o + a] * D[o];
    ms += wq[q] * B[o + a] * B[o];
  }
  const double v = ks - k2 * ms;
  f[i] = make_double2(-g.x * v, -g.y * v);
}

iga_status iga_load_dirichlet(iga_ctx* ctx, double g_re, double g_im, iga_c128* f) {
  CHECK_CTX(); CHECK_PTR(f);
  if (!ctx->prm.robin) return set_err(ctx, IGA_E_INVALID, "iga_load_dirichlet needs a context with robin = 1");
  const LevelData& L = ctx->lv[0];
  CK(cudaMemsetAsync(f, 0, sizeof(double2) * L.n, ctx->st));
  k_dirichlet_lift<<<1, 32, 0, ctx->st>>>(ctx->p, L.nx, L.wq, L.B, L.D, ctx->k2const, make_double2(g_re, g_im),
                                          (double2*)f); iga_count_launch();
  CKL();
  return IGA_OK;
}

iga_status iga_load_point_source(iga_ctx* ctx, double x0, double y0, iga_c128* f) {
  CHECK_CTX(); CHECK_PTR(f);
  if (!(x0 >= 0.0 && x0 <= 1.0) || (ctx->dim == 2 && !(y0 >= 0.0 && y0 <= 1.0)))
    return set_err(ctx, IGA_E_INVALID, "source outside the domain");
  const LevelData& L = ctx->lv[0];
  CK(cudaMemsetAsync(f, 0, sizeof(double2) * L.n, ctx->st));
  k_point_source<<<1, 32, 0, ctx->st>>>(L.knots, L.n_el, ctx->p, L.nx, ctx->dim, x0, y0, (double2*)f); iga_count_launch();
  CKL();
  return IGA_OK;
}

iga_status iga_mgs(iga_ctx* ctx, const iga_c128* V, size_t ldv, int j, iga_c128* w, iga_c128* h) {
  CHECK_CTX(); CHECK_PTR(V); CHECK_PTR(w); CHECK_PTR(h);
  if (j < 0 || ldv < iga_ndof(ctx)) return set_err(ctx, IGA_E_INVALID, "j / ldv");
  return kry_mgs(ctx, (const double2*)V, ldv, j, (double2*)w, (double2*)h);
}

iga_status iga_solve(iga_ctx* ctx, const iga_c128* rhs, iga_c128* x, double tol, int maxit, int* iters,
                     double* res_hist, double* true_res) {
  CHECK_CTX(); CHECK_SOLVE(); CHECK_PTR(rhs); CHECK_PTR(x);
  if (maxit < 1 || maxit > 1000 || !(tol >= 0.0)) return set_err(ctx, IGA_E_INVALID, "tol / maxit");
  if ((const void*)rhs == (const void*)x) return set_err(ctx, IGA_E_INVALID, "rhs and x alias");
  return kry_solve(ctx, (const double2*)rhs, (double2*)x, tol, maxit, iters, res_hist, true_res);
}

iga_status iga_set_wait_limit(iga_ctx* ctx, long long polls, int phantom_arrivals) {
  CHECK_CTX();
  return kry_set_wait_limit(ctx, polls, phantom_arrivals);
}

iga_status iga_solve_host(iga_ctx* ctx, const iga_c128* rhs_host, iga_c128* x_host, double tol, int maxit,
                          int* iters, double* res_hist, double* true_res) {
  CHECK_CTX(); CHECK_SOLVE();
  if (!rhs_host || !x_host) return set_err(ctx, IGA_E_INVALID, "NULL host pointer");
  if (ctx->maxit_alloc < 0 && maxit > 0) { /* workspace is allocated by the solve itself */ }
  size_t n = ctx->lv[0].n;
  double2* f = ctx->hf;
  double2* u = ctx->hu;
  if (!f) {
    ctx->hf = f = dalloc<double2>(ctx, n);
    ctx->hu = u = dalloc<double2>(ctx, n);
    if (!f || !u) return set_err(ctx, IGA_E_OOM, "host-solve buffers");
  }
  CK(cudaMemcpyAsync(f, rhs_host, sizeof(double2) * n, cudaMemcpyHostToDevice, ctx->st));
  iga_status s = kry_solve(ctx, f, u, tol, maxit, iters, res_hist, true_res);
  if (s < 0) return s;
  CK(cudaMemcpyAsync(x_host, u, sizeof(double2) * n, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return s;
}

}  // extern "C"

// Point-source load: f_i = Phi_i(x0, y0), evaluated by Cox-de Boor on the span
// that contains the source (the right end point belongs to the last span).
__global__ void k_point_source(const double* t, int n_el, int p, int nx, int dim, double x0, double y0,
                               double2* f) {
  if (threadIdx.x != 0) return;
  double vx[IGA_MAXP + 1], vy[IGA_MAXP + 1], d[IGA_MAXP + 1];
  int sx = find_span(t, n_el, p, x0);
  active_basis(t, p, sx, x0, vx, d);
  if (dim == 1) {
    for (int a = 0; a <= p; ++a) {
      int i = sx - p + a - 1;        // interior index of full function sx-p+a
      if (i >= 0 && i < nx) f[i] = make_double2(vx[a], 0.0);
    }
    return;
  }
  int sy = find_span(t, n_el, p, y0);
  active_basis(t, p, sy, y0, vy, d);
  for (int b = 0; b <= p; ++b) {
    int iy = sy - p + b - 1;
    if (iy < 0 || iy >= nx) continue;
    for (int a = 0; a <= p; ++a) {
      int ix = sx - p + a - 1;
      if (ix >= 0 && ix < nx) f[(size_t)iy * nx + ix] = make_double2(vy[b] * vx[a], 0.0);
    }
  }
}
