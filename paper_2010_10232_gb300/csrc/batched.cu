// Batched solves: many independent instances (each with its own context, wave
// number, order p and mesh) and several right-hand sides per instance, solved
// by ONE CUDA-graph launch.
//
// Graph layout: for instance b and right-hand side r the chain
//     init(f_br) -> WHILE(cond_br) { one FGMRES/GMRES iteration } -> finish(f_br, x_br) -> record
// is appended to the graph.  Right-hand side r > 0 of an instance runs on the
// instance's workspace clone r - 1 (same setup, its own vectors; created at
// the first batched call that needs it and kept by the context), so no chain
// has an edge to another and all of them run concurrently (an instance with a
// network attached keeps one workspace: its chains follow each other).  Each
// WHILE node stops on its own convergence flag; the init kernel sets the
// condition so that a zero right-hand side runs no iteration.
#include "common.cuh"
#include <vector>

iga_status solve_init(iga_ctx* ctx, const double2* f, double tol, bool flex, cudaGraphConditionalHandle cond,
                      int use_cond);
iga_status solve_finish(iga_ctx* ctx, const double2* f, double2* x, bool flex, bool true_res);
iga_status capture_body(iga_ctx* ctx, cudaGraph_t body, bool flex, int maxit, cudaGraphConditionalHandle cond,
                        unsigned long long* nkern);
iga_status kry_prepare(iga_ctx* ctx, int maxit, bool flex);
__global__ void k_record(const int* kint, const int* flag, int* out, int slot);

namespace {

struct GraphGuard {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  ~GraphGuard() {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
  }
};

// Capture `fn` (which enqueues on ctx->st) into graph g after the nodes `deps`;
// on return `deps` holds the leaves of the captured work.
template <typename F>
iga_status capture_after(iga_ctx* ctx, cudaGraph_t g, std::vector<cudaGraphNode_t>& deps, F fn) {
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  cudaStream_t saved = ctx->st;
  ctx->st = ctx->cap_stream;
  cudaError_t e = cudaStreamBeginCaptureToGraph(ctx->st, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                                cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) { ctx->st = saved; return set_err(ctx, IGA_E_CUDA, "capture: %s", cudaGetErrorString(e)); }
  iga_status s = fn();
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* leaves = nullptr;
  size_t nleaves = 0;
  cudaError_t e1 = cudaStreamGetCaptureInfo(ctx->st, &cs, nullptr, nullptr, &leaves, nullptr, &nleaves);
  std::vector<cudaGraphNode_t> out;
  if (e1 == cudaSuccess && leaves) out.assign(leaves, leaves + nleaves);
  cudaGraph_t gout = g;
  cudaError_t e2 = cudaStreamEndCapture(ctx->st, &gout);
  ctx->st = saved;
  if (s != IGA_OK) return s;
  if (e1 != cudaSuccess) return set_err(ctx, IGA_E_CUDA, "capture info: %s", cudaGetErrorString(e1));
  if (e2 != cudaSuccess) return set_err(ctx, IGA_E_CUDA, "end capture: %s", cudaGetErrorString(e2));
  deps = out;
  return IGA_OK;
}

}  // namespace

extern "C" iga_status iga_solve_batched(iga_ctx* const* ctxs, int nb, const iga_c128* const* rhs,
                                        iga_c128* const* x, const int* nrhs, double tol, int maxit, int* iters,
                                        int* status, void* stream) {
  if (!ctxs || nb < 1 || !rhs || !x || !nrhs || !iters || maxit < 1 || maxit > 1000 || !(tol >= 0.0))
    return IGA_E_INVALID;
  int dev = -1;
  int total = 0;
  for (int b = 0; b < nb; ++b) {
    iga_ctx* c = ctxs[b];
    if (!c || c->prm.skip_deflation || c->prm.deflation != 1 || nrhs[b] < 1 || !rhs[b] || !x[b]) return IGA_E_INVALID;
    if (((uintptr_t)rhs[b] & 15u) || ((uintptr_t)x[b] & 15u)) return IGA_E_INVALID;
    if (dev < 0) dev = c->device;
    if (c->device != dev) return IGA_E_INVALID;
    for (int a = 0; a < b; ++a)
      if (ctxs[a] == c) return IGA_E_INVALID;   // one chain per context
    total += nrhs[b];
  }
  iga_ctx* ctx = ctxs[0];   // error reporting and the record buffer
  // the workspace of right-hand side r of instance b
  auto chain_ctx = [&](int b, int r) -> iga_ctx* {
    iga_ctx* c = ctxs[b];
    return (r == 0 || c->net) ? c : c->clones[r - 1];
  };
  for (int b = 0; b < nb; ++b) {
    iga_ctx* c = ctxs[b];
    if (!c->arnoldi_cgs) {       // the single-solve graph (if any) used the other Arnoldi form
      c->arnoldi_cgs = true;
      if (c->gexec) cudaGraphExecDestroy(c->gexec);
      if (c->graph) cudaGraphDestroy(c->graph);
      c->gexec = nullptr;
      c->graph = nullptr;
    }
    if (!c->net)
      while ((int)c->clones.size() < nrhs[b] - 1) {
        CK(cudaStreamSynchronize(c->st));
        iga_ctx* k = clone_workspace(c);
        if (!k) return set_err(ctx, IGA_E_OOM, "workspace for right-hand side %zu of instance %d", c->clones.size() + 2, b);
        c->clones.push_back(k);
      }
    bool flex = c->prm.precision != 0 || c->prm.flexible != 0;
    for (int r = 0; r < nrhs[b]; ++r) {
      iga_ctx* w = chain_ctx(b, r);
      if (r > 0 && w == c) break;
      iga_status s = kry_prepare(w, maxit, flex);
      if (s != IGA_OK) return s;
    }
  }
  if (ctx->brec_cap < total) {
    ctx->brec = dalloc<int>(ctx, 4 * (size_t)total);
    if (!ctx->brec) return set_err(ctx, IGA_E_OOM, "batch record");
    ctx->brec_cap = total;
  }
  GraphGuard G;
  CK(cudaGraphCreate(&G.g, 0));
  unsigned long long before = iga_launch_count();
  std::vector<unsigned long long> body_k(total, 0);
  int slot = 0;
  for (int b = 0; b < nb; ++b) {
    const bool flex = ctxs[b]->prm.precision != 0 || ctxs[b]->prm.flexible != 0;
    const size_t n = ctxs[b]->lv[0].n;
    std::vector<cudaGraphNode_t> deps;
    for (int r = 0; r < nrhs[b]; ++r, ++slot) {
      iga_ctx* c = chain_ctx(b, r);
      if (c != ctxs[b] || r == 0) deps.clear();     // a chain on its own workspace depends on nothing
      const double2* f = (const double2*)rhs[b] + (size_t)r * n;
      double2* xo = (double2*)x[b] + (size_t)r * n;
      cudaGraphConditionalHandle h;
      CK(cudaGraphConditionalHandleCreate(&h, G.g, 0, cudaGraphCondAssignDefault));
      TRY(capture_after(c, G.g, deps, [&]() { return solve_init(c, f, tol, flex, h, 1); }));
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t wnode;
      CK(cudaGraphAddNode(&wnode, G.g, deps.data(), nullptr, deps.size(), &np));
      TRY(capture_body(c, np.conditional.phGraph_out[0], flex, maxit, h, &body_k[slot]));   // nets itself out
      deps.assign(1, wnode);
      int* rec = ctx->brec;
      int sl = slot;
      TRY(capture_after(c, G.g, deps, [&]() {
        TRY(solve_finish(c, f, xo, flex, false));
        k_record<<<1, 32, 0, c->st>>>(c->kint, c->gflag, rec, sl); iga_count_launch();
        return IGA_OK;
      }));
    }
  }
  unsigned long long outside = iga_launch_count() - before;   // init + finish kernels, executed once each
  iga_add_launches(-(long long)outside);
  CK(cudaGraphInstantiate(&G.e, G.g, 0));
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaGraphLaunch(G.e, st));
  std::vector<int> rec(4 * (size_t)total);
  CK(cudaMemcpyAsync(rec.data(), ctx->brec, sizeof(int) * rec.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  unsigned long long executed = outside;
  iga_status worst = IGA_OK;
  for (int i = 0; i < total; ++i) {
    iters[i] = rec[4 * i];
    int st_i = rec[4 * i + 3] ? IGA_E_TIMEOUT : rec[4 * i + 2] ? IGA_E_NONFINITE : rec[4 * i + 1] ? IGA_OK : IGA_NOT_CONVERGED;
    if (status) status[i] = st_i;
    if (st_i < 0) worst = (iga_status)st_i;
    else if (st_i == IGA_NOT_CONVERGED && worst == IGA_OK) worst = IGA_NOT_CONVERGED;
    executed += body_k[i] * (unsigned long long)rec[4 * i];
  }
  iga_add_launches((long long)executed);
  return worst;
}
