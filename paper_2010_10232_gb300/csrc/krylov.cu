// GMRES / flexible GMRES on the deflated, CSLP-preconditioned IgA system
// (Section 3: GMRES with P and M^{-1}; Section 4.3: stop at relative residual
// 1e-7, at most 100 iterations).
//
// Reading of the deflated system (DEF1): GMRES on M~^{-1} P A x^ = M~^{-1} P f
// from x^ = 0, then u = Q f + P^T x^ = x^ + Q (f - A x^).  FGMRES (right
// preconditioning, stored z_j) is used when the preconditioner is not a fixed
// FP64 operator (the FP32 V-cycle).
//
// Arnoldi is modified Gram-Schmidt with the Hermitian inner product.  Every
// reduction is deterministic: each block reduces a grid-strided slice in a
// fixed order, and every consumer re-reduces the per-block partial sums in
// the same fixed order.  Hessenberg least squares by complex Givens
// rotations [c, s; -conj(s), c] with real c.
#include "common.cuh"
#include <cmath>

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// block-wide sum of (a, b) pairs; result valid in thread 0
__device__ double2 block_sum2(double a, double b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sa[wid] = a; sb[wid] = b; }
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
  __syncthreads();
  return make_double2(a, b);
}
// every block re-reduces the nb partial pairs in the same order; result in all threads
__device__ double2 reduce_partials(const double* part, int nb) {
  __shared__ double2 res;
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) { a += part[2 * t]; b += part[2 * t + 1]; }
  double2 s = block_sum2(a, b);
  if (threadIdx.x == 0) res = s;
  __syncthreads();
  double2 r = res;
  __syncthreads();
  return r;
}

// MGS step i of column j: w -= h_{i-1} v_{i-1} (i > 0, h_{i-1} from the previous
// step's partials), then partial sums of v_i^H w (i <= j) or ||w||^2 (i = j+1).
__global__ void k_mgs_step(const double2* V, size_t ldv, size_t n, int i, int j, double2* w,
                           const double* part_in, double* part_out, double2* h) {
  double2 hp = make_double2(0.0, 0.0);
  if (i > 0) {
    hp = reduce_partials(part_in, gridDim.x);
    if (blockIdx.x == 0 && threadIdx.x == 0) h[i - 1] = hp;
  }
  const double2* vprev = V + (size_t)(i - 1) * ldv;
  const double2* vi = V + (size_t)i * ldv;
  double a = 0.0, b = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double2 we = w[e];
    if (i > 0) {
      we = we - cmul(hp, vprev[e]);
      w[e] = we;
    }
    if (i <= j) {
      double2 c = cconjmul(vi[e], we);
      a += c.x;
      b += c.y;
    } else {
      a += we.x * we.x + we.y * we.y;
    }
  }
  double2 s = block_sum2(a, b);
  if (threadIdx.x == 0) { part_out[2 * blockIdx.x] = s.x; part_out[2 * blockIdx.x + 1] = s.y; }
}

// partial sums of ||x||^2
__global__ void k_norm2_part(const double2* x, size_t n, double* part) {
  double a = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    a += x[e].x * x[e].x + x[e].y * x[e].y;
  double2 s = block_sum2(a, 0.0);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s.x; part[2 * blockIdx.x + 1] = 0.0; }
}
__global__ void k_finish_norm(const double* part, int nb, double* out) {
  double2 s = reduce_partials(part, nb);
  if (threadIdx.x == 0) *out = sqrt(s.x);
}
__global__ void k_finish_h(const double* part, int nb, double2* h) {
  double2 s = reduce_partials(part, nb);
  if (threadIdx.x == 0) *h = make_double2(sqrt(s.x), 0.0);
}

struct GState {
  double* cs;      // [maxit]
  double2* sn;     // [maxit]
  double2* g;      // [maxit+1]
  double* hist;    // [maxit+1]
  double* scal;    // [0] beta, [1] tol
  int* flag;       // [0] converged, [1] nonfinite
};

// New rotation for column j (H[j][j], H[j+1][j] after the previous rotations),
// applied to the column and to g; residual estimate and flags.
__device__ void givens_new(double2* Hj, int j, GState gs) {
  double2 a = Hj[j], b = Hj[j + 1];
  double aa = hypot(a.x, a.y), ab = hypot(b.x, b.y);
  double c;
  double2 s;
  if (ab == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0;
    s = make_double2(b.x / ab, -b.y / ab);
  } else {
    double t = hypot(aa, ab);
    c = aa / t;
    double2 ph = make_double2(a.x / aa, a.y / aa);
    double2 cb = make_double2(b.x / t, -b.y / t);
    s = cmul(ph, cb);
  }
  gs.cs[j] = c;
  gs.sn[j] = s;
  Hj[j] = c * a + cmul(s, b);
  Hj[j + 1] = make_double2(0.0, 0.0);
  double2 gj = gs.g[j];
  gs.g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));   // -conj(s) g_j
  gs.g[j] = c * gj;
  double res = hypot(gs.g[j + 1].x, gs.g[j + 1].y) / gs.scal[0];
  gs.hist[j + 1] = res;
  if (!isfinite(res)) gs.flag[1] = 1;
  if (res <= gs.scal[1]) gs.flag[0] = 1;
}

// Previous rotations applied to column j, then the new one (one thread).
__device__ void givens_update(double2* Hj, int j, GState gs) {
  for (int i = 0; i < j; ++i) {
    double c = gs.cs[i];
    double2 s = gs.sn[i];
    double2 t = c * Hj[i] + cmul(s, Hj[i + 1]);
    Hj[i + 1] = c * Hj[i + 1] - cconjmul(s, Hj[i]);
    Hj[i] = t;
  }
  givens_new(Hj, j, gs);
}

// The same with the rotations' four real outputs (Re t, Im t, Re h, Im h) on
// four lanes of one warp (called by all 32 lanes of the warp): every output
// is c X + Y1 Z1 + Y2 Z2 with lane-selected operands, so a rotation costs
// three FP64 instructions of the warp instead of twenty on one thread.
__device__ void givens_update_warp(double2* Hj, int j, GState gs) {
  const int lane = threadIdx.x & 31, k = lane & 3;
  double2 a = Hj[0];                           // running H[i][j] after the previous rotations
  for (int i = 0; i < j; ++i) {
    const double c = gs.cs[i];
    const double2 s = gs.sn[i], b = Hj[i + 1];
    // t = c a + s b;  h = c b - conj(s) a
    const double X = k == 0 ? a.x : k == 1 ? a.y : k == 2 ? b.x : b.y;
    const double Y1 = k < 2 ? s.x : -s.x;
    const double Z1 = k == 0 ? b.x : k == 1 ? b.y : k == 2 ? a.x : a.y;
    const double Y2 = (k == 0 || k == 2) ? -s.y : s.y;
    const double Z2 = k == 0 ? b.y : k == 1 ? b.x : k == 2 ? a.y : a.x;
    const double o = fma(Y2, Z2, fma(Y1, Z1, c * X));
    const double t_re = __shfl_sync(0xffffffffu, o, 0), t_im = __shfl_sync(0xffffffffu, o, 1);
    const double h_re = __shfl_sync(0xffffffffu, o, 2), h_im = __shfl_sync(0xffffffffu, o, 3);
    if (lane == 0) Hj[i] = make_double2(t_re, t_im);
    a = make_double2(h_re, h_im);
  }
  if (lane == 0) {
    Hj[j] = a;
    givens_new(Hj, j, gs);
  }
  __syncwarp();
}

// v_{j+1} = w / ||w|| (w already holds the orthogonalised vector), H[j+1][j] =
// ||w||, then the Givens update of column j (block 0, thread 0).
__global__ void k_normalize_givens(double2* w, size_t n, const double* part, double2* Hj, int j, GState gs,
                                   int do_givens) {
  double2 s = reduce_partials(part, gridDim.x);
  double hn = sqrt(s.x);
  double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    w[e] = inv * w[e];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Hj[j + 1] = make_double2(hn, 0.0);
    if (do_givens) givens_update(Hj, j, gs);
  }
}

// initial vector: v0 = b / ||b||, g0 = beta, hist0 = 1; optionally sets the
// loop condition of the following WHILE node (run only if beta is finite and
// non-zero).
__global__ void k_init_v0(double2* v, size_t n, const double* part, GState gs, double2* vcur,
                          cudaGraphConditionalHandle cond, int use_cond) {
  double2 s = reduce_partials(part, gridDim.x);
  double beta = sqrt(s.x);
  double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double2 u = inv * v[e];
    v[e] = u;
    if (vcur) vcur[e] = u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    gs.scal[0] = beta;
    gs.g[0] = make_double2(beta, 0.0);
    gs.hist[0] = 1.0;
    gs.flag[0] = (beta == 0.0) ? 1 : 0;
    gs.flag[1] = isfinite(beta) ? 0 : 1;
    if (use_cond) cudaGraphSetConditional(cond, (beta > 0.0 && isfinite(beta)) ? 1u : 0u);
  }
}

// per-solve state reset (kernel form so that it can live inside a graph)
__global__ void k_solve_reset(double2* H, size_t nh, int* kint, unsigned* kbar, double* scal, double tol) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < nh) H[i] = make_double2(0.0, 0.0);
  if (i < 4) kint[i] = 0;
  if (i < 2) kbar[i] = 0u;
  if (i == 0) scal[1] = tol;
}
// copy the iteration count and flags of a finished solve into slot `slot`
__global__ void k_record(const int* kint, const int* flag, int* out, int slot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    out[4 * slot + 0] = kint[0];
    out[4 * slot + 1] = flag[0];
    out[4 * slot + 2] = flag[1];
    out[4 * slot + 3] = kint[1];
  }
}

// R y = g (R upper triangular, column-major with leading dimension ldh)
__global__ void k_backsolve(const double2* H, int ldh, const double2* g, double2* y, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int r = k - 1; r >= 0; --r) {
    double2 s = g[r];
    for (int c = r + 1; c < k; ++c) s = s - cmul(H[(size_t)c * ldh + r], y[c]);
    double2 d = H[(size_t)r * ldh + r];
    y[r] = cmul(s, cinv(d));
  }
}

// x = sum_k Vk y_k (+ x0 if add)
__global__ void k_combine(const double2* V, size_t ldv, size_t n, const double2* y, int k, double2* x) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int c = 0; c < k; ++c) acc = acc + cmul(y[c], V[(size_t)c * ldv + e]);
  x[e] = acc;
}
__global__ void k_add(const double2* a, const double2* b, double2* out, size_t n) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < n) out[e] = a[e] + b[e];
}

// ------------------------------------------------------------------ device-resident iteration
// Bounded grid barrier for a cooperative launch (all blocks co-resident).  The
// barrier opens when `expect` blocks have arrived (the grid size; a test sets
// one more, which never arrives).  A block that has polled `limit` times
// (default 2^24, ~1 s) sets *err and returns false; every other waiting block
// sees *err and returns false too, and the host reports IGA_E_TIMEOUT.
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned expect, int* err, unsigned long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile int* verr = err;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    ok = 1;
    if (arrived == expect - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == g) {
        if (*verr || ++spins > limit) { atomicExch(err, 1); ok = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

struct ArnoldiArgs {
  double2* V;          // basis, column i at V + i*ldv
  size_t ldv, n;
  double2* w;          // candidate vector; orthogonalised in place
  double2* vcur;       // receives v_{j+1} (input of the next iteration)
  double2* H;          // (maxit+1) x maxit, column-major, leading dimension ldh
  int ldh, maxit;
  GState gs;
  int* jptr;           // current column j, advanced by this kernel
  double* part;        // 2 x gridDim.x (re, im) partial sums
  unsigned* bar;       // grid barrier {count, generation}
  int* err;            // barrier timeout flag
  unsigned long long spin_limit;   // polls before a barrier wait gives up
  unsigned phantom;    // extra arrivals the barrier waits for (0; a test sets 1)
  cudaGraphConditionalHandle cond;
  int use_cond;
};

// One Arnoldi step of column j = *jptr in a single cooperative launch:
// modified Gram-Schmidt (i = 0..j: h_ij = v_i^H w, w -= h_ij v_i, one grid
// barrier per coefficient), h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}, the
// Givens update of column j, j <- j + 1 and the loop condition.
// A barrier that gave up (now or in an earlier iteration) ends the step in
// every block; block 0 then clears the loop condition, so the WHILE node stops.
__global__ void __launch_bounds__(256) k_arnoldi_coop(ArnoldiArgs a) {
  const int j = *a.jptr;
  const unsigned nb = gridDim.x;
  if (*(volatile int*)a.err) {
    if (a.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
    return;
  }
  double2* hcol = a.H + (size_t)j * a.ldh;
  double2 hp = make_double2(0.0, 0.0);
  for (int i = 0; i <= j + 1; ++i) {
    const double2* vprev = a.V + (size_t)(i > 0 ? i - 1 : 0) * a.ldv;
    const double2* vi = a.V + (size_t)(i <= j ? i : 0) * a.ldv;
    double sa = 0.0, sb = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < a.n; e += (size_t)nb * blockDim.x) {
      double2 we = a.w[e];
      if (i > 0) {
        we = we - cmul(hp, vprev[e]);
        a.w[e] = we;
      }
      if (i <= j) {
        double2 c = cconjmul(vi[e], we);
        sa += c.x;
        sb += c.y;
      } else {
        sa += we.x * we.x + we.y * we.y;
      }
    }
    double2 s = block_sum2(sa, sb);
    double* pb = a.part + (size_t)(i & 1) * 2 * nb;
    if (threadIdx.x == 0) { pb[2 * blockIdx.x] = s.x; pb[2 * blockIdx.x + 1] = s.y; }
    if (!grid_sync(a.bar, nb + a.phantom, a.err, a.spin_limit)) {
      if (a.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
      return;
    }
    hp = reduce_partials(pb, nb);
    if (i <= j && blockIdx.x == 0 && threadIdx.x == 0) hcol[i] = hp;
  }
  double hn = sqrt(hp.x);
  double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  double2* vnext = a.V + (size_t)(j + 1) * a.ldv;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < a.n; e += (size_t)nb * blockDim.x) {
    double2 v = inv * a.w[e];
    vnext[e] = v;
    a.vcur[e] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    hcol[j + 1] = make_double2(hn, 0.0);
    givens_update(hcol, j, a.gs);
    *a.jptr = j + 1;
    unsigned go = (a.gs.flag[0] == 0 && a.gs.flag[1] == 0 && j + 1 < a.maxit) ? 1u : 0u;
    if (a.use_cond) cudaGraphSetConditional(a.cond, go);
  }
}

// ------------------------------------------------------------------ CGS2 Arnoldi (no grid barrier)
// Classical Gram-Schmidt with one reorthogonalisation: h = V^H w (all j+1
// projections in one pass), w -= V h, twice; H[:, j] = h1 + h2.  Six launches
// per iteration whatever j is, and no kernel waits on another block, so
// concurrent solves in one graph can overlap:
//   dots(w) | reduce | update + dots(w) | reduce | update + ||w||^2 | normalise (+ Givens in the last block)
// FP64 on this part retires one warp instruction per 64 cycles per SM
// sub-partition, so the reductions are arranged to issue few FP64 adds.
constexpr int CGS_T = 128;      // threads per block (4 warps)
constexpr int CGS_CH = 8;       // projections accumulated per sweep

// Sum 16 per-thread values (8 complex partial sums, re in v[0..7], im in
// v[8..15]) over a warp with a halving butterfly: 16 FP64 adds per warp instead
// of 80 for one shuffle tree per value.  Afterwards lane L holds the total of
// value bfly_index(L) (lanes L and L^1 hold the same).
__device__ __forceinline__ int bfly_index(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}
__device__ __forceinline__ double warp_bfly16(double* v, int lane) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool up = lane & 16;
    double keep = up ? v[8 + k] : v[k], send = up ? v[k] : v[8 + k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 8;
    double keep = up ? v[4 + k] : v[k], send = up ? v[k] : v[4 + k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 4;
    double keep = up ? v[2 + k] : v[k], send = up ? v[k] : v[2 + k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool up = lane & 2;
    double keep = up ? v[1] : v[0], send = up ? v[0] : v[1];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Block partials of v_i^H w for i = i0 .. i0 + 7 (i <= j) -> part[blk][2 i .. 2 i + 1]
__device__ __forceinline__ void cgs_store_partials(double* v, int i0, int j, double* part, int stride) {
  __shared__ double red[CGS_T / 32][16];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const double s = warp_bfly16(v, lane);
  if ((lane & 1) == 0) red[wp][bfly_index(lane)] = s;
  __syncthreads();
  if (threadIdx.x < 16) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < CGS_T / 32; ++q) t += red[q][threadIdx.x];
    const int c = threadIdx.x & 7, i = i0 + c;
    if (i <= j) part[(size_t)blockIdx.x * stride + 2 * i + (threadIdx.x >> 3)] = t;
  }
  __syncthreads();
}

// conj(v) w accumulated with FMAs: re += vx wx + vy wy, im += vx wy - vy wx
__device__ __forceinline__ void cacc_conj(double* v, int c, double2 a, double2 b) {
  v[c] = fma(a.x, b.x, v[c]);
  v[c] = fma(a.y, b.y, v[c]);
  v[8 + c] = fma(a.x, b.y, v[8 + c]);
  v[8 + c] = fma(-a.y, b.x, v[8 + c]);
}

// pass 1: partial projections of w
__global__ void __launch_bounds__(CGS_T) k_cgs_dots(const double2* V, size_t ldv, size_t n, const int* jptr,
                                                    const double2* w, double* part, int stride) {
  const int j = *jptr;
  for (int i0 = 0; i0 <= j; i0 += CGS_CH) {
    double v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = 0.0;
    for (size_t e = blockIdx.x * (size_t)CGS_T + threadIdx.x; e < n; e += (size_t)gridDim.x * CGS_T) {
      const double2 we = w[e];
#pragma unroll
      for (int c = 0; c < CGS_CH; ++c)
        if (i0 + c <= j) cacc_conj(v, c, V[(size_t)(i0 + c) * ldv + e], we);
    }
    cgs_store_partials(v, i0, j, part, stride);
  }
}

// h_i = sum over blocks in a fixed order (one block per coefficient); the
// first pass stores H[:, j] = h, the second adds to it
__global__ void __launch_bounds__(CGS_T) k_cgs_reduce(const double* part, int nb, int stride, const int* jptr,
                                                      double2* h, double2* H, int ldh, int second) {
  const int i = blockIdx.x;
  if (i > *jptr) return;
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < nb; t += CGS_T) {
    a += part[(size_t)t * stride + 2 * i];
    b += part[(size_t)t * stride + 2 * i + 1];
  }
  double2 s = block_sum2(a, b);
  if (threadIdx.x == 0) {
    h[i] = s;
    double2* hc = H + (size_t)(*jptr) * ldh;
    hc[i] = second ? hc[i] + s : s;
  }
}

// w -= sum_{i <= j} h_i v_i, then (NORM) partial ||w||^2 or (else) the second
// pass's partial projections of the updated w, over the same elements
template <bool NORM>
__global__ void __launch_bounds__(CGS_T) k_cgs_update(const double2* V, size_t ldv, size_t n, const int* jptr,
                                                      const double2* h, double2* w, double* part, int stride) {
  const int j = *jptr;
  double nrm = 0.0;
  for (size_t e = blockIdx.x * (size_t)CGS_T + threadIdx.x; e < n; e += (size_t)gridDim.x * CGS_T) {
    double2 we = w[e];
    for (int i = 0; i <= j; ++i) {
      const double2 hv = h[i], vv = V[(size_t)i * ldv + e];
      we.x = fma(-hv.x, vv.x, fma(hv.y, vv.y, we.x));
      we.y = fma(-hv.x, vv.y, fma(-hv.y, vv.x, we.y));
    }
    w[e] = we;
    if (NORM) nrm = fma(we.x, we.x, fma(we.y, we.y, nrm));
  }
  if (NORM) {
    double2 s = block_sum2(nrm, 0.0);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s.x; part[2 * blockIdx.x + 1] = 0.0; }
    return;
  }
  __syncthreads();      // every thread's w is written before it is read back below
  for (int i0 = 0; i0 <= j; i0 += CGS_CH) {
    double v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = 0.0;
    for (size_t e = blockIdx.x * (size_t)CGS_T + threadIdx.x; e < n; e += (size_t)gridDim.x * CGS_T) {
      const double2 we = w[e];
#pragma unroll
      for (int c = 0; c < CGS_CH; ++c)
        if (i0 + c <= j) cacc_conj(v, c, V[(size_t)(i0 + c) * ldv + e], we);
    }
    cgs_store_partials(v, i0, j, part, stride);
  }
}

// v_{j+1} = w / ||w|| into V[:, j+1] and vcur (every block re-reduces ||w||^2).
// The block that finishes last (ticket counter, no waiting) then sets
// H[j+1][j] = ||w||, applies the Givens update of column j, advances j and
// sets the loop condition: by then every block has read j.
__global__ void __launch_bounds__(CGS_T) k_cgs_normalize(double2* V, size_t ldv, size_t n, const double2* w,
                                                         double2* vcur, const double* part, int* jptr,
                                                         unsigned* ticket, double2* H, int ldh, int maxit, GState gs,
                                                         cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ bool last;
  const int j = *jptr;
  double2 s = reduce_partials(part, gridDim.x);
  const double hn = sqrt(s.x);
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  double2* vnext = V + (size_t)(j + 1) * ldv;
  for (size_t e = blockIdx.x * (size_t)CGS_T + threadIdx.x; e < n; e += (size_t)gridDim.x * CGS_T) {
    double2 v = inv * w[e];
    vnext[e] = v;
    vcur[e] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {            // one warp of the last block
    __threadfence();
    double2* hcol = H + (size_t)j * ldh;
    if (threadIdx.x == 0) {
      *ticket = 0u;
      hcol[j + 1] = make_double2(hn, 0.0);
    }
    __syncwarp();
    givens_update_warp(hcol, j, gs);
    if (threadIdx.x == 0) {
      *jptr = j + 1;
      unsigned go = (gs.flag[0] == 0 && gs.flag[1] == 0 && j + 1 < maxit) ? 1u : 0u;
      if (use_cond) cudaGraphSetConditional(cond, go);
    }
  }
}

// z_j -> column j = *jptr of Zb
__global__ void k_store_col(double2* Zb, size_t ldv, size_t n, const int* jptr, const double2* z) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < n) Zb[(size_t)(*jptr) * ldv + e] = z[e];
}
// back substitution and combination with the device-side iteration count
__global__ void k_backsolve_dev(const double2* H, int ldh, const double2* g, double2* y, const int* jptr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = *jptr;
  for (int r = k - 1; r >= 0; --r) {
    double2 s = g[r];
    for (int c = r + 1; c < k; ++c) s = s - cmul(H[(size_t)c * ldh + r], y[c]);
    y[r] = cmul(s, cinv(H[(size_t)r * ldh + r]));
  }
}
__global__ void k_combine_dev(const double2* V, size_t ldv, size_t n, const double2* y, const int* jptr, double2* x) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  int k = *jptr;
  double2 acc = make_double2(0.0, 0.0);
  for (int c = 0; c < k; ++c) acc = acc + cmul(y[c], V[(size_t)c * ldv + e]);
  x[e] = acc;
}

// ------------------------------------------------------------------ host
static int red_blocks(iga_ctx* ctx) { return 2 * ctx->num_sms; }

iga_status vec_norm(iga_ctx* ctx, const double2* x, size_t n, double* dev_out) {
  int nb = red_blocks(ctx);
  k_norm2_part<<<nb, IGA_RED_THREADS, 0, ctx->st>>>(x, n, ctx->partials); iga_count_launch();
  k_finish_norm<<<1, IGA_RED_THREADS, 0, ctx->st>>>(ctx->partials, nb, dev_out); iga_count_launch();
  CKL();
  return IGA_OK;
}

// MGS of w against columns 0..j of V; h[0..j] projections, h[j+1] = ||w||
// (w is NOT normalised).
iga_status kry_mgs(iga_ctx* ctx, const double2* V, size_t ldv, int j, double2* w, double2* h) {
  int nb = red_blocks(ctx);
  size_t n = ctx->lv[0].n;
  double* pa = ctx->partials;
  double* pb = ctx->partials + 2 * nb;
  for (int i = 0; i <= j + 1; ++i) {
    const double* pin = (i & 1) ? pa : pb;
    double* pout = (i & 1) ? pb : pa;
    k_mgs_step<<<nb, IGA_RED_THREADS, 0, ctx->st>>>(V, ldv, n, i, j, w, pin, pout, h); iga_count_launch();
  }
  const double* plast = ((j + 1) & 1) ? pb : pa;
  k_finish_h<<<1, IGA_RED_THREADS, 0, ctx->st>>>(plast, nb, h + j + 1); iga_count_launch();
  CKL();
  return IGA_OK;
}

static void drop_graph(iga_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->gexec = nullptr;
  ctx->graph = nullptr;
}

static iga_status ensure_krylov(iga_ctx* ctx, int maxit, bool flexible) {
  size_t n = ctx->lv[0].n;
  if (!ctx->kvec) {
    ctx->kvec = dalloc<double2>(ctx, 3 * n);        // vcur, zcur, wnext
    ctx->kint = dalloc<int>(ctx, 4);                 // j, barrier err
    ctx->kbar = dalloc<unsigned>(ctx, 2);
    if (!ctx->kvec || !ctx->kint || !ctx->kbar) return set_err(ctx, IGA_E_OOM, "krylov vectors");
    CK(cudaMemsetAsync(ctx->kbar, 0, 2 * sizeof(unsigned), ctx->st));
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_arnoldi_coop, 256, 0);
    // co-resident blocks for the cooperative Arnoldi step, sized to the problem
    // (about 2048 entries per block) so that small batched instances leave room
    // for each other
    int cap = std::max(1, std::min(occ, 2)) * ctx->num_sms;
    ctx->coop_blocks = (int)std::max<size_t>(1, std::min<size_t>(cap, cdiv(n, 2048)));
  }
  if (ctx->maxit_alloc >= maxit && (!flexible || ctx->Zb)) return IGA_OK;
  drop_graph(ctx);
  int m = std::max(maxit, ctx->maxit_alloc);
  ctx->Vb = dalloc<double2>(ctx, n * (size_t)(m + 1));
  ctx->Zb = flexible || ctx->Zb ? dalloc<double2>(ctx, n * (size_t)m) : nullptr;
  ctx->H = dalloc<double2>(ctx, (size_t)(m + 1) * m);
  ctx->gstate = dalloc<double>(ctx, (size_t)m + (m + 1) + 4);
  ctx->gsn = dalloc<double2>(ctx, m);
  ctx->gg = dalloc<double2>(ctx, m + 1);
  ctx->gy = dalloc<double2>(ctx, m);
  ctx->gflag = dalloc<int>(ctx, 4);
  // FP64-bound passes: two 4-warp blocks per SM where n allows
  ctx->cgs_blocks = (int)std::max<size_t>(1, std::min<size_t>(2 * ctx->num_sms, cdiv(n, 128)));
  ctx->cgs_part = dalloc<double>(ctx, (size_t)ctx->cgs_blocks * 2 * (m + 1) + 16);
  ctx->cgs_h = dalloc<double2>(ctx, m + 1);
  if (!ctx->cgs_ticket) {
    ctx->cgs_ticket = dalloc<unsigned>(ctx, 1);
    if (ctx->cgs_ticket) CK(cudaMemset(ctx->cgs_ticket, 0, sizeof(unsigned)));
  }
  if (!ctx->cgs_part || !ctx->cgs_h || !ctx->cgs_ticket) return set_err(ctx, IGA_E_OOM, "cgs workspace");
  if (!ctx->Vb || (flexible && !ctx->Zb) || !ctx->H || !ctx->gstate || !ctx->gsn || !ctx->gg || !ctx->gy || !ctx->gflag)
    return set_err(ctx, IGA_E_OOM, "krylov workspace (n=%zu, maxit=%d)", n, m);
  ctx->maxit_alloc = m;
  return IGA_OK;
}

// z = M~^{-1} r: the exact CSLP inverse (C_ex), z = r without a CSLP
// (n_vcycles = 0: deflation alone), else the V-cycles in the context's precision
static iga_status precond(iga_ctx* ctx, const double2* r, double2* z) {
  LevelData& L = ctx->lv[0];
  if (ctx->prm.precond == 1) return cslp_exact_solve(ctx, r, z);
  if (ctx->prm.n_vcycles < 1) {
    CK(cudaMemcpyAsync(z, r, sizeof(double2) * L.n, cudaMemcpyDeviceToDevice, ctx->st));
    return IGA_OK;
  }
  if (ctx->prm.precision == 0) return mg_vcycle<double>(ctx, r, z);
  if (!ctx->net) return mg_vcycle32_c128(ctx, r, z);
  launch_convert_d2f(r, ctx->fin, L.n, ctx->st);
  TRY(mg_vcycle<float>(ctx, ctx->fin, ctx->fout));
  if (ctx->net) TRY(net_correct(ctx, ctx->fin, ctx->fout));
  launch_convert_f2d(ctx->fout, z, L.n, ctx->st);
  CKL();
  return IGA_OK;
}

static GState gstate_of(iga_ctx* ctx) {
  GState gs;
  gs.cs = ctx->gstate;
  gs.hist = ctx->gstate + ctx->maxit_alloc;
  gs.scal = gs.hist + ctx->maxit_alloc + 1;
  gs.sn = ctx->gsn;
  gs.g = ctx->gg;
  gs.flag = ctx->gflag;
  return gs;
}

static ArnoldiArgs arnoldi_args(iga_ctx* ctx, int maxit) {
  ArnoldiArgs a;
  a.V = ctx->Vb;
  a.ldv = ctx->lv[0].n;
  a.n = ctx->lv[0].n;
  a.w = ctx->kvec + 2 * a.n;
  a.vcur = ctx->kvec;
  a.H = ctx->H;
  a.ldh = ctx->maxit_alloc + 1;
  a.maxit = maxit;
  a.gs = gstate_of(ctx);
  a.jptr = ctx->kint;
  a.part = ctx->partials;
  a.bar = ctx->kbar;
  a.err = ctx->kint + 1;
  a.spin_limit = ctx->wait_polls;
  a.phantom = (unsigned)ctx->wait_phantom;
  a.cond = ctx->gcond;
  a.use_cond = 0;
  return a;
}

static iga_status launch_arnoldi_cgs(iga_ctx* ctx, ArnoldiArgs a) {
  cudaStream_t st = ctx->st;
  const int nb = ctx->cgs_blocks;
  const int stride = 2 * (ctx->maxit_alloc + 1);
  double* part = ctx->cgs_part;
  double2* h = ctx->cgs_h;
  k_cgs_dots<<<nb, CGS_T, 0, st>>>(a.V, a.ldv, a.n, a.jptr, a.w, part, stride); iga_count_launch();
  k_cgs_reduce<<<a.maxit + 1, CGS_T, 0, st>>>(part, nb, stride, a.jptr, h, a.H, a.ldh, 0); iga_count_launch();
  k_cgs_update<false><<<nb, CGS_T, 0, st>>>(a.V, a.ldv, a.n, a.jptr, h, a.w, part, stride); iga_count_launch();
  k_cgs_reduce<<<a.maxit + 1, CGS_T, 0, st>>>(part, nb, stride, a.jptr, h, a.H, a.ldh, 1); iga_count_launch();
  k_cgs_update<true><<<nb, CGS_T, 0, st>>>(a.V, a.ldv, a.n, a.jptr, h, a.w, part, stride); iga_count_launch();
  k_cgs_normalize<<<nb, CGS_T, 0, st>>>(a.V, a.ldv, a.n, a.w, a.vcur, part, a.jptr, ctx->cgs_ticket, a.H, a.ldh,
                                        a.maxit, a.gs, a.cond, a.use_cond); iga_count_launch();
  CKL();
  return IGA_OK;
}

static iga_status launch_arnoldi(iga_ctx* ctx, ArnoldiArgs a) {
  if (ctx->arnoldi_cgs) return launch_arnoldi_cgs(ctx, a);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctx->coop_blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = ctx->st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CK(cudaLaunchKernelEx(&cfg, k_arnoldi_coop, a));
  iga_count_launch();
  return IGA_OK;
}

iga_status kry_precond(iga_ctx* ctx, const double2* r, double2* z) { return precond(ctx, r, z); }

// One iteration's work after v_j is in vcur, then the Arnoldi step:
//   deflation 1 (DEF1): w = M~^{-1} P A v_j (left) or z_j = M~^{-1} v_j, w = P A z_j (flexible);
//   deflation 0 (none): w = M~^{-1} A v_j (left) or w = A M~^{-1} v_j (flexible);
//   deflation 2 (literal, left only): w = P^T M~^{-1} A v_j.
static iga_status iteration_body(iga_ctx* ctx, bool flex, ArnoldiArgs a) {
  const size_t n = ctx->lv[0].n;
  const int defl = ctx->prm.deflation;
  double2* vcur = ctx->kvec;
  double2* zcur = ctx->kvec + n;
  double2* wnext = ctx->kvec + 2 * n;
  if (flex) {
    TRY(precond(ctx, vcur, zcur));
    k_store_col<<<cdiv(n, 256), 256, 0, ctx->st>>>(ctx->Zb, n, n, ctx->kint, zcur); iga_count_launch();
    if (defl == 1) {
      TRY(op_apply<double>(ctx, 0, OP_A, zcur, ctx->w1, nullptr, EPI_Y, nullptr, 0.0));
      TRY(defl_apply(ctx, ctx->w1, wnext));
    } else {
      TRY(op_apply<double>(ctx, 0, OP_A, zcur, wnext, nullptr, EPI_Y, nullptr, 0.0));
    }
  } else {
    TRY(op_apply<double>(ctx, 0, OP_A, vcur, ctx->w1, nullptr, EPI_Y, nullptr, 0.0));
    if (defl == 1) {
      TRY(defl_apply(ctx, ctx->w1, ctx->w2));
      TRY(precond(ctx, ctx->w2, wnext));
    } else if (defl == 0) {
      TRY(precond(ctx, ctx->w1, wnext));
    } else {
      TRY(precond(ctx, ctx->w1, ctx->w2));
      TRY(defl_apply_T(ctx, ctx->w2, wnext, ctx->w1, ctx->w3));
    }
  }
  return launch_arnoldi(ctx, a);
}

// Build (once per workspace) the graph WHILE(cond) { iteration }.  Capture runs
// on a private stream; ctx->st is restored afterwards.
iga_status capture_body(iga_ctx* ctx, cudaGraph_t body, bool flex, int maxit, cudaGraphConditionalHandle cond,
                        unsigned long long* nkern);

// Build (once per workspace) the graph WHILE(cond) { iteration }.
static iga_status build_loop_graph(iga_ctx* ctx, bool flex, int maxit) {
  drop_graph(ctx);
  CK(cudaGraphCreate(&ctx->graph, 0));
  CK(cudaGraphConditionalHandleCreate(&ctx->gcond, ctx->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = ctx->gcond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, ctx->graph, nullptr, nullptr, 0, &np));
  TRY(capture_body(ctx, np.conditional.phGraph_out[0], flex, maxit, ctx->gcond, &ctx->body_kernels));
  CK(cudaGraphInstantiate(&ctx->gexec, ctx->graph, 0));
  ctx->graph_flex = flex;
  ctx->graph_maxit = maxit;
  return IGA_OK;
}

// Phase 1 (kernels only): reset the solve state and form v0.
iga_status solve_init(iga_ctx* ctx, const double2* f, double tol, bool flex, cudaGraphConditionalHandle cond,
                      int use_cond) {
  cudaStream_t st = ctx->st;
  const size_t n = ctx->lv[0].n;
  const int ldh = ctx->maxit_alloc + 1;
  const int nb = red_blocks(ctx);
  GState gs = gstate_of(ctx);
  size_t nh = (size_t)ldh * ctx->maxit_alloc;
  k_solve_reset<<<cdiv(nh, 256), 256, 0, st>>>(ctx->H, nh, ctx->kint, ctx->kbar, gs.scal, tol); iga_count_launch();
  if (ctx->cgs_ticket) CK(cudaMemsetAsync(ctx->cgs_ticket, 0, sizeof(unsigned), st));
  double2* V = ctx->Vb;
  const int defl = ctx->prm.deflation;
  if (flex) {
    if (defl == 1) TRY(defl_apply(ctx, f, V));
    else CK(cudaMemcpyAsync(V, f, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
  } else if (defl == 1) {
    TRY(defl_apply(ctx, f, ctx->w0));
    TRY(precond(ctx, ctx->w0, V));
  } else if (defl == 0) {
    TRY(precond(ctx, f, V));
  } else {
    TRY(precond(ctx, f, ctx->w0));
    TRY(defl_apply_T(ctx, ctx->w0, V, ctx->w1, ctx->w2));
  }
  k_norm2_part<<<nb, IGA_RED_THREADS, 0, st>>>(V, n, ctx->partials); iga_count_launch();
  k_init_v0<<<nb, IGA_RED_THREADS, 0, st>>>(V, n, ctx->partials, gs, ctx->kvec, cond, use_cond); iga_count_launch();
  CKL();
  return IGA_OK;
}

// Phase 3 (kernels only): x^ = V y (Z y), u = x^ + Q (f - A x^) (DEF1) or
// u = x^ (no deflation, literal ordering), optional true-residual norms into
// scal[2], scal[3].
iga_status solve_finish(iga_ctx* ctx, const double2* f, double2* x, bool flex, bool true_res) {
  cudaStream_t st = ctx->st;
  const size_t n = ctx->lv[0].n;
  const int ldh = ctx->maxit_alloc + 1;
  GState gs = gstate_of(ctx);
  k_backsolve_dev<<<1, 1, 0, st>>>(ctx->H, ldh, gs.g, ctx->gy, ctx->kint); iga_count_launch();
  if (ctx->prm.deflation == 1) {
    k_combine_dev<<<cdiv(n, 256), 256, 0, st>>>(flex ? ctx->Zb : ctx->Vb, n, n, ctx->gy, ctx->kint, ctx->w0); iga_count_launch();
    TRY(op_apply<double>(ctx, 0, OP_A, ctx->w0, ctx->w1, f, EPI_ZMINUS, nullptr, 0.0));
    TRY(defl_q(ctx, ctx->w1, ctx->w2));
    k_add<<<cdiv(n, 256), 256, 0, st>>>(ctx->w0, ctx->w2, x, n); iga_count_launch();
  } else {
    k_combine_dev<<<cdiv(n, 256), 256, 0, st>>>(flex ? ctx->Zb : ctx->Vb, n, n, ctx->gy, ctx->kint, x); iga_count_launch();
  }
  CKL();
  if (true_res) {
    TRY(op_apply<double>(ctx, 0, OP_A, x, ctx->w1, f, EPI_ZMINUS, nullptr, 0.0));
    TRY(vec_norm(ctx, ctx->w1, n, gs.scal + 2));
    TRY(vec_norm(ctx, f, n, gs.scal + 3));
  }
  return IGA_OK;
}

// Capture one iteration into `body` (the body graph of a WHILE node) with the
// Arnoldi step driving `cond`.  Returns the number of kernels in the body.
iga_status capture_body(iga_ctx* ctx, cudaGraph_t body, bool flex, int maxit, cudaGraphConditionalHandle cond,
                        unsigned long long* nkern) {
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  cudaStream_t saved = ctx->st;
  ctx->st = ctx->cap_stream;
  unsigned long long before = iga_launch_count();
  cudaError_t e = cudaStreamBeginCaptureToGraph(ctx->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) { ctx->st = saved; return set_err(ctx, IGA_E_CUDA, "capture: %s", cudaGetErrorString(e)); }
  ArnoldiArgs a = arnoldi_args(ctx, maxit);
  a.cond = cond;
  a.use_cond = 1;
  iga_status s = iteration_body(ctx, flex, a);
  cudaGraph_t cap = body;
  cudaError_t e2 = cudaStreamEndCapture(ctx->st, &cap);
  ctx->st = saved;
  *nkern = iga_launch_count() - before;
  iga_add_launches(-(long long)*nkern);   // capture executes nothing
  if (s != IGA_OK) return s;
  if (e2 != cudaSuccess) return set_err(ctx, IGA_E_CUDA, "end capture: %s", cudaGetErrorString(e2));
  return IGA_OK;
}

iga_status kry_prepare(iga_ctx* ctx, int maxit, bool flex) { return ensure_krylov(ctx, maxit, flex); }

iga_status kry_set_wait_limit(iga_ctx* ctx, long long polls, int phantom) {
  if (polls < 0 || phantom < 0 || phantom > 1) return set_err(ctx, IGA_E_INVALID, "wait limit");
  CK(cudaStreamSynchronize(ctx->st));
  ctx->wait_polls = polls == 0 ? (1ull << 24) : (unsigned long long)polls;
  ctx->wait_phantom = phantom;
  drop_graph(ctx);                       // the captured Arnoldi step holds the old limit
  return IGA_OK;
}

iga_status kry_solve(iga_ctx* ctx, const double2* f, double2* x, double tol, int maxit, int* iters, double* hist,
                     double* true_res) {
  const bool flex = ctx->prm.precision != 0 || ctx->prm.flexible != 0;
  TRY(ensure_krylov(ctx, maxit, flex));
  cudaStream_t st = ctx->st;
  GState gs = gstate_of(ctx);
  TRY(solve_init(ctx, f, tol, flex, 0, 0));
  int hflag[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(hflag, gs.flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (!hflag[0] && !hflag[1]) {
    if (ctx->use_graph) {
      if (!ctx->gexec || ctx->graph_flex != flex || ctx->graph_maxit != maxit) {
        iga_status s = build_loop_graph(ctx, flex, maxit);
        if (s != IGA_OK) {                 // keep going without the graph
          fprintf(stderr, "iga_solve: loop graph unavailable (%s); iterating from the host\n", ctx->err.c_str());
          drop_graph(ctx);
          ctx->use_graph = false;
          cudaGetLastError();
        }
      }
    }
    if (ctx->use_graph) {
      CK(cudaGraphLaunch(ctx->gexec, st));
    } else {
      ArnoldiArgs a = arnoldi_args(ctx, maxit);
      for (int j = 0; j < maxit; ++j) {
        TRY(iteration_body(ctx, flex, a));
        CK(cudaMemcpyAsync(hflag, gs.flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hflag + 2, ctx->kint, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (hflag[0] || hflag[1] || hflag[3]) break;
      }
    }
  }
  TRY(solve_finish(ctx, f, x, flex, true_res != nullptr));
  double hn[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(hflag, gs.flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hflag + 2, ctx->kint, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (true_res) CK(cudaMemcpyAsync(hn, gs.scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int jdone = hflag[2];
  if (ctx->use_graph) iga_add_launches((long long)ctx->body_kernels * jdone);
  if (hist) CK(cudaMemcpy(hist, gs.hist, sizeof(double) * (jdone + 1), cudaMemcpyDeviceToHost));
  if (true_res) *true_res = hn[1] > 0 ? hn[0] / hn[1] : 0.0;
  if (iters) *iters = jdone;
  if (hflag[3]) return set_err(ctx, IGA_E_TIMEOUT, "grid barrier timed out in the Arnoldi step");
  if (hflag[1]) return set_err(ctx, IGA_E_NONFINITE, "non-finite residual at iteration %d", jdone);
  return hflag[0] ? IGA_OK : IGA_NOT_CONVERGED;
}
