/*
 * iga_helmholtz.h — C ABI of the GB300 (sm_103a) IgA Helmholtz solver.
 *
 * Method: arXiv 2010.10232 (Dwarka, Tielen, Moller, Vuik).  GMRES on the
 * B-spline Galerkin system A u = f with A = S - M^{k^2} (Section 2.3, Eq.
 * linearsystem1, read with the sign of the model problems), preconditioned by
 * multigrid V-cycles of the complex shifted Laplacian (Section 3, CSLP
 * equation; damped Jacobi omega = 0.6) and deflated with P = I - A Q,
 * Q = Z E^{-1} Z^T, E = Z^T A Z (Section 3, Eq. adef1, quadratic Bezier Z).
 *
 * Conventions (all entry points):
 *  - Vectors hold the interior (Dirichlet-eliminated) B-spline coefficients,
 *    lexicographic with x fastest: entry (ix, iy) at iy * n_x + ix, n_x =
 *    n_el + p - 2.  Complex values are interleaved (re, im) pairs.
 *  - Unless stated otherwise every pointer argument is a DEVICE pointer,
 *    allocated and owned by the caller, 16-byte aligned (8-byte for
 *    iga_c64), on the device that was current at iga_setup.  A misaligned or
 *    NULL pointer returns IGA_E_INVALID and launches nothing.
 *  - Work is enqueued on params.stream (NULL = the legacy default stream) and
 *    is asynchronous with respect to the host, except where a function says it
 *    synchronises.
 *  - No exception crosses the ABI.  Errors are returned; the most recent
 *    error text of a context is available from iga_last_error().
 *  - The context owns its device workspace (allocated in iga_setup and
 *    iga_solve, released in iga_destroy).
 */
#ifndef IGA_HELMHOLTZ_H
#define IGA_HELMHOLTZ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } iga_c128;
typedef struct { float re, im; } iga_c64;

typedef enum {
  IGA_OK = 0,
  IGA_NOT_CONVERGED = 1,   /* solve reached maxit; outputs are still valid          */
  IGA_E_INVALID = -1,      /* bad argument (NULL, misaligned, out of range)          */
  IGA_E_CUDA = -2,         /* a CUDA runtime call failed                              */
  IGA_E_OOM = -3,          /* device allocation failed                                */
  IGA_E_BREAKDOWN = -4,    /* Arnoldi produced an unusable basis vector               */
  IGA_E_NONFINITE = -5,    /* NaN or Inf met in the iteration                         */
  IGA_E_TIMEOUT = -6,      /* a bounded device wait gave up                           */
  IGA_E_UNSUPPORTED = -7   /* valid request that this build does not implement       */
} iga_status;

#define IGA_MAX_LINES 8

/* Problem and solver parameters.  Fill with iga_default_params() first. */
typedef struct {
  int dim;                 /* 1 or 2 (unit interval / unit square)                        */
  int p;                   /* B-spline degree, 1..5 (Section 2.3.1)                       */
  int n_el;                /* elements per direction; open uniform knots i/n_el           */
  /* wave number: k(x,y) = k_values[#lines with a*x + b*y + c >= 0]; n_lines = 0 is
     the constant k_values[0].  Lines must not cross inside the domain.        */
  int n_lines;             /* 0..IGA_MAX_LINES (2D only when > 0)                         */
  double lines[IGA_MAX_LINES][3];
  double k_values[IGA_MAX_LINES + 1];
  double beta1, beta2;     /* CSLP M = S - (beta1 - i beta2) M^{k^2}                       */
  double eps;              /* ADP weight epsilon (Section 3, weighted stencil)            */
  int nu_pre, nu_post;     /* damped-Jacobi sweeps before / after coarse correction        */
  double omega;            /* Jacobi damping, 0.6 in the paper                            */
  int n_vcycles;           /* V-cycles per preconditioner application                     */
  int precision;           /* 0: FP64 throughout, GMRES left-preconditioned
                              1: FP32 V-cycle (FP32 storage and accumulation) inside
                                 FP64 flexible GMRES                                      */
  int flexible;            /* 1: right-preconditioned FGMRES even in FP64 (precision 1
                              implies it)                                                 */
  int skip_deflation;      /* 1: operator / V-cycle context only (no Z, E); deflation and
                              solve entry points then return IGA_E_INVALID                 */
  int arnoldi;             /* 0: modified Gram-Schmidt, all projections of an
                              iteration in one cooperative launch (grid barriers);
                              1 (default): classical Gram-Schmidt with one
                              reorthogonalisation (CGS2, barrier-free, a fixed number
                              of launches per iteration; batched solves always use it) */
  int fused_vcycle;        /* 0 (default): one kernel per V-cycle operation;
                              1: the FP32 V-cycle (2D, constant k, nu_pre = nu_post = 1)
                              runs each level as two fused kernels (residual +
                              restriction; prolongation + post-smoothing), the
                              pre-smoothing sweep recomputed where needed: half the
                              DRAM bytes, more instructions (slower on GB300 as
                              measured, kept for bandwidth-starved parts)               */
  int host_loop;           /* 0 (default): the GMRES loop runs on the device as a CUDA
                              graph with a WHILE conditional node; 1: the host launches
                              each iteration and reads the convergence flag (profiling)   */
  void* stream;            /* cudaStream_t for all work of this context                   */
  int precond;             /* preconditioner M~^{-1} of the solve (Section 4.3 list):
                              0 (default): n_vcycles multigrid V-cycles of the CSLP
                                 (C_MG^j); n_vcycles = 0 means no CSLP at all (the
                                 deflation-only D / D_eps of Section 4.3.1);
                              1: the CSLP matrix inverted exactly (C_ex).  1D: band LU
                                 with partial pivoting (any size, any k); 2D: constant
                                 k, n_x <= 2048, by fast diagonalisation of the finest
                                 level with FP64 iterative refinement               */
  int deflation;           /* 1 (default): ADP deflation, GMRES on M~^{-1} P A x^ =
                              M~^{-1} P f, u = Q f + P^T x^ (the DEF1 reading of Section
                              3's deflated system); 0: no deflation (GMRES on M~^{-1} A,
                              C_ex / C_MG alone); 2: the literal ordering P^T M~^{-1} A u =
                              P^T M~^{-1} f, iterate used as u (precision 0, flexible 0) */
  int robin;               /* 1D only.  0 (default): homogeneous Dirichlet at both ends;
                              1: MP 1-A (Section 2.1): Sommerfeld u' - i k u = 0 at x = 1
                              (the last basis function is an unknown, A = S - k^2 M -
                              i k N with the boundary mass N of Section 2.3; the CSLP
                              levels carry the same boundary term), Dirichlet at x = 0
                              with its value entered by iga_load_dirichlet.  Constant
                              k (n_lines = 0).                                            */
} iga_params;

typedef struct iga_ctx iga_ctx;

/* Fill *prm with the defaults: dim 2, p 3, n_el 32, k 10, beta (1, 0.5), eps 0,
   nu 1/1, omega 0.6, one V-cycle, FP64, DEF1 deflation, stream NULL. Host
   pointer. */
void iga_default_params(iga_params* prm);

/* Build everything the solve needs on the device (Sections 2.3, 3): knots,
   Gauss tables, 1D band matrices and transfer operators per multigrid level,
   the coarsest-level inverse, Z and the factorised E.  The coarsest level is
   inverted densely up to 2048 dofs; beyond that 2D setups are refused and 1D
   ones factorise its band.  E: fast diagonalisation for constant k in 2D and
   for small constant-k 1D problems without a Sommerfeld end (m_x <= 192),
   block LU for variable k in 2D, otherwise (1D) a band factorisation
   (partitioned LU with partial pivoting).  Synchronises.
   prm is a host pointer; *out receives a context to release with iga_destroy.
   Errors: IGA_E_INVALID for out-of-range parameters, IGA_E_OOM, IGA_E_CUDA. */
iga_status iga_setup(const iga_params* prm, iga_ctx** out);
void iga_destroy(iga_ctx* ctx);

/* Sizes.  n = n_x^dim fine dofs, m = floor(n_x/2)^dim deflation dofs. */
size_t iga_ndof(const iga_ctx* ctx);
size_t iga_coarse_ndof(const iga_ctx* ctx);
int iga_num_levels(const iga_ctx* ctx);
int iga_level_nx(const iga_ctx* ctx, int level);       /* interior functions per direction */
int iga_level_nel(const iga_ctx* ctx, int level);
const char* iga_status_str(iga_status s);
/* Number of kernels this library has launched in the process so far (host
   counter, incremented at every launch site). */
unsigned long long iga_launch_count(void);
const char* iga_last_error(const iga_ctx* ctx);

/* Copy the open knot vector of multigrid level `level` (n_el_l + 2p + 1 doubles,
   computed on the device as i/n_el_l) to the HOST buffer out (capacity cap).
   Synchronises. */
iga_status iga_get_knots(iga_ctx* ctx, int level, double* out, int cap);
/* Copy the 1D interior band matrix of level `level` to the HOST buffer out:
   which = 0 stiffness K, 1 mass M; layout [n_x][2p+1], out[i*(2p+1)+d+p] =
   Mat[i][i+d] (zero outside the matrix). Synchronises. */
iga_status iga_get_band(iga_ctx* ctx, int level, int which, double* out, size_t cap);
/* Copy the knot-insertion prolongation of level l -> l+1 as a dense HOST
   matrix [n_x(l)][n_x(l+1)] (interior rows and columns). Synchronises. */
iga_status iga_get_prolongation(iga_ctx* ctx, int level, double* out, size_t cap);

/* y = A x, A = S - M^{k^2} (Section 2.3), matrix-free: constant k by banded
   1D passes (K_x, M_x then M_y, K_y), variable k by per-element sum-factorised
   quadrature with k evaluated at the Gauss points.  x, y: n complex128, must
   not alias. */
iga_status iga_apply_A(iga_ctx* ctx, const iga_c128* x, iga_c128* y);

/* y = M_beta x on multigrid level `level` (0 = finest), M_beta =
   S_l - (beta1 - i beta2) M^{k^2}_l by rediscretisation (Section 3, CSLP
   equation).  FP64. */
iga_status iga_apply_Mshift(iga_ctx* ctx, int level, const iga_c128* x, iga_c128* y);

/* x_out = x_in + omega D^{-1} (b - M_beta x_in), D = diag(M_beta), `sweeps`
   times on level `level` (Section 3: damped Jacobi).  x_out receives the
   result; x_in is used as scratch and overwritten when sweeps > 1. FP64. */
iga_status iga_jacobi(iga_ctx* ctx, int level, const iga_c128* b, iga_c128* x_in,
                      iga_c128* x_out, int sweeps);

/* FP32 forms of the two operators above, as the FP32 V-cycle (precision 1)
   applies them: y = M_beta x and one damped Jacobi sweep x_out = x_in +
   omega D^{-1} (b - M_beta x_in) on level `level`, with FP32 bands and
   FP32 accumulation (single rounding per fused multiply-add).  Vectors:
   complex64, DEVICE, 8-byte aligned; x_in and x_out must not alias. */
iga_status iga_apply_Mshift32(iga_ctx* ctx, int level, const iga_c64* x, iga_c64* y);
iga_status iga_jacobi32(iga_ctx* ctx, int level, const iga_c64* b, const iga_c64* x_in, iga_c64* x_out);

/* Multigrid transfers between level l (fine) and l+1 (coarse): knot-insertion
   prolongation P_l (Section 4.2: linear interpolation is the p = 1 case).
   restrict: coarse = P_l^T fine.  prolong_add: fine += P_l coarse.  FP64. */
iga_status iga_restrict(iga_ctx* ctx, int level, const iga_c128* fine, iga_c128* coarse);
iga_status iga_prolong_add(iga_ctx* ctx, int level, const iga_c128* coarse, iga_c128* fine);

/* Coarsest-level solve x = M_beta^{-1} b with the dense inverse built at setup. */
iga_status iga_coarse_solve(iga_ctx* ctx, const iga_c128* b, iga_c128* x);

/* z ~ M_beta^{-1} r by n_vcycles V-cycles (Section 3; Section 4.2). r, z: n
   complex128.  In precision 1 the cycle runs in FP32 and r, z are converted. */
iga_status iga_vcycle_cslp(iga_ctx* ctx, const iga_c128* r, iga_c128* z);

/* z = M~^{-1} r, the preconditioner the solve applies (Section 4.3 list):
   n_vcycles V-cycles (as iga_vcycle_cslp), the exact CSLP inverse M_beta^{-1}
   (precond = 1; FP64 to ~1e-12 relative), or z = r (n_vcycles = 0).  r, z: n
   complex128, must not alias. */
iga_status iga_precond(iga_ctx* ctx, const iga_c128* r, iga_c128* z);

/* Deflation pieces (Section 3, Eq. adef1 and the Z / Z^T stencils):
   zt: c = Z^T x (n -> m);  z: x = Z c (m -> n);  esolve: s = E^{-1} t (m);
   deflate: y = P x = x - A Z E^{-1} Z^T x (n). */
iga_status iga_zt(iga_ctx* ctx, const iga_c128* x, iga_c128* c);
iga_status iga_z(iga_ctx* ctx, const iga_c128* c, iga_c128* x);
iga_status iga_esolve(iga_ctx* ctx, const iga_c128* t, iga_c128* s);
iga_status iga_deflate(iga_ctx* ctx, const iga_c128* x, iga_c128* y);

/* Right-hand side of the inhomogeneous Dirichlet value u(0) = g (context
   with robin = 1; Section 2.1, MP 1-A): f = -g A[unknowns, first basis
   function], non-zero in the first p entries (the first, interpolatory
   coefficient of the solution is g).  f: n complex128, overwritten. */
iga_status iga_load_dirichlet(iga_ctx* ctx, double g_re, double g_im, iga_c128* f);

/* Unit load vector of a point source at (x0, y0): f_i = Phi_i(x0, y0)
   (y0 ignored in 1D).  f: n complex128. */
iga_status iga_load_point_source(iga_ctx* ctx, double x0, double y0, iga_c128* f);

/* One modified Gram-Schmidt sweep (Arnoldi, Section 3 GMRES): for i = 0..j,
   h[i] = v_i^H w, w -= h[i] v_i; then h[j+1] = ||w||.  V: column-major,
   column i at V + i*ldv, n entries each.  w (n) is updated in place; h
   (j+2 entries) is written in DEVICE memory.  Uses context scratch. */
iga_status iga_mgs(iga_ctx* ctx, const iga_c128* V, size_t ldv, int j, iga_c128* w,
                   iga_c128* h);

/* Deflated, preconditioned GMRES (DEF1 reading of Section 3's deflated
   system): GMRES on M~^{-1} P A x^ = M~^{-1} P f from x^ = 0 (or FGMRES on
   P A M~^{-1} y = P f), then u = Q f + P^T x^.  Stops when the residual
   GMRES minimises has dropped by `tol` (1e-7 in Section 4.3) or after maxit.
   rhs, x: device, n complex128.  iters, res_hist (maxit+1 doubles, relative
   residual estimate per iteration, entry 0 = 1) and true_res
   (||f - A u|| / ||f||) are HOST pointers; res_hist and true_res may be NULL.
   Synchronises.  Returns IGA_OK or IGA_NOT_CONVERGED, or an error. */
iga_status iga_solve(iga_ctx* ctx, const iga_c128* rhs, iga_c128* x, double tol, int maxit,
                     int* iters, double* res_hist, double* true_res);

/* Same as iga_solve, but rhs and x are HOST pointers: the host->device and
   device->host copies are part of the call. */
iga_status iga_solve_host(iga_ctx* ctx, const iga_c128* rhs_host, iga_c128* x_host, double tol,
                          int maxit, int* iters, double* res_hist, double* true_res);

/* Operator tile shape chosen by the setup-time autotuner for `level` and
   precision (0 FP64, 1 FP32): 0 = 32x16, 1 = 16x16, 2 = 32x8 outputs per
   256-thread block, 3 = 8x8 per 64-thread block; FP64 only: 4 = 8x8 per
   256-thread block and 5 = 8x4 per 128-thread block with the real and
   imaginary parts of each value on a lane pair; -1 = not tuned (heuristic),
   -2 = bad argument.  The autotuner times every shape on each level with
   n_x >= 8 (constant k, 2D), as dependent launches in one CUDA graph, and
   caches the choice per (p, precision, n_x) for the process.  The E-residual
   sweep on the deflation grid takes the FP64 choice of the level of nearest
   n_x.  Constant k, 2D only (other operators have one kernel). */
int iga_tile_choice(const iga_ctx* ctx, int level, int precision);

/* Override the tile shape of `level` and `precision` (codes as above, -1 =
   heuristic) for the calls that follow; every shape computes the same
   operator.  Returns IGA_E_INVALID for a level or precision out of range or
   a code the precision does not have.  Not stream-ordered: call it between
   solves, not while work of this context is in flight or captured. */
iga_status iga_set_tile(iga_ctx* ctx, int level, int precision, int tile);

/* Bounded device waits (failure detection without a GPU fault; not in the
   paper).  The one wait in this library is the grid barrier of the
   cooperative MGS Arnoldi step (arnoldi = 0); it gives up after `polls`
   polls of ~64 ns (0 = the default 2^24, about one second), every block of
   the step returns, the solve stops and iga_solve returns IGA_E_TIMEOUT with
   the iterations done so far; the context stays usable.  phantom_arrivals = 1
   makes the barrier wait for one block more than the grid has, which never
   arrives: every wait then runs out (the deterministic way to exercise the
   timeout path); 0 restores normal barriers.  Synchronises; takes effect
   from the next solve. */
iga_status iga_set_wait_limit(iga_ctx* ctx, long long polls, int phantom_arrivals);

/* Batched solves in one CUDA-graph launch (not in the paper; the batched form of
   the method): instance b (context ctxs[b], each with its own k, p, mesh and
   precision) solves nrhs[b] right-hand sides stored back to back at rhs[b]
   (nrhs[b] * n_b complex128, DEVICE) into x[b] (same layout).  Every
   right-hand side runs as its own chain, concurrently with all others: the
   second and later right-hand sides of an instance use workspace clones of
   its context (the setup shared, the solve vectors and Krylov workspace of
   their own; created by the first call that needs them and freed by
   iga_destroy of the context), except for a context with a network attached,
   whose chains run in order.  Each right-hand side stops on its own
   convergence test (tol, maxit as iga_solve).
   iters and status (HOST, sum(nrhs) entries, instance-major; status may be
   NULL) receive per right-hand side the iteration count and IGA_OK /
   IGA_NOT_CONVERGED / error.  Contexts must be distinct, on one device, built
   with deflation.  Arnoldi runs as CGS2 (barrier-free) in this entry point so
   that the instances' kernels can overlap.  Work is launched on `stream`; the
   call synchronises.
   Returns the worst per-right-hand-side status. */
iga_status iga_solve_batched(iga_ctx* const* ctxs, int nb, const iga_c128* const* rhs, iga_c128* const* x,
                             const int* nrhs, double tol, int maxit, int* iters, int* status, void* stream);

/* ------------------------------------------------------------------ learned correction
   Not in the paper: a 3x3 convolutional network (channels 3 -> 32 -> 32 -> 32 -> 2,
   ReLU after the first three layers, BF16 weights/activations, FP32
   accumulation on the tensor cores) that corrects the FP32 CSLP V-cycle inside
   FGMRES: z = V(v) + gamma s NN(r~ / s), r~ = v - M_beta V(v), s = RMS(r~).
   A correction with any non-finite entry is dropped (the plain V-cycle result
   is used).  Input tensors are NHWC bf16 [B][H][W][16]: channels (Re r~ / s,
   Im r~ / s, (k h)^2 at the dof's Greville point, 13 zeros); outputs and
   targets FP32 [B][H][W][2].  Parameters: one flat FP32 vector, layer by layer
   W[co][3][3][ci] then bias[co] (iga_net_num_params() floats). */
typedef struct iga_net iga_net;
int iga_net_num_params(void);
/* He-initialised network (counter-based normal draws from `seed`). */
iga_status iga_net_create(unsigned long long seed, iga_net** out);
void iga_net_destroy(iga_net* net);
const char* iga_net_last_error(const iga_net* net);
/* HOST copies of the FP32 parameters (checkpoint / restore; set resets Adam). */
iga_status iga_net_get_params(iga_net* net, float* host, int cap);
iga_status iga_net_set_params(iga_net* net, const float* host, int count);
/* y = NN(x) for B images of H x W (x: DEVICE bf16 NHWC-16, y: DEVICE FP32 NHWC-2). */
iga_status iga_net_forward(iga_net* net, const void* x, float* y, int B, int H, int W, void* stream);
/* Batch loss mean_b ||NN(x_b) - t_b||^2 / ||t_b||^2 and its gradient (grad_host:
   HOST, iga_net_num_params() floats; loss_host: HOST; either may be NULL).
   Synchronises. */
iga_status iga_net_grad(iga_net* net, const void* x, const float* t, int B, int H, int W, float* grad_host,
                        float* loss_host, void* stream);
/* One Adam step (lr, beta 0.9 / 0.999, eps 1e-8) on the batch loss; loss_host
   (HOST, may be NULL) receives the loss before the step. */
iga_status iga_net_train_step(iga_net* net, const void* x, const float* t, int B, int H, int W, float lr,
                              float* loss_host, void* stream);
/* Attach (or detach with NULL) a network to a 2D context in precision 1. */
iga_status iga_attach_net(iga_ctx* ctx, iga_net* net, double gamma);
/* Training pair from a preconditioner input v (DEVICE, n complex128) by the
   error propagation of the FP32 V-cycle V: e = V(v), then `cycles` times
   e <- e - V(M_beta e); rt = M_beta e (so e = M_beta^{-1} rt exactly). */
iga_status iga_precond_pair(iga_ctx* ctx, const iga_c128* v, iga_c128* rt, iga_c128* e, int cycles);
/* Crop [y0, y0+Hc) x [x0, x0+Wc) of rt (and e) into a network input X (DEVICE
   bf16 [Hc][Wc][16]) and target T = e / (RMS(rt) gamma) (DEVICE FP32
   [Hc][Wc][2]; skipped when e or T is NULL). */
iga_status iga_net_pack(iga_ctx* ctx, const iga_c128* rt, const iga_c128* e, int x0, int y0, int Hc, int Wc,
                        void* X, float* T, double gamma);

/* Allocation-free variant of iga_mgs, for callers that cannot call cudaMalloc
   (for example code inside a framework whose caching allocator owns the device
   memory, or a latency-critical loop that must not pay cudaMalloc's implicit
   device synchronisation).  The paper has no counterpart: it is a property of
   this library, not of the method.
   Same sweep as iga_mgs, without a context: for i = 0..j, h[i] = v_i^H w,
   w -= h[i] v_i; then h[j+1] = ||w||.  V (column i at V + i*ldv, n entries),
   w (n, updated in place) and h (j+2 entries) are DEVICE pointers owned by the
   caller, 16-byte aligned; work is enqueued on `stream`.
   Scratch: the per-block partial sums live in one file-scope device array of
   32 KiB (4096 doubles, enough for 1024 reduction blocks; the sweep uses two
   blocks per SM).  Every GPU that loads the library holds that array until the
   process exits.  The function allocates nothing and calls no allocating
   library routine.  The first call on a device looks up the array's device
   address (cudaGetSymbolAddress) with that device current and keeps it for
   the rest of the process; make that first call before any stream capture,
   and do not call the function on a device after cudaDeviceReset (the kept
   address would no longer be valid).  All calls share the one array and it keeps
   the last call's contents (every entry is written before it is read), so two
   calls whose work overlaps on the GPU race: order them on one stream.
   Errors (no text is printed; there is no context to hold a message):
   IGA_E_INVALID for NULL/misaligned pointers, n = 0, ldv < n, j < 0, or a
   device with more than 512 SMs, whose reduction grid would exceed the
   1024-block scratch;
   IGA_E_CUDA if the symbol lookup or a launch fails. */
iga_status iga_mgs_noalloc(const iga_c128* V, size_t ldv, size_t n, int j, iga_c128* w, iga_c128* h,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IGA_HELMHOLTZ_H */
