// Shared device helpers and the internal context of the IgA Helmholtz library.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <functional>
#include <vector>

#include "../../include/iga_helmholtz.h"

#define IGA_MAXP 5
#define IGA_MAXQ (IGA_MAXP + 1)
#define IGA_MAX_LEVELS 16

// ------------------------------------------------------------------ complex
template <typename T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float>  { using t = float2; };

__host__ __device__ __forceinline__ double2 mkc(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2  mkc(float r, float i)  { return make_float2(r, i); }
template <typename C> __host__ __device__ __forceinline__ C czero();
template <> __host__ __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __host__ __device__ __forceinline__ float2  czero<float2>()  { return make_float2(0.f, 0.f); }

__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2  operator+(float2 a, float2 b)   { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2  operator-(float2 a, float2 b)   { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a)  { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2  operator*(float s, float2 a)    { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ float2  cmul(float2 a, float2 b)   { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
__host__ __device__ __forceinline__ double2 cconjmul(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
// acc + s * a   (real s)
__host__ __device__ __forceinline__ double2 cfma(double s, double2 a, double2 acc) { return make_double2(fma(s, a.x, acc.x), fma(s, a.y, acc.y)); }
__host__ __device__ __forceinline__ float2  cfma(float s, float2 a, float2 acc)    { return make_float2(fmaf(s, a.x, acc.x), fmaf(s, a.y, acc.y)); }
__host__ __device__ __forceinline__ double2 cinv(double2 a) { double d = a.x * a.x + a.y * a.y; return make_double2(a.x / d, -a.y / d); }
__host__ __device__ __forceinline__ float2  cinv(float2 a)  {   // one correctly rounded reciprocal on the device
  float d = a.x * a.x + a.y * a.y;
#ifdef __CUDA_ARCH__
  float m = __frcp_rn(d);
#else
  float m = 1.0f / d;
#endif
  return make_float2(a.x * m, -a.y * m);
}
__host__ __device__ __forceinline__ double2 tod(float2 a) { return make_double2((double)a.x, (double)a.y); }
__host__ __device__ __forceinline__ float2  tof(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <typename C> __host__ __device__ __forceinline__ C cconv(double2 a);
template <> __host__ __device__ __forceinline__ double2 cconv<double2>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2  cconv<float2>(double2 a)  { return tof(a); }

// ------------------------------------------------------------------ k field
struct KFieldDev {
  int n_lines;
  double lines[IGA_MAX_LINES][3];
  double k2[IGA_MAX_LINES + 1];   // squared wave numbers per layer
};

// k^2 at (x, y): layer = number of lines with ((a*x) + (b*y)) + c >= 0, evaluated
// without contraction so that both sides of a comparison round identically.
__device__ __forceinline__ double kfield_k2(const KFieldDev& kf, double x, double y) {
  int cnt = 0;
  for (int l = 0; l < kf.n_lines; ++l) {
    double s = __dadd_rn(__dadd_rn(__dmul_rn(kf.lines[l][0], x), __dmul_rn(kf.lines[l][1], y)), kf.lines[l][2]);
    cnt += (s >= 0.0);
  }
  return kf.k2[cnt];
}

// ------------------------------------------------------------------ context
// Fast diagonalisation of a tensor-product operator Op = M (x) K + K (x) M
// + c M (x) M (2D; K + c M in 1D) from the generalised eigenpairs of the 1D
// pencil (K, M): Op^{-1} = (V (x) V) diag(1 / (lam_i + lam_j + c)) (V (x) V)^T.
struct FdmData {
  int n = 0;                         // 1D size
  double* V = nullptr;               // generalised eigenvectors [n][n], row-major V[i][k]
  double* lam = nullptr;             // eigenvalues [n] (Rayleigh quotients)
  float* Vf = nullptr;               // FP32 copies of V and of V^T
  float* Vtf = nullptr;
  float2* dinv = nullptr;            // 1 / (lam_i + lam_j + c), formed in FP64, rounded once
  float2* w1 = nullptr;              // FP32 transform scratch (n^dim each)
  float2* w2 = nullptr;
  int refine = 2;                    // FP64 iterative refinement steps per solve
};

// LU factors of a complex band matrix (half bandwidth b <= 5) in P row
// partitions with spikes and the interface system (banded.cu)
struct BandLU {
  int n = 0, b = 0, s = 0, P = 0;
  double2* lu = nullptr;             // [n][3b+1] U rows of the partition blocks, column c at (c - r + b)
  double2* lm = nullptr;             // [n][b] multipliers of elimination step j (rows j+1 .. j+b)
  double2* rdiag = nullptr;          // [n] 1 / U(r, r)
  int* ipiv = nullptr;               // [n] pivot row of step j
  double2* ucs = nullptr;            // [n][2b] column j of U above the diagonal scaled by 1 / U(j, j):
                                     //   U(j-1-q, j) / U(j, j), zero above the partition's first row
  double2* V = nullptr;              // [n][b] right spikes A_i^{-1} [0; B_i]
  double2* Wl = nullptr;             // [n][b] left spikes A_i^{-1} [C_i; 0]
  double2* y = nullptr;              // [n] partition solutions
  int nr = 0, br = 0;                // interface system: 2 b P unknowns, half bandwidth 3b
  double2 *rlu = nullptr, *rlm = nullptr, *rrdiag = nullptr, *rucs = nullptr, *rz = nullptr, *rz2 = nullptr;
  int* ripiv = nullptr;
};

struct LevelData {
  int n_el = 0, nx = 0, ny = 1, n = 0;
  double* knots = nullptr;       // n_el + 2p + 1
  double* xq = nullptr;          // [n_el][Q] Gauss points
  double* wq = nullptr;          // [n_el][Q] Gauss weights (scaled by span length / 2)
  double* B = nullptr;           // [n_el][Q][p+1] basis values at Gauss points
  double* D = nullptr;           // [n_el][Q][p+1] derivatives
  float* Bf = nullptr;           // FP32 copies for the mixed-precision operator
  float* wqf = nullptr;
  double* K = nullptr;           // band [nx][2p+1]
  double* M = nullptr;
  float* Kf = nullptr;
  // FP32 interior stencil of K and M (uniform knots: every band row at least
  // 2p from either end), copied to the host at setup (kernel parameters)
  float sK[2 * IGA_MAXP + 1] = {}, sM[2 * IGA_MAXP + 1] = {};
  bool has_stencil = false;
  float* Mf = nullptr;
  // transfer to the next coarser level (absent on the coarsest)
  int wP = 0, wR = 0;
  double* Pw = nullptr; int* Plo = nullptr;   // fine row i: coarse cols Plo[i] .. +wP
  double* Rw = nullptr; int* Rlo = nullptr;   // coarse row j: fine rows Rlo[j] .. +wR
  float* Pwf = nullptr; float* Rwf = nullptr;
  float* k2qf = nullptr;                      // (unused unless variable k) reserved
  int vc_fmax = 0, vc_cmax = 0;               // fused V-cycle: fine footprint / coarse patch bounds
  // uniform-knot interior of the restriction table to the next level (host
  // copy, 2D tiled transfers): coarse rows j in [rj0, rj1] have
  // Rlo[j] = 2j + roff and the weights r
  struct {
    double r[8] = {};
    int roff = 0, rj0 = 0, rj1 = -1;
  } tst;
  int tr_fmax = 0, tp_cmax = 0;               // tiled 2D transfers (0: per-point kernels)
  // variable k: inverse diagonal of M_beta
  double2* dinv = nullptr;
  float2* dinvf = nullptr;
  // V-cycle work vectors
  double2 *vb = nullptr, *vx = nullptr, *vy = nullptr, *vr = nullptr;
  float2 *fb = nullptr, *fx = nullptr, *fy = nullptr, *fr = nullptr;
};

struct iga_net;

struct DevBuf {   // tracked allocation list
  std::vector<void*> ptrs;
  ~DevBuf() { for (void* p : ptrs) cudaFree(p); }
};

struct iga_ctx {
  iga_params prm{};
  int dim = 2, p = 3, L = 0, Q = 4;
  bool vark = false;
  KFieldDev kf{};
  double k2const = 0.0;              // k^2 when constant
  double robin_k = 0.0;              // 1D Sommerfeld end at x = 1: the -i k N coefficient (0: none)
  double2 sig{};                     // beta1 - i beta2
  LevelData lv[IGA_MAX_LEVELS];
  int tile[IGA_MAX_LEVELS][2];       // operator tile shape per level and precision (-1: heuristic)
  cudaStream_t st = nullptr;
  int device = 0;
  int num_sms = 148;
  // coarsest level: dense inverse, or (1D, more than IGA_MAX_COARSEST dofs) band LU
  int nc = 0;
  double2* cinv = nullptr;
  float2* cinvf = nullptr;
  bool coarse_banded = false;
  BandLU bandC;
  double2* cband_t = nullptr;        // FP32 V-cycle: the coarse right-hand side and solution in FP64
  double2* cband_x = nullptr;
  // 1D: band LU of E (deflation) and of the finest M_beta (exact CSLP)
  BandLU bandE;
  BandLU bandX;
  // deflation (ADP)
  int mx = 0;
  size_t m = 0;
  double* kc = nullptr;              // 1D coarse Z^T K Z  [mx][mx] dense
  double* mc = nullptr;              // 1D coarse Z^T M Z
  double2* ct = nullptr;             // m-sized scratch
  double2* cs = nullptr;
  double2* cw = nullptr;
  double2* ce1 = nullptr;            // refinement residual / correction
  double2* ce2 = nullptr;
  FdmData fdmE;                      // fast diagonalisation of E (constant k)
  FdmData fdmC;                      // of the fine-level CSLP matrix (exact CSLP, constant k)
  double2* cxr = nullptr;            // exact-CSLP refinement residual (n)
  double* kcb = nullptr;             // banded 1D coarse matrices (half width (p+4)/2)
  double* mcb = nullptr;
  float2* ctf = nullptr;             // FP32 copies of Z^T x and of the refinement residual
  float2* cef = nullptr;
  // variable-k E (block tridiagonal, banded in y): see deflation.cu
  int eblk = 0, enb = 0, els = 0;   // block size (lines per block * mx), number of blocks, lines
  double2* eDinv = nullptr;          // [enb][bs][bs] inverse diagonal blocks D_I^{-1}
  double2* eOff = nullptr;           // [enb][bs][bs] lower off-diagonal blocks E_{I,I-1}
  double2* eF = nullptr;             // [enb][bs][bs] D_I^{-1} E_{I,I+1}
  double2 *ep_t = nullptr, *ep_g = nullptr, *ep_v = nullptr;   // padded solve vectors
  // solve workspace
  double2* w0 = nullptr;             // n-sized vectors
  double2* w1 = nullptr;
  double2* w2 = nullptr;
  double2* w3 = nullptr;
  float2* fin = nullptr;             // FP32 V-cycle input / output at level 0
  float2* fout = nullptr;
  double2* hf = nullptr;             // device copies for the host-pointer solve
  double2* hu = nullptr;
  double* partials = nullptr;        // reduction scratch [2 * IGA_RED_BLOCKS + 16]
  int maxit_alloc = -1;
  double2* Vb = nullptr;             // Krylov basis (n x (maxit+1))
  double2* Zb = nullptr;             // FGMRES preconditioned vectors (n x maxit)
  double2* H = nullptr;              // (maxit+1) x maxit, column-major
  double* gstate = nullptr;          // cs[maxit], residual hist[maxit+1], scalars
  double2* gsn = nullptr;            // sn[maxit]
  double2* gg = nullptr;             // g[maxit+1]
  double2* gy = nullptr;             // y[maxit]
  int* gflag = nullptr;              // [0] converged, [1] nonfinite, [2] breakdown
  int* hflag = nullptr;              // pinned host copy
  // device-resident iteration (CUDA graph with a WHILE conditional node)
  double2* kvec = nullptr;           // vcur, zcur, wnext (3 n)
  int* kint = nullptr;               // [0] j, [1] barrier timeout
  unsigned* kbar = nullptr;          // grid barrier state
  int coop_blocks = 0;
  unsigned long long wait_polls = 1ull << 24;   // bounded device waits: polls before giving up
  int wait_phantom = 0;              // test hook: arrivals a grid barrier waits for beyond the grid
  bool vc_fused = false;             // V-cycle by the fused level kernels
  bool arnoldi_cgs = false;          // CGS2 Arnoldi (no grid barrier) instead of cooperative MGS
  int cgs_blocks = 0;
  double* cgs_part = nullptr;        // [cgs_blocks][2 (maxit+1)] partial projections
  double2* cgs_h = nullptr;          // current projections
  unsigned* cgs_ticket = nullptr;    // finished-block counter of the normalisation
  bool use_graph = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle gcond = 0;
  bool graph_flex = false;
  int graph_maxit = 0;
  unsigned long long body_kernels = 0;
  // learned correction of the FP32 V-cycle (precision 1 with a network attached)
  iga_net* net = nullptr;
  double net_gamma = 1.0;
  double* net_rms = nullptr;
  int* net_bad = nullptr;
  int* brec = nullptr;               // batched solve: per right-hand side {iters, conv, nonfinite, timeout}
  int brec_cap = 0;
  double* hres = nullptr;            // pinned host copy of residual
  // batched solves: workspace clones for the 2nd, 3rd, ... right-hand side of
  // this instance (every setup table and factor shared read-only with this
  // context, every vector a solve writes their own); owned and destroyed here
  std::vector<iga_ctx*> clones;
  DevBuf bufs;
  std::string err;
};

#define IGA_RED_BLOCKS 296
#define IGA_RED_THREADS 256
#define IGA_MAX_COARSEST 2048      // largest coarsest-level system inverted densely at setup

// ------------------------------------------------------------------ host helpers
// Every kernel launch site calls this once per launch (process-wide counter,
// read with iga_launch_count()).
void iga_count_launch();
void iga_add_launches(long long n);
iga_status set_err(iga_ctx* c, iga_status s, const char* fmt, ...);
template <typename T> inline T* dalloc(iga_ctx* c, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  c->bufs.ptrs.push_back(p);
  return (T*)p;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e__ = (call);                                                               \
    if (e__ != cudaSuccess) return set_err(ctx, IGA_E_CUDA, "%s: %s", #call, cudaGetErrorString(e__)); \
  } while (0)
#define CKL()                                                                               \
  do {                                                                                      \
    cudaError_t e__ = cudaGetLastError();                                                   \
    if (e__ != cudaSuccess) return set_err(ctx, IGA_E_CUDA, "launch: %s", cudaGetErrorString(e__)); \
  } while (0)
#define TRY(x) do { iga_status s__ = (x); if (s__ != IGA_OK) return s__; } while (0)

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------------ internal API
// setup.cu
iga_status setup_levels(iga_ctx* ctx);
// operator.cu
template <typename T>
iga_status op_apply(iga_ctx* ctx, int level, int which, const typename cplx<T>::t* x,
                    typename cplx<T>::t* y, const typename cplx<T>::t* z, int epi,
                    const typename cplx<T>::t* b, double omega);
iga_status setup_vark_diag(iga_ctx* ctx, int level);
iga_status autotune_tiles(iga_ctx* ctx);
// constant-coefficient tensor operator with explicit 1D bands (half width P)
iga_status op_apply_bands(iga_ctx* ctx, int P, int nx, int ny, const double* K, const double* M, double2 c,
                          const double2* x, double2* y, const double2* z, int epi,
                          float2* yf = nullptr);
// op "which": 0 = A (c = -1), 1 = M_beta (c = -sigma)
enum { OP_A = 0, OP_MB = 1 };
// epilogues
enum { EPI_Y = 0, EPI_ZMINUS = 1, EPI_JACOBI = 2, EPI_JACOBI_OUT64 = 3 /* FP32 sweep, FP64 output (sweep32.cu) */ };
// mg.cu
template <typename T> iga_status mg_vcycle(iga_ctx* ctx, const typename cplx<T>::t* r, typename cplx<T>::t* z);
// FP32 V-cycle with complex128 input and output (conversions fused into the
// first and last finest-level kernels where the register-stencil sweep runs)
iga_status mg_vcycle32_c128(iga_ctx* ctx, const double2* r, double2* z);
// sweep32.cu: one FP32 damped Jacobi sweep of M_beta on `level` writing its
// result in complex128 (the V-cycle's last post-sweep)
iga_status sweep32_jacobi_out64(iga_ctx* ctx, int level, const float2* x, double2* y64, const float2* b);
template <typename T> iga_status mg_restrict(iga_ctx* ctx, int l, const typename cplx<T>::t* f, typename cplx<T>::t* c);
template <typename T> iga_status mg_prolong_add(iga_ctx* ctx, int l, const typename cplx<T>::t* c, typename cplx<T>::t* f);
template <typename T> iga_status mg_coarse(iga_ctx* ctx, const typename cplx<T>::t* b, typename cplx<T>::t* x);
template <typename T> iga_status mg_vcycle_fused(iga_ctx* ctx, const typename cplx<T>::t* r, typename cplx<T>::t* z);
iga_status setup_fused_vcycle(iga_ctx* ctx);
iga_status setup_const_dinv(iga_ctx* ctx);
iga_status setup_tiled_transfers(iga_ctx* ctx);
template <typename T> iga_status mg_jacobi0(iga_ctx* ctx, int l, const typename cplx<T>::t* b, typename cplx<T>::t* x);
iga_status setup_coarse_inverse(iga_ctx* ctx);
// deflation.cu
iga_status setup_deflation(iga_ctx* ctx);
iga_status defl_zt(iga_ctx* ctx, const double2* x, double2* c, float2* cf = nullptr);
iga_status defl_z(iga_ctx* ctx, const double2* c, double2* x);
iga_status defl_esolve(iga_ctx* ctx, const double2* t, double2* s, const float2* tf = nullptr);
iga_status defl_apply(iga_ctx* ctx, const double2* x, double2* y);        // y = P x
iga_status defl_q(iga_ctx* ctx, const double2* x, double2* y);            // y = Q x
// y = P^T x = x - Q A x (tmp: n-sized scratch distinct from x, y)
iga_status defl_apply_T(iga_ctx* ctx, const double2* x, double2* y, double2* tmp1, double2* tmp2);
// exact CSLP (constant k): z = M_beta^{-1} r on the finest level
iga_status setup_exact_cslp(iga_ctx* ctx);
iga_status band_setup(iga_ctx* ctx, BandLU& F, const double2* Ab, int n, int b);
iga_status band_clone_scratch(iga_ctx* ctx, BandLU& F);
iga_ctx* clone_workspace(iga_ctx* parent);
iga_status band_solve(iga_ctx* ctx, const BandLU& F, const double2* t, double2* x);
iga_status band_probe(iga_ctx* ctx, int n, int b, const std::function<iga_status(const double2*, double2*)>& apply,
                      double2* x, double2* y, double2* Ab);
iga_status setup_robin_dinv(iga_ctx* ctx);         // mg.cu
iga_status cslp_exact_solve(iga_ctx* ctx, const double2* r, double2* z);
// ecoarse.cu (variable k)
iga_status setup_block_E(iga_ctx* ctx);
iga_status block_E_solve(iga_ctx* ctx, const double2* t, double2* s);
// cnn.cu
iga_status net_correct(iga_ctx* ctx, const float2* r, float2* z);
// krylov.cu
iga_status kry_mgs(iga_ctx* ctx, const double2* V, size_t ldv, int j, double2* w, double2* h);
iga_status kry_solve(iga_ctx* ctx, const double2* f, double2* x, double tol, int maxit, int* iters,
                     double* hist, double* true_res);
iga_status vec_norm(iga_ctx* ctx, const double2* x, size_t n, double* dev_out);
iga_status kry_precond(iga_ctx* ctx, const double2* r, double2* z);   // M~^{-1} as configured
iga_status kry_set_wait_limit(iga_ctx* ctx, long long polls, int phantom);
void launch_convert_d2f(const double2* a, float2* b, size_t n, cudaStream_t st);
void launch_convert_f2d(const float2* a, double2* b, size_t n, cudaStream_t st);
