// Direct solver for complex band matrices (1D problems): the deflation matrix
// E = Z^T A Z (Section 3, Eq. adef1: E is inverted exactly), the exactly
// inverted CSLP C_ex (Section 4.3) and the coarsest multigrid level.
//
// A 1D band matrix of size n and half bandwidth b is split into P partitions
// of s consecutive rows (the last takes the remainder, s >= 4 b).  Each
// partition's diagonal block A_i is factorised by Gaussian elimination with
// partial pivoting inside the band (L unpermuted, the row interchanges kept
// per step).  The couplings to the neighbouring partitions enter through the
// spikes V_i = A_i^{-1} [0; B_i] and W_i = A_i^{-1} [C_i; 0] (B_i: the block of
// the next partition's first b columns in this partition's last b rows, C_i:
// the previous partition's last b columns in this partition's first b rows).
// With y_i = A_i^{-1} t_i the solution is
//     x_i = y_i - V_i top(x_{i+1}) - W_i bot(x_{i-1}),
// top/bot = first/last b entries; evaluated at the partition ends this is a
// band system of size 2 b P (half bandwidth 3 b) for the interface values,
// factorised the same way as one partition.  A solve is: a warp per
// partition for y (forward and back substitution with register windows), one
// warp for the interface system, and a thread per row for x.  Sequential
// depth ~ 2 (s + 2 b P) steps with s ~ sqrt(2 b n), each step reading its
// coefficients from shared memory (staged chunk by chunk with cp.async);
// setup runs on the device.
#include "common.cuh"

#include <cmath>
#include <functional>

namespace {

__device__ __forceinline__ double2 bz() { return make_double2(0.0, 0.0); }

// entry (r, c) of a band matrix stored [n][2b+1] (zero outside the band)
__device__ __forceinline__ double2 band_at(const double2* Ab, int n, int b, int r, int c) {
  const int d = c - r;
  if (r < 0 || r >= n || c < 0 || c >= n || d < -b || d > b) return bz();
  return Ab[(size_t)r * (2 * b + 1) + d + b];
}

__device__ __forceinline__ void part_rows(int i, int n, int s, int P, int& r0, int& r1) {
  r0 = i * s;
  r1 = (i == P - 1) ? n : r0 + s;
}

// LU with partial pivoting of every partition's diagonal block (thread per
// partition).  lu row r holds columns r - b .. r + 2b at (c - r + b).
__global__ void k_band_factor(const double2* __restrict__ Ab, int n, int b, int s, int P, double2* lu, double2* lm,
                              double2* rdiag, int* ipiv, int* info) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  int r0, r1;
  part_rows(i, n, s, P, r0, r1);
  const int W = 3 * b + 1;
  for (int r = r0; r < r1; ++r)
    for (int q = 0; q < W; ++q) {
      const int c = r - b + q;
      lu[(size_t)r * W + q] = (c >= r0 && c < r1 && c <= r + b) ? band_at(Ab, n, b, r, c) : bz();
    }
  for (int j = r0; j < r1; ++j) {
    const int rmax = min(j + b, r1 - 1), cmax = min(j + 2 * b, r1 - 1);
    int p = j;
    double best = -1.0;
    for (int r = j; r <= rmax; ++r) {
      const double2 v = lu[(size_t)r * W + j - r + b];
      const double a = v.x * v.x + v.y * v.y;
      if (a > best) { best = a; p = r; }
    }
    ipiv[j] = p;
    if (p != j)
      for (int c = j; c <= cmax; ++c) {
        const double2 t = lu[(size_t)j * W + c - j + b];
        lu[(size_t)j * W + c - j + b] = lu[(size_t)p * W + c - p + b];
        lu[(size_t)p * W + c - p + b] = t;
      }
    const double2 d = lu[(size_t)j * W + b];
    double2 dinv = bz();
    if (d.x == 0.0 && d.y == 0.0) atomicExch(info, 1);
    else dinv = cinv(d);
    rdiag[j] = dinv;
    for (int q = 0; q < b; ++q) {
      const int r = j + 1 + q;
      double2 l = bz();
      if (r <= rmax) {
        l = cmul(lu[(size_t)r * W + j - r + b], dinv);
        lu[(size_t)r * W + j - r + b] = bz();
        for (int c = j + 1; c <= cmax; ++c)
          lu[(size_t)r * W + c - r + b] = lu[(size_t)r * W + c - r + b] - cmul(l, lu[(size_t)j * W + c - j + b]);
      }
      lm[(size_t)j * b + q] = l;
    }
  }
}

// x = A_i^{-1} x in place for rows r0 .. r1-1 of one partition (global memory;
// setup only)
__device__ void part_solve_gm(int r0, int r1, int b, const double2* lu, const double2* lm, const double2* rdiag,
                              const int* ipiv, double2* x) {
  const int W = 3 * b + 1;
  for (int j = r0; j < r1; ++j) {
    const int p = ipiv[j];
    if (p != j) { const double2 t = x[j]; x[j] = x[p]; x[p] = t; }
    for (int q = 0; q < b && j + 1 + q < r1; ++q) x[j + 1 + q] = x[j + 1 + q] - cmul(lm[(size_t)j * b + q], x[j]);
  }
  for (int j = r1 - 1; j >= r0; --j) {
    double2 acc = x[j];
    for (int c = j + 1; c <= min(j + 2 * b, r1 - 1); ++c) acc = acc - cmul(lu[(size_t)j * W + c - j + b], x[c]);
    x[j] = cmul(acc, rdiag[j]);
  }
}

// spikes (thread per partition, column and side); col-th column of V_i
// (side 0) or W_i (side 1), written to V / Wl [n][b]; scratch [2b][n] holds
// the right-hand sides
__global__ void k_band_spikes(const double2* __restrict__ Ab, int n, int b, int s, int P, const double2* lu,
                              const double2* lm, const double2* rdiag, const int* ipiv, double2* scratch, double2* V,
                              double2* Wl) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P * 2 * b) return;
  const int i = t / (2 * b), rem = t - i * 2 * b, side = rem / b, col = rem - side * b;
  int r0, r1;
  part_rows(i, n, s, P, r0, r1);
  double2* x = scratch + (size_t)(side * b + col) * n;      // column (side, col) of an n-long scratch panel
  for (int r = r0; r < r1; ++r) x[r] = bz();
  const bool present = side == 0 ? (i < P - 1) : (i > 0);
  if (present) {
    if (side == 0)
      for (int q = 0; q < b; ++q) x[r1 - b + q] = band_at(Ab, n, b, r1 - b + q, r1 + col);
    else
      for (int q = 0; q < b; ++q) x[r0 + q] = band_at(Ab, n, b, r0 + q, r0 - b + col);
    part_solve_gm(r0, r1, b, lu, lm, rdiag, ipiv, x);
  }
  double2* out = side == 0 ? V : Wl;
  for (int r = r0; r < r1; ++r) out[(size_t)r * b + col] = x[r];
}

// interface system R (2 b P unknowns: top_i = x[r0 .. r0+b), bot_i =
// x[r1-b .. r1)), band [nr][2 br + 1], br = 3b (thread per partition)
__global__ void k_band_reduced(int n, int b, int s, int P, const double2* V, const double2* Wl, double2* R) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  int r0, r1;
  part_rows(i, n, s, P, r0, r1);
  const int br = 3 * b, WR = 2 * br + 1;
  for (int a = 0; a < 2 * b; ++a) {
    const int row = 2 * b * i + a;
    const int lr = a < b ? r0 + a : r1 - b + (a - b);          // local row of the partition
    double2* Rrow = R + (size_t)row * WR;
    for (int q = 0; q < WR; ++q) Rrow[q] = bz();
    Rrow[br] = make_double2(1.0, 0.0);
    for (int c = 0; c < b; ++c) {
      if (i < P - 1) Rrow[2 * b * (i + 1) + c - row + br] = V[(size_t)lr * b + c];
      if (i > 0) Rrow[2 * b * (i - 1) + b + c - row + br] = Wl[(size_t)lr * b + c];
    }
  }
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// rows of coefficients staged per chunk (two chunks in flight per warp)
__host__ __device__ constexpr int band_chunk(int b) { return b <= 5 ? 128 : 64; }
__host__ __device__ constexpr size_t band_smem(int b) {
  return 2 * ((size_t)band_chunk(b) * (2 * b + 2) * sizeof(double2) + (size_t)band_chunk(b) * sizeof(int));
}

// y = A_i^{-1} t for every partition: one warp per partition (one warp per
// block).  The 32 lanes copy the next chunk of the partition's coefficient
// rows (multipliers, pivots and entering right-hand sides for the forward
// sweep; U rows, 1/U(r,r) and forward results for the back sweep) into shared
// memory with cp.async while lane 0 runs the sequential recurrence on the
// current chunk with register windows (forward: rows j .. j+b; back: the last
// 2b solution values).  BM >= b.  t, y and rz must not overlap.  rz
// (optional): the partition's first and last b solution values, as the
// interface system's right-hand side.
template <int BM>
__global__ void __launch_bounds__(32) k_band_solve_local(int n, int b, int s, int P, const double2* __restrict__ lu,
                                                         const double2* __restrict__ lm,
                                                         const double2* __restrict__ rdiag,
                                                         const int* __restrict__ ipiv, const double2* __restrict__ t,
                                                         double2* __restrict__ y, double2* __restrict__ rz) {
  const int i = blockIdx.x, lane = threadIdx.x;
  if (i >= P) return;
  int r0, r1;
  part_rows(i, n, s, P, r0, r1);
  const int len = r1 - r0, W = 3 * b + 1, CH = band_chunk(b);
  extern __shared__ __align__(16) unsigned char band_sm[];
  // buffer q: A [CH][2b] complex, B [CH], C [CH] complex, I [CH] int
  const size_t buf_bytes = (size_t)CH * (2 * b + 2) * sizeof(double2) + (size_t)CH * sizeof(int);
  auto bufA = [&](int q) { return reinterpret_cast<double2*>(band_sm + q * buf_bytes); };
  auto bufB = [&](int q) { return bufA(q) + (size_t)CH * 2 * b; };
  auto bufC = [&](int q) { return bufB(q) + CH; };
  auto bufI = [&](int q) { return reinterpret_cast<int*>(bufC(q) + CH); };
  const int nch = (len + CH - 1) / CH;

  // ---- forward sweep: chunk c = rows j0 .. j0 + CH - 1
  auto load_fwd = [&](int c, int q) {
    const int j0 = c * CH, rows = min(CH, len - j0);
    double2* A = bufA(q);
    for (int e = lane; e < rows * b; e += 32) cpa16(A + e, lm + (size_t)(r0 + j0) * b + e);
    double2* Bv = bufB(q);
    for (int e = lane; e < rows; e += 32) {
      const int idx = j0 + e + b + 1;
      if (idx < len) cpa16(Bv + e, t + r0 + idx);
    }
    int* I = bufI(q);
    for (int e = lane; e < rows; e += 32) cpa4(I + e, ipiv + r0 + j0 + e);
  };
  double2 w[BM + 1];
#pragma unroll
  for (int q = 0; q <= BM; ++q) w[q] = (lane == 0 && q <= b && q < len) ? t[r0 + q] : bz();
  load_fwd(0, 0);
  cpa_commit();
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) load_fwd(c + 1, (c + 1) & 1);
    cpa_commit();
    cpa_wait1();
    __syncwarp();
    if (lane == 0) {
      const int j0 = c * CH, rows = min(CH, len - j0);
      const double2* A = bufA(c & 1);
      const double2* Bv = bufB(c & 1);
      const int* I = bufI(c & 1);
      for (int jj = 0; jj < rows; ++jj) {
        const int j = j0 + jj, g = r0 + j;
        const int pj = I[jj] - g;
        const double2 w0 = w[0];
        double2 sel = w0;
#pragma unroll
        for (int q = 1; q <= BM; ++q) {           // interchange rows j and ipiv[j] (selects, no indexing)
          const bool hit = q == pj;
          const double2 wq = w[q];
          sel = hit ? wq : sel;
          w[q] = hit ? w0 : wq;
        }
        w[0] = sel;
        y[g] = sel;
#pragma unroll
        for (int q = 1; q <= BM; ++q)
          if (q <= b) w[q] = w[q] - cmul(A[jj * b + q - 1], sel);
#pragma unroll
        for (int q = 0; q < BM; ++q) w[q] = w[q + 1];
        w[BM] = bz();
        const double2 tn = (j + 1 + b < len) ? Bv[jj] : bz();
#pragma unroll
        for (int q = 0; q <= BM; ++q) w[q] = q == b ? tn : w[q];
      }
    }
    __syncwarp();                                  // the buffer is refilled two chunks later
  }
  // forward results are read back by every lane's copies
  if (lane == 0) __threadfence();
  __syncwarp();

  // ---- back sweep: chunk c = rows jlo .. jhi, taken from the end
  auto back_range = [&](int c, int& jlo, int& rows) {
    const int jhi = len - c * CH - 1;
    jlo = max(0, jhi - CH + 1);
    rows = jhi - jlo + 1;
  };
  auto load_back = [&](int c, int q) {
    int jlo, rows;
    back_range(c, jlo, rows);
    double2* A = bufA(q);
    for (int e = lane; e < rows * 2 * b; e += 32) {
      const int row = e / (2 * b), qq = e - row * 2 * b;
      cpa16(A + e, lu + (size_t)(r0 + jlo + row) * W + b + 1 + qq);
    }
    double2* Bv = bufB(q);
    double2* Cv = bufC(q);
    for (int e = lane; e < rows; e += 32) {
      cpa16(Bv + e, rdiag + r0 + jlo + e);
      cpa16(Cv + e, y + r0 + jlo + e);
    }
  };
  double2 x[2 * BM];
#pragma unroll
  for (int q = 0; q < 2 * BM; ++q) x[q] = bz();
  load_back(0, 0);
  cpa_commit();
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) load_back(c + 1, (c + 1) & 1);
    cpa_commit();
    cpa_wait1();
    __syncwarp();
    if (lane == 0) {
      int jlo, rows;
      back_range(c, jlo, rows);
      const double2* A = bufA(c & 1);
      const double2* Bv = bufB(c & 1);
      const double2* Cv = bufC(c & 1);
      for (int jj = rows - 1; jj >= 0; --jj) {
        double2 a0 = Cv[jj], a1 = bz();            // two partial sums shorten the dependent chain
#pragma unroll
        for (int q = 0; q < 2 * BM; q += 2) {
          if (q < 2 * b) a0 = a0 - cmul(A[jj * 2 * b + q], x[q]);
          if (q + 1 < 2 * b) a1 = a1 - cmul(A[jj * 2 * b + q + 1], x[q + 1]);
        }
        const double2 xj = cmul(a0 + a1, Bv[jj]);
#pragma unroll
        for (int q = 2 * BM - 1; q > 0; --q) x[q] = x[q - 1];
        x[0] = xj;
        y[r0 + jlo + jj] = xj;
      }
    }
    __syncwarp();
  }
  if (rz && lane == 0)
    for (int a = 0; a < b; ++a) {
      rz[2 * b * i + a] = y[r0 + a];
      rz[2 * b * i + b + a] = y[r1 - b + a];
    }
}

// x_r = y_r - V_r top(x_{i+1}) - W_r bot(x_{i-1}) (thread per row)
__global__ void k_band_update(int n, int b, int s, int P, const double2* __restrict__ V,
                              const double2* __restrict__ Wl, const double2* __restrict__ z,
                              const double2* __restrict__ y, double2* __restrict__ x) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int i = min(r / s, P - 1);
  double2 acc = y[r];
  if (i < P - 1)
    for (int c = 0; c < b; ++c) acc = acc - cmul(V[(size_t)r * b + c], z[2 * b * (i + 1) + c]);
  if (i > 0)
    for (int c = 0; c < b; ++c) acc = acc - cmul(Wl[(size_t)r * b + c], z[2 * b * (i - 1) + b + c]);
  x[r] = acc;
}

// probing: x = sum of e_j over j = c (mod 2b+1); the band entries of column
// class c from y = A x
__global__ void k_probe_vec(double2* x, int n, int stride, int c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = make_double2(i % stride == c ? 1.0 : 0.0, 0.0);
}
__global__ void k_probe_scatter(const double2* y, int n, int b, int c, double2* Ab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int stride = 2 * b + 1, lo = i - b;
  const int j = lo + (((c - lo) % stride) + stride) % stride;       // the one column of class c in [i-b, i+b]
  if (j >= 0 && j < n) Ab[(size_t)i * stride + j - i + b] = y[i];
}

// forward and back substitution of every partition (b <= 5: the matrices;
// b <= 15: the interface system, half bandwidth 3b)
template <int BM>
void launch_local(int n, int b, int s, int P, const double2* lu, const double2* lm, const double2* rdiag,
                  const int* ipiv, const double2* t, double2* y, double2* rz, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_band_solve_local<BM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_smem(BM));
    attr = true;
  }
  k_band_solve_local<BM><<<P, 32, band_smem(b), st>>>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz);
  iga_count_launch();
}

// forward and back substitution of every partition with the narrowest window
// that holds b (b <= 5: the matrices; 3, 6, 9, 12, 15: interface systems)
void solve_parts(int n, int b, int s, int P, const double2* lu, const double2* lm, const double2* rdiag,
                 const int* ipiv, const double2* t, double2* y, double2* rz, cudaStream_t st) {
  switch (b) {
    case 1: launch_local<1>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
    case 2: launch_local<2>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
    case 3: launch_local<3>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
    case 4: launch_local<4>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
    case 5: launch_local<5>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
    case 6: launch_local<6>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
    case 9: launch_local<9>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
    case 12: launch_local<12>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
    default: launch_local<15>(n, b, s, P, lu, lm, rdiag, ipiv, t, y, rz, st); break;
  }
}

}  // namespace

// Band of an operator by probing: 2b+1 applications to class vectors.
iga_status band_probe(iga_ctx* ctx, int n, int b, const std::function<iga_status(const double2*, double2*)>& apply,
                      double2* x, double2* y, double2* Ab) {
  CK(cudaMemsetAsync(Ab, 0, sizeof(double2) * (size_t)n * (2 * b + 1), ctx->st));
  for (int c = 0; c < 2 * b + 1; ++c) {
    k_probe_vec<<<cdiv(n, 256), 256, 0, ctx->st>>>(x, n, 2 * b + 1, c); iga_count_launch();
    TRY(apply(x, y));
    k_probe_scatter<<<cdiv(n, 256), 256, 0, ctx->st>>>(y, n, b, c, Ab); iga_count_launch();
  }
  CKL();
  return IGA_OK;
}

iga_status band_setup(iga_ctx* ctx, BandLU& F, const double2* Ab, int n, int b) {
  if (n < 1 || b < 1 || b > 5) return set_err(ctx, IGA_E_INVALID, "band solver: n = %d, b = %d", n, b);
  int s = (int)std::ceil(std::sqrt((double)n * 2.0 * b));
  if (s < 4 * b) s = 4 * b;
  int P = n / s;
  if (P <= 1) { P = 1; s = n; }
  F.n = n; F.b = b; F.s = s; F.P = P;
  const int W = 3 * b + 1;
  F.lu = dalloc<double2>(ctx, (size_t)n * W);
  F.y = dalloc<double2>(ctx, n);
  F.lm = dalloc<double2>(ctx, (size_t)n * b);
  F.rdiag = dalloc<double2>(ctx, n);
  F.ipiv = dalloc<int>(ctx, n);
  int* info = dalloc<int>(ctx, 2);
  if (!F.lu || !F.y || !F.lm || !F.rdiag || !F.ipiv || !info) return set_err(ctx, IGA_E_OOM, "band solver");
  CK(cudaMemsetAsync(info, 0, 2 * sizeof(int), ctx->st));
  k_band_factor<<<cdiv(P, 32), 32, 0, ctx->st>>>(Ab, n, b, s, P, F.lu, F.lm, F.rdiag, F.ipiv, info); iga_count_launch();
  CKL();
  if (P > 1) {
    F.V = dalloc<double2>(ctx, (size_t)n * b);
    F.Wl = dalloc<double2>(ctx, (size_t)n * b);
    double2* scratch = dalloc<double2>(ctx, (size_t)n * 2 * b);
    F.nr = 2 * b * P;
    F.br = 3 * b;
    double2* R = dalloc<double2>(ctx, (size_t)F.nr * (2 * F.br + 1));
    const int WR = 3 * F.br + 1;
    F.rlu = dalloc<double2>(ctx, (size_t)F.nr * WR);
    F.rlm = dalloc<double2>(ctx, (size_t)F.nr * F.br);
    F.rrdiag = dalloc<double2>(ctx, F.nr);
    F.ripiv = dalloc<int>(ctx, F.nr);
    F.rz = dalloc<double2>(ctx, F.nr);
    F.rz2 = dalloc<double2>(ctx, F.nr);
    if (!F.V || !F.Wl || !scratch || !R || !F.rlu || !F.rlm || !F.rrdiag || !F.ripiv || !F.rz || !F.rz2)
      return set_err(ctx, IGA_E_OOM, "band solver spikes");
    k_band_spikes<<<cdiv(P * 2 * b, 64), 64, 0, ctx->st>>>(Ab, n, b, s, P, F.lu, F.lm, F.rdiag, F.ipiv, scratch, F.V,
                                                          F.Wl); iga_count_launch();
    k_band_reduced<<<cdiv(P, 64), 64, 0, ctx->st>>>(n, b, s, P, F.V, F.Wl, R); iga_count_launch();
    k_band_factor<<<1, 32, 0, ctx->st>>>(R, F.nr, F.br, F.nr, 1, F.rlu, F.rlm, F.rrdiag, F.ripiv, info + 1);
    iga_count_launch();
    CKL();
  }
  int hinfo[2] = {0, 0};
  CK(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (hinfo[0] || hinfo[1])
    return set_err(ctx, IGA_E_INVALID, "band solver: singular %s block", hinfo[0] ? "partition" : "interface");
  return IGA_OK;
}

// fresh solve scratch (y, rz, rz2) for a workspace clone sharing the factors
iga_status band_clone_scratch(iga_ctx* ctx, BandLU& F) {
  if (F.n == 0) return IGA_OK;
  F.y = dalloc<double2>(ctx, F.n);
  if (!F.y) return set_err(ctx, IGA_E_OOM, "band solver scratch");
  if (F.P > 1) {
    F.rz = dalloc<double2>(ctx, F.nr);
    F.rz2 = dalloc<double2>(ctx, F.nr);
    if (!F.rz || !F.rz2) return set_err(ctx, IGA_E_OOM, "band solver scratch");
  }
  return IGA_OK;
}

// x = A^{-1} t (t and x may be the same vector)
iga_status band_solve(iga_ctx* ctx, const BandLU& F, const double2* t, double2* x) {
  if (F.P == 1 && x != t) {
    solve_parts(F.n, F.b, F.s, 1, F.lu, F.lm, F.rdiag, F.ipiv, t, x, nullptr, ctx->st);
  } else {
    solve_parts(F.n, F.b, F.s, F.P, F.lu, F.lm, F.rdiag, F.ipiv, t, F.y, F.P > 1 ? F.rz : nullptr, ctx->st);
    if (F.P > 1) {
      solve_parts(F.nr, F.br, F.nr, 1, F.rlu, F.rlm, F.rrdiag, F.ripiv, F.rz, F.rz2, nullptr, ctx->st);
      k_band_update<<<cdiv(F.n, 256), 256, 0, ctx->st>>>(F.n, F.b, F.s, F.P, F.V, F.Wl, F.rz2, F.y, x);
      iga_count_launch();
    } else {
      CK(cudaMemcpyAsync(x, F.y, sizeof(double2) * F.n, cudaMemcpyDeviceToDevice, ctx->st));
    }
  }
  CKL();
  return IGA_OK;
}
