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
// partition for y (forward and back substitution, the elimination window
// spread over the warp's lanes), one warp for the interface system, and a
// thread per row for x.  Sequential depth ~ 2 (s + 2 b P) steps with
// s ~ sqrt(2 b n), each step reading its coefficients from shared memory
// (staged chunk by chunk with cp.async); setup runs on the device.
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

__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
// w - a s with four fused multiply-adds (dependent depth two)
__device__ __forceinline__ double2 cfms(double2 w, double2 a, double2 s) {
  return make_double2(fma(-a.x, s.x, fma(a.y, s.y, w.x)), fma(-a.x, s.y, fma(-a.y, s.x, w.y)));
}

// rows of coefficients staged per chunk (two chunks in flight per warp), a
// multiple of the warp width; a stage holds [CH][2b] coefficients, [CH]
// entering values and [CH] pivots
__host__ __device__ constexpr int band_chunk(int b) { return b <= 5 ? 128 : 64; }
__host__ __device__ constexpr size_t band_stage(int b) {
  return (size_t)band_chunk(b) * (2 * b + 1) * sizeof(double2) + (size_t)band_chunk(b) * sizeof(int);
}
__host__ __device__ constexpr size_t band_smem(int b) { return 2 * band_stage(b); }

__device__ __forceinline__ double flip_sign(double v, bool neg) {
  return __hiloint2double(__double2hiint(v) ^ (neg ? (int)0x80000000 : 0), __double2loint(v));
}

// Forward sweep of one partition (rows r0 .. r0 + len - 1), y = L^{-1} Pi t,
// with the real and imaginary parts of the row in slot j mod 16 in lanes
// 2 slot and 2 slot + 1: a step is three shuffles (the pivot row's two parts
// to every lane, row j's part to the pivot row's lanes) and one complex
// multiply-add of two FP64 warp instructions in the b rows below; the lanes of
// a finished row take row j + 16.  b <= 15.  Ends with the results visible to
// the back sweep's cp.async copies.
__device__ __forceinline__ void band_fwd_pair(int b, int r0, int len, const double2* __restrict__ lm,
                                              const int* __restrict__ ipiv, const double2* __restrict__ t,
                                              double2* __restrict__ y, unsigned char* band_sm, int lane) {
  const int slot = lane >> 1, c = lane & 1, b2 = 2 * b, CH = band_chunk(b);
  const double* td = reinterpret_cast<const double*>(t);
  double* yd = reinterpret_cast<double*>(y);
  const size_t sb = band_stage(b);
  auto bufA = [&](int q) { return reinterpret_cast<double2*>(band_sm + q * sb); };
  auto bufE = [&](int q) { return bufA(q) + (size_t)CH * b2; };
  auto bufI = [&](int q) { return reinterpret_cast<int*>(bufE(q) + CH); };
  const int nch = (len + CH - 1) / CH;
  auto load_fwd = [&](int ch, int q) {
    const int j0 = ch * CH, rows = min(CH, len - j0);
    double2* A = bufA(q);
    for (int e = lane; e < rows * b; e += 32) cpa16(A + e, lm + (size_t)(r0 + j0) * b + e);
    double2* Ev = bufE(q);
    for (int e = lane; e < rows; e += 32) {
      const int idx = j0 + e + 16;
      if (idx < len) cpa16(Ev + e, t + r0 + idx);
      else Ev[e] = bz();
    }
    int* I = bufI(q);
    for (int e = lane; e < rows; e += 32) cpa4(I + e, ipiv + r0 + j0 + e);
  };
  double w = slot < len ? td[2 * (size_t)(r0 + slot) + c] : 0.0;
  double fin = 0.0;
  load_fwd(0, 0);
  cpa_commit();
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) load_fwd(ch + 1, (ch + 1) & 1);
    cpa_commit();
    cpa_wait1();
    __syncwarp();
    const int j0 = ch * CH, rows = min(CH, len - j0);
    const double2* A = bufA(ch & 1);
    const double* Ev = reinterpret_cast<const double*>(bufE(ch & 1));
    const int* I = bufI(ch & 1);
#pragma unroll 4
    for (int jj = 0; jj < rows; ++jj) {
      const int j = j0 + jj, me = j & 15;
      const int pl = (I[jj] - r0) & 15;            // slot of the pivot row
      const double sc = __shfl_sync(0xffffffffu, w, 2 * pl + c);       // pivot value, this lane's part
      const double so = __shfl_sync(0xffffffffu, w, 2 * pl + 1 - c);   // and the other part
      const double rj = __shfl_sync(0xffffffffu, w, 2 * me + c);       // row j, for the pivot row's lanes
      if (slot == pl) w = rj;
      const int d = (slot - me) & 15;              // this lane holds row j + d
      if (d >= 1 && d <= b) {
        const double2 a = A[jj * b + d - 1];
        w = fma(-a.x, sc, fma(flip_sign(a.y, c), so, w));
      }
      if (slot == me) { fin = sc; w = Ev[2 * jj + c]; }
      if (me == 15 || j == len - 1) {
        const int row = (j & ~15) + slot;
        if (row <= j) yd[2 * (size_t)(r0 + row) + c] = fin;
      }
    }
    __syncwarp();
  }
  __threadfence();
  __syncwarp();
}

// y = A_i^{-1} t for every partition: one warp per partition (one warp per
// block), b <= 15.  The forward sweep is band_fwd_pair.  The back sweep runs
// column by column with row j in lane j mod 32 for as long as it is in the
// window (so no step shifts the window): step j broadcasts the finished sum
// acc_j of row j (one shuffle) and subtracts U(r, j) x_j = (U(r, j) / U(j, j))
// acc_j from rows j-1 .. j-2b in their lanes (one complex multiply-add, four
// FP64 warp instructions, whatever b; the columns of U are scaled at setup),
// so that x_j = acc_j / U(j, j) is formed 32 rows at a time, off the
// dependent chain.  The next chunk of coefficients is copied into shared
// memory with cp.async while the current one is swept.  t, y and rz must not
// overlap.  rz (optional): the partition's first and last b solution values,
// as the interface system's right-hand side.
__global__ void __launch_bounds__(32) k_band_solve_warp(int n, int b, int s, int P, const double2* __restrict__ lm,
                                                        const int* __restrict__ ipiv, const double2* __restrict__ ucs,
                                                        const double2* __restrict__ rdiag,
                                                        const double2* __restrict__ t, double2* __restrict__ y,
                                                        double2* __restrict__ rz) {
  const int i = blockIdx.x, lane = threadIdx.x;
  if (i >= P) return;
  int r0, r1;
  part_rows(i, n, s, P, r0, r1);
  const int len = r1 - r0, b2 = 2 * b, CH = band_chunk(b);
  extern __shared__ __align__(16) unsigned char band_sm[];
  const size_t sb = band_stage(b);
  auto bufA = [&](int q) { return reinterpret_cast<double2*>(band_sm + q * sb); };
  auto bufE = [&](int q) { return bufA(q) + (size_t)CH * b2; };
  const int nch = (len + CH - 1) / CH;

  band_fwd_pair(b, r0, len, lm, ipiv, t, y, band_sm, lane);

  // ---- back sweep over m = len - 1 - j; chunk c = m0 .. m0 + CH - 1; row
  // j = len - 1 - m lives in lane m mod 32
  auto load_back = [&](int c, int q) {
    const int m0 = c * CH, rows = min(CH, len - m0);
    double2* A = bufA(q);
    for (int e = lane; e < rows * b2; e += 32) {
      const int mm = e / b2, qq = e - mm * b2;
      cpa16(A + e, ucs + (size_t)(r0 + len - 1 - m0 - mm) * b2 + qq);
    }
    double2* Ev = bufE(q);
    for (int e = lane; e < rows; e += 32) {
      const int jn = len - 1 - m0 - e - 32;
      if (jn >= 0) cpa16(Ev + e, y + r0 + jn);
      else Ev[e] = bz();
    }
  };
  double2 acc = lane < len ? y[r0 + len - 1 - lane] : bz();
  double2 fin = bz(), dv = bz();
  load_back(0, 0);
  cpa_commit();
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) load_back(c + 1, (c + 1) & 1);
    cpa_commit();
    cpa_wait1();
    __syncwarp();
    const int m0 = c * CH, rows = min(CH, len - m0);
    const double2* A = bufA(c & 1);
    const double2* Ev = bufE(c & 1);
#pragma unroll 4
    for (int mm = 0; mm < rows; ++mm) {
      const int m = m0 + mm, me = m & 31;
      if (me == 0) {                               // 1 / U(j, j) of this lane's row in the coming group
        const int jr = len - 1 - m - lane;
        dv = jr >= 0 ? rdiag[r0 + jr] : bz();
      }
      const double2 a = shfl2(acc, me);            // acc_j, final
      const int d = (lane - me) & 31;              // this lane holds row j - d
      if (d >= 1 && d <= b2) acc = cfms(acc, A[mm * b2 + d - 1], a);
      if (lane == me) { fin = a; acc = Ev[mm]; }
      if (me == 31 || m == len - 1) {              // rows of m = (m & ~31) .. m are final
        const int mr = (m & ~31) + lane;
        if (mr <= m) y[r0 + len - 1 - mr] = cmul(fin, dv);
      }
    }
    __syncwarp();
  }
  if (rz) {
    __syncwarp();
    for (int a = lane; a < b2; a += 32) rz[b2 * i + a] = a < b ? y[r0 + a] : y[r1 - b2 + a];
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


// The same solve with the back sweep also on two lanes per row (lane
// 2 slot + c holds part c of the row in slot m mod 16): a complex
// multiply-add is then two FP64 warp instructions instead of four.  The back
// sweep's window of 2b + 1 rows must fit in 16 slots: b <= 7.  Arguments as
// k_band_solve_warp.
__global__ void __launch_bounds__(32) k_band_solve_pair(int n, int b, int s, int P, const double2* __restrict__ lm,
                                                        const int* __restrict__ ipiv, const double2* __restrict__ ucs,
                                                        const double2* __restrict__ rdiag,
                                                        const double2* __restrict__ t, double2* __restrict__ y,
                                                        double2* __restrict__ rz) {
  const int i = blockIdx.x, lane = threadIdx.x, slot = lane >> 1, c = lane & 1;
  if (i >= P) return;
  int r0, r1;
  part_rows(i, n, s, P, r0, r1);
  const int len = r1 - r0, b2 = 2 * b, CH = band_chunk(b);
  double* yd = reinterpret_cast<double*>(y);
  extern __shared__ __align__(16) unsigned char band_sm[];
  const size_t sb = band_stage(b);
  auto bufA = [&](int q) { return reinterpret_cast<double2*>(band_sm + q * sb); };
  auto bufE = [&](int q) { return bufA(q) + (size_t)CH * b2; };
  const int nch = (len + CH - 1) / CH;

  band_fwd_pair(b, r0, len, lm, ipiv, t, y, band_sm, lane);

  // ---- back sweep over m = len - 1 - j; row j in slot m mod 16
  auto load_back = [&](int ch, int q) {
    const int m0 = ch * CH, rows = min(CH, len - m0);
    double2* A = bufA(q);
    for (int e = lane; e < rows * b2; e += 32) {
      const int mm = e / b2, qq = e - mm * b2;
      cpa16(A + e, ucs + (size_t)(r0 + len - 1 - m0 - mm) * b2 + qq);
    }
    double2* Ev = bufE(q);
    for (int e = lane; e < rows; e += 32) {
      const int jn = len - 1 - m0 - e - 16;
      if (jn >= 0) cpa16(Ev + e, y + r0 + jn);
      else Ev[e] = bz();
    }
  };
  double acc = slot < len ? yd[2 * (size_t)(r0 + len - 1 - slot) + c] : 0.0;
  double fx = 0.0, fy = 0.0;
  double2 dv = bz();
  load_back(0, 0);
  cpa_commit();
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) load_back(ch + 1, (ch + 1) & 1);
    cpa_commit();
    cpa_wait1();
    __syncwarp();
    const int m0 = ch * CH, rows = min(CH, len - m0);
    const double2* A = bufA(ch & 1);
    const double* Ev = reinterpret_cast<const double*>(bufE(ch & 1));
#pragma unroll 4
    for (int mm = 0; mm < rows; ++mm) {
      const int m = m0 + mm, me = m & 15;
      if (me == 0) {
        const int jr = len - 1 - m - slot;
        dv = jr >= 0 ? rdiag[r0 + jr] : bz();
      }
      const double ac = __shfl_sync(0xffffffffu, acc, 2 * me + c);     // acc_j, this lane's part
      const double ao = __shfl_sync(0xffffffffu, acc, 2 * me + 1 - c);
      const int d = (slot - me) & 15;              // this lane holds row j - d
      if (d >= 1 && d <= b2) {
        const double2 u = A[mm * b2 + d - 1];
        acc = fma(-u.x, ac, fma(flip_sign(u.y, c), ao, acc));
      }
      if (slot == me) {
        fx = c ? ao : ac;
        fy = c ? ac : ao;
        acc = Ev[2 * mm + c];
      }
      if (me == 15 || m == len - 1) {              // x = acc_j / U(j, j), part c
        const int mr = (m & ~15) + slot;
        if (mr <= m)
          yd[2 * (size_t)(r0 + len - 1 - mr) + c] = fma(fx, c ? dv.y : dv.x, flip_sign(fy, !c) * (c ? dv.x : dv.y));
      }
    }
    __syncwarp();
  }
  if (rz) {
    __syncwarp();
    for (int a = lane; a < b2; a += 32) rz[b2 * i + a] = a < b ? y[r0 + a] : y[r1 - b2 + a];
  }
}

// U(j-1-q, j) / U(j, j), q < 2b, inside each partition (thread per row)
__global__ void k_band_ucols(int n, int b, int s, int P, const double2* __restrict__ lu,
                             const double2* __restrict__ rdiag, double2* __restrict__ ucs) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int i = min(g / s, P - 1), r0 = i * s, W = 3 * b + 1;
  const double2 dj = rdiag[g];
  for (int q = 0; q < 2 * b; ++q) {
    const int r = g - 1 - q;
    ucs[(size_t)g * 2 * b + q] = r >= r0 ? cmul(lu[(size_t)r * W + q + 1 + b], dj) : bz();
  }
}

// forward and back substitution of every partition (b <= 5: the matrices;
// b <= 15: interface systems, half bandwidth 3b); two lanes per row where the
// window fits (b <= 7)
void solve_parts(int n, int b, int s, int P, const double2* lm, const int* ipiv, const double2* ucs,
                 const double2* rdiag, const double2* t, double2* y, double2* rz, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_band_solve_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_smem(15));
    cudaFuncSetAttribute(k_band_solve_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_smem(15));
    attr = true;
  }
  if (b <= 7) k_band_solve_pair<<<P, 32, band_smem(b), st>>>(n, b, s, P, lm, ipiv, ucs, rdiag, t, y, rz);
  else k_band_solve_warp<<<P, 32, band_smem(b), st>>>(n, b, s, P, lm, ipiv, ucs, rdiag, t, y, rz);
  iga_count_launch();
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
  F.ucs = dalloc<double2>(ctx, (size_t)n * 2 * b);
  if (!F.ucs) return set_err(ctx, IGA_E_OOM, "band solver");
  k_band_ucols<<<cdiv(n, 256), 256, 0, ctx->st>>>(n, b, s, P, F.lu, F.rdiag, F.ucs); iga_count_launch();
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
    F.rucs = dalloc<double2>(ctx, (size_t)F.nr * 2 * F.br);
    F.rz = dalloc<double2>(ctx, F.nr);
    F.rz2 = dalloc<double2>(ctx, F.nr);
    if (!F.V || !F.Wl || !scratch || !R || !F.rlu || !F.rlm || !F.rrdiag || !F.ripiv || !F.rucs || !F.rz || !F.rz2)
      return set_err(ctx, IGA_E_OOM, "band solver spikes");
    k_band_spikes<<<cdiv(P * 2 * b, 64), 64, 0, ctx->st>>>(Ab, n, b, s, P, F.lu, F.lm, F.rdiag, F.ipiv, scratch, F.V,
                                                          F.Wl); iga_count_launch();
    k_band_reduced<<<cdiv(P, 64), 64, 0, ctx->st>>>(n, b, s, P, F.V, F.Wl, R); iga_count_launch();
    k_band_factor<<<1, 32, 0, ctx->st>>>(R, F.nr, F.br, F.nr, 1, F.rlu, F.rlm, F.rrdiag, F.ripiv, info + 1);
    iga_count_launch();
    k_band_ucols<<<cdiv(F.nr, 256), 256, 0, ctx->st>>>(F.nr, F.br, F.nr, 1, F.rlu, F.rrdiag, F.rucs);
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
    solve_parts(F.n, F.b, F.s, 1, F.lm, F.ipiv, F.ucs, F.rdiag, t, x, nullptr, ctx->st);
  } else {
    solve_parts(F.n, F.b, F.s, F.P, F.lm, F.ipiv, F.ucs, F.rdiag, t, F.y, F.P > 1 ? F.rz : nullptr, ctx->st);
    if (F.P > 1) {
      solve_parts(F.nr, F.br, F.nr, 1, F.rlm, F.ripiv, F.rucs, F.rrdiag, F.rz, F.rz2, nullptr, ctx->st);
      k_band_update<<<cdiv(F.n, 256), 256, 0, ctx->st>>>(F.n, F.b, F.s, F.P, F.V, F.Wl, F.rz2, F.y, x);
      iga_count_launch();
    } else {
      CK(cudaMemcpyAsync(x, F.y, sizeof(double2) * F.n, cudaMemcpyDeviceToDevice, ctx->st));
    }
  }
  CKL();
  return IGA_OK;
}
