// FP32 constant-k 2D operator sweep for large multigrid levels (the CSLP
// V-cycle of Section 3 in single precision): y = Op x, y = z - Op x, or one
// damped Jacobi sweep x_out = x + omega D^{-1} (b - Op x), with
// Op = M_y (x) (K_x + c M_x) + K_y (x) M_x as in operator.cu.
//
// Designed to be bound by HBM rather than by instruction issue:
//  - interior tiles take the banded stencils from registers: with uniform
//    knots every band row at least 2p rows from either end is the same
//    stencil, so only tiles touching those edge rows read per-row
//    coefficients;
//  - both banded passes run as sliding windows (every input value is read
//    from shared memory once per thread and scattered into the outputs that
//    use it);
//  - the complex-by-real taps use packed FP32 pair FMAs (fma.rn.f32x2): one
//    instruction applies two real coefficients to one input, e.g. (M_y, K_y)
//    to Re x in the first pass and (K_x, M_x) to (Re u, Re w) in the second;
//  - the epilogue reads the right-hand side and writes the result with
//    consecutive threads on consecutive columns.
// Tile: 64 - 2p columns x 32 rows of outputs per 256-thread block; the x tile
// with its p-wide halo is exactly 64 columns wide.
#include "common.cuh"

namespace {

constexpr int SW_SX = 64, SW_TY = 32, SW_NT = 256, SW_OUT = 8;

__device__ __forceinline__ unsigned long long pk2(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
// (a.x * b.x + c.x, a.y * b.y + c.y), each correctly rounded once
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(d);
}

// padded column position: one spare slot every 8 columns, so the 8 threads
// of a quarter-warp that read 16-byte elements 8 columns apart hit 8
// different bank groups
__device__ __forceinline__ int swpos(int c) { return c + (c >> 3); }

template <int P> struct SwGeom {
  static constexpr int W = 2 * P + 1;
  static constexpr int TX = SW_SX - 2 * P;          // output columns per tile
  static constexpr int SY = SW_TY + 2 * P;          // x-tile rows
  static constexpr int UWC = SW_SX + 2 * P;         // (u, w) columns read by the second pass
  static constexpr int RSU = UWC + (UWC >> 3) + 1;  // padded (u, w) row length, 16-byte elements
  static constexpr size_t xs_bytes = sizeof(float2) * SY * SW_SX;
  static constexpr size_t uw_bytes = sizeof(float4) * SW_TY * RSU;
  static constexpr size_t cf_bytes = sizeof(float2) * (SW_TY + SW_SX) * W + sizeof(float2) * (SW_TY + SW_SX);
  static constexpr size_t smem = xs_bytes + uw_bytes + cf_bytes;
};

}  // namespace

template <int P> size_t sweep32_smem() { return SwGeom<P>::smem; }

// First pass for 8 output rows of one x-tile column (sliding window down the
// column): EDGE takes the (M, K) band pair of every output row from the tile
// table cy, otherwise the interior stencil of band row ci from registers.
template <int P, bool EDGE>
__device__ __forceinline__ void sweep_ypass(const float2* xs, float4* uw, const float2* cy, const float* K,
                                            const float* M, int ci, float2 cm, int tid) {
  using G = SwGeom<P>;
  constexpr int W = G::W, RSU = G::RSU, SX = SW_SX;
  const int c = tid & 63, r0 = (tid >> 6) * SW_OUT;
  float2 creg[W];
  if constexpr (!EDGE) {
#pragma unroll
    for (int d = 0; d < W; ++d) creg[d] = make_float2(M[(size_t)ci * W + d], K[(size_t)ci * W + d]);
  }
  float2 aR[SW_OUT], aI[SW_OUT];   // (Re s1, Re s2), (Im s1, Im s2)
#pragma unroll
  for (int j = 0; j < SW_OUT; ++j) aR[j] = aI[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < SW_OUT + 2 * P; ++q) {
    const float2 v = xs[(r0 + q) * SX + c];
    const float2 vr = make_float2(v.x, v.x), vi = make_float2(v.y, v.y);
#pragma unroll
    for (int d = 0; d < W; ++d) {
      const int j = q - d;
      if (j >= 0 && j < SW_OUT) {
        float2 cf;
        if constexpr (EDGE) cf = cy[(r0 + j) * W + d];
        else cf = creg[d];
        aR[j] = ffma2(cf, vr, aR[j]);
        aI[j] = ffma2(cf, vi, aI[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < SW_OUT; ++j) {
    const float s1r = aR[j].x, s1i = aI[j].x;
    const float wr = fmaf(cm.x, s1r, fmaf(-cm.y, s1i, aR[j].y));
    const float wi = fmaf(cm.x, s1i, fmaf(cm.y, s1r, aI[j].y));
    uw[(r0 + j) * RSU + swpos(c)] = make_float4(s1r, wr, s1i, wi);
  }
}

// Second pass for 8 consecutive outputs of one tile row (sliding window along
// the row): (K, M) band pairs per output column from cx (EDGE) or registers.
template <int P, bool EDGE>
__device__ __forceinline__ void sweep_xpass(const float4* uw, const float2* cx, const float* K, const float* M, int ci,
                                            int tid, float2* res) {
  using G = SwGeom<P>;
  constexpr int W = G::W, RSU = G::RSU, SX = SW_SX;
  const int rr = tid >> 3, s0 = (tid & 7) * SW_OUT;
  float2 creg[W];
  if constexpr (!EDGE) {
#pragma unroll
    for (int d = 0; d < W; ++d) creg[d] = make_float2(K[(size_t)ci * W + d], M[(size_t)ci * W + d]);
  }
  float2 aR[SW_OUT], aI[SW_OUT];   // (K Re u, M Re w), (K Im u, M Im w)
#pragma unroll
  for (int t = 0; t < SW_OUT; ++t) aR[t] = aI[t] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < SW_OUT + 2 * P; ++q) {
    const float4 e = uw[rr * RSU + swpos(s0 + q)];
    const float2 pr = make_float2(e.x, e.y), pi = make_float2(e.z, e.w);
#pragma unroll
    for (int d = 0; d < W; ++d) {
      const int t = q - d;
      if (t >= 0 && t < SW_OUT) {
        float2 cf;
        if constexpr (EDGE) cf = cx[min(s0 + t, SX - 1) * W + d];
        else cf = creg[d];
        aR[t] = ffma2(cf, pr, aR[t]);
        aI[t] = ffma2(cf, pi, aI[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < SW_OUT; ++t) res[t] = make_float2(aR[t].x + aR[t].y, aI[t].x + aI[t].y);
}

// a: operator arguments as in operator.cu (FP32 bands of the level); EPI as there.
template <int P, int EPI>
__global__ void __launch_bounds__(SW_NT) k_sweep32(int nx, int ny, const float* __restrict__ K,
                                                   const float* __restrict__ M, float2 cm,
                                                   const float2* __restrict__ x, float2* y, const float2* z,
                                                   float omega) {
  using G = SwGeom<P>;
  constexpr int W = G::W, TX = G::TX, SY = G::SY, RSU = G::RSU, TY = SW_TY, SX = SW_SX;
  extern __shared__ __align__(16) unsigned char sw_smem[];
  float2* xs = reinterpret_cast<float2*>(sw_smem);                            // [SY][SX]
  float4* uw = reinterpret_cast<float4*>(sw_smem + G::xs_bytes);              // [TY][RSU] (Re u, Re w, Im u, Im w)
  float2* ys = reinterpret_cast<float2*>(uw);                                 // [TY][RSU] after the second pass
  float2* cy = reinterpret_cast<float2*>(sw_smem + G::xs_bytes + G::uw_bytes);   // [TY][W] (M_y, K_y) per tile row
  float2* cx = cy + TY * W;                                                   // [SX][W] (K_x, M_x) per output column
  float2* dy = cx + SX * W;                                                   // [TY] (M, K) diagonals
  float2* dx = dy + TY;                                                       // [SX] (K, M) diagonals

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  // interior stencil rows: at least 2p from either end (uniform B-splines only)
  const bool inner_ok = nx > 4 * P + 1 && ny > 4 * P + 1;
  const bool yedge = !inner_ok || y0 < 2 * P || y0 + TY - 1 > ny - 1 - 2 * P;
  const bool xedge = !inner_ok || x0 < 2 * P || x0 + TX - 1 > nx - 1 - 2 * P;

  // ---- right-hand side of the epilogue (prefetched with the x tile: one
  // round of global latency per block)
  constexpr int NE = (TY * TX + SW_NT - 1) / SW_NT;
  float2 zv[NE];
  if (EPI != EPI_Y) {
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      const int i = tid + k * SW_NT, r = i / TX, c = i - r * TX;
      const int gy = y0 + r, gx = x0 + c;
      zv[k] = (i < TY * TX && gy < ny && gx < nx) ? z[(size_t)gy * nx + gx] : make_float2(0.f, 0.f);
    }
  }
  // ---- x tile with halo (zero outside the grid), all loads issued first
  {
    constexpr int TOT = SY * SX, IT = (TOT + SW_NT - 1) / SW_NT;
    float2 v[IT];
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int i = tid + k * SW_NT;
      const int r = i >> 6, c = i & 63;
      const int gy = y0 - P + r, gx = x0 - P + c;
      v[k] = (i < TOT && gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? x[(size_t)gy * nx + gx] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int i = tid + k * SW_NT;
      if (i < TOT) xs[i] = v[k];
    }
  }
  if (yedge) {
    for (int i = tid; i < TY * W; i += SW_NT) {
      const int r = i / W, d = i - r * W, gy = y0 + r;
      cy[i] = gy < ny ? make_float2(M[(size_t)gy * W + d], K[(size_t)gy * W + d]) : make_float2(0.f, 0.f);
    }
  }
  if (xedge) {
    for (int i = tid; i < SX * W; i += SW_NT) {
      const int j = i / W, d = i - j * W, gx = x0 + j;
      cx[i] = gx < nx ? make_float2(K[(size_t)gx * W + d], M[(size_t)gx * W + d]) : make_float2(0.f, 0.f);
    }
  }
  if (EPI == EPI_JACOBI && (yedge || xedge)) {
    if (tid < TY) {
      const int gy = min(y0 + tid, ny - 1);
      dy[tid] = make_float2(M[(size_t)gy * W + P], K[(size_t)gy * W + P]);
    } else if (tid < TY + SX) {
      const int gx = min(x0 + tid - TY, nx - 1);
      dx[tid - TY] = make_float2(K[(size_t)gx * W + P], M[(size_t)gx * W + P]);
    }
  }
  __syncthreads();

  // ---- pass along y: (s1, s2) = (M_y x, K_y x); u = s1, w = c s1 + s2
  if (yedge) sweep_ypass<P, true>(xs, uw, cy, nullptr, nullptr, 0, cm, tid);
  else sweep_ypass<P, false>(xs, uw, cy, K, M, ny >> 1, cm, tid);
  __syncthreads();

  // ---- pass along x: Op x = K_x u + M_x w
  float2 res[SW_OUT];
  const int rr = tid >> 3, s0 = (tid & 7) * SW_OUT;
  if (xedge) sweep_xpass<P, true>(uw, cx, nullptr, nullptr, 0, tid, res);
  else sweep_xpass<P, false>(uw, cx, K, M, nx >> 1, tid, res);
  __syncthreads();   // every thread is done reading (u, w): the results go to the same space
#pragma unroll
  for (int t = 0; t < SW_OUT; ++t)
    if (s0 + t < TX) ys[rr * (2 * RSU) + swpos(s0 + t)] = res[t];
  __syncthreads();

  // ---- epilogue: consecutive threads on consecutive columns
  float2 dint = make_float2(0.f, 0.f);
  if (EPI == EPI_JACOBI && !(yedge || xedge)) {
    const int ci = nx >> 1;
    const float kd = K[(size_t)ci * W + P], md = M[(size_t)ci * W + P];
    const float2 diag = md * (make_float2(kd, 0.f) + md * cm) + make_float2(kd * md, 0.f);
    dint = cinv(diag);
  }
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    const int i = tid + k * SW_NT, r = i / TX, c = i - r * TX;
    const int gy = y0 + r, gx = x0 + c;
    if (i >= TY * TX || gy >= ny || gx >= nx) continue;
    const size_t o = (size_t)gy * nx + gx;
    const float2 acc = ys[r * (2 * RSU) + swpos(c)];
    if (EPI == EPI_Y) {
      y[o] = acc;
    } else if (EPI == EPI_ZMINUS) {
      y[o] = zv[k] - acc;
    } else {
      float2 di = dint;
      if (yedge || xedge) {
        const float2 dyr = dy[r], dxc = dx[c];
        const float2 diag = dyr.x * (make_float2(dxc.x, 0.f) + dxc.y * cm) + make_float2(dyr.y * dxc.y, 0.f);
        di = cinv(diag);
      }
      const float2 xo = xs[(r + P) * SX + c + P];
      y[o] = xo + omega * cmul(di, zv[k] - acc);
    }
  }
}

template <int P, int EPI>
static void launch_sweep(int nx, int ny, const float* K, const float* M, float2 cm, const float2* x, float2* y,
                         const float2* z, float omega, cudaStream_t st) {
  using G = SwGeom<P>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sweep32<P, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
    attr = true;
  }
  dim3 grid(cdiv(nx, G::TX), cdiv(ny, SW_TY));
  k_sweep32<P, EPI><<<grid, SW_NT, G::smem, st>>>(nx, ny, K, M, cm, x, y, z, omega);
  iga_count_launch();
}

template <int P>
static void launch_sweep_epi(int epi, int nx, int ny, const float* K, const float* M, float2 cm, const float2* x,
                             float2* y, const float2* z, float omega, cudaStream_t st) {
  if (epi == EPI_Y) launch_sweep<P, EPI_Y>(nx, ny, K, M, cm, x, y, z, omega, st);
  else if (epi == EPI_ZMINUS) launch_sweep<P, EPI_ZMINUS>(nx, ny, K, M, cm, x, y, z, omega, st);
  else launch_sweep<P, EPI_JACOBI>(nx, ny, K, M, cm, x, y, z, omega, st);
}

// dispatch by degree (operator.cu: tile code 6 of the FP32 constant-k operator)
void sweep32_launch(int p, int epi, int nx, int ny, const float* K, const float* M, float2 cm, const float2* x,
                    float2* y, const float2* z, float omega, cudaStream_t st) {
  switch (p) {
    case 1: launch_sweep_epi<1>(epi, nx, ny, K, M, cm, x, y, z, omega, st); break;
    case 2: launch_sweep_epi<2>(epi, nx, ny, K, M, cm, x, y, z, omega, st); break;
    case 3: launch_sweep_epi<3>(epi, nx, ny, K, M, cm, x, y, z, omega, st); break;
    case 4: launch_sweep_epi<4>(epi, nx, ny, K, M, cm, x, y, z, omega, st); break;
    default: launch_sweep_epi<5>(epi, nx, ny, K, M, cm, x, y, z, omega, st); break;
  }
}
