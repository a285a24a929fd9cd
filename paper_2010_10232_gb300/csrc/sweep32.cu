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
//  - the complex-by-real taps use packed FP32 pair FMAs (fma.rn.f32x2) on
//    operands kept packed in 64-bit registers: one instruction applies two
//    real coefficients to one input, (M_y, K_y) to Re x in the first pass and
//    (K_x, M_x) to (Re u, Re w) in the second;
//  - the right-hand side is fetched together with the x tile (one round of
//    global latency per block), every thread loading one tile column with
//    pointer increments; the epilogue runs one warp per output row with
//    predicated stores.
// Tile: 64 - 2p columns x 32 rows of outputs per 256-thread block (three
// blocks per SM); the x tile with its p-wide halo is exactly 64 columns wide.
// (Measured on GB300 against a persistent, cp.async double-buffered form with
// one 512-thread block per SM: that form issued fewer instructions but ran
// slower, with half the warps per SM and more barrier stalls.)
#include "common.cuh"

namespace {

constexpr int SW_SX = 64, SW_TY = 32, SW_NT = 256, SW_OUT = 8;
typedef unsigned long long u64;

// two floats packed in one 64-bit register (lo in the low half)
__device__ __forceinline__ u64 pk2(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk2(u64 r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
// (a.lo * b.lo + c.lo, a.hi * b.hi + c.hi), each correctly rounded once
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
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
  static constexpr int NE = 2 * SW_TY / (SW_NT / 32);   // epilogue slots per thread: rows x 2 column halves
  static constexpr size_t xs_bytes = sizeof(float2) * SY * SW_SX;
  static constexpr size_t uw_bytes = sizeof(float4) * SW_TY * RSU;
  static constexpr size_t cf_bytes = sizeof(float2) * (SW_TY + SW_SX) * W + sizeof(float2) * (SW_TY + SW_SX);
  static constexpr size_t smem = xs_bytes + uw_bytes + cf_bytes;
  static_assert(3 * (smem + 1024) <= 233472, "three blocks per SM");
};

}  // namespace

// The level's interior stencil (band row at least 2p from either end), passed
// by value so that it comes from the constant bank, not from global memory.
struct SwStencil {
  float k[2 * IGA_MAXP + 1], m[2 * IGA_MAXP + 1];
  int valid;       // the level has interior rows (n_x > 4p + 1)
};

// First pass for 8 output rows of one x-tile column (sliding window down the
// column): EDGE takes the (M, K) band pair of every output row from the tile
// table cy, otherwise the interior stencil creg.
template <int P, bool EDGE>
__device__ __forceinline__ void sweep_ypass(const float2* xs, float4* uw, const u64* cy, const u64* creg, float2 cm,
                                            int tid) {
  using G = SwGeom<P>;
  constexpr int W = G::W, RSU = G::RSU, SX = SW_SX;
  const int c = tid & 63, r0 = (tid >> 6) * SW_OUT;
  u64 aR[SW_OUT], aI[SW_OUT];   // (Re s1, Re s2), (Im s1, Im s2)
#pragma unroll
  for (int j = 0; j < SW_OUT; ++j) aR[j] = aI[j] = 0ull;
#pragma unroll
  for (int q = 0; q < SW_OUT + 2 * P; ++q) {
    const float2 v = xs[(r0 + q) * SX + c];
    const u64 vr = pk2(v.x, v.x), vi = pk2(v.y, v.y);
#pragma unroll
    for (int d = 0; d < W; ++d) {
      const int j = q - d;
      if (j >= 0 && j < SW_OUT) {
        u64 cf;
        if constexpr (EDGE) cf = cy[(r0 + j) * W + d];
        else cf = creg[d];
        aR[j] = ffma2(cf, vr, aR[j]);
        aI[j] = ffma2(cf, vi, aI[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < SW_OUT; ++j) {
    const float2 re = upk2(aR[j]), im = upk2(aI[j]);   // (s1, s2) real and imaginary parts
    const float wr = fmaf(cm.x, re.x, fmaf(-cm.y, im.x, re.y));
    const float wi = fmaf(cm.x, im.x, fmaf(cm.y, re.x, im.y));
    uw[(r0 + j) * RSU + swpos(c)] = make_float4(re.x, wr, im.x, wi);
  }
}

// Second pass for 8 consecutive outputs of one tile row (sliding window along
// the row): (K, M) band pairs per output column from cx (EDGE) or creg.
// The (u, w) element (Re u, Re w, Im u, Im w) is read as two packed pairs.
template <int P, bool EDGE>
__device__ __forceinline__ void sweep_xpass(const float4* uw, const u64* cx, const u64* creg, int tid, float2* res) {
  using G = SwGeom<P>;
  constexpr int W = G::W, RSU = G::RSU, SX = SW_SX;
  const int rr = tid >> 3, s0 = (tid & 7) * SW_OUT;
  const ulonglong2* uwp = reinterpret_cast<const ulonglong2*>(uw) + rr * RSU;
  u64 aR[SW_OUT], aI[SW_OUT];   // (K Re u, M Re w), (K Im u, M Im w)
#pragma unroll
  for (int t = 0; t < SW_OUT; ++t) aR[t] = aI[t] = 0ull;
#pragma unroll
  for (int q = 0; q < SW_OUT + 2 * P; ++q) {
    const ulonglong2 e = uwp[swpos(s0 + q)];
#pragma unroll
    for (int d = 0; d < W; ++d) {
      const int t = q - d;
      if (t >= 0 && t < SW_OUT) {
        u64 cf;
        if constexpr (EDGE) cf = cx[min(s0 + t, SX - 1) * W + d];
        else cf = creg[d];
        aR[t] = ffma2(cf, e.x, aR[t]);
        aI[t] = ffma2(cf, e.y, aI[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < SW_OUT; ++t) {
    const float2 re = upk2(aR[t]), im = upk2(aI[t]);
    res[t] = make_float2(re.x + re.y, im.x + im.y);
  }
}

// K, M: FP32 bands [nx][2p+1] of the level; cm: mass coefficient; EPI as in
// operator.cu (z: minuend for EPI_ZMINUS, right-hand side b for EPI_JACOBI).
// x, y and z are distinct vectors.
template <int P, int EPI>
__global__ void __launch_bounds__(SW_NT, 3) k_sweep32(int nx, int ny, const float* __restrict__ K,
                                                      const float* __restrict__ M, float2 cm,
                                                      const float2* __restrict__ x, float2* __restrict__ y,
                                                      const float2* __restrict__ z, float omega,
                                                      double2* __restrict__ y64, const SwStencil stn) {
  using G = SwGeom<P>;
  constexpr int W = G::W, TX = G::TX, SY = G::SY, RSU = G::RSU, TY = SW_TY, SX = SW_SX, NE = G::NE;
  constexpr int RSTEP = SW_NT / 64;                   // tile rows loaded per round (one thread per column)
  extern __shared__ __align__(16) unsigned char sw_smem[];
  float2* xs = reinterpret_cast<float2*>(sw_smem);                            // [SY][SX]
  float4* uw = reinterpret_cast<float4*>(sw_smem + G::xs_bytes);              // [TY][RSU] (Re u, Re w, Im u, Im w)
  float2* ys = reinterpret_cast<float2*>(uw);                                 // [TY][2 RSU] after the second pass
  u64* cy = reinterpret_cast<u64*>(sw_smem + G::xs_bytes + G::uw_bytes);      // [TY][W] (M_y, K_y) per tile row
  u64* cx = cy + TY * W;                                                      // [SX][W] (K_x, M_x) per output column
  float2* dy = reinterpret_cast<float2*>(cx + SX * W);                        // [TY] (M, K) diagonals
  float2* dx = dy + TY;                                                       // [SX] (K, M) diagonals

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  // interior stencil rows: at least 2p from either end (uniform B-splines only)
  const bool inner_ok = stn.valid && nx > 4 * P + 1 && ny > 4 * P + 1;
  const bool yedge = !inner_ok || y0 < 2 * P || y0 + TY - 1 > ny - 1 - 2 * P;
  const bool xedge = !inner_ok || x0 < 2 * P || x0 + TX - 1 > nx - 1 - 2 * P;

  // ---- right-hand side of the epilogue (slot k: row warp + 8 (k / 2),
  // column lane + 32 (k % 2)), fetched together with the x tile
  float2 zv[NE];
  if (EPI != EPI_Y) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h, gx = x0 + c;
      const bool colok = c < TX && gx < nx;
      int gy = y0 + warp;
      const float2* src = z + (ptrdiff_t)gy * nx + gx;
#pragma unroll
      for (int k = 0; k < NE / 2; ++k) {
        zv[2 * k + h] = (colok && gy < ny) ? *src : make_float2(0.f, 0.f);
        gy += SW_NT / 32;
        src += (ptrdiff_t)(SW_NT / 32) * nx;
      }
    }
  }
  // ---- x tile with halo (zero outside the grid): one column per thread, all
  // loads issued before the stores
  {
    constexpr int IT = (SY + RSTEP - 1) / RSTEP;
    const int c = tid & 63, r0 = tid >> 6;
    const int gx = x0 - P + c;
    const bool colok = gx >= 0 && gx < nx;
    int gy = y0 - P + r0;
    const float2* src = x + (ptrdiff_t)gy * nx + gx;
    float2 v[IT];
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      v[k] = (colok && gy >= 0 && gy < ny && r0 + RSTEP * k < SY) ? *src : make_float2(0.f, 0.f);
      gy += RSTEP;
      src += (ptrdiff_t)RSTEP * nx;
    }
#pragma unroll
    for (int k = 0; k < IT; ++k)
      if (r0 + RSTEP * k < SY) xs[(r0 + RSTEP * k) * SX + c] = v[k];
  }
  if (yedge) {
    for (int i = tid; i < TY * W; i += SW_NT) {
      const int r = i / W, d = i - r * W, gy = y0 + r;
      cy[i] = gy < ny ? pk2(M[(size_t)gy * W + d], K[(size_t)gy * W + d]) : 0ull;
    }
  }
  if (xedge) {
    for (int i = tid; i < SX * W; i += SW_NT) {
      const int j = i / W, d = i - j * W, gx = x0 + j;
      cx[i] = gx < nx ? pk2(K[(size_t)gx * W + d], M[(size_t)gx * W + d]) : 0ull;
    }
  }
  constexpr bool JAC = EPI == EPI_JACOBI || EPI == EPI_JACOBI_OUT64;
  if (JAC && (yedge || xedge)) {
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
  {
    u64 creg[W];
    if (!yedge) {
#pragma unroll
      for (int d = 0; d < W; ++d) creg[d] = pk2(stn.m[d], stn.k[d]);
      sweep_ypass<P, false>(xs, uw, cy, creg, cm, tid);
    } else {
      sweep_ypass<P, true>(xs, uw, cy, creg, cm, tid);
    }
  }
  __syncthreads();

  // ---- pass along x: Op x = K_x u + M_x w
  float2 res[SW_OUT];
  const int rr = tid >> 3, s0 = (tid & 7) * SW_OUT;
  {
    u64 creg[W];
    if (!xedge) {
#pragma unroll
      for (int d = 0; d < W; ++d) creg[d] = pk2(stn.k[d], stn.m[d]);
      sweep_xpass<P, false>(uw, cx, creg, tid, res);
    } else {
      sweep_xpass<P, true>(uw, cx, creg, tid, res);
    }
  }
  __syncthreads();   // every thread is done reading (u, w): the results go to the same space
#pragma unroll
  for (int q = 0; q < SW_OUT; ++q)
    if (s0 + q < TX) ys[rr * (2 * RSU) + swpos(s0 + q)] = res[q];
  __syncthreads();

  // ---- epilogue: one warp per output row, consecutive lanes on consecutive
  // columns; every slot computes (shared-memory reads stay inside the tile
  // buffers), only the store is predicated
  float2 dint = make_float2(0.f, 0.f);
  if (JAC && !(yedge || xedge)) {
    const float kd = stn.k[P], md = stn.m[P];
    const float2 diag = md * (make_float2(kd, 0.f) + md * cm) + make_float2(kd * md, 0.f);
    dint = cinv(diag);
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = lane + 32 * h, gx = x0 + c;
    const int cc = min(c, TX - 1);
    const bool colok = c < TX && gx < nx;
    int gy = y0 + warp;
    float2* dst = y + (ptrdiff_t)gy * nx + gx;
    double2* dst64 = y64 + (ptrdiff_t)gy * nx + gx;
#pragma unroll
    for (int k = 0; k < NE / 2; ++k) {
      const int r = warp + (SW_NT / 32) * k;
      const float2 acc = ys[r * (2 * RSU) + swpos(cc)];
      float2 out;
      if (EPI == EPI_Y) {
        out = acc;
      } else if (EPI == EPI_ZMINUS) {
        out = zv[2 * k + h] - acc;
      } else {
        float2 di = dint;
        if (yedge || xedge) {
          const float2 dyr = dy[r], dxc = dx[cc];
          const float2 diag = dyr.x * (make_float2(dxc.x, 0.f) + dxc.y * cm) + make_float2(dyr.y * dxc.y, 0.f);
          di = cinv(diag);
        }
        const float2 xo = xs[(r + P) * SX + cc + P];
        out = xo + omega * cmul(di, zv[2 * k + h] - acc);
      }
      if (colok && gy < ny) {
        if (EPI == EPI_JACOBI_OUT64) *dst64 = tod(out);
        else *dst = out;
      }
      gy += SW_NT / 32;
      dst += (ptrdiff_t)(SW_NT / 32) * nx;
      dst64 += (ptrdiff_t)(SW_NT / 32) * nx;
    }
  }
}

template <int P, int EPI>
static void launch_sweep(int nx, int ny, const float* K, const float* M, float2 cm, const float2* x, float2* y,
                         const float2* z, float omega, double2* y64, const SwStencil& stn, cudaStream_t st) {
  using G = SwGeom<P>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sweep32<P, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
    // the largest shared-memory carveout, so that three blocks fit on an SM
    cudaFuncSetAttribute(k_sweep32<P, EPI>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = true;
  }
  dim3 grid(cdiv(nx, G::TX), cdiv(ny, SW_TY));
  k_sweep32<P, EPI><<<grid, SW_NT, G::smem, st>>>(nx, ny, K, M, cm, x, y, z, omega, y64, stn);
  iga_count_launch();
}

template <int P>
static void launch_sweep_epi(int epi, int nx, int ny, const float* K, const float* M, float2 cm, const float2* x,
                             float2* y, const float2* z, float omega, double2* y64, const SwStencil& stn, cudaStream_t st) {
  if (epi == EPI_Y) launch_sweep<P, EPI_Y>(nx, ny, K, M, cm, x, y, z, omega, y64, stn, st);
  else if (epi == EPI_ZMINUS) launch_sweep<P, EPI_ZMINUS>(nx, ny, K, M, cm, x, y, z, omega, y64, stn, st);
  else if (epi == EPI_JACOBI) launch_sweep<P, EPI_JACOBI>(nx, ny, K, M, cm, x, y, z, omega, y64, stn, st);
  else launch_sweep<P, EPI_JACOBI_OUT64>(nx, ny, K, M, cm, x, y, z, omega, y64, stn, st);
}

static void sweep_dispatch(int p, int epi, int nx, int ny, const float* K, const float* M, float2 cm,
                           const float2* x, float2* y, const float2* z, float omega, double2* y64, const SwStencil& stn, cudaStream_t st) {
  switch (p) {
    case 1: launch_sweep_epi<1>(epi, nx, ny, K, M, cm, x, y, z, omega, y64, stn, st); break;
    case 2: launch_sweep_epi<2>(epi, nx, ny, K, M, cm, x, y, z, omega, y64, stn, st); break;
    case 3: launch_sweep_epi<3>(epi, nx, ny, K, M, cm, x, y, z, omega, y64, stn, st); break;
    case 4: launch_sweep_epi<4>(epi, nx, ny, K, M, cm, x, y, z, omega, y64, stn, st); break;
    default: launch_sweep_epi<5>(epi, nx, ny, K, M, cm, x, y, z, omega, y64, stn, st); break;
  }
}

static SwStencil level_stencil(const LevelData& L, int p) {
  SwStencil s{};
  for (int d = 0; d < 2 * p + 1; ++d) {
    s.k[d] = L.sK[d];
    s.m[d] = L.sM[d];
  }
  s.valid = L.has_stencil ? 1 : 0;
  return s;
}

// operator.cu: tile code 6 of the FP32 constant-k operator
void sweep32_launch(const LevelData& L, int p, int epi, const float2* x, float2* y, const float2* z, float2 cm,
                    float omega, cudaStream_t st) {
  sweep_dispatch(p, epi, L.nx, L.ny, L.Kf, L.Mf, cm, x, y, z, omega, nullptr, level_stencil(L, p), st);
}

iga_status sweep32_jacobi_out64(iga_ctx* ctx, int level, const float2* x, double2* y64, const float2* b) {
  const LevelData& L = ctx->lv[level];
  double2 c = make_double2(-ctx->sig.x * ctx->k2const, -ctx->sig.y * ctx->k2const);   // M_beta mass coefficient
  sweep_dispatch(ctx->p, EPI_JACOBI_OUT64, L.nx, L.ny, L.Kf, L.Mf, tof(c), x, nullptr, b, (float)ctx->prm.omega, y64,
                 level_stencil(L, ctx->p), ctx->st);
  CKL();
  return IGA_OK;
}
