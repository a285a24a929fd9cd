// Fused V-cycle levels for the 2D constant-k CSLP with one pre- and one
// post-smoothing sweep (Section 3: damped Jacobi, omega = 0.6; Section 4.2:
// V-cycle between nested spline spaces, transfers by knot insertion).
//
// The pre-smoothing sweep starts from zero, so it is pointwise:
// x = omega D^{-1} b.  It is never stored: both kernels of a level recompute
// it from b on the tile (plus halo) they need.  A level then takes two
// launches instead of five, and reads b twice instead of moving five vectors:
//   down(l): c_{l+1} = R_l (b_l - M_l x)                       (residual + restriction)
//   up(l):   x <- x + P_l xc_{l+1};  x_out = x + omega D^{-1} (b_l - M_l x)
// V-cycle = down(0 .. L-2), dense solve on the coarsest level, up(L-2 .. 0).
// Mathematically identical to the per-operation sequence in mg.cu (the sums
// are taken in the same order); rounding differs only by where values are
// kept (shared memory instead of global vectors).
#include "common.cuh"

template <typename T> struct FusedArgs {
  using C = typename cplx<T>::t;
  int nxf, nyf, nxc, nyc;     // this level (fine) and the next coarser one
  const T* K;                 // fine 1D bands [nxf][2p+1] (the same in x and y)
  const T* M;
  C c;                        // mass coefficient of M_beta
  const C* dinv;              // fine D^{-1} (FP64 levels) or nullptr (formed from the bands)
  T omega;
  const C* b;                 // fine right-hand side
  // down
  const T* Rw; const int* Rlo; int wR;
  C* cout;                    // coarse right-hand side
  int fmax;                   // largest fine footprint of a coarse tile (per direction)
  // up
  const T* Pw; const int* Plo; int wP;
  const C* xc;                // coarse correction
  C* xout;                    // fine result
  int cmax;                   // largest coarse patch of a fine tile (per direction)
};

// 1/D for D = m_y (k_x + c m_x) + k_y m_x (the diagonal of M_beta, the same
// expression as the Jacobi epilogue of the operator kernels).  FP32: one
// correctly rounded reciprocal of |D|^2; FP64: the quotient.
template <typename T>
__device__ __forceinline__ typename cplx<T>::t diag_inv_of(T kx, T mx, T ky, T my, typename cplx<T>::t c) {
  using C = typename cplx<T>::t;
  C d = my * (mkc(kx, (T)0) + mx * c) + mkc(ky * mx, (T)0);
  if constexpr (sizeof(T) == 4) {
    float m = __frcp_rn(d.x * d.x + d.y * d.y);
    return make_float2(d.x * m, -d.y * m);
  } else {
    return cinv(d);
  }
}

// Thread layout of both kernels: 8 warps; a warp walks rows, its lanes walk
// columns, so global rows are read and written coalesced and each lane keeps
// the band coefficients of its column in registers.
constexpr int VC_NW = 8;

// coarse tile of the down kernel: its fine footprint 2 (CT - 1) + (p + 3) is
// at most one warp wide in the interior
__host__ __device__ constexpr int down_ct(int P) { return (32 - (P + 3)) / 2 + 1; }

template <typename C, typename T>
__host__ __device__ inline size_t down_smem(int P, int fmax) {
  const int W = 2 * P + 1, H = fmax + 2 * P, CT = down_ct(P), WR = P + 3;
  return sizeof(C) * ((size_t)H * H + 2 * (size_t)H * fmax) +
         sizeof(T) * (4 * (size_t)fmax * W + 4 * (size_t)H + 2 * (size_t)CT * WR) + sizeof(int) * 2 * CT;
}

template <int P, typename T>
__global__ void __launch_bounds__(256) k_vc_down(FusedArgs<T> a) {
  using C = typename cplx<T>::t;
  constexpr int W = 2 * P + 1, CT = down_ct(P), WR = P + 3;
  extern __shared__ __align__(16) unsigned char vsm[];
  const int fm = a.fmax, H = fm + 2 * P;
  C* xs = reinterpret_cast<C*>(vsm);            // [H][H] x on the halo tile; later the residual [FY][fm]
  C* us = xs + (size_t)H * H;                   // [H][fm] x-pass; later the x-restricted rows [FY][cxn]
  C* ts = us + (size_t)H * fm;
  T* kxs = reinterpret_cast<T*>(ts + (size_t)H * fm);   // bands of the footprint columns / rows
  T* mxs = kxs + fm * W;
  T* kys = mxs + fm * W;
  T* mys = kys + fm * W;
  T* kdx = mys + fm * W;                        // diagonal entries of the halo columns / rows
  T* mdx = kdx + H;
  T* kdy = mdx + H;
  T* mdy = kdy + H;
  T* Rwx = mdy + H;                             // [CT][WR]
  T* Rwy = Rwx + CT * WR;
  int* Rlox = reinterpret_cast<int*>(Rwy + CT * WR);   // window starts relative to the footprint
  int* Rloy = Rlox + CT;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int nxf = a.nxf, nyf = a.nyf, nxc = a.nxc;
  const int cx0 = blockIdx.x * CT, cy0 = blockIdx.y * CT;
  const int cxn = min(CT, nxc - cx0), cyn = min(CT, a.nyc - cy0);
  const int fx0 = max(0, a.Rlo[cx0]), fx1 = min(nxf, a.Rlo[cx0 + cxn - 1] + WR);
  const int fy0 = max(0, a.Rlo[cy0]), fy1 = min(nyf, a.Rlo[cy0 + cyn - 1] + WR);
  const int FX = fx1 - fx0, FY = fy1 - fy0, HX = FX + 2 * P, HY = FY + 2 * P;
  if (FX > fm || FY > fm || FX < 1 || FY < 1) return;     // cannot happen: fmax is the maximum over tiles
  for (int i = tid; i < FX * W; i += 256) {
    kxs[i] = a.K[(size_t)fx0 * W + i];
    mxs[i] = a.M[(size_t)fx0 * W + i];
  }
  for (int i = tid; i < FY * W; i += 256) {
    kys[i] = a.K[(size_t)fy0 * W + i];
    mys[i] = a.M[(size_t)fy0 * W + i];
  }
  for (int i = tid; i < HX; i += 256) {
    int g = fx0 - P + i;
    bool in = g >= 0 && g < nxf;
    kdx[i] = in ? a.K[(size_t)g * W + P] : (T)0;
    mdx[i] = in ? a.M[(size_t)g * W + P] : (T)0;
  }
  for (int i = tid; i < HY; i += 256) {
    int g = fy0 - P + i;
    bool in = g >= 0 && g < nyf;
    kdy[i] = in ? a.K[(size_t)g * W + P] : (T)0;
    mdy[i] = in ? a.M[(size_t)g * W + P] : (T)0;
  }
  for (int i = tid; i < cxn * WR; i += 256) Rwx[i] = a.Rw[(size_t)cx0 * WR + i];
  for (int i = tid; i < cyn * WR; i += 256) Rwy[i] = a.Rw[(size_t)cy0 * WR + i];
  if (tid < cxn) Rlox[tid] = a.Rlo[cx0 + tid] - fx0;
  if (tid < cyn) Rloy[tid] = a.Rlo[cy0 + tid] - fy0;
  __syncthreads();
  // pre-smoothed x = omega D^{-1} b on the halo tile (zero outside the grid)
  for (int r = wp; r < HY; r += VC_NW) {
    const int gy = fy0 - P + r;
    const bool rin = gy >= 0 && gy < nyf;
    for (int c = lane; c < HX; c += 32) {
      const int gx = fx0 - P + c;
      C v = czero<C>();
      if (rin && gx >= 0 && gx < nxf) {
        const size_t o = (size_t)gy * nxf + gx;
        C di = a.dinv ? a.dinv[o] : diag_inv_of<T>(kdx[c], mdx[c], kdy[r], mdy[r], a.c);
        v = a.omega * cmul(di, a.b[o]);
      }
      xs[r * H + c] = v;
    }
  }
  __syncthreads();
  // x-pass: every halo row, footprint columns (the column's band in registers)
  for (int c = lane; c < FX; c += 32) {
    T kr[W], mr[W];
#pragma unroll
    for (int d = 0; d < W; ++d) { kr[d] = kxs[c * W + d]; mr[d] = mxs[c * W + d]; }
    for (int r = wp; r < HY; r += VC_NW) {
      C s1 = czero<C>(), s2 = czero<C>();
#pragma unroll
      for (int d = 0; d < W; ++d) {
        C v = xs[r * H + c + d];
        s1 = cfma(kr[d], v, s1);
        s2 = cfma(mr[d], v, s2);
      }
      us[r * fm + c] = s1 + cmul(a.c, s2);
      ts[r * fm + c] = s2;
    }
  }
  __syncthreads();
  // y-pass: residual b - M_beta x on the footprint (into xs, row stride fm)
  for (int r = wp; r < FY; r += VC_NW) {
    T kb[W], mb[W];
#pragma unroll
    for (int d = 0; d < W; ++d) { kb[d] = kys[r * W + d]; mb[d] = mys[r * W + d]; }
    for (int c = lane; c < FX; c += 32) {
      C acc = czero<C>();
#pragma unroll
      for (int d = 0; d < W; ++d) {
        acc = cfma(mb[d], us[(r + d) * fm + c], acc);
        acc = cfma(kb[d], ts[(r + d) * fm + c], acc);
      }
      xs[r * fm + c] = a.b[(size_t)(fy0 + r) * nxf + fx0 + c] - acc;
    }
  }
  __syncthreads();
  // restriction along x: half a warp per footprint row, a lane per coarse column
  {
    const int jx = lane & 15, sub = lane >> 4;
    if (jx < cxn) {
      T wr[WR];
#pragma unroll
      for (int t = 0; t < WR; ++t) wr[t] = Rwx[jx * WR + t];
      const int j0 = Rlox[jx];
      for (int r = 2 * wp + sub; r < FY; r += 2 * VC_NW) {
        C acc = czero<C>();
#pragma unroll
        for (int t = 0; t < WR; ++t) {
          const int f = j0 + t;
          if (f >= 0 && f < FX) acc = cfma(wr[t], xs[r * fm + f], acc);
        }
        us[r * cxn + jx] = acc;
      }
    }
  }
  __syncthreads();
  // restriction along y
  for (int i = tid; i < cyn * cxn; i += 256) {
    const int jy = i / cxn, jx = i - jy * cxn;
    const int j0 = Rloy[jy];
    C acc = czero<C>();
#pragma unroll
    for (int t = 0; t < WR; ++t) {
      const int f = j0 + t;
      if (f >= 0 && f < FY) acc = cfma(Rwy[jy * WR + t], us[f * cxn + jx], acc);
    }
    a.cout[(size_t)(cy0 + jy) * nxc + cx0 + jx] = acc;
  }
}

template <typename C, typename T>
__host__ __device__ inline size_t up_smem(int P, int TY, int cmax) {
  const int TX = 32, W = 2 * P + 1, SX = TX + 2 * P, SY = TY + 2 * P, WP = P / 2 + 3, CP = cmax + WP;
  return sizeof(C) * ((size_t)SY * SX + 2 * (size_t)SY * TX + (size_t)CP * SX + (size_t)CP * CP) +
         sizeof(T) * ((size_t)2 * SX + 2 * SY + 2 * (size_t)TY * W + (size_t)(SX + SY) * WP) + sizeof(int) * (SX + SY);
}

template <int P, typename T, int TY>
__global__ void __launch_bounds__(256) k_vc_up(FusedArgs<T> a) {
  using C = typename cplx<T>::t;
  constexpr int TX = 32, W = 2 * P + 1, SX = TX + 2 * P, SY = TY + 2 * P, WP = P / 2 + 3;
  extern __shared__ __align__(16) unsigned char vsm[];
  const int cm = a.cmax, CP = cm + WP;          // coarse patch, zero-padded by a window
  C* xs = reinterpret_cast<C*>(vsm);            // [SY][SX] x on the halo tile
  C* us = xs + SY * SX;                         // [SY][TX]
  C* ts = us + SY * TX;
  C* t1 = ts + SY * TX;                         // [CP][SX] coarse rows prolonged along x
  C* xcs = t1 + (size_t)CP * SX;                // [CP][CP]
  T* kdx = reinterpret_cast<T*>(xcs + (size_t)CP * CP);   // diagonal entries of halo columns / rows
  T* mdx = kdx + SX;
  T* kdy = mdx + SX;
  T* mdy = kdy + SY;
  T* kyb = mdy + SY;                            // [TY][W] bands of the tile rows
  T* myb = kyb + TY * W;
  T* Pwx = myb + TY * W;                        // [SX][WP]
  T* Pwy = Pwx + SX * WP;                       // [SY][WP]
  int* Plox = reinterpret_cast<int*>(Pwy + SY * WP);   // window starts relative to the patch
  int* Ploy = Plox + SX;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int nxf = a.nxf, nyf = a.nyf, nxc = a.nxc, nyc = a.nyc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int gxl = max(0, x0 - P), gxh = min(nxf, x0 + TX + P);
  const int gyl = max(0, y0 - P), gyh = min(nyf, y0 + TY + P);
  const int cxa = max(0, a.Plo[gxl]), cxb = min(nxc, a.Plo[gxh - 1] + WP);
  const int cya = max(0, a.Plo[gyl]), cyb = min(nyc, a.Plo[gyh - 1] + WP);
  const int CXN = cxb - cxa, CYN = cyb - cya;
  if (CXN > cm || CYN > cm) return;             // cannot happen: cmax is the maximum over tiles
  for (int i = tid; i < CP * CP; i += 256) {
    const int r = i / CP, c = i - r * CP;
    xcs[i] = (r < CYN && c < CXN) ? a.xc[(size_t)(cya + r) * nxc + cxa + c] : czero<C>();
  }
  for (int i = tid; i < SX; i += 256) {
    const int g = x0 - P + i;
    const bool in = g >= 0 && g < nxf;
    Plox[i] = in ? max(0, a.Plo[g] - cxa) : 0;
#pragma unroll
    for (int t = 0; t < WP; ++t) Pwx[i * WP + t] = in ? a.Pw[(size_t)g * WP + t] : (T)0;
    kdx[i] = in ? a.K[(size_t)g * W + P] : (T)0;
    mdx[i] = in ? a.M[(size_t)g * W + P] : (T)0;
  }
  for (int i = tid; i < SY; i += 256) {
    const int g = y0 - P + i;
    const bool in = g >= 0 && g < nyf;
    Ploy[i] = in ? max(0, a.Plo[g] - cya) : 0;
#pragma unroll
    for (int t = 0; t < WP; ++t) Pwy[i * WP + t] = in ? a.Pw[(size_t)g * WP + t] : (T)0;
    kdy[i] = in ? a.K[(size_t)g * W + P] : (T)0;
    mdy[i] = in ? a.M[(size_t)g * W + P] : (T)0;
  }
  for (int i = tid; i < TY * W; i += 256) {
    const int r = i / W;
    kyb[i] = y0 + r < nyf ? a.K[(size_t)y0 * W + i] : (T)0;
    myb[i] = y0 + r < nyf ? a.M[(size_t)y0 * W + i] : (T)0;
  }
  __syncthreads();
  // pre-smoothed x on the halo tile; coarse rows prolonged along x
  for (int r = wp; r < SY; r += VC_NW) {
    const int gy = y0 - P + r;
    const bool rin = gy >= 0 && gy < nyf;
    for (int c = lane; c < SX; c += 32) {
      const int gx = x0 - P + c;
      C v = czero<C>();
      if (rin && gx >= 0 && gx < nxf) {
        const size_t o = (size_t)gy * nxf + gx;
        C di = a.dinv ? a.dinv[o] : diag_inv_of<T>(kdx[c], mdx[c], kdy[r], mdy[r], a.c);
        v = a.omega * cmul(di, a.b[o]);
      }
      xs[r * SX + c] = v;
    }
  }
  for (int c = lane; c < SX; c += 32) {
    T wv[WP];
#pragma unroll
    for (int t = 0; t < WP; ++t) wv[t] = Pwx[c * WP + t];
    const int j0 = Plox[c];
    for (int r = wp; r < CP; r += VC_NW) {
      C acc = czero<C>();
#pragma unroll
      for (int t = 0; t < WP; ++t) acc = cfma(wv[t], xcs[r * CP + j0 + t], acc);
      t1[r * SX + c] = acc;
    }
  }
  __syncthreads();
  // prolongation along y, added to x
  for (int r = wp; r < SY; r += VC_NW) {
    T wv[WP];
#pragma unroll
    for (int t = 0; t < WP; ++t) wv[t] = Pwy[r * WP + t];
    const int j0 = Ploy[r];
    for (int c = lane; c < SX; c += 32) {
      C acc = czero<C>();
#pragma unroll
      for (int t = 0; t < WP; ++t) acc = cfma(wv[t], t1[(j0 + t) * SX + c], acc);
      xs[r * SX + c] = xs[r * SX + c] + acc;    // zero weights keep out-of-grid points at zero
    }
  }
  __syncthreads();
  // post-smoothing sweep: x-pass (lane = tile column, band in registers)
  {
    const int c = lane, gx = x0 + c;
    T kr[W], mr[W];
#pragma unroll
    for (int d = 0; d < W; ++d) {
      kr[d] = gx < nxf ? a.K[(size_t)gx * W + d] : (T)0;
      mr[d] = gx < nxf ? a.M[(size_t)gx * W + d] : (T)0;
    }
    for (int r = wp; r < SY; r += VC_NW) {
      C s1 = czero<C>(), s2 = czero<C>();
#pragma unroll
      for (int d = 0; d < W; ++d) {
        C v = xs[r * SX + c + d];
        s1 = cfma(kr[d], v, s1);
        s2 = cfma(mr[d], v, s2);
      }
      us[r * TX + c] = s1 + cmul(a.c, s2);
      ts[r * TX + c] = s2;
    }
  }
  __syncthreads();
  // y-pass and x_out = x + omega D^{-1} (b - M_beta x)
  {
    const int c = lane, gx = x0 + c;
    for (int r = wp; r < TY; r += VC_NW) {
      const int gy = y0 + r;
      if (gy >= nyf || gx >= nxf) continue;
      C acc = czero<C>();
#pragma unroll
      for (int d = 0; d < W; ++d) {
        acc = cfma(myb[r * W + d], us[(r + d) * TX + c], acc);
        acc = cfma(kyb[r * W + d], ts[(r + d) * TX + c], acc);
      }
      const size_t o = (size_t)gy * nxf + gx;
      C di = a.dinv ? a.dinv[o] : diag_inv_of<T>(kdx[c + P], mdx[c + P], kdy[r + P], mdy[r + P], a.c);
      a.xout[o] = xs[(r + P) * SX + c + P] + a.omega * cmul(di, a.b[o] - acc);
    }
  }
}

// D^{-1} of M_beta on a constant-k level (FP64 levels keep it in memory)
__global__ void k_const_dinv(int nx, int ny, int p, const double* K, const double* M, double2 c, double2* out) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nx * ny) return;
  const int W = 2 * p + 1;
  int iy = (int)(i / nx), ix = (int)(i - (size_t)iy * nx);
  double kxd = K[(size_t)ix * W + p], mxd = M[(size_t)ix * W + p];
  double kyd = K[(size_t)iy * W + p], myd = M[(size_t)iy * W + p];
  double2 d = myd * (mkc(kxd, 0.0) + mxd * c) + mkc(kyd * mxd, 0.0);
  out[i] = cinv(d);
}

// ------------------------------------------------------------------ host side
template <typename T> struct FusedBufs;
template <> struct FusedBufs<double> {
  static const double* K(LevelData& L) { return L.K; }
  static const double* M(LevelData& L) { return L.M; }
  static const double* Rw(LevelData& L) { return L.Rw; }
  static const double* Pw(LevelData& L) { return L.Pw; }
  static const double2* dinv(LevelData& L) { return L.dinv; }
  static double2* b(LevelData& L) { return L.vb; }
  static double2* x(LevelData& L) { return L.vx; }
};
template <> struct FusedBufs<float> {
  static const float* K(LevelData& L) { return L.Kf; }
  static const float* M(LevelData& L) { return L.Mf; }
  static const float* Rw(LevelData& L) { return L.Rwf; }
  static const float* Pw(LevelData& L) { return L.Pwf; }
  static const float2* dinv(LevelData&) { return nullptr; }
  static float2* b(LevelData& L) { return L.fb; }
  static float2* x(LevelData& L) { return L.fx; }
};

static int up_ty(const LevelData& F) { return F.nx >= 256 ? 16 : 8; }

template <int P, typename T>
static void set_fused_attrs(int maxsm) {
  cudaFuncSetAttribute(k_vc_down<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
  cudaFuncSetAttribute(k_vc_up<P, T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
  cudaFuncSetAttribute(k_vc_up<P, T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
}

// FP64 D^{-1} of M_beta on every constant-k 2D level (the FP64 Jacobi sweeps
// read it instead of dividing: FP64 division is slow on this part)
iga_status setup_const_dinv(iga_ctx* ctx) {
  if (ctx->dim != 2 || ctx->vark) return IGA_OK;
  const double2 cm = ctx->k2const * make_double2(-ctx->sig.x, -ctx->sig.y);
  for (int l = 0; l < ctx->L; ++l) {
    LevelData& F = ctx->lv[l];
    if (F.dinv) continue;
    F.dinv = dalloc<double2>(ctx, F.n);
    if (!F.dinv) return set_err(ctx, IGA_E_OOM, "D^-1 of level %d", l);
    k_const_dinv<<<cdiv(F.n, 256), 256, 0, ctx->st>>>(F.nx, F.ny, ctx->p, F.K, F.M, cm, F.dinv); iga_count_launch();
    CKL();
  }
  return IGA_OK;
}

// Decide whether the fused V-cycle applies, and size its tiles from the
// transfer tables (copied to the host once).
iga_status setup_fused_vcycle(iga_ctx* ctx) {
  ctx->vc_fused = false;
  const iga_params& P = ctx->prm;
  if (!P.fused_vcycle || ctx->dim != 2 || ctx->vark || P.nu_pre != 1 || P.nu_post != 1 || ctx->L < 2) return IGA_OK;
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  const int p = ctx->p;
  for (int l = 0; l + 1 < ctx->L; ++l) {
    LevelData& F = ctx->lv[l];
    LevelData& Cl = ctx->lv[l + 1];
    std::vector<int> Rlo(Cl.nx), Plo(F.nx);
    CK(cudaMemcpy(Rlo.data(), F.Rlo, sizeof(int) * Cl.nx, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(Plo.data(), F.Plo, sizeof(int) * F.nx, cudaMemcpyDeviceToHost));
    for (int j = 1; j < Cl.nx; ++j)
      if (Rlo[j] < Rlo[j - 1]) return IGA_OK;     // the tiles assume monotone windows
    for (int i = 1; i < F.nx; ++i)
      if (Plo[i] < Plo[i - 1]) return IGA_OK;
    if (F.wR != p + 3 || F.wP != p / 2 + 3) return IGA_OK;   // the kernels fix the window widths
    const int CT = down_ct(p);
    int fmax = 1;
    for (int c0 = 0; c0 < Cl.nx; c0 += CT) {
      int cn = std::min(CT, Cl.nx - c0);
      int f0 = std::max(0, Rlo[c0]), f1 = std::min(F.nx, Rlo[c0 + cn - 1] + F.wR);
      fmax = std::max(fmax, f1 - f0);
    }
    const int TY = up_ty(F);
    int cmax = 1;
    for (int dirn = 0; dirn < 2; ++dirn) {
      const int T_ = dirn == 0 ? 32 : TY;
      for (int x0 = 0; x0 < F.nx; x0 += T_) {
        int gl = std::max(0, x0 - p), gh = std::min(F.nx, x0 + T_ + p);
        int ca = std::max(0, Plo[gl]), cb = std::min(Cl.nx, Plo[gh - 1] + F.wP);
        cmax = std::max(cmax, cb - ca);
      }
    }
    F.vc_fmax = fmax;
    F.vc_cmax = cmax;
    const size_t need = std::max(down_smem<double2, double>(p, fmax), up_smem<double2, double>(p, TY, cmax));
    if (need > (size_t)maxsm) return IGA_OK;
  }
  switch (p) {
    case 1: set_fused_attrs<1, double>(maxsm); set_fused_attrs<1, float>(maxsm); break;
    case 2: set_fused_attrs<2, double>(maxsm); set_fused_attrs<2, float>(maxsm); break;
    case 3: set_fused_attrs<3, double>(maxsm); set_fused_attrs<3, float>(maxsm); break;
    case 4: set_fused_attrs<4, double>(maxsm); set_fused_attrs<4, float>(maxsm); break;
    case 5: set_fused_attrs<5, double>(maxsm); set_fused_attrs<5, float>(maxsm); break;
    default: return IGA_OK;
  }
  cudaGetLastError();
  ctx->vc_fused = true;
  return IGA_OK;
}

template <typename T>
static FusedArgs<T> fused_args(iga_ctx* ctx, int l) {
  using C = typename cplx<T>::t;
  LevelData& F = ctx->lv[l];
  LevelData& Cl = ctx->lv[l + 1];
  FusedArgs<T> a;
  a.nxf = F.nx; a.nyf = F.ny; a.nxc = Cl.nx; a.nyc = Cl.ny;
  a.K = FusedBufs<T>::K(F);
  a.M = FusedBufs<T>::M(F);
  a.c = cconv<C>(ctx->k2const * make_double2(-ctx->sig.x, -ctx->sig.y));
  a.dinv = FusedBufs<T>::dinv(F);
  a.omega = (T)ctx->prm.omega;
  a.b = nullptr;
  a.Rw = FusedBufs<T>::Rw(F); a.Rlo = F.Rlo; a.wR = F.wR; a.cout = nullptr; a.fmax = F.vc_fmax;
  a.Pw = FusedBufs<T>::Pw(F); a.Plo = F.Plo; a.wP = F.wP; a.xc = nullptr; a.xout = nullptr; a.cmax = F.vc_cmax;
  return a;
}

template <int P, typename T>
static void launch_down(iga_ctx* ctx, const FusedArgs<T>& a) {
  using C = typename cplx<T>::t;
  constexpr int CT = down_ct(P);
  dim3 g(cdiv(a.nxc, CT), cdiv(a.nyc, CT));
  k_vc_down<P, T><<<g, 256, down_smem<C, T>(P, a.fmax), ctx->st>>>(a); iga_count_launch();
}

template <int P, typename T>
static void launch_up(iga_ctx* ctx, const LevelData& F, const FusedArgs<T>& a) {
  using C = typename cplx<T>::t;
  if (up_ty(F) == 16) {
    dim3 g(cdiv(a.nxf, 32), cdiv(a.nyf, 16));
    k_vc_up<P, T, 16><<<g, 256, up_smem<C, T>(P, 16, a.cmax), ctx->st>>>(a);
  } else {
    dim3 g(cdiv(a.nxf, 32), cdiv(a.nyf, 8));
    k_vc_up<P, T, 8><<<g, 256, up_smem<C, T>(P, 8, a.cmax), ctx->st>>>(a);
  }
  iga_count_launch();
}

template <int P, typename T>
static iga_status vcycle_fused_p(iga_ctx* ctx, const typename cplx<T>::t* r, typename cplx<T>::t* z) {
  using C = typename cplx<T>::t;
  const int L = ctx->L;
  for (int l = 0; l + 1 < L; ++l) {
    FusedArgs<T> a = fused_args<T>(ctx, l);
    a.b = l == 0 ? r : FusedBufs<T>::b(ctx->lv[l]);
    a.cout = FusedBufs<T>::b(ctx->lv[l + 1]);
    launch_down<P, T>(ctx, a);
  }
  LevelData& Lc = ctx->lv[L - 1];
  TRY(mg_coarse<T>(ctx, FusedBufs<T>::b(Lc), FusedBufs<T>::x(Lc)));
  for (int l = L - 2; l >= 0; --l) {
    FusedArgs<T> a = fused_args<T>(ctx, l);
    a.b = l == 0 ? r : FusedBufs<T>::b(ctx->lv[l]);
    a.xc = FusedBufs<T>::x(ctx->lv[l + 1]);
    a.xout = l == 0 ? z : FusedBufs<T>::x(ctx->lv[l]);
    launch_up<P, T>(ctx, ctx->lv[l], a);
  }
  CKL();
  return IGA_OK;
}

// One V-cycle z = V(r) from z = 0 with the fused level kernels.
template <typename T>
iga_status mg_vcycle_fused(iga_ctx* ctx, const typename cplx<T>::t* r, typename cplx<T>::t* z) {
  switch (ctx->p) {
    case 1: return vcycle_fused_p<1, T>(ctx, r, z);
    case 2: return vcycle_fused_p<2, T>(ctx, r, z);
    case 3: return vcycle_fused_p<3, T>(ctx, r, z);
    case 4: return vcycle_fused_p<4, T>(ctx, r, z);
    case 5: return vcycle_fused_p<5, T>(ctx, r, z);
    default: return set_err(ctx, IGA_E_INVALID, "p out of range");
  }
}

template iga_status mg_vcycle_fused<double>(iga_ctx*, const double2*, double2*);
template iga_status mg_vcycle_fused<float>(iga_ctx*, const float2*, float2*);
