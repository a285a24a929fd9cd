// Geometric multigrid V-cycle for the CSLP (Section 3: damped Jacobi,
// omega = 0.6; Section 4.2: V-cycle with coarse correction between nested
// spline spaces).  Transfers are knot insertion (B-spline refinement), whose
// p = 1 case is the paper's linear interpolation; restriction is its
// transpose.  The coarsest level is solved with a dense inverse built at setup
// (1D above IGA_MAX_COARSEST dofs: the band solver of banded.cu).
#include "common.cuh"
#include <algorithm>
#include <cmath>
#include <vector>

// ------------------------------------------------------------------ kernels
// First Jacobi sweep from x = 0:  x = omega D^{-1} b.
template <typename T>
__global__ void k_jacobi0(int nx, int ny, int p, const T* K, const T* M, typename cplx<T>::t c,
                          const typename cplx<T>::t* dinv, const typename cplx<T>::t* b,
                          typename cplx<T>::t* x, T omega) {
  using C = typename cplx<T>::t;
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;      // levels hold < 2^31 dofs
  if (i >= (unsigned)nx * (unsigned)ny) return;
  C di;
  if (dinv) {
    di = dinv[i];
  } else {
    int W = 2 * p + 1;
    int iy = (int)(i / (unsigned)nx), ix = (int)(i - (unsigned)iy * nx);
    T kx = K[(size_t)ix * W + p], mx = M[(size_t)ix * W + p];
    C d;
    if (ny == 1) {
      d = mkc(kx, (T)0) + mx * c;
    } else {
      T ky = K[(size_t)iy * W + p], my = M[(size_t)iy * W + p];
      d = my * (mkc(kx, (T)0) + mx * c) + mkc(ky * mx, (T)0);
    }
    di = cinv(d);
  }
  x[i] = omega * cmul(di, b[i]);
}

// The same first sweep on the finest FP32 level of a constant-k 2D problem,
// fed by the complex128 right-hand side: b32 = (float) b is stored for the
// later sweeps and x = omega D^{-1} b32 (the conversion and the sweep in one
// pass; results equal to converting first).
__global__ void k_jacobi0_in128(int nx, int ny, int p, const float* K, const float* M, float2 c, const double2* b,
                                float2* b32, float2* x, float omega) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)nx * (unsigned)ny) return;
  const int W = 2 * p + 1;
  const int iy = (int)(i / (unsigned)nx), ix = (int)(i - (unsigned)iy * nx);
  const float kx = K[(size_t)ix * W + p], mx = M[(size_t)ix * W + p];
  const float ky = K[(size_t)iy * W + p], my = M[(size_t)iy * W + p];
  const float2 d = my * (mkc(kx, 0.f) + mx * c) + mkc(ky * mx, 0.f);
  const float2 bv = tof(b[i]);
  b32[i] = bv;
  x[i] = omega * cmul(cinv(d), bv);
}

// coarse = P^T fine  (2D: tensor product of the 1D restriction rows)
// With xc != nullptr the same kernel also performs the coarse level's first
// damped Jacobi sweep from zero, xc = omega D_c^{-1} c (D_c from the coarse 1D
// band diagonals, or dinv for variable k).
template <typename T>
__global__ void k_restrict(int nxf, int nyf, int nxc, int nyc, int wR, const T* Rw, const int* Rlo,
                           const typename cplx<T>::t* f, typename cplx<T>::t* c, typename cplx<T>::t* xc, int p,
                           const T* Kc, const T* Mc, typename cplx<T>::t cm, const typename cplx<T>::t* dinv,
                           T omega) {
  using C = typename cplx<T>::t;
  size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (j >= (size_t)nxc * nyc) return;
  int jy = (int)(j / nxc), jx = (int)(j - (size_t)jy * nxc);
  C acc = czero<C>();
  int lx = Rlo[jx];
  if (nyc == 1) {
    for (int kx = 0; kx < wR; ++kx) {
      int ix = lx + kx;
      T w = Rw[(size_t)jx * wR + kx];
      if (w != (T)0 && ix >= 0 && ix < nxf) acc = cfma(w, f[ix], acc);
    }
  } else {
    int ly = Rlo[jy];
    for (int ky = 0; ky < wR; ++ky) {
      int iy = ly + ky;
      T wy = Rw[(size_t)jy * wR + ky];
      if (wy == (T)0 || iy < 0 || iy >= nyf) continue;
      C row = czero<C>();
      for (int kx = 0; kx < wR; ++kx) {
        int ix = lx + kx;
        T w = Rw[(size_t)jx * wR + kx];
        if (w != (T)0 && ix >= 0 && ix < nxf) row = cfma(w, f[(size_t)iy * nxf + ix], row);
      }
      acc = cfma(wy, row, acc);
    }
  }
  c[j] = acc;
  if (xc) {
    C di;
    if (dinv) {
      di = dinv[j];
    } else {
      int W = 2 * p + 1;
      T kx = Kc[(size_t)jx * W + p], mx = Mc[(size_t)jx * W + p];
      C d;
      if (nyc == 1) {
        d = mkc(kx, (T)0) + mx * cm;
      } else {
        T ky = Kc[(size_t)jy * W + p], my = Mc[(size_t)jy * W + p];
        d = my * (mkc(kx, (T)0) + mx * cm) + mkc(ky * mx, (T)0);
      }
      di = cinv(d);
    }
    xc[j] = omega * cmul(di, acc);
  }
}

// fine += P coarse
template <typename T>
__global__ void k_prolong_add(int nxf, int nyf, int nxc, int nyc, int wP, const T* Pw, const int* Plo,
                              const typename cplx<T>::t* c, typename cplx<T>::t* f) {
  using C = typename cplx<T>::t;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nxf * nyf) return;
  int iy = (int)(i / nxf), ix = (int)(i - (size_t)iy * nxf);
  C acc = czero<C>();
  int lx = Plo[ix];
  if (nyf == 1) {
    for (int kx = 0; kx < wP; ++kx) {
      int jx = lx + kx;
      T w = Pw[(size_t)ix * wP + kx];
      if (w != (T)0 && jx >= 0 && jx < nxc) acc = cfma(w, c[jx], acc);
    }
  } else {
    int ly = Plo[iy];
    for (int ky = 0; ky < wP; ++ky) {
      int jy = ly + ky;
      T wy = Pw[(size_t)iy * wP + ky];
      if (wy == (T)0 || jy < 0 || jy >= nyc) continue;
      C row = czero<C>();
      for (int kx = 0; kx < wP; ++kx) {
        int jx = lx + kx;
        T w = Pw[(size_t)ix * wP + kx];
        if (w != (T)0 && jx >= 0 && jx < nxc) row = cfma(w, c[(size_t)jy * nxc + jx], row);
      }
      acc = cfma(wy, row, acc);
    }
  }
  f[i] = f[i] + acc;
}

// ------------------------------------------------------------------ tiled 2D transfers
// Separable tensor-product transfers through shared memory: each pass runs
// one 1D window (p + 3 or p/2 + 3 taps) per output instead of the 2D window,
// so a thread's dependent chain is a few FMAs (FP64 retires one warp
// instruction per 64 cycles per SM sub-partition on this part).
constexpr int TR_CT = 16;            // coarse tile of the restriction (TR_CT^2 = 256 threads)
constexpr int TP_TX = 32, TP_TY = 32; // fine tile of the prolongation (32 x 8 on small levels)

template <typename C, typename T>
__host__ __device__ inline size_t tr_smem(int fmax, int wR) {
  return sizeof(C) * ((size_t)fmax * fmax + (size_t)fmax * TR_CT) + sizeof(T) * 2 * TR_CT * wR + sizeof(int) * 2 * TR_CT;
}

// Interior stencil of the restriction table, passed by value (kernel
// parameter space): weights r with Rlo[j] = 2j + roff for coarse j in
// [rj0, rj1] (valid = 0: tables only)
template <typename T> struct TrStencil {
  T r[8];
  int roff, rj0, rj1, valid;
};

template <typename T>
static TrStencil<T> tr_stencil(const LevelData& F) {
  TrStencil<T> st{};
  for (int t = 0; t < 8; ++t) st.r[t] = (T)F.tst.r[t];
  st.roff = F.tst.roff; st.rj0 = F.tst.rj0; st.rj1 = F.tst.rj1;
  st.valid = F.tst.rj1 >= F.tst.rj0;
  return st;
}

// c = R f on a coarse TR_CT^2 tile; with xc also xc = omega D_c^{-1} c.
// WR > 0 (= wR): tiles whose coarse columns (rows) lie in the stencil's
// interior range make the x (y) pass with the interior weights from the
// parameter space and fixed offsets (no weight loads, no bounds tests).
template <typename T, int WR>
__global__ void __launch_bounds__(256) k_restrict_tiled(int nxf, int nyf, int nxc, int nyc, int wR, const T* Rw,
                                                        const int* Rlo, int fmax, const typename cplx<T>::t* f,
                                                        typename cplx<T>::t* c, typename cplx<T>::t* xc,
                                                        const typename cplx<T>::t* dinv, T omega, int p,
                                                        const T* Kc, const T* Mc, typename cplx<T>::t cm,
                                                        TrStencil<T> st) {
  using C = typename cplx<T>::t;
  extern __shared__ __align__(16) unsigned char rsm[];
  C* fs = reinterpret_cast<C*>(rsm);                 // [FY][FX] fine footprint
  C* rx = fs + (size_t)fmax * fmax;                  // [FY][TR_CT] restricted along x
  T* Rwx = reinterpret_cast<T*>(rx + (size_t)fmax * TR_CT);
  T* Rwy = Rwx + TR_CT * wR;
  int* Rlox = reinterpret_cast<int*>(Rwy + TR_CT * wR);
  int* Rloy = Rlox + TR_CT;
  const int tid = threadIdx.x;
  const int cx0 = blockIdx.x * TR_CT, cy0 = blockIdx.y * TR_CT;
  const int cxn = min(TR_CT, nxc - cx0), cyn = min(TR_CT, nyc - cy0);
  const int fx0 = max(0, Rlo[cx0]), fx1 = min(nxf, Rlo[cx0 + cxn - 1] + wR);
  const int fy0 = max(0, Rlo[cy0]), fy1 = min(nyf, Rlo[cy0 + cyn - 1] + wR);
  const int FX = fx1 - fx0, FY = fy1 - fy0;
  if (FX > fmax || FY > fmax || FX < 1 || FY < 1) return;   // cannot happen: fmax is the maximum over tiles
  const float rFX = 1.0f / (float)FX;
  for (int i = tid; i < FY * FX; i += 256) {         // flat over the footprint (measured faster than warp rows)
    // i / FX without a division: (i + 1/2) / FX is at least 1/(2 FX) away from
    // an integer, far above the float rounding of the product (FX, FY < 2^8)
    const int r = __float2int_rz(((float)i + 0.5f) * rFX), q = i - r * FX;
    fs[i] = f[(size_t)(fy0 + r) * nxf + fx0 + q];
  }
  const bool xin = WR > 0 && st.valid && cx0 >= st.rj0 && cx0 + cxn - 1 <= st.rj1;
  const bool yin = WR > 0 && st.valid && cy0 >= st.rj0 && cy0 + cyn - 1 <= st.rj1;
  for (int i = tid; i < cxn * wR; i += 256) Rwx[i] = Rw[(size_t)cx0 * wR + i];
  for (int i = tid; i < cyn * wR; i += 256) Rwy[i] = Rw[(size_t)cy0 * wR + i];
  if (tid < cxn) Rlox[tid] = Rlo[cx0 + tid] - fx0;
  if (tid < cyn) Rloy[tid] = Rlo[cy0 + tid] - fy0;
  __syncthreads();
  {
    const int jx = tid & (TR_CT - 1);                // a thread per coarse column and every 16th row
    if (jx < cxn) {
      if (xin) {
        const int q0 = 2 * (cx0 + jx) + st.roff - fx0;
        for (int r = tid / TR_CT; r < FY; r += 256 / TR_CT) {
          const C* fr = fs + r * FX + q0;
          C acc = czero<C>();
#pragma unroll
          for (int t = 0; t < (WR > 0 ? WR : 1); ++t) acc = cfma(st.r[t], fr[t], acc);
          rx[r * TR_CT + jx] = acc;
        }
      } else {
        for (int r = tid / TR_CT; r < FY; r += 256 / TR_CT) {
          C acc = czero<C>();
          for (int t = 0; t < wR; ++t) {
            const T w = Rwx[jx * wR + t];
            const int q = Rlox[jx] + t;
            if (w != (T)0 && q >= 0 && q < FX) acc = cfma(w, fs[r * FX + q], acc);
          }
          rx[r * TR_CT + jx] = acc;
        }
      }
    }
  }
  __syncthreads();
  {
    const int jy = tid / TR_CT, jx = tid & (TR_CT - 1);   // TR_CT^2 = 256: one coarse output per thread
    if (jy >= cyn || jx >= cxn) return;
    C acc = czero<C>();
    if (yin) {
      const C* rc = rx + (2 * (cy0 + jy) + st.roff - fy0) * TR_CT + jx;
#pragma unroll
      for (int t = 0; t < (WR > 0 ? WR : 1); ++t) acc = cfma(st.r[t], rc[t * TR_CT], acc);
    } else {
      for (int t = 0; t < wR; ++t) {
        const T w = Rwy[jy * wR + t];
        const int q = Rloy[jy] + t;
        if (w != (T)0 && q >= 0 && q < FY) acc = cfma(w, rx[q * TR_CT + jx], acc);
      }
    }
    const size_t o = (size_t)(cy0 + jy) * nxc + cx0 + jx;
    c[o] = acc;
    if (xc) {
      C di;
      if (dinv) {
        di = dinv[o];
      } else {          // D_c from the coarse 1D band diagonals
        const int W = 2 * p + 1, gx = cx0 + jx, gy = cy0 + jy;
        const T kxd = Kc[gx * W + p], mxd = Mc[gx * W + p], kyd = Kc[gy * W + p], myd = Mc[gy * W + p];
        di = cinv(myd * (mkc(kxd, (T)0) + mxd * cm) + mkc(kyd * mxd, (T)0));
      }
      xc[o] = omega * cmul(di, acc);
    }
  }
}

template <typename C, typename T>
__host__ __device__ inline size_t tp_smem(int cmax, int wP, int ty) {
  return sizeof(C) * ((size_t)cmax * cmax + (size_t)cmax * TP_TX) + sizeof(T) * (TP_TX + ty) * wP +
         sizeof(int) * (TP_TX + ty);
}

// f += P c on a fine TP_TX x TY tile: a lane per fine column, a warp per row;
// the tile's f values are fetched first so their latency overlaps the
// coarse-patch work
template <typename T, int TY>
__global__ void __launch_bounds__(256) k_prolong_tiled(int nxf, int nyf, int nxc, int nyc, int wP, const T* Pw,
                                                       const int* Plo, int cmax, const typename cplx<T>::t* c,
                                                       typename cplx<T>::t* f) {
  using C = typename cplx<T>::t;
  constexpr int RPW = TY / 8;                        // fine rows per warp
  extern __shared__ __align__(16) unsigned char psm[];
  C* cs = reinterpret_cast<C*>(psm);                 // [CYN][CXN] coarse patch
  C* t1 = cs + (size_t)cmax * cmax;                  // [CYN][TP_TX] prolonged along x
  T* Pwx = reinterpret_cast<T*>(t1 + (size_t)cmax * TP_TX);
  T* Pwy = Pwx + TP_TX * wP;
  int* Plox = reinterpret_cast<int*>(Pwy + TY * wP);
  int* Ploy = Plox + TP_TX;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int x0 = blockIdx.x * TP_TX, y0 = blockIdx.y * TY;
  const int xn = min(TP_TX, nxf - x0), yn = min(TY, nyf - y0);
  const int cxa = max(0, Plo[x0]), cxb = min(nxc, Plo[x0 + xn - 1] + wP);
  const int cya = max(0, Plo[y0]), cyb = min(nyc, Plo[y0 + yn - 1] + wP);
  const int CXN = cxb - cxa, CYN = cyb - cya;
  if (CXN > cmax || CYN > cmax || CXN < 1 || CYN < 1) return;   // cannot happen: cmax is the maximum over tiles
  C fv[RPW];
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int r = wp + 8 * k;
    fv[k] = (r < yn && lane < xn) ? f[(size_t)(y0 + r) * nxf + x0 + lane] : czero<C>();
  }
  for (int r = wp; r < CYN; r += 8)
    for (int q = lane; q < CXN; q += 32) cs[r * CXN + q] = c[(size_t)(cya + r) * nxc + cxa + q];
  for (int i = tid; i < xn * wP; i += 256) Pwx[i] = Pw[(size_t)x0 * wP + i];
  for (int i = tid; i < yn * wP; i += 256) Pwy[i] = Pw[(size_t)y0 * wP + i];
  if (tid < xn) Plox[tid] = Plo[x0 + tid] - cxa;
  if (tid < yn) Ploy[tid] = Plo[y0 + tid] - cya;
  __syncthreads();
  if (lane < xn) {
    for (int r = wp; r < CYN; r += 8) {
      C acc = czero<C>();
      for (int t = 0; t < wP; ++t) {
        const T w = Pwx[lane * wP + t];
        const int j = Plox[lane] + t;
        if (w != (T)0 && j >= 0 && j < CXN) acc = cfma(w, cs[r * CXN + j], acc);
      }
      t1[r * TP_TX + lane] = acc;
    }
  }
  __syncthreads();
  if (lane >= xn) return;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int r = wp + 8 * k;
    if (r >= yn) break;
    C acc = czero<C>();
    for (int t = 0; t < wP; ++t) {
      const T w = Pwy[r * wP + t];
      const int j = Ploy[r] + t;
      if (w != (T)0 && j >= 0 && j < CYN) acc = cfma(w, t1[j * TP_TX + lane], acc);
    }
    f[(size_t)(y0 + r) * nxf + x0 + lane] = fv[k] + acc;
  }
}

// Tile extents of the tiled transfers of level l -> l+1 (from the host copies
// of the window tables).  0 when a window table is not monotone.
iga_status setup_tiled_transfers(iga_ctx* ctx) {
  if (ctx->dim != 2) return IGA_OK;
  for (int l = 0; l + 1 < ctx->L; ++l) {
    LevelData& F = ctx->lv[l];
    LevelData& Cl = ctx->lv[l + 1];
    std::vector<int> Rlo(Cl.nx), Plo(F.nx);
    CK(cudaMemcpy(Rlo.data(), F.Rlo, sizeof(int) * Cl.nx, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(Plo.data(), F.Plo, sizeof(int) * F.nx, cudaMemcpyDeviceToHost));
    bool mono = true;
    for (int j = 1; j < Cl.nx; ++j) mono = mono && Rlo[j] >= Rlo[j - 1];
    for (int i = 1; i < F.nx; ++i) mono = mono && Plo[i] >= Plo[i - 1];
    F.tr_fmax = F.tp_cmax = 0;
    F.tst = {};
    if (!mono) continue;
    {
      // interior stencil of the restriction: the contiguous range around the
      // middle whose rows equal the middle row shifted by 2 per coarse row,
      // with the whole window inside the grid
      std::vector<double> Rw((size_t)Cl.nx * F.wR);
      CK(cudaMemcpy(Rw.data(), F.Rw, sizeof(double) * Rw.size(), cudaMemcpyDeviceToHost));
      auto& st = F.tst;
      if (F.wR <= 8 && Cl.nx >= 3) {
        const int jm = Cl.nx / 2;
        st.roff = Rlo[jm] - 2 * jm;
        for (int t = 0; t < F.wR; ++t) st.r[t] = Rw[(size_t)jm * F.wR + t];
        auto rok = [&](int j) {
          if (Rlo[j] != 2 * j + st.roff || Rlo[j] < 0 || Rlo[j] + F.wR > F.nx) return false;
          for (int t = 0; t < F.wR; ++t)      // the knot-insertion weights of interior rows agree to rounding
            if (std::fabs(Rw[(size_t)j * F.wR + t] - st.r[t]) > 1e-13) return false;
          return true;
        };
        if (rok(jm)) {
          st.rj0 = st.rj1 = jm;
          while (st.rj0 > 0 && rok(st.rj0 - 1)) --st.rj0;
          while (st.rj1 + 1 < Cl.nx && rok(st.rj1 + 1)) ++st.rj1;
        }
      }
    }
    int fmax = 1, cmax = 1;
    for (int c0 = 0; c0 < Cl.nx; c0 += TR_CT) {
      int cn = std::min(TR_CT, Cl.nx - c0);
      fmax = std::max(fmax, std::min(F.nx, Rlo[c0 + cn - 1] + F.wR) - std::max(0, Rlo[c0]));
    }
    for (int T_ : {TP_TX, TP_TY})
      for (int x0 = 0; x0 < F.nx; x0 += T_) {
        int xn = std::min(T_, F.nx - x0);
        cmax = std::max(cmax, std::min(Cl.nx, Plo[x0 + xn - 1] + F.wP) - std::max(0, Plo[x0]));
      }
    if (tr_smem<double2, double>(fmax, F.wR) <= 48 * 1024 && tp_smem<double2, double>(cmax, F.wP, TP_TY) <= 48 * 1024) {
      F.tr_fmax = fmax;
      F.tp_cmax = cmax;
    }
  }
  return IGA_OK;
}

// x = Minv b, dense: one warp per row, lanes over the columns, shuffle sum
// (a row's dependent chain is a few FMAs instead of n)
template <typename C>
__global__ void k_dense_mv(int n, const C* Minv, const C* b, C* x) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  C acc = czero<C>();
  for (int j = lane; j < n; j += 32) acc = acc + cmul(Minv[(size_t)row * n + j], b[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) x[row] = acc;
}

// Gauss-Jordan inversion with partial pivoting (one block): A (n x n, row
// major, destroyed), Inv starts as the identity.
__global__ void k_gauss_jordan(double2* A, double2* Inv, int n, int* info) {
  extern __shared__ double2 fcol[];
  __shared__ int piv;
  __shared__ double2 pinv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int best = k;
      double bv = -1.0;
      for (int i = k; i < n; ++i) {
        double2 v = A[(size_t)i * n + k];
        double m = v.x * v.x + v.y * v.y;
        if (m > bv) { bv = m; best = i; }
      }
      piv = best;
      if (!(bv > 0.0)) *info = 1;
    }
    __syncthreads();
    if (piv != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double2 t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)piv * n + j]; A[(size_t)piv * n + j] = t;
        t = Inv[(size_t)k * n + j]; Inv[(size_t)k * n + j] = Inv[(size_t)piv * n + j]; Inv[(size_t)piv * n + j] = t;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) pinv = cinv(A[(size_t)k * n + k]);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      A[(size_t)k * n + j] = cmul(pinv, A[(size_t)k * n + j]);
      Inv[(size_t)k * n + j] = cmul(pinv, Inv[(size_t)k * n + j]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = A[(size_t)i * n + k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      int i = idx / n, j = idx - i * n;
      if (i == k) continue;
      double2 f = fcol[i];
      A[(size_t)i * n + j] = A[(size_t)i * n + j] - cmul(f, A[(size_t)k * n + j]);
      Inv[(size_t)i * n + j] = Inv[(size_t)i * n + j] - cmul(f, Inv[(size_t)k * n + j]);
    }
    __syncthreads();
  }
}

__global__ void k_unit(double2* e, int n, int j) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) e[i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}
__global__ void k_eye(double2* e, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * n) e[i] = make_double2((i / n) == (i % n) ? 1.0 : 0.0, 0.0);
}
// columns (stored as rows of colsT) -> row-major matrix
__global__ void k_transpose_c(const double2* colsT, double2* A, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * n) { int r = i / n, c = i % n; A[(size_t)r * n + c] = colsT[(size_t)c * n + r]; }
}
__global__ void k_c2f(const double2* a, float2* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = tof(a[i]);
}
__global__ void k_f2d(const float2* a, double2* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = tod(a[i]);
}
template <typename C>
__global__ void k_axpy1(C* y, const C* x, size_t n) {   // y += x
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = y[i] + x[i];
}

void launch_convert_d2f(const double2* a, float2* b, size_t n, cudaStream_t st) {
  k_c2f<<<cdiv(n, 256), 256, 0, st>>>(a, b, n); iga_count_launch();
}
void launch_convert_f2d(const float2* a, double2* b, size_t n, cudaStream_t st) {
  k_f2d<<<cdiv(n, 256), 256, 0, st>>>(a, b, n); iga_count_launch();
}

// ------------------------------------------------------------------ host
iga_status setup_coarse_inverse(iga_ctx* ctx) {
  int l = ctx->L - 1;
  LevelData& L = ctx->lv[l];
  int n = L.n;
  ctx->nc = n;
  if (n > IGA_MAX_COARSEST && ctx->dim == 1) {
    // 1D: M_beta is a band matrix (half bandwidth p); probe its band and
    // factorise it with the band solver
    ctx->coarse_banded = true;
    double2* Ab = dalloc<double2>(ctx, (size_t)n * (2 * ctx->p + 1));
    ctx->cband_t = dalloc<double2>(ctx, n);
    ctx->cband_x = dalloc<double2>(ctx, n);
    if (!Ab || !ctx->cband_t || !ctx->cband_x) return set_err(ctx, IGA_E_OOM, "coarse band alloc");
    auto apply = [ctx, l](const double2* x, double2* y) -> iga_status {
      return op_apply<double>(ctx, l, OP_MB, x, y, nullptr, EPI_Y, nullptr, 0.0);
    };
    TRY(band_probe(ctx, n, ctx->p, apply, L.vx, L.vy, Ab));
    return band_setup(ctx, ctx->bandC, Ab, n, ctx->p);
  }
  // one block inverts the coarsest matrix (a row of it in shared memory)
  if (n > IGA_MAX_COARSEST)
    return set_err(ctx, IGA_E_INVALID,
                   "coarsest level has %d dofs (> %d): n_el must halve to a coarsest mesh of at most ~%d "
                   "elements per direction", n, IGA_MAX_COARSEST, 40);
  double2* cols = dalloc<double2>(ctx, (size_t)n * n);   // row j = M_beta e_j
  double2* A = dalloc<double2>(ctx, (size_t)n * n);
  double2* e = dalloc<double2>(ctx, n);
  ctx->cinv = dalloc<double2>(ctx, (size_t)n * n);
  ctx->cinvf = dalloc<float2>(ctx, (size_t)n * n);
  int* info = dalloc<int>(ctx, 1);
  if (!cols || !A || !e || !ctx->cinv || !ctx->cinvf || !info) return set_err(ctx, IGA_E_OOM, "coarse alloc");
  for (int j = 0; j < n; ++j) {
    k_unit<<<cdiv(n, 128), 128, 0, ctx->st>>>(e, n, j); iga_count_launch();
    TRY(op_apply<double>(ctx, l, OP_MB, e, cols + (size_t)j * n, nullptr, EPI_Y, nullptr, 0.0));
  }
  k_transpose_c<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(cols, A, n); iga_count_launch();
  k_eye<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(ctx->cinv, n); iga_count_launch();
  CK(cudaMemsetAsync(info, 0, sizeof(int), ctx->st));
  k_gauss_jordan<<<1, 256, n * sizeof(double2), ctx->st>>>(A, ctx->cinv, n, info); iga_count_launch();
  CKL();
  k_c2f<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(ctx->cinv, ctx->cinvf, (size_t)n * n); iga_count_launch();
  int hinfo = 0;
  CK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (hinfo) return set_err(ctx, IGA_E_INVALID, "coarsest CSLP matrix is singular");
  return IGA_OK;
}

template <typename T> struct LvBuf;
template <> struct LvBuf<double> {
  static double2* b(LevelData& L) { return L.vb; }
  static double2* x(LevelData& L) { return L.vx; }
  static double2* y(LevelData& L) { return L.vy; }
  static double2* r(LevelData& L) { return L.vr; }
  static const double* K(LevelData& L) { return L.K; }
  static const double* M(LevelData& L) { return L.M; }
  static const double2* dinv(LevelData& L) { return L.dinv; }
  static const double* Pw(LevelData& L) { return L.Pw; }
  static const double* Rw(LevelData& L) { return L.Rw; }
  static const double2* cinv(iga_ctx* c) { return c->cinv; }
};
template <> struct LvBuf<float> {
  static float2* b(LevelData& L) { return L.fb; }
  static float2* x(LevelData& L) { return L.fx; }
  static float2* y(LevelData& L) { return L.fy; }
  static float2* r(LevelData& L) { return L.fr; }
  static const float* K(LevelData& L) { return L.Kf; }
  static const float* M(LevelData& L) { return L.Mf; }
  static const float2* dinv(LevelData& L) { return L.dinvf; }
  static const float* Pw(LevelData& L) { return L.Pwf; }
  static const float* Rw(LevelData& L) { return L.Rwf; }
  static const float2* cinv(iga_ctx* c) { return c->cinvf; }
};

// D^{-1} for the Jacobi sweeps where it is kept in memory: every 2D FP64 level
// (FP64 division is slow), FP32 only with variable k, and every level of a 1D
// problem with a Sommerfeld end (its last diagonal entry carries -i k); else
// formed on the fly
template <typename T>
static const typename cplx<T>::t* jac_dinv(iga_ctx* ctx, LevelData& L) {
  if (ctx->dim != 2) return ctx->robin_k != 0.0 ? LvBuf<T>::dinv(L) : nullptr;
  if (sizeof(T) == 8 || ctx->vark) return LvBuf<T>::dinv(L);
  return nullptr;
}

// 1D with a Sommerfeld end: D = K_ii + c M_ii (- i k on the last row), inverted
// in FP64 and, from the FP32 bands, in FP32
__global__ void k_robin_dinv(int nx, int p, const double* K, const double* M, const float* Kf, const float* Mf,
                             double2 c, double rk, double2* dinv, float2* dinvf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  const int W = 2 * p + 1;
  double2 d = mkc(K[(size_t)i * W + p], 0.0) + M[(size_t)i * W + p] * c;
  float2 df = mkc(Kf[(size_t)i * W + p], 0.f) + Mf[(size_t)i * W + p] * tof(c);
  if (i == nx - 1) {
    d = d + mkc(0.0, -rk);
    df = df + mkc(0.f, (float)-rk);
  }
  dinv[i] = cinv(d);
  dinvf[i] = cinv(df);
}

iga_status setup_robin_dinv(iga_ctx* ctx) {
  if (ctx->robin_k == 0.0) return IGA_OK;
  const double2 c = make_double2(-ctx->sig.x * ctx->k2const, -ctx->sig.y * ctx->k2const);
  for (int l = 0; l < ctx->L; ++l) {
    LevelData& L = ctx->lv[l];
    L.dinv = dalloc<double2>(ctx, L.n);
    L.dinvf = dalloc<float2>(ctx, L.n);
    if (!L.dinv || !L.dinvf) return set_err(ctx, IGA_E_OOM, "robin dinv");
    k_robin_dinv<<<cdiv(L.nx, 128), 128, 0, ctx->st>>>(L.nx, ctx->p, L.K, L.M, L.Kf, L.Mf, c, ctx->robin_k, L.dinv,
                                                       L.dinvf); iga_count_launch();
    CKL();
  }
  return IGA_OK;
}

template <typename T>
iga_status mg_jacobi0(iga_ctx* ctx, int l, const typename cplx<T>::t* b, typename cplx<T>::t* x) {
  using C = typename cplx<T>::t;
  LevelData& L = ctx->lv[l];
  double2 cm = make_double2(-ctx->sig.x, -ctx->sig.y);
  if (!ctx->vark) cm = ctx->k2const * cm;
  const C* dinv = jac_dinv<T>(ctx, L);
  k_jacobi0<T><<<cdiv(L.n, 256), 256, 0, ctx->st>>>(L.nx, L.ny, ctx->p, LvBuf<T>::K(L), LvBuf<T>::M(L),
                                                    cconv<C>(cm), dinv, b, x, (T)ctx->prm.omega); iga_count_launch();
  CKL();
  return IGA_OK;
}

template <typename T>
static void launch_restrict_tiled(iga_ctx* ctx, int l, const typename cplx<T>::t* f, typename cplx<T>::t* c,
                                  typename cplx<T>::t* xc, const typename cplx<T>::t* dinv) {
  using C = typename cplx<T>::t;
  LevelData& F = ctx->lv[l];
  LevelData& Cc = ctx->lv[l + 1];
  const C cm = cconv<C>(ctx->k2const * make_double2(-ctx->sig.x, -ctx->sig.y));
  dim3 g(cdiv(Cc.nx, TR_CT), cdiv(Cc.ny, TR_CT));
  const size_t sm = tr_smem<C, T>(F.tr_fmax, F.wR);
  const TrStencil<T> st = tr_stencil<T>(F);
#define IGA_RESTRICT(W_)                                                                                          \
  k_restrict_tiled<T, W_><<<g, 256, sm, ctx->st>>>(F.nx, F.ny, Cc.nx, Cc.ny, F.wR, LvBuf<T>::Rw(F), F.Rlo,       \
                                                   F.tr_fmax, f, c, xc, dinv, (T)ctx->prm.omega, ctx->p,        \
                                                   LvBuf<T>::K(Cc), LvBuf<T>::M(Cc), cm, st)
  switch (F.wR) {
    case 4: IGA_RESTRICT(4); break;
    case 5: IGA_RESTRICT(5); break;
    case 6: IGA_RESTRICT(6); break;
    case 7: IGA_RESTRICT(7); break;
    case 8: IGA_RESTRICT(8); break;
    default: IGA_RESTRICT(0); break;
  }
#undef IGA_RESTRICT
  iga_count_launch();
}

template <typename T>
iga_status mg_restrict(iga_ctx* ctx, int l, const typename cplx<T>::t* f, typename cplx<T>::t* c) {
  LevelData& F = ctx->lv[l];
  LevelData& Cc = ctx->lv[l + 1];
  if (F.tr_fmax > 0) {
    launch_restrict_tiled<T>(ctx, l, f, c, nullptr, nullptr);
    CKL();
    return IGA_OK;
  }
  k_restrict<T><<<cdiv(Cc.n, 256), 256, 0, ctx->st>>>(F.nx, F.ny, Cc.nx, Cc.ny, F.wR, LvBuf<T>::Rw(F), F.Rlo, f, c,
                                                     nullptr, 0, nullptr, nullptr, czero<typename cplx<T>::t>(),
                                                     nullptr, (T)0); iga_count_launch();
  CKL();
  return IGA_OK;
}

// c = P^T f and xc = omega D_c^{-1} c (the coarse level's first Jacobi sweep)
template <typename T>
static iga_status mg_restrict_j0(iga_ctx* ctx, int l, const typename cplx<T>::t* f, typename cplx<T>::t* c,
                                 typename cplx<T>::t* xc) {
  using C = typename cplx<T>::t;
  LevelData& F = ctx->lv[l];
  LevelData& Cc = ctx->lv[l + 1];
  double2 cm = make_double2(-ctx->sig.x, -ctx->sig.y);
  if (!ctx->vark) cm = ctx->k2const * cm;
  const C* dinv = jac_dinv<T>(ctx, Cc);
  if (F.tr_fmax > 0 && (dinv || !ctx->vark)) {   // D_c^{-1} in memory, or from constant-k bands
    launch_restrict_tiled<T>(ctx, l, f, c, xc, dinv);
    CKL();
    return IGA_OK;
  }
  k_restrict<T><<<cdiv(Cc.n, 256), 256, 0, ctx->st>>>(F.nx, F.ny, Cc.nx, Cc.ny, F.wR, LvBuf<T>::Rw(F), F.Rlo, f, c, xc,
                                                     ctx->p, LvBuf<T>::K(Cc), LvBuf<T>::M(Cc), cconv<C>(cm), dinv,
                                                     (T)ctx->prm.omega); iga_count_launch();
  CKL();
  return IGA_OK;
}

template <typename T>
iga_status mg_prolong_add(iga_ctx* ctx, int l, const typename cplx<T>::t* c, typename cplx<T>::t* f) {
  using C = typename cplx<T>::t;
  LevelData& F = ctx->lv[l];
  LevelData& Cc = ctx->lv[l + 1];
  if (F.tp_cmax > 0) {
    if (F.nx >= 1024) {        // large level: 32 x 32 tiles, four rows per warp
      dim3 g(cdiv(F.nx, TP_TX), cdiv(F.ny, 32));
      k_prolong_tiled<T, 32><<<g, 256, tp_smem<C, T>(F.tp_cmax, F.wP, 32), ctx->st>>>(
          F.nx, F.ny, Cc.nx, Cc.ny, F.wP, LvBuf<T>::Pw(F), F.Plo, F.tp_cmax, c, f);
    } else {                   // enough blocks to fill the GPU on small levels
      dim3 g(cdiv(F.nx, TP_TX), cdiv(F.ny, 8));
      k_prolong_tiled<T, 8><<<g, 256, tp_smem<C, T>(F.tp_cmax, F.wP, 8), ctx->st>>>(
          F.nx, F.ny, Cc.nx, Cc.ny, F.wP, LvBuf<T>::Pw(F), F.Plo, F.tp_cmax, c, f);
    }
    iga_count_launch();
    CKL();
    return IGA_OK;
  }
  k_prolong_add<T><<<cdiv(F.n, 256), 256, 0, ctx->st>>>(F.nx, F.ny, Cc.nx, Cc.ny, F.wP, LvBuf<T>::Pw(F), F.Plo, c, f); iga_count_launch();
  CKL();
  return IGA_OK;
}

template <typename T>
iga_status mg_coarse(iga_ctx* ctx, const typename cplx<T>::t* b, typename cplx<T>::t* x) {
  using C = typename cplx<T>::t;
  if (ctx->coarse_banded) {
    if constexpr (sizeof(T) == 8) return band_solve(ctx, ctx->bandC, b, x);
    else {
      launch_convert_f2d(b, ctx->cband_t, ctx->nc, ctx->st);
      TRY(band_solve(ctx, ctx->bandC, ctx->cband_t, ctx->cband_x));
      launch_convert_d2f(ctx->cband_x, x, ctx->nc, ctx->st);
      CKL();
      return IGA_OK;
    }
  }
  k_dense_mv<C><<<cdiv(ctx->nc, 8), 256, 0, ctx->st>>>(ctx->nc, LvBuf<T>::cinv(ctx), b, x); iga_count_launch();
  CKL();
  return IGA_OK;
}

// One V-cycle on level l for M_beta x = b from x = 0.  The result is written to
// `out`; `alt` is a second level-sized buffer used for Jacobi ping-pong.
// Buffer (out or alt) in which level l's pre-smoothing starts, so that the
// last post-sweep lands in `out`.
static int start_buffer(iga_ctx* ctx) {
  const int nu1 = ctx->prm.nu_pre, nu2 = ctx->prm.nu_post;
  const int before_post = nu2 & 1;
  return (nu1 >= 1) ? (before_post ^ ((nu1 - 1) & 1)) : before_post;
}

// pre_done: the first Jacobi sweep (from zero) was already written into the
// start buffer by the parent's fused restriction.
template <typename T>
static iga_status vcycle_level(iga_ctx* ctx, int l, const typename cplx<T>::t* b, typename cplx<T>::t* out,
                               typename cplx<T>::t* alt, bool pre_done = false) {
  using C = typename cplx<T>::t;
  LevelData& L = ctx->lv[l];
  if (l == ctx->L - 1) return mg_coarse<T>(ctx, b, out);
  const int nu1 = ctx->prm.nu_pre, nu2 = ctx->prm.nu_post;
  const double om = ctx->prm.omega;
  // Choose the buffer the pre-smoother starts in so that, after the nu2
  // post-sweeps (each flips the buffer), the result lands in `out`.
  C* bufs[2] = {out, alt};
  int cur = start_buffer(ctx);
  if (nu1 >= 1) {
    if (!pre_done) TRY(mg_jacobi0<T>(ctx, l, b, bufs[cur]));
    for (int s = 1; s < nu1; ++s) {
      TRY(op_apply<T>(ctx, l, OP_MB, bufs[cur], bufs[cur ^ 1], nullptr, EPI_JACOBI, b, om));
      cur ^= 1;
    }
  } else {
    CK(cudaMemsetAsync(bufs[cur], 0, sizeof(C) * L.n, ctx->st));
  }
  C* r = LvBuf<T>::r(L);
  if (nu1 >= 1) {
    TRY(op_apply<T>(ctx, l, OP_MB, bufs[cur], r, b, EPI_ZMINUS, nullptr, 0.0));
  } else {
    CK(cudaMemcpyAsync(r, b, sizeof(C) * L.n, cudaMemcpyDeviceToDevice, ctx->st));
  }
  LevelData& Cl = ctx->lv[l + 1];
  if (nu1 >= 1 && l + 1 < ctx->L - 1) {
    C* cstart = start_buffer(ctx) ? LvBuf<T>::y(Cl) : LvBuf<T>::x(Cl);
    TRY(mg_restrict_j0<T>(ctx, l, r, LvBuf<T>::b(Cl), cstart));
    TRY(vcycle_level<T>(ctx, l + 1, LvBuf<T>::b(Cl), LvBuf<T>::x(Cl), LvBuf<T>::y(Cl), true));
  } else {
    TRY(mg_restrict<T>(ctx, l, r, LvBuf<T>::b(Cl)));
    TRY(vcycle_level<T>(ctx, l + 1, LvBuf<T>::b(Cl), LvBuf<T>::x(Cl), LvBuf<T>::y(Cl)));
  }
  TRY(mg_prolong_add<T>(ctx, l, LvBuf<T>::x(Cl), bufs[cur]));
  for (int s = 0; s < nu2; ++s) {
    TRY(op_apply<T>(ctx, l, OP_MB, bufs[cur], bufs[cur ^ 1], nullptr, EPI_JACOBI, b, om));
    cur ^= 1;
  }
  if (cur != 0) CK(cudaMemcpyAsync(out, bufs[cur], sizeof(C) * L.n, cudaMemcpyDeviceToDevice, ctx->st));
  return IGA_OK;
}

// z = n_vcycles V-cycles applied to r on the finest level (stationary
// iteration z <- z + V(r - M_beta z) from z = 0).
// one V-cycle from zero on the finest level: the fused level kernels where they
// apply (2D, constant k, one pre- and one post-sweep, FP32), else operation by
// operation
// (in FP64 the halo recomputation costs more FP64 work than the saved
// launches are worth)
template <typename T>
static iga_status vcycle0(iga_ctx* ctx, const typename cplx<T>::t* b, typename cplx<T>::t* out) {
  if (ctx->vc_fused && sizeof(T) == 4) return mg_vcycle_fused<T>(ctx, b, out);
  return vcycle_level<T>(ctx, 0, b, out, LvBuf<T>::y(ctx->lv[0]));
}

template <typename T>
iga_status mg_vcycle(iga_ctx* ctx, const typename cplx<T>::t* r, typename cplx<T>::t* z) {
  using C = typename cplx<T>::t;
  LevelData& L = ctx->lv[0];
  TRY(vcycle0<T>(ctx, r, z));
  for (int c = 1; c < ctx->prm.n_vcycles; ++c) {
    C* res = LvBuf<T>::b(L);
    C* e = LvBuf<T>::x(L);
    TRY(op_apply<T>(ctx, 0, OP_MB, z, res, r, EPI_ZMINUS, nullptr, 0.0));
    TRY(vcycle0<T>(ctx, res, e));
    k_axpy1<C><<<cdiv(L.n, 256), 256, 0, ctx->st>>>(z, e, L.n); iga_count_launch();
    CKL();
  }
  return IGA_OK;
}

// FP32 V-cycle z ~ M_beta^{-1} r with complex128 r and z.  Where the finest
// level's FP32 sweeps run on the register-stencil kernel (2D, constant k, one
// pre-sweep, one V-cycle, per-operation V-cycle) the conversions are folded
// into the first and last finest-level kernels: the pre-sweep from zero reads
// r and also stores its FP32 copy, the last post-sweep writes z in
// complex128.  The operations are those of converting, the FP32 V-cycle and
// converting back (the compiler may contract them differently, so the two
// agree to FP32 rounding); otherwise that is what runs.
iga_status mg_vcycle32_c128(iga_ctx* ctx, const double2* r, double2* z) {
  LevelData& L = ctx->lv[0];
  const int nu2 = ctx->prm.nu_post;
  const bool fold = ctx->dim == 2 && !ctx->vark && !ctx->vc_fused && ctx->L > 1 && ctx->prm.nu_pre == 1 &&
                    nu2 >= 1 && ctx->prm.n_vcycles == 1 && ctx->tile[0][1] == 6;
  if (!fold) {
    launch_convert_d2f(r, ctx->fin, L.n, ctx->st);
    TRY(mg_vcycle<float>(ctx, ctx->fin, ctx->fout));
    launch_convert_f2d(ctx->fout, z, L.n, ctx->st);
    CKL();
    return IGA_OK;
  }
  float2* b32 = ctx->fin;
  float2* bufs[2] = {ctx->fout, L.fy};
  int cur = 0;
  const double2 cm = make_double2(-ctx->sig.x * ctx->k2const, -ctx->sig.y * ctx->k2const);
  k_jacobi0_in128<<<cdiv(L.n, 256), 256, 0, ctx->st>>>(L.nx, L.ny, ctx->p, L.Kf, L.Mf, tof(cm), r, b32, bufs[cur],
                                                       (float)ctx->prm.omega); iga_count_launch();
  TRY(op_apply<float>(ctx, 0, OP_MB, bufs[cur], L.fr, b32, EPI_ZMINUS, nullptr, 0.0));
  LevelData& Cl = ctx->lv[1];
  if (ctx->L > 2) {
    float2* cstart = start_buffer(ctx) ? Cl.fy : Cl.fx;
    TRY(mg_restrict_j0<float>(ctx, 0, L.fr, Cl.fb, cstart));
    TRY(vcycle_level<float>(ctx, 1, Cl.fb, Cl.fx, Cl.fy, true));
  } else {
    TRY(mg_restrict<float>(ctx, 0, L.fr, Cl.fb));
    TRY(vcycle_level<float>(ctx, 1, Cl.fb, Cl.fx, Cl.fy));
  }
  TRY(mg_prolong_add<float>(ctx, 0, Cl.fx, bufs[cur]));
  for (int s = 0; s + 1 < nu2; ++s) {
    TRY(op_apply<float>(ctx, 0, OP_MB, bufs[cur], bufs[cur ^ 1], nullptr, EPI_JACOBI, b32, ctx->prm.omega));
    cur ^= 1;
  }
  return sweep32_jacobi_out64(ctx, 0, bufs[cur], z, b32);
}

template iga_status mg_vcycle<double>(iga_ctx*, const double2*, double2*);
template iga_status mg_vcycle<float>(iga_ctx*, const float2*, float2*);
template iga_status mg_restrict<double>(iga_ctx*, int, const double2*, double2*);
template iga_status mg_prolong_add<double>(iga_ctx*, int, const double2*, double2*);
template iga_status mg_coarse<double>(iga_ctx*, const double2*, double2*);
template iga_status mg_coarse<float>(iga_ctx*, const float2*, float2*);
template iga_status mg_jacobi0<double>(iga_ctx*, int, const double2*, double2*);
