// Matrix-free IgA Helmholtz operators (Section 2.3, Eq. linearsystem1 with
// A = S - M^{k^2}; Section 3, CSLP M_beta = S - (beta1 - i beta2) M^{k^2}).
//
// Constant k: Op = M_y (x) (K_x + c M_x) + K_y (x) M_x applied as two banded
// 1D passes through a shared-memory tile with a p-wide halo:
//   y-pass  u = M_y x,  w = c u + K_y x     (tile rows, columns of tile + halo)
//   x-pass  y = K_x u + M_x w
// c = -k^2 for A and -(beta1 - i beta2) k^2 for M_beta.
//
// Variable k: S by the same banded passes, the k^2-mass by per-element
// sum factorisation in the tile: interpolate to the Gauss points along x,
// then y, weight by w_x w_y k^2(x_q, y_q), project back along y, then x.
//
// Epilogues fuse what follows the apply: y = Op x, y = z - Op x (residual,
// deflation), or one damped Jacobi sweep x_out = x + omega D^{-1} (b - Op x).
#include "common.cuh"

template <typename T> struct OpArgs {
  using C = typename cplx<T>::t;
  int nx, ny, n_el;
  const T* K;          // bands [nx][2p+1]
  const T* M;
  C c;                 // coefficient of the (k^2-)mass term
  const C* x;
  C* y;
  const C* z;          // EPI_ZMINUS: minuend; EPI_JACOBI: right-hand side b
  const C* dinv;       // EPI_JACOBI with variable k: precomputed D^{-1}
  float2* yf;          // EPI_ZMINUS: optional FP32 copy of y (nullptr: none)
  T omega;
  T rk;                // 1D Sommerfeld end: the last row adds -i rk x_last (0: none)
  // variable k
  const T* B;          // [n_el][Q][p+1]
  const T* wq;         // [n_el][Q]
  const double* xq;    // [n_el][Q]
};

struct KFieldF {
  int n_lines;
  float lines[IGA_MAX_LINES][3];
  float k2[IGA_MAX_LINES + 1];
};

template <typename T> struct KSel;
template <> struct KSel<double> {
  using KF = KFieldDev;
  static __device__ __forceinline__ double k2(const KFieldDev& kf, double x, double y) { return kfield_k2(kf, x, y); }
};
template <> struct KSel<float> {
  using KF = KFieldF;
  static __device__ __forceinline__ float k2(const KFieldF& kf, double xd, double yd) {
    float x = (float)xd, y = (float)yd;
    int cnt = 0;
    for (int l = 0; l < kf.n_lines; ++l) {
      float s = __fadd_rn(__fadd_rn(__fmul_rn(kf.lines[l][0], x), __fmul_rn(kf.lines[l][1], y)), kf.lines[l][2]);
      cnt += (s >= 0.f);
    }
    return kf.k2[cnt];
  }
};

template <typename T, int EPI>
__device__ __forceinline__ void epilogue(const OpArgs<T>& a, size_t o, typename cplx<T>::t acc,
                                         typename cplx<T>::t xo, typename cplx<T>::t diag) {
  using C = typename cplx<T>::t;
  if (EPI == EPI_Y) {
    a.y[o] = acc;
  } else if (EPI == EPI_ZMINUS) {
    const C v = a.z[o] - acc;
    a.y[o] = v;
    if constexpr (sizeof(T) == 8) {
      if (a.yf) a.yf[o] = tof(v);
    }
  } else {
    C r = a.z[o] - acc;
    C di = a.dinv ? a.dinv[o] : cinv(diag);
    a.y[o] = xo + a.omega * cmul(di, r);
  }
}

// ------------------------------------------------------------------ 1D
template <int P, typename T, int EPI>
__global__ void __launch_bounds__(256) k_kron1d(OpArgs<T> a) {
  using C = typename cplx<T>::t;
  constexpr int W = 2 * P + 1;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nx) return;
  C s1 = czero<C>(), s2 = czero<C>();
#pragma unroll
  for (int d = 0; d < W; ++d) {
    int j = i + d - P;
    if (j >= 0 && j < a.nx) {
      C v = a.x[j];
      s1 = cfma(a.K[(size_t)i * W + d], v, s1);
      s2 = cfma(a.M[(size_t)i * W + d], v, s2);
    }
  }
  C acc = s1 + cmul(a.c, s2);
  const bool bnd = a.rk != (T)0 && i == a.nx - 1;   // boundary mass N at the Sommerfeld end
  if (bnd) {
    const C v = a.x[i];
    acc = acc + mkc(a.rk * v.y, -a.rk * v.x);       // - i rk x_last
  }
  C diag = czero<C>();
  if (EPI == EPI_JACOBI) {
    T kd = a.K[(size_t)i * W + P], md = a.M[(size_t)i * W + P];
    diag = mkc(kd, (T)0) + md * a.c;
    if (bnd) diag = diag + mkc((T)0, -a.rk);
  }
  epilogue<T, EPI>(a, i, acc, EPI == EPI_JACOBI ? a.x[i] : czero<C>(), diag);
}

// ------------------------------------------------------------------ 2D constant k
// Tile shapes (TX x TY outputs per 256-thread block): 32 x 16 for large grids,
// 16 x 16 when the large tile would leave the SMs under-filled.
template <int P, typename T, int TX, int TY>
constexpr size_t kron2d_smem() {
  using C = typename cplx<T>::t;
  return sizeof(C) * ((TY + 2 * P) * (TX + 2 * P) + 2 * TY * (TX + 2 * P)) + sizeof(T) * (2 * TX + 2 * TY) * (2 * P + 1);
}

template <int P, typename T, int EPI, int TX, int TY, int NT = 256>
__global__ void __launch_bounds__(NT) k_kron2d(OpArgs<T> a) {
  using C = typename cplx<T>::t;
  constexpr int W = 2 * P + 1, SX = TX + 2 * P, SY = TY + 2 * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* xs = (C*)smem_raw;
  C* us = xs + SY * SX;           // [TY][SX]  M_y x
  C* ws = us + TY * SX;           // [TY][SX]  c M_y x + K_y x
  T* kx = (T*)(ws + TY * SX);
  T* mx = kx + TX * W;
  T* ky = mx + TX * W;
  T* my = ky + TY * W;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nx = a.nx, ny = a.ny;
  for (int i = tid; i < SY * SX; i += NT) {
    int r = i / SX, c = i - r * SX;
    int gy = y0 - P + r, gx = x0 - P + c;
    xs[i] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? a.x[(size_t)gy * nx + gx] : czero<C>();
  }
  for (int i = tid; i < TX * W; i += NT) {
    int c = i / W, gx = x0 + c;
    kx[i] = gx < nx ? a.K[(size_t)x0 * W + i] : (T)0;
    mx[i] = gx < nx ? a.M[(size_t)x0 * W + i] : (T)0;
  }
  for (int i = tid; i < TY * W; i += NT) {
    int r = i / W, gy = y0 + r;
    ky[i] = gy < ny ? a.K[(size_t)y0 * W + i] : (T)0;
    my[i] = gy < ny ? a.M[(size_t)y0 * W + i] : (T)0;
  }
  __syncthreads();
  // pass along y over the tile rows and all halo columns (the halo of the
  // wider tile side is the one recomputed, so the first pass does the least
  // redundant work): u = M_y x, w = c u + K_y x
  for (int i = tid; i < TY * SX; i += NT) {
    int r = i / SX, c = i - r * SX;
    C s1 = czero<C>(), s2 = czero<C>();
#pragma unroll
    for (int d = 0; d < W; ++d) {
      C v = xs[(r + d) * SX + c];
      s1 = cfma(my[r * W + d], v, s1);
      s2 = cfma(ky[r * W + d], v, s2);
    }
    us[i] = s1;
    ws[i] = cmul(a.c, s1) + s2;
  }
  __syncthreads();
  // pass along x: Op x = K_x u + M_x w
  for (int i = tid; i < TY * TX; i += NT) {
    int r = i / TX, c = i - r * TX;
    int gy = y0 + r, gx = x0 + c;
    if (gy >= ny || gx >= nx) continue;
    C acc = czero<C>();
#pragma unroll
    for (int d = 0; d < W; ++d) {
      acc = cfma(kx[c * W + d], us[r * SX + c + d], acc);
      acc = cfma(mx[c * W + d], ws[r * SX + c + d], acc);
    }
    C diag = czero<C>();
    if (EPI == EPI_JACOBI) {
      T kxd = kx[c * W + P], mxd = mx[c * W + P], kyd = ky[r * W + P], myd = my[r * W + P];
      diag = myd * (mkc(kxd, (T)0) + mxd * a.c) + mkc(kyd * mxd, (T)0);
    }
    epilogue<T, EPI>(a, (size_t)gy * nx + gx, acc, xs[(r + P) * SX + c + P], diag);
  }
}

// ------------------------------------------------------------------ 2D constant k, FP64 lane pairs
// The same two banded passes for small FP64 grids, with the real and the
// imaginary part of every complex value on a lane pair (lane ^ 1): a thread
// carries half as many FP64 FMA chains per pass.  On a small level the
// time is the FP64 warp instructions each SM sub-partition issues (one per
// 64 cycles on this part), and those are what the split halves.  The complex
// factors (the mass coefficient c, D^{-1}) take the partner's component by a
// shuffle.  Every thread runs the same number of rounds, so the shuffles see
// full warps.
template <int P, int TX, int TY>
constexpr size_t kron2d_pair_smem() {
  return sizeof(double2) * (TY + 2 * P) * (TX + 2 * P) + sizeof(double) * 4 * TY * (TX + 2 * P) +
         sizeof(double) * (2 * TX + 2 * TY) * (2 * P + 1);
}

template <int P, int EPI, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_kron2d_pair(OpArgs<double> a) {
  constexpr int W = 2 * P + 1, SX = TX + 2 * P, SY = TY + 2 * P;
  static_assert(NT % 32 == 0, "whole warps");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* xs = (double2*)smem_raw;            // [SY][SX]
  double* us = (double*)(xs + SY * SX);         // [TY][SX][re, im]  M_y x
  double* ws = us + 2 * TY * SX;                // [TY][SX][re, im]  c M_y x + K_y x
  double* kx = ws + 2 * TY * SX;
  double* mx = kx + TX * W;
  double* ky = mx + TX * W;
  double* my = ky + TY * W;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nx = a.nx, ny = a.ny;
  for (int i = tid; i < SY * SX; i += NT) {
    int r = i / SX, c = i - r * SX;
    int gy = y0 - P + r, gx = x0 - P + c;
    xs[i] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? a.x[(size_t)gy * nx + gx] : make_double2(0.0, 0.0);
  }
  for (int i = tid; i < TX * W; i += NT) {
    int c = i / W, gx = x0 + c;
    kx[i] = gx < nx ? a.K[(size_t)x0 * W + i] : 0.0;
    mx[i] = gx < nx ? a.M[(size_t)x0 * W + i] : 0.0;
  }
  for (int i = tid; i < TY * W; i += NT) {
    int r = i / W, gy = y0 + r;
    ky[i] = gy < ny ? a.K[(size_t)y0 * W + i] : 0.0;
    my[i] = gy < ny ? a.M[(size_t)y0 * W + i] : 0.0;
  }
  __syncthreads();
  const double* xd = (const double*)xs;
  const double cre = a.c.x, cim = a.c.y;
  // pass along y (tile rows, all halo columns); task q = 2 * point + component
  constexpr int NY = 2 * TY * SX;
  for (int base = 0; base < NY; base += NT) {
    const int t = base + tid;
    const int q = t < NY ? t : 0;
    const int comp = q & 1, pt = q >> 1;
    const int r = pt / SX, c = pt - r * SX;
    double s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int d = 0; d < W; ++d) {
      const double v = xd[2 * ((r + d) * SX + c) + comp];
      s1 = fma(my[r * W + d], v, s1);
      s2 = fma(ky[r * W + d], v, s2);
    }
    // w = c u + K_y x:  re = cre u_re - cim u_im + s2_re,  im = cre u_im + cim u_re + s2_im
    const double so = __shfl_xor_sync(0xffffffffu, s1, 1);
    const double w = fma(cre, s1, fma(comp ? cim : -cim, so, s2));
    if (t < NY) {
      us[q] = s1;
      ws[q] = w;
    }
  }
  __syncthreads();
  // pass along x: Op x = K_x u + M_x w, then the epilogue per component
  constexpr int NXT = 2 * TY * TX;
  for (int base = 0; base < NXT; base += NT) {
    const int t = base + tid;
    const int q = t < NXT ? t : 0;
    const int comp = q & 1, pt = q >> 1;
    const int r = pt / TX, c = pt - r * TX;
    const int gy = y0 + r, gx = x0 + c;
    const bool ok = t < NXT && gy < ny && gx < nx;
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < W; ++d) {
      const int s = 2 * (r * SX + c + d) + comp;
      acc = fma(kx[c * W + d], us[s], acc);
      acc = fma(mx[c * W + d], ws[s], acc);
    }
    // clamped into the grid so that every lane may read (only `ok` lanes store)
    const size_t o = (size_t)min(gy, ny - 1) * nx + min(gx, nx - 1);
    if (EPI == EPI_Y) {
      if (ok) ((double*)(a.y + o))[comp] = acc;
    } else if (EPI == EPI_ZMINUS) {
      if (ok) {
        const double v = ((const double*)(a.z + o))[comp] - acc;
        ((double*)(a.y + o))[comp] = v;
        if (a.yf) ((float*)(a.yf + o))[comp] = (float)v;
      }
    } else {
      // x_out = x + omega D^{-1} (b - Op x)
      const double res = ((const double*)(a.z + o))[comp] - acc;
      const double ro = __shfl_xor_sync(0xffffffffu, res, 1);
      double2 di;
      if (a.dinv) {
        di = a.dinv[o];
      } else {
        const double kxd = kx[c * W + P], mxd = mx[c * W + P], kyd = ky[r * W + P], myd = my[r * W + P];
        di = cinv(myd * (make_double2(kxd, 0.0) + mxd * a.c) + make_double2(kyd * mxd, 0.0));
      }
      const double dr = fma(di.x, res, (comp ? di.y : -di.y) * ro);
      if (ok) ((double*)(a.y + o))[comp] = fma(a.omega, dr, xd[2 * ((r + P) * SX + c + P) + comp]);
    }
  }
}

// ------------------------------------------------------------------ 2D variable k
constexpr int EL_T = 8;

template <int P, typename T>
constexpr size_t elem2d_smem() {
  using C = typename cplx<T>::t;
  constexpr int Q = P + 1, E = EL_T + P, SX = EL_T + 2 * P;
  return sizeof(C) * (SX * SX + SX * E * Q + (E * Q) * (E * Q) + EL_T * EL_T) + sizeof(double) * 2 * E * Q +
         sizeof(T) * (2 * E * Q * Q + 2 * E * Q);
}

template <int P, typename T, int EPI>
__global__ void __launch_bounds__(256) k_elem2d(OpArgs<T> a, typename KSel<T>::KF kf) {
  using C = typename cplx<T>::t;
  constexpr int Q = P + 1, TT = EL_T, E = TT + P, SX = TT + 2 * P, W = 2 * P + 1, EQ = E * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* X = (C*)smem_raw;          // [SX][SX]
  C* V = X + SX * SX;           // [SX][E][Q]  (also stiffness temporaries, then T4)
  C* U = V + SX * E * Q;        // [E][Q][E][Q]
  C* Ys = U + EQ * EQ;          // [TT][TT]
  double* xqx = (double*)(Ys + TT * TT);
  double* xqy = xqx + EQ;
  T* Bx = (T*)(xqy + EQ);       // [E][Q][Q]
  T* By = Bx + E * Q * Q;
  T* wx = By + E * Q * Q;       // [E][Q]
  T* wy = wx + EQ;
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny, N = a.n_el;
  const int ix0 = blockIdx.x * TT, iy0 = blockIdx.y * TT;
  const int ex0 = ix0 + 1 - P, ey0 = iy0 + 1 - P;   // first element of the tile (may be < 0)

  for (int i = tid; i < SX * SX; i += 256) {
    int r = i / SX, c = i - r * SX;
    int gy = iy0 - P + r, gx = ix0 - P + c;
    X[i] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? a.x[(size_t)gy * nx + gx] : czero<C>();
  }
  for (int i = tid; i < E * Q * Q; i += 256) {
    int el = i / (Q * Q), rest = i - el * Q * Q;
    int ex = ex0 + el, ey = ey0 + el;
    Bx[i] = (ex >= 0 && ex < N) ? a.B[(size_t)ex * Q * Q + rest] : (T)0;
    By[i] = (ey >= 0 && ey < N) ? a.B[(size_t)ey * Q * Q + rest] : (T)0;
  }
  for (int i = tid; i < EQ; i += 256) {
    int el = i / Q, q = i - el * Q;
    int ex = ex0 + el, ey = ey0 + el;
    bool vx = ex >= 0 && ex < N, vy = ey >= 0 && ey < N;
    wx[i] = vx ? a.wq[ex * Q + q] : (T)0;
    wy[i] = vy ? a.wq[ey * Q + q] : (T)0;
    xqx[i] = vx ? a.xq[ex * Q + q] : 0.0;
    xqy[i] = vy ? a.xq[ey * Q + q] : 0.0;
  }
  __syncthreads();

  // stiffness S = M_y (x) K_x + K_y (x) M_x on the tile
  C* t1 = V;
  C* t2 = V + SX * TT;
  for (int i = tid; i < SX * TT; i += 256) {
    int r = i / TT, c = i - r * TT;
    int gx = ix0 + c;
    C s1 = czero<C>(), s2 = czero<C>();
    if (gx < nx) {
#pragma unroll
      for (int d = 0; d < W; ++d) {
        C v = X[r * SX + c + d];
        s1 = cfma(a.K[(size_t)gx * W + d], v, s1);
        s2 = cfma(a.M[(size_t)gx * W + d], v, s2);
      }
    }
    t1[i] = s1;
    t2[i] = s2;
  }
  __syncthreads();
  for (int i = tid; i < TT * TT; i += 256) {
    int r = i / TT, c = i - r * TT;
    int gy = iy0 + r;
    C acc = czero<C>();
    if (gy < ny) {
#pragma unroll
      for (int d = 0; d < W; ++d) {
        acc = cfma(a.M[(size_t)gy * W + d], t1[(r + d) * TT + c], acc);
        acc = cfma(a.K[(size_t)gy * W + d], t2[(r + d) * TT + c], acc);
      }
    }
    Ys[i] = acc;
  }
  __syncthreads();

  // S2: interpolate along x: V[ry][el][qx] = sum_a Bx[el][qx][a] X[ry][el + a]
  for (int i = tid; i < SX * EQ; i += 256) {
    int ry = i / EQ, rest = i - ry * EQ;
    int el = rest / Q, q = rest - el * Q;
    C s = czero<C>();
#pragma unroll
    for (int aa = 0; aa <= P; ++aa) s = cfma(Bx[(el * Q + q) * Q + aa], X[ry * SX + el + aa], s);
    V[i] = s;
  }
  __syncthreads();
  // S3: interpolate along y and weight: U[ely][qy][elx][qx]
  for (int i = tid; i < EQ * EQ; i += 256) {
    int ry = i / EQ, cx = i - ry * EQ;        // ry = ely*Q + qy, cx = elx*Q + qx
    int ely = ry / Q, qy = ry - ely * Q;
    C s = czero<C>();
#pragma unroll
    for (int b = 0; b <= P; ++b) s = cfma(By[(ely * Q + qy) * Q + b], V[(ely + b) * EQ + cx], s);
    T w = wx[cx] * wy[ry];
    T k2 = (w != (T)0) ? KSel<T>::k2(kf, xqx[cx], xqy[ry]) : (T)0;
    U[i] = (w * k2) * s;
  }
  __syncthreads();
  // S4: project along y onto the output rows: T4[r][elx][qx]
  C* T4 = V;
  for (int i = tid; i < TT * EQ; i += 256) {
    int r = i / EQ, cx = i - r * EQ;
    C s = czero<C>();
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      int ely = r + P - b;
      if (ely >= 0 && ely < E) {
#pragma unroll
        for (int qy = 0; qy < Q; ++qy) s = cfma(By[(ely * Q + qy) * Q + b], U[(ely * Q + qy) * EQ + cx], s);
      }
    }
    T4[i] = s;
  }
  __syncthreads();
  // S5: project along x, add the stiffness part, epilogue
  for (int i = tid; i < TT * TT; i += 256) {
    int r = i / TT, c = i - r * TT;
    int gy = iy0 + r, gx = ix0 + c;
    if (gy >= ny || gx >= nx) continue;
    C s = czero<C>();
#pragma unroll
    for (int aa = 0; aa <= P; ++aa) {
      int elx = c + P - aa;
      if (elx >= 0 && elx < E) {
#pragma unroll
        for (int qx = 0; qx < Q; ++qx) s = cfma(Bx[(elx * Q + qx) * Q + aa], T4[r * EQ + elx * Q + qx], s);
      }
    }
    C acc = Ys[i] + cmul(a.c, s);
    epilogue<T, EPI>(a, (size_t)gy * nx + gx, acc, X[(r + P) * SX + c + P], czero<C>());
  }
}

// Inverse diagonal of M_beta = S - sigma M^{k^2} for variable k, thread per dof.
__global__ void k_vark_diag(int nx, int n_el, int p, const double* K, const double* M, const double* B,
                            const double* wq, const double* xq, KFieldDev kf, double2 c, double2* dinv,
                            float2* dinvf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx * nx) return;
  int iy = i / nx, ix = i - iy * nx;
  int W = 2 * p + 1, Q = p + 1;
  double s = M[(size_t)iy * W + p] * K[(size_t)ix * W + p] + K[(size_t)iy * W + p] * M[(size_t)ix * W + p];
  int bx = ix + 1, by = iy + 1;
  double mk = 0.0;
  for (int ey = max(by - p, 0); ey <= min(by, n_el - 1); ++ey)
    for (int ex = max(bx - p, 0); ex <= min(bx, n_el - 1); ++ex)
      for (int qy = 0; qy < Q; ++qy)
        for (int qx = 0; qx < Q; ++qx) {
          double vx = B[((size_t)ex * Q + qx) * Q + (bx - ex)];
          double vy = B[((size_t)ey * Q + qy) * Q + (by - ey)];
          double k2 = kfield_k2(kf, xq[ex * Q + qx], xq[ey * Q + qy]);
          mk += wq[ex * Q + qx] * wq[ey * Q + qy] * k2 * vx * vx * vy * vy;
        }
  double2 d = make_double2(s, 0.0) + mk * c;
  double2 di = cinv(d);
  dinv[i] = di;
  dinvf[i] = tof(di);
}

// ------------------------------------------------------------------ host dispatch
template <int P, typename T, int EPI, int TX, int TY, int NT = 256>
static void launch_kron_tile(const OpArgs<T>& a, cudaStream_t st) {
  constexpr size_t sm = kron2d_smem<P, T, TX, TY>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_kron2d<P, T, EPI, TX, TY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  dim3 grid(cdiv(a.nx, TX), cdiv(a.ny, TY));
  k_kron2d<P, T, EPI, TX, TY, NT><<<grid, NT, sm, st>>>(a); iga_count_launch();
}

// 8 x 8 tiles with 64 threads: on small levels (and the coarse E grid) more,
// smaller blocks spread the FP64 dependency chains over more SMs
template <int P, typename T, int EPI>
static void launch_kron_small(const OpArgs<T>& a, cudaStream_t st) { launch_kron_tile<P, T, EPI, 8, 8, 64>(a, st); }

// FP64 lane-pair tiles: 4 = 8 x 8 outputs per 256-thread block, 5 = 8 x 4 per 128
template <int P, int EPI, int TX, int TY, int NT>
static void launch_kron_pair_tile(const OpArgs<double>& a, cudaStream_t st) {
  constexpr size_t sm = kron2d_pair_smem<P, TX, TY>();
  static_assert(sm <= 48 * 1024, "default shared-memory limit");
  dim3 grid(cdiv(a.nx, TX), cdiv(a.ny, TY));
  k_kron2d_pair<P, EPI, TX, TY, NT><<<grid, NT, sm, st>>>(a); iga_count_launch();
}

template <int P, int EPI>
static void launch_kron_pair(const OpArgs<double>& a, cudaStream_t st, int tile) {
  if (tile == 4) launch_kron_pair_tile<P, EPI, 8, 8, 256>(a, st);
  else launch_kron_pair_tile<P, EPI, 8, 4, 128>(a, st);
}

void sweep32_launch(const LevelData& L, int p, int epi, const float2* x, float2* y, const float2* z, float2 cm,
                    float omega, cudaStream_t st);

template <int P, typename T, int EPI>
static void launch_op(iga_ctx* ctx, const OpArgs<T>& a, int level) {
  cudaStream_t st = ctx->st;
  if (ctx->dim == 1) {
    k_kron1d<P, T, EPI><<<cdiv(a.nx, 256), 256, 0, st>>>(a); iga_count_launch();
  } else if (!ctx->vark) {
    int tile = ctx->tile[level][sizeof(T) == 8 ? 0 : 1];
    if (tile < 0) {   // untuned: heuristic
      size_t big = (size_t)cdiv(a.nx, 32) * cdiv(a.ny, 16);
      size_t mid = (size_t)cdiv(a.nx, 16) * cdiv(a.ny, 16);
      // FP64 dependency chains favour more, smaller blocks on small grids
      tile = big >= (size_t)3 * ctx->num_sms ? 0 : (mid >= (size_t)ctx->num_sms || sizeof(T) == 4 ? 1 : 3);
    }
    if constexpr (sizeof(T) == 4) {
      if (tile == 6) {
        sweep32_launch(ctx->lv[level], P, EPI, a.x, a.y, a.z, a.c, a.omega, st);
        return;
      }
    }
    if (tile == 0) launch_kron_tile<P, T, EPI, 32, 16>(a, st);
    else if (tile == 1) launch_kron_tile<P, T, EPI, 16, 16>(a, st);
    else if (tile == 2) launch_kron_tile<P, T, EPI, 32, 8>(a, st);
    else if (tile == 3) launch_kron_small<P, T, EPI>(a, st);
    else if constexpr (sizeof(T) == 8) launch_kron_pair<P, EPI>(a, st, tile);
    else launch_kron_small<P, T, EPI>(a, st);
  } else {
    constexpr size_t sm = elem2d_smem<P, T>();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_elem2d<P, T, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      attr = true;
    }
    dim3 grid(cdiv(a.nx, EL_T), cdiv(a.ny, EL_T));
    typename KSel<T>::KF kf;
    if constexpr (sizeof(T) == 8) {
      kf = ctx->kf;
    } else {
      kf.n_lines = ctx->kf.n_lines;
      for (int l = 0; l < IGA_MAX_LINES; ++l)
        for (int c = 0; c < 3; ++c) kf.lines[l][c] = (float)ctx->kf.lines[l][c];
      for (int l = 0; l <= IGA_MAX_LINES; ++l) kf.k2[l] = (float)ctx->kf.k2[l];
    }
    k_elem2d<P, T, EPI><<<grid, 256, sm, st>>>(a, kf); iga_count_launch();
  }
  (void)level;
}

template <int P, typename T>
static void launch_epi(iga_ctx* ctx, const OpArgs<T>& a, int level, int epi) {
  if (epi == EPI_Y) launch_op<P, T, EPI_Y>(ctx, a, level);
  else if (epi == EPI_ZMINUS) launch_op<P, T, EPI_ZMINUS>(ctx, a, level);
  else launch_op<P, T, EPI_JACOBI>(ctx, a, level);
}

template <typename T>
iga_status op_apply(iga_ctx* ctx, int level, int which, const typename cplx<T>::t* x, typename cplx<T>::t* y,
                    const typename cplx<T>::t* z, int epi, const typename cplx<T>::t* b, double omega) {
  using C = typename cplx<T>::t;
  const LevelData& L = ctx->lv[level];
  OpArgs<T> a{};
  a.nx = L.nx;
  a.ny = L.ny;
  a.n_el = L.n_el;
  constexpr bool dbl = sizeof(T) == 8;
  if constexpr (dbl) {
    a.K = (const T*)L.K; a.M = (const T*)L.M; a.B = (const T*)L.B; a.wq = (const T*)L.wq;
  } else {
    a.K = (const T*)L.Kf; a.M = (const T*)L.Mf; a.B = (const T*)L.Bf; a.wq = (const T*)L.wqf;
  }
  a.xq = L.xq;
  // mass coefficient: A: -1 (times k^2); M_beta: -(beta1 - i beta2) (times k^2)
  double2 cm = (which == OP_A) ? make_double2(-1.0, 0.0) : make_double2(-ctx->sig.x, -ctx->sig.y);
  if (!ctx->vark) cm = ctx->k2const * cm;
  a.c = cconv<C>(cm);
  a.x = x;
  a.y = y;
  a.z = (epi == EPI_JACOBI) ? b : z;
  a.dinv = nullptr;     // D^{-1} from memory: 2D FP64 levels, FP32 with variable k
  if (epi == EPI_JACOBI && ctx->dim == 2) {
    if constexpr (dbl) a.dinv = (const C*)L.dinv; else if (ctx->vark) a.dinv = (const C*)L.dinvf;
  } else if (epi == EPI_JACOBI && ctx->robin_k != 0.0) {   // 1D, Sommerfeld end: stored D^{-1}
    if constexpr (dbl) a.dinv = (const C*)L.dinv; else a.dinv = (const C*)L.dinvf;
  }
  a.omega = (T)omega;
  a.rk = (T)ctx->robin_k;      // the Sommerfeld term belongs to A and to the CSLP levels alike
  switch (ctx->p) {
    case 1: launch_epi<1, T>(ctx, a, level, epi); break;
    case 2: launch_epi<2, T>(ctx, a, level, epi); break;
    case 3: launch_epi<3, T>(ctx, a, level, epi); break;
    case 4: launch_epi<4, T>(ctx, a, level, epi); break;
    case 5: launch_epi<5, T>(ctx, a, level, epi); break;
    default: return set_err(ctx, IGA_E_INVALID, "p out of range");
  }
  CKL();
  return IGA_OK;
}

template iga_status op_apply<double>(iga_ctx*, int, int, const double2*, double2*, const double2*, int,
                                     const double2*, double);
template iga_status op_apply<float>(iga_ctx*, int, int, const float2*, float2*, const float2*, int,
                                    const float2*, double);

iga_status setup_vark_diag(iga_ctx* ctx, int level) {
  LevelData& L = ctx->lv[level];
  L.dinv = dalloc<double2>(ctx, L.n);
  L.dinvf = dalloc<float2>(ctx, L.n);
  if (!L.dinv || !L.dinvf) return set_err(ctx, IGA_E_OOM, "dinv");
  double2 c = make_double2(-ctx->sig.x, -ctx->sig.y);
  k_vark_diag<<<cdiv(L.n, 128), 128, 0, ctx->st>>>(L.nx, L.n_el, ctx->p, L.K, L.M, L.B, L.wq, L.xq, ctx->kf, c,
                                                   L.dinv, L.dinvf); iga_count_launch();
  CKL();
  return IGA_OK;
}

// Constant-coefficient tensor operator with explicit bands (used for the
// deflation coarse matrix E, which has the same Kronecker structure as A).
template <int P>
static void launch_bands(iga_ctx* ctx, const OpArgs<double>& a, int epi) {
  cudaStream_t st = ctx->st;
  if (a.ny == 1) {
    if (epi == EPI_Y) { k_kron1d<P, double, EPI_Y><<<cdiv(a.nx, 256), 256, 0, st>>>(a); iga_count_launch(); }
    else { k_kron1d<P, double, EPI_ZMINUS><<<cdiv(a.nx, 256), 256, 0, st>>>(a); iga_count_launch(); }
    return;
  }
  // the coarse grid is small (m_x ~ n_x / 2): the small-tile shape the autotuner
  // chose for the FP64 level of nearest size, else 8 x 8 tiles unless 16 x 16
  // already fills the GPU
  int tile = -1, dist = 1 << 30;
  for (int l = 0; l < ctx->L; ++l) {
    const int dd = abs(ctx->lv[l].nx - a.nx);
    if (ctx->tile[l][0] >= 0 && dd < dist) { dist = dd; tile = ctx->tile[l][0]; }
  }
  const bool small = (size_t)cdiv(a.nx, 16) * cdiv(a.ny, 16) < (size_t)ctx->num_sms;
  if (tile >= 4) {
    if (epi == EPI_Y) launch_kron_pair<P, EPI_Y>(a, st, tile); else launch_kron_pair<P, EPI_ZMINUS>(a, st, tile);
  } else if (epi == EPI_Y) {
    if (small) launch_kron_small<P, double, EPI_Y>(a, st); else launch_kron_tile<P, double, EPI_Y, 16, 16>(a, st);
  } else {
    if (small) launch_kron_small<P, double, EPI_ZMINUS>(a, st); else launch_kron_tile<P, double, EPI_ZMINUS, 16, 16>(a, st);
  }
}

iga_status op_apply_bands(iga_ctx* ctx, int P, int nx, int ny, const double* K, const double* M, double2 c,
                          const double2* x, double2* y, const double2* z, int epi, float2* yf) {
  OpArgs<double> a{};
  a.yf = yf;
  a.nx = nx;
  a.ny = ny;
  a.K = K;
  a.M = M;
  a.c = c;
  a.x = x;
  a.y = y;
  a.z = z;
  switch (P) {
    case 1: launch_bands<1>(ctx, a, epi); break;
    case 2: launch_bands<2>(ctx, a, epi); break;
    case 3: launch_bands<3>(ctx, a, epi); break;
    case 4: launch_bands<4>(ctx, a, epi); break;
    case 5: launch_bands<5>(ctx, a, epi); break;
    default: return set_err(ctx, IGA_E_INVALID, "band width");
  }
  CKL();
  return IGA_OK;
}

// ------------------------------------------------------------------ tile autotuner
// For constant k in 2D the operator kernel has six tile shapes: 32x16, 16x16,
// 32x8 outputs per 256-thread block, 8x8 per 64-thread block, and (FP64 only)
// the lane-pair kernel with 8x8 outputs per 256 threads or 8x4 per 128; FP32
// has in their place the register-stencil sweep of sweep32.cu (code 6).  At
// setup every level times each shape on its own operator, FP64 and FP32, as
// the solve runs it: TUNE_REPS dependent launches captured in one CUDA graph
// per shape (host launch costs, which would hide the small levels'
// differences, stay out of the measurement).  The graphs are timed in
// TUNE_ROUNDS interleaved rounds and each shape keeps its fastest round, so a
// clock ramp or a stray delay does not decide the choice.  Results are cached
// per (p, precision, n_x) for the whole process, so batched instances of
// equal size are tuned once.
#include <map>
#include <mutex>
#include <tuple>

static std::map<std::tuple<int, int, int>, int> g_tile_cache;
static std::mutex g_tile_mu;
constexpr int TUNE_REPS = 24, TUNE_ROUNDS = 5, TUNE_MAX_TILES = 6;

// graph of TUNE_REPS applies of M_beta on level l with the current tile
template <typename T>
static iga_status capture_applies(iga_ctx* ctx, int l, const typename cplx<T>::t* x, typename cplx<T>::t* y,
                                  cudaGraphExec_t* out) {
  *out = nullptr;
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  cudaStream_t saved = ctx->st;
  // one untimed launch outside the capture (first-use attributes of the kernel)
  TRY(op_apply<T>(ctx, l, OP_MB, x, y, nullptr, EPI_Y, nullptr, 0.0));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->st = ctx->cap_stream;
  const unsigned long long before = iga_launch_count();
  cudaError_t e = cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) { ctx->st = saved; return set_err(ctx, IGA_E_CUDA, "tune capture: %s", cudaGetErrorString(e)); }
  iga_status s = IGA_OK;
  for (int r = 0; r < TUNE_REPS && s == IGA_OK; ++r) s = op_apply<T>(ctx, l, OP_MB, x, y, nullptr, EPI_Y, nullptr, 0.0);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(ctx->st, &g);
  ctx->st = saved;
  iga_add_launches(-(long long)(iga_launch_count() - before));   // capture executes nothing
  if (s != IGA_OK) { if (g) cudaGraphDestroy(g); return s; }
  if (e2 != cudaSuccess) return set_err(ctx, IGA_E_CUDA, "tune end capture: %s", cudaGetErrorString(e2));
  cudaError_t e3 = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) { *out = nullptr; return set_err(ctx, IGA_E_CUDA, "tune instantiate: %s", cudaGetErrorString(e3)); }
  return IGA_OK;
}

template <typename T>
static iga_status tune_level(iga_ctx* ctx, int l, int slot) {
  using C = typename cplx<T>::t;
  LevelData& L = ctx->lv[l];
  auto key = std::make_tuple(ctx->p, slot, L.nx);
  {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    auto it = g_tile_cache.find(key);
    if (it != g_tile_cache.end()) { ctx->tile[l][slot] = it->second; return IGA_OK; }
  }
  C* x = (C*)(slot == 0 ? (void*)L.vb : (void*)L.fb);
  C* y = (C*)(slot == 0 ? (void*)L.vx : (void*)L.fx);
  CK(cudaMemsetAsync(x, 0, sizeof(C) * L.n, ctx->st));
  // candidate shapes: FP64 0..5; FP32 0..3 and the register-stencil sweep (6)
  static const int cand64[] = {0, 1, 2, 3, 4, 5}, cand32[] = {0, 1, 2, 3, 6};
  const int* cand = sizeof(T) == 8 ? cand64 : cand32;
  const int ntiles = sizeof(T) == 8 ? 6 : 5;
  cudaGraphExec_t ge[TUNE_MAX_TILES] = {};
  cudaEvent_t ev[2 * TUNE_MAX_TILES] = {};
  float best_ms[TUNE_MAX_TILES];
  iga_status s = IGA_OK;
  for (int t = 0; t < ntiles && s == IGA_OK; ++t) {
    ctx->tile[l][slot] = cand[t];
    best_ms[t] = 1e30f;
    s = capture_applies<T>(ctx, l, x, y, &ge[t]);
  }
  for (int i = 0; i < 2 * ntiles && s == IGA_OK; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) s = set_err(ctx, IGA_E_CUDA, "tune events");
  // one warm-up round, then TUNE_ROUNDS timed rounds over all shapes
  for (int round = 0; round <= TUNE_ROUNDS && s == IGA_OK; ++round) {
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < ntiles && e == cudaSuccess; ++t) {
      e = cudaEventRecord(ev[2 * t], ctx->st);
      if (e == cudaSuccess) e = cudaGraphLaunch(ge[t], ctx->st);
      if (e == cudaSuccess) e = cudaEventRecord(ev[2 * t + 1], ctx->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    for (int t = 0; t < ntiles && e == cudaSuccess && round > 0; ++t) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[2 * t], ev[2 * t + 1]);
      if (e == cudaSuccess && ms < best_ms[t]) best_ms[t] = ms;
    }
    if (e != cudaSuccess) s = set_err(ctx, IGA_E_CUDA, "tune launch: %s", cudaGetErrorString(e));
  }
  for (int t = 0; t < ntiles; ++t)
    if (ge[t]) cudaGraphExecDestroy(ge[t]);
  for (int i = 0; i < 2 * ntiles; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (s != IGA_OK) { ctx->tile[l][slot] = -1; return s; }
  int best_tile = 0;
  for (int t = 1; t < ntiles; ++t)
    if (best_ms[t] < best_ms[best_tile]) best_tile = t;
  ctx->tile[l][slot] = cand[best_tile];
  std::lock_guard<std::mutex> lock(g_tile_mu);
  g_tile_cache[key] = cand[best_tile];
  return IGA_OK;
}

iga_status autotune_tiles(iga_ctx* ctx) {
  if (ctx->dim != 2 || ctx->vark) return IGA_OK;
  for (int l = 0; l < ctx->L; ++l) {
    if (ctx->lv[l].nx < 8) continue;
    TRY(tune_level<double>(ctx, l, 0));
    TRY(tune_level<float>(ctx, l, 1));
  }
  return IGA_OK;
}

extern "C" iga_status iga_set_tile(iga_ctx* ctx, int level, int precision, int tile) {
  if (!ctx) return IGA_E_INVALID;
  if (level < 0 || level >= ctx->L || precision < 0 || precision > 1)
    return set_err(ctx, IGA_E_INVALID, "iga_set_tile: level %d / precision %d out of range", level, precision);
  const bool ok = tile >= -1 && (precision == 0 ? tile <= 5 : (tile <= 3 || tile == 6));
  if (!ok) return set_err(ctx, IGA_E_INVALID, "iga_set_tile: tile %d not available in this precision", tile);
  ctx->tile[level][precision] = tile;
  // the cached loop graph captured the previous kernels
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->gexec = nullptr;
  ctx->graph = nullptr;
  return IGA_OK;
}

extern "C" int iga_tile_choice(const iga_ctx* ctx, int level, int precision) {
  if (!ctx || level < 0 || level >= ctx->L || precision < 0 || precision > 1) return -2;
  return ctx->tile[level][precision];
}
