// Deflation coarse matrix E = Z^T A Z for a variable wave number (Section 3,
// Eq. adef1), where E has no Kronecker structure.
//
// Assembly by coloured probing: coarse dof j couples to i only if
// |i_x - j_x| <= b and |i_y - j_y| <= b with b = floor((p + 4) / 2) (the ADP
// stencil is 5 fine dofs wide, A is 2p+1 wide).  For each of the (2b+1)^2
// colours (j_x mod 2b+1, j_y mod 2b+1) the probe vector c (ones on the colour)
// gives r = Z^T A Z c, and r_i is exactly E_{i, j*(i)} for the unique colour
// member j* within reach of i.
//
// Factorisation: grouping s = b coarse grid lines per block makes E block
// tridiagonal (blocks of bs = s * m_x).  Block LU (block Thomas):
//   D_0 = E_00,  D_I = E_II - E_{I,I-1} D_{I-1}^{-1} E_{I-1,I},
// with D_I^{-1} formed by Gauss-Jordan elimination with partial pivoting and
// F_I = D_I^{-1} E_{I,I+1} kept for the back substitution.  E is complex
// symmetric, so E_{I-1,I} = E_{I,I-1}^T.  The grid is padded to nb * s lines
// with identity rows.
#include "common.cuh"

__global__ void k_probe(int mx, int S, int cx, int cy, double2* c) {
  size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (j >= (size_t)mx * mx) return;
  int jy = (int)(j / mx), jx = (int)(j - (size_t)jy * mx);
  c[j] = make_double2((jx % S == cx && jy % S == cy) ? 1.0 : 0.0, 0.0);
}

__device__ __forceinline__ int colour_partner(int i, int cc, int S, int b) {
  int d = ((cc - i) % S + S) % S;
  return d <= b ? i + d : i + d - S;
}

// Scatter probe results r (coarse, length mx*mx) into the diagonal and lower
// off-diagonal blocks (row-major bs x bs each).
__global__ void k_scatter_E(int mx, int S, int b, int s, int bs, int cx, int cy, const double2* r, double2* Ed,
                            double2* El) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)mx * mx) return;
  int iy = (int)(i / mx), ix = (int)(i - (size_t)iy * mx);
  int jx = colour_partner(ix, cx, S, b), jy = colour_partner(iy, cy, S, b);
  if (jx < 0 || jx >= mx || jy < 0 || jy >= mx) return;
  int I = iy / s, J = jy / s;
  size_t row = (size_t)(iy - I * s) * mx + ix;
  size_t col = (size_t)(jy - J * s) * mx + jx;
  size_t blk = (size_t)bs * bs;
  if (J == I) Ed[(size_t)I * blk + row * bs + col] = r[i];
  else if (J == I - 1) El[(size_t)I * blk + row * bs + col] = r[i];
}

// identity on the padded rows of the last diagonal block
__global__ void k_pad_identity(double2* Ed_last, int bs, int first_pad) {
  int i = first_pad + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < bs) Ed_last[(size_t)i * bs + i] = make_double2(1.0, 0.0);
}

// C = beta C + alpha * A * op(B)   (complex, row-major n x n; TB: op(B) = B^T)
template <bool TB>
__global__ void __launch_bounds__(256) k_zgemm(int n, double2 alpha, const double2* A, const double2* B, double beta,
                                               double2* C) {
  constexpr int TS = 32, TK = 16;
  __shared__ double2 As[TS][TK + 1];
  __shared__ double2 Bs[TK][TS + 1];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int r0 = blockIdx.y * TS, c0 = blockIdx.x * TS;
  double2 acc[2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
  for (int k0 = 0; k0 < n; k0 += TK) {
    for (int t = threadIdx.x; t < TS * TK; t += 256) {
      int rr = t / TK, kk = t - rr * TK;
      int gr = r0 + rr, gk = k0 + kk;
      As[rr][kk] = (gr < n && gk < n) ? A[(size_t)gr * n + gk] : make_double2(0.0, 0.0);
      int kb = t / TS, cc = t - kb * TS;
      int gkb = k0 + kb, gc = c0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (gkb < n && gc < n) v = TB ? B[(size_t)gc * n + gkb] : B[(size_t)gkb * n + gc];
      Bs[kb][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double2 a0 = As[ty][kk], a1 = As[ty + 16][kk];
      double2 b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = acc[0][0] + cmul(a0, b0);
      acc[0][1] = acc[0][1] + cmul(a0, b1);
      acc[1][0] = acc[1][0] + cmul(a1, b0);
      acc[1][1] = acc[1][1] + cmul(a1, b1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int gr = r0 + ty + 16 * a, gc = c0 + tx + 16 * b;
      if (gr < n && gc < n) {
        size_t o = (size_t)gr * n + gc;
        double2 v = cmul(alpha, acc[a][b]);
        C[o] = beta == 0.0 ? v : beta * C[o] + v;
      }
    }
}

// Gauss-Jordan step k, part 1 (one block): pivot search, row swap, scaling of
// row k, and the saved column k (multipliers).
__global__ void k_gj_pivot(double2* A, double2* Inv, int n, int k, double2* fcol, int* info) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  __shared__ double2 pinv;
  double best = -1.0;
  int besti = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    double2 v = A[(size_t)i * n + k];
    double m = v.x * v.x + v.y * v.y;
    if (m > best) { best = m; besti = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double o = bv[threadIdx.x + s];
      int oi = bi[threadIdx.x + s];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) { bv[threadIdx.x] = o; bi[threadIdx.x] = oi; }
    }
    __syncthreads();
  }
  int p = bi[0];
  if (threadIdx.x == 0 && !(bv[0] > 0.0)) *info = 1;
  if (p != k) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double2 t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)p * n + j]; A[(size_t)p * n + j] = t;
      t = Inv[(size_t)k * n + j]; Inv[(size_t)k * n + j] = Inv[(size_t)p * n + j]; Inv[(size_t)p * n + j] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) pinv = bv[0] > 0.0 ? cinv(A[(size_t)k * n + k]) : make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    A[(size_t)k * n + j] = cmul(pinv, A[(size_t)k * n + j]);
    Inv[(size_t)k * n + j] = cmul(pinv, Inv[(size_t)k * n + j]);
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = (i == k) ? make_double2(0.0, 0.0) : A[(size_t)i * n + k];
}

// Gauss-Jordan step k, part 2: eliminate column k from every other row.
__global__ void k_gj_elim(double2* A, double2* Inv, int n, int k, const double2* fcol) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t tot = (size_t)n * n;
  if (idx >= tot) return;
  int i = (int)(idx / n), j = (int)(idx - (size_t)i * n);
  double2 f = fcol[i];
  if (f.x == 0.0 && f.y == 0.0) return;
  if (j >= k) A[idx] = A[idx] - cmul(f, A[(size_t)k * n + j]);
  Inv[idx] = Inv[idx] - cmul(f, Inv[(size_t)k * n + j]);
}

__global__ void k_eye_c(double2* e, int n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < (size_t)n * n) e[i] = make_double2((i / n) == (i % n) ? 1.0 : 0.0, 0.0);
}

// y = z - A x   (sub) or y = A x ; A dense complex n x n row-major; one warp per row
template <bool SUB>
__global__ void k_zgemv(int n, const double2* A, const double2* x, const double2* z, double2* y) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double2* a = A + (size_t)warp * n;
  double re = 0.0, im = 0.0;
  for (int k = lane; k < n; k += 32) {
    double2 v = a[k], w = x[k];
    re += v.x * w.x - v.y * w.y;
    im += v.x * w.y + v.y * w.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if (lane == 0) y[warp] = SUB ? make_double2(z[warp].x - re, z[warp].y - im) : make_double2(re, im);
}

static iga_status gj_invert(iga_ctx* ctx, double2* A, double2* Inv, int n, double2* fcol, int* info) {
  k_eye_c<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(Inv, n); iga_count_launch();
  for (int k = 0; k < n; ++k) {
    k_gj_pivot<<<1, 256, 0, ctx->st>>>(A, Inv, n, k, fcol, info); iga_count_launch();
    k_gj_elim<<<cdiv((size_t)n * n, 256), 256, 0, ctx->st>>>(A, Inv, n, k, fcol); iga_count_launch();
  }
  CKL();
  return IGA_OK;
}

iga_status setup_block_E(iga_ctx* ctx) {
  const int mx = ctx->mx, p = ctx->p;
  const int b = (p + 4) / 2, S = 2 * b + 1, s = b;
  const int bs = s * mx, nb = (mx + s - 1) / s;
  ctx->eblk = bs;
  ctx->enb = nb;
  ctx->els = s;
  size_t blk = (size_t)bs * bs;
  ctx->eDinv = dalloc<double2>(ctx, blk * nb);
  ctx->eOff = dalloc<double2>(ctx, blk * nb);
  ctx->eF = dalloc<double2>(ctx, blk * nb);
  double2* work = dalloc<double2>(ctx, blk);
  double2* fcol = dalloc<double2>(ctx, bs);
  int* info = dalloc<int>(ctx, 1);
  ctx->ep_t = dalloc<double2>(ctx, (size_t)nb * bs);
  ctx->ep_g = dalloc<double2>(ctx, (size_t)nb * bs);
  ctx->ep_v = dalloc<double2>(ctx, bs);
  if (!ctx->eDinv || !ctx->eOff || !ctx->eF || !work || !fcol || !info || !ctx->ep_t || !ctx->ep_g || !ctx->ep_v)
    return set_err(ctx, IGA_E_OOM, "block E (%d blocks of %d)", nb, bs);
  cudaStream_t st = ctx->st;
  // assemble: diagonal blocks go to eF (scratch for now), lower blocks to eOff
  CK(cudaMemsetAsync(ctx->eF, 0, sizeof(double2) * blk * nb, st));
  CK(cudaMemsetAsync(ctx->eOff, 0, sizeof(double2) * blk * nb, st));
  CK(cudaMemsetAsync(info, 0, sizeof(int), st));
  size_t m = ctx->m;
  LevelData& L = ctx->lv[0];
  for (int cy = 0; cy < S; ++cy)
    for (int cx = 0; cx < S; ++cx) {
      k_probe<<<cdiv(m, 256), 256, 0, st>>>(mx, S, cx, cy, ctx->ct); iga_count_launch();
      TRY(defl_z(ctx, ctx->ct, ctx->w3));
      TRY(op_apply<double>(ctx, 0, OP_A, ctx->w3, ctx->w2, nullptr, EPI_Y, nullptr, 0.0));
      TRY(defl_zt(ctx, ctx->w2, ctx->cs));
      k_scatter_E<<<cdiv(m, 256), 256, 0, st>>>(mx, S, b, s, bs, cx, cy, ctx->cs, ctx->eF, ctx->eOff); iga_count_launch();
    }
  int first_pad = (mx - (nb - 1) * s) * mx;
  if (first_pad < bs) k_pad_identity<<<cdiv(bs - first_pad, 128), 128, 0, st>>>(ctx->eF + blk * (nb - 1), bs, first_pad); iga_count_launch();
  CKL();
  (void)L;
  dim3 gg(cdiv(bs, 32), cdiv(bs, 32));
  for (int I = 0; I < nb; ++I) {
    double2* EdI = ctx->eF + blk * I;          // E_II (overwritten by D_I)
    if (I > 0) {
      // T = D_{I-1}^{-1} E_{I-1,I} = Dinv_{I-1} El_I^T  -> stored as F_{I-1} in `work` first
      k_zgemm<true><<<gg, 256, 0, st>>>(bs, make_double2(1.0, 0.0), ctx->eDinv + blk * (I - 1), ctx->eOff + blk * I, 0.0,
                                        work); iga_count_launch();
      // D_I = E_II - El_I T
      k_zgemm<false><<<gg, 256, 0, st>>>(bs, make_double2(-1.0, 0.0), ctx->eOff + blk * I, work, 1.0, EdI); iga_count_launch();
      // F_{I-1} = T  (E_{I-1,I-1} storage is free again: it holds D_{I-1} which is no longer needed)
      CK(cudaMemcpyAsync(ctx->eF + blk * (I - 1), work, sizeof(double2) * blk, cudaMemcpyDeviceToDevice, st));
    }
    // Dinv_I = D_I^{-1}; D_I stays in eF[I] (destroyed by elimination) until F_I overwrites it
    TRY(gj_invert(ctx, EdI, ctx->eDinv + blk * I, bs, fcol, info));
  }
  int hinfo = 0;
  CK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hinfo) return set_err(ctx, IGA_E_INVALID, "singular block in the coarse deflation matrix");
  return IGA_OK;
}

// s = E^{-1} t by block forward / back substitution
iga_status block_E_solve(iga_ctx* ctx, const double2* t, double2* s) {
  const int bs = ctx->eblk, nb = ctx->enb;
  const size_t blk = (size_t)bs * bs, m = ctx->m;
  cudaStream_t st = ctx->st;
  double2* tp = ctx->ep_t;
  double2* g = ctx->ep_g;
  CK(cudaMemcpyAsync(tp, t, sizeof(double2) * m, cudaMemcpyDeviceToDevice, st));
  if ((size_t)nb * bs > m) CK(cudaMemsetAsync(tp + m, 0, sizeof(double2) * ((size_t)nb * bs - m), st));
  unsigned gv = cdiv((size_t)bs * 32, 256);
  for (int I = 0; I < nb; ++I) {
    const double2* rhs = tp + (size_t)I * bs;
    if (I > 0) {
      k_zgemv<true><<<gv, 256, 0, st>>>(bs, ctx->eOff + blk * I, g + (size_t)(I - 1) * bs, rhs, ctx->ep_v); iga_count_launch();
      rhs = ctx->ep_v;
    }
    k_zgemv<false><<<gv, 256, 0, st>>>(bs, ctx->eDinv + blk * I, rhs, nullptr, g + (size_t)I * bs); iga_count_launch();
  }
  // back substitution in place on g: s_I = g_I - F_I s_{I+1} (each output is read
  // and written by the same lane, so the update is in place)
  for (int I = nb - 2; I >= 0; --I)
    k_zgemv<true><<<gv, 256, 0, st>>>(bs, ctx->eF + blk * I, g + (size_t)(I + 1) * bs, g + (size_t)I * bs,
                                      g + (size_t)I * bs); iga_count_launch();
  CK(cudaMemcpyAsync(s, g, sizeof(double2) * m, cudaMemcpyDeviceToDevice, st));
  CKL();
  return IGA_OK;
}
