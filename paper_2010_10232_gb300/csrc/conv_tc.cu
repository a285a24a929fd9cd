// 3x3 convolution layer of the learned correction network on the fifth-
// generation tensor cores (tcgen05.mma, accumulator in tensor memory).  Not in
// the paper; see cnn.cu for the network.
//
// Implicit GEMM per output tile of 8 x 16 pixels (M = 128 rows = pixels,
// row m <-> pixel (m % 8, m / 8)):  D[m][n] = sum over the 9 taps and the input
// channels of X[pixel(m) + tap][c] * Wt[n][tap][c], N = output channels, K
// consumed 16 channels per instruction, all 9 * CIN / 16 instructions issued
// by one thread into one TMEM accumulator of N columns.
//
// Operands live in shared memory in the canonical no-swizzle K-major layout
// of the UMMA descriptors: core matrices of 8 rows x 16 bytes (8 bf16 of K),
// 128 contiguous bytes each.
//   A (input halo tile, 10 x 18 pixels): byte (cb, hy, hx) at
//     ((cb * 18 + hy) * 10 + hx) * 16, cb = channel block of 8.  For tap
//     (dy, dx) the A core matrix of output row py is the 8 pixels
//     (hy = py + dy, hx = dx .. dx + 7): SBO (next 8 rows = next pixel row) =
//     160 B, LBO (next 8 channels) = 18 * 10 * 16 B, start offset
//     ((cb * 18 + dy) * 10 + dx) * 16.
//   B (weights, all taps, loaded once per block): byte (t, cb, n) at
//     ((t * CB + cb) * N + n) * 16: SBO (next 8 output channels) = 128 B,
//     LBO (next 8 input channels) = N * 16 B.
// The MMA completion is signalled by tcgen05.commit on an mbarrier; every wait
// is bounded (on timeout the block records an error, frees its tensor memory
// and returns).
#include "common.cuh"
#include <cuda_bf16.h>

typedef __nv_bfloat16 bf16;

namespace {

constexpr int TC_TX = 8, TC_TY = 16, TC_HX = TC_TX + 2, TC_HY = TC_TY + 2, TC_NT = 128;
constexpr unsigned TC_WAIT_LIMIT = 1u << 22;      // mbarrier polls before a block gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// UMMA shared-memory matrix descriptor, no swizzle (layout type 0)
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;                                  // descriptor version of this architecture
  return d;
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr unsigned umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int CIN, int N> struct TcGeom {
  static constexpr int CB = CIN / 8;
  static constexpr size_t a_bytes = (size_t)CB * TC_HY * TC_HX * 16;
  static constexpr size_t b_bytes = (size_t)9 * CB * N * 16;
  static constexpr size_t smem = 2 * a_bytes + b_bytes + 32;   // + two mbarriers and the TMEM address slot
  static constexpr int ACC_COLS = 32;                           // one accumulator (>= N FP32 columns)
  static constexpr int TMEM_COLS = 2 * ACC_COLS;                // two, alternating between tiles
  static_assert(N == 16 || N == 32, "accumulator width");
  static_assert(CIN % 16 == 0, "K chunks of 16 channels");
};

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// bounded wait on an mbarrier phase; false if the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(unsigned a, unsigned parity) {
  unsigned polls = 0;
  while (!mbar_try_wait(a, parity)) {
    if (++polls > TC_WAIT_LIMIT) return false;
    __nanosleep(32);
  }
  return true;
}

}  // namespace

// X: NHWC bf16 [B][H][W][CIN]; Wt: [COUTP][9][CIN] bf16 (COUTP >= COUT real
// output channels, rows beyond COUTP read as zero up to N); EPI as in cnn.cu:
// 0 + bias, ReLU, bf16 [px][N]; 1 + bias, FP32 [px][2]; 2 times (mask > 0),
// bf16 [px][N].  err: set to 1 if a wait gave up.
//
// Persistent blocks take tiles blockIdx.x, blockIdx.x + gridDim.x, ... in a
// two-stage pipeline: iteration i issues the MMAs of tile i into accumulator
// i % 2 (from A buffer i % 2), then waits for tile i - 1's MMAs, reads its
// accumulator, starts the cp.async halo load of tile i + 1 into the A buffer
// tile i - 1 used, and stores tile i - 1's outputs.  The tensor core works
// on one tile while the block loads the next and writes the previous.
template <int CIN, int N, int EPI>
__global__ void __launch_bounds__(TC_NT) k_conv3x3_tc(const bf16* __restrict__ X, const bf16* __restrict__ Wt,
                                                      int coutp, const float* __restrict__ bias,
                                                      const bf16* __restrict__ mask, void* Yout, int B, int H,
                                                      int W, int* err) {
  using G = TcGeom<CIN, N>;
  constexpr int CB = G::CB;
  extern __shared__ __align__(128) unsigned char tc_smem[];
  unsigned char* Bs = tc_smem + 2 * G::a_bytes;
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(Bs + G::b_bytes);
  unsigned* tslot = reinterpret_cast<unsigned*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    mbar_init(smem_u32(mbar + 1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights into the B layout: chunk (t, cb, n) = Wt[n][t][8 cb .. 8 cb + 7]
  for (int i = tid; i < 9 * CB * N; i += TC_NT) {
    const int n = i % N, tcb = i / N, cb = tcb % CB, t = tcb / CB;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (n < coutp) v = *reinterpret_cast<const uint4*>(Wt + ((size_t)n * 9 + t) * CIN + cb * 8);
    *reinterpret_cast<uint4*>(Bs + (size_t)((t * CB + cb) * N + n) * 16) = v;
  }
  const unsigned a_base0 = smem_u32(tc_smem), b_base = smem_u32(Bs);
  constexpr unsigned idesc = umma_idesc_bf16(128, N);
  constexpr unsigned A_LBO = TC_HY * TC_HX * 16, A_SBO = TC_HX * 16, B_LBO = N * 16, B_SBO = 8 * 16;

  const int tiles_x = (W + TC_TX - 1) / TC_TX, tiles_y = (H + TC_TY - 1) / TC_TY;
  const int per_img = tiles_x * tiles_y, ntiles = per_img * B;

  // input halo tile into the A layout (16-byte chunks of 8 channels, zero-filled outside the image)
  auto load_tile = [&](int tile, unsigned a_dst) {
    const int b = tile / per_img, rem = tile - b * per_img;
    const int ty = rem / tiles_x, tx = rem - ty * tiles_x;
    const int x0 = tx * TC_TX, y0 = ty * TC_TY;
    const size_t img = (size_t)b * H * W;
    for (int i = tid; i < CB * TC_HY * TC_HX; i += TC_NT) {
      const int hx = i % TC_HX, r = i / TC_HX, hy = r % TC_HY, cb = r / TC_HY;
      const int gy = y0 - 1 + hy, gx = x0 - 1 + hx;
      const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
      const bf16* src = in ? X + (img + (size_t)gy * W + gx) * CIN + cb * 8 : X;
      cp_async16(a_dst + (unsigned)i * 16u, src, in ? 16u : 0u);
    }
  };

  if ((int)blockIdx.x < ntiles) load_tile(blockIdx.x, a_base0);
  cp_async_commit();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tslot;
  const unsigned mb0 = smem_u32(mbar);

  unsigned phase = 0u, pending = 0u;     // bit b: parity to wait for / MMAs outstanding on mbarrier b
  bool failed = false;
  for (int it = 0;; ++it) {
    const int cur = (int)blockIdx.x + it * (int)gridDim.x;
    const bool have_cur = cur < ntiles;
    if (!have_cur && it == 0) break;
    const int s = it & 1;
    // tile cur's operands landed (the only outstanding cp.async group) and
    // every thread finished reading the accumulator this tile overwrites
    cp_async_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (have_cur) {
      if (tid == 0) {
        tc_fence_after();
        const unsigned a_base = a_base0 + (unsigned)(s * G::a_bytes);
        const unsigned d_tmem = tmem + (unsigned)(s * G::ACC_COLS);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int dy = t / 3, dx = t % 3;
#pragma unroll
          for (int kc = 0; kc < CIN / 16; ++kc) {
            const unsigned a_off = (unsigned)((((2 * kc) * TC_HY + dy) * TC_HX + dx) * 16);
            const unsigned b_off = (unsigned)((t * CB + 2 * kc) * N * 16);
            tc_mma(d_tmem, umma_desc(a_base + a_off, A_LBO, A_SBO), umma_desc(b_base + b_off, B_LBO, B_SBO), idesc,
                   (t | kc) != 0 ? 1u : 0u);
          }
        }
        tc_commit(mb0 + 8u * (unsigned)s);
      }
      pending |= 1u << s;
    }
    const bool have_prev = it > 0;
    const int q = s ^ 1;
    float acc[N];
    if (have_prev) {
      // the give-up decision is made for the whole block
      const bool done = mbar_wait_bounded(mb0 + 8u * (unsigned)q, (phase >> q) & 1u);
      if (__syncthreads_or(!done)) {
        failed = true;
        if (tid == 0) atomicExch(err, 1);
        break;
      }
      phase ^= 1u << q;
      pending &= ~(1u << q);
      tc_fence_after();
      const unsigned trow = tmem + (unsigned)(q * G::ACC_COLS) + ((unsigned)(32 * warp) << 16);
      tc_ld16(trow, acc);
      if constexpr (N == 32) tc_ld16(trow + 16, acc + 16);
    }
    // A buffer q is free once tile cur - gridDim.x's MMAs completed
    const int nxt = cur + (int)gridDim.x;
    if (have_cur && nxt < ntiles) load_tile(nxt, a_base0 + (unsigned)(q * G::a_bytes));
    cp_async_commit();
    if (have_prev) {
      // epilogue: thread <-> TMEM lane 32 warp + lane <-> pixel (m % 8, m / 8)
      const int prev = cur - (int)gridDim.x;
      const int b = prev / per_img, rem = prev - b * per_img;
      const int ty = rem / tiles_x, tx = rem - ty * tiles_x;
      const int m = 32 * warp + lane;
      const int gx = tx * TC_TX + (m & 7), gy = ty * TC_TY + (m >> 3);
      if (gx < W && gy < H) {
        const size_t p = (size_t)b * H * W + (size_t)gy * W + gx;
        if (EPI == 0) {
          __nv_bfloat162 o[N / 2];
#pragma unroll
          for (int c = 0; c < N; c += 2)
            o[c / 2] = __floats2bfloat162_rn(fmaxf(acc[c] + bias[c], 0.f), fmaxf(acc[c + 1] + bias[c + 1], 0.f));
#pragma unroll
          for (int v = 0; v < N / 8; ++v)
            reinterpret_cast<uint4*>((bf16*)Yout + p * N)[v] = reinterpret_cast<const uint4*>(o)[v];
        } else if (EPI == 1) {
          *reinterpret_cast<float2*>((float*)Yout + p * 2) = make_float2(acc[0] + bias[0], acc[1] + bias[1]);
        } else {
          __nv_bfloat162 o[N / 2];
          const __nv_bfloat162* mk = reinterpret_cast<const __nv_bfloat162*>(mask + p * N);
#pragma unroll
          for (int c = 0; c < N; c += 2) {
            const __nv_bfloat162 mv = mk[c / 2];
            o[c / 2] = __floats2bfloat162_rn(__bfloat162float(mv.x) > 0.f ? acc[c] : 0.f,
                                             __bfloat162float(mv.y) > 0.f ? acc[c + 1] : 0.f);
          }
#pragma unroll
          for (int v = 0; v < N / 8; ++v)
            reinterpret_cast<uint4*>((bf16*)Yout + p * N)[v] = reinterpret_cast<const uint4*>(o)[v];
        }
      }
    }
    if (!have_cur) break;
  }
  cp_async_wait_all();
  // a block that gave up waits (bounded) for its own MMAs before freeing TMEM
  if (failed) {
#pragma unroll
    for (int b = 0; b < 2; ++b)
      if ((pending >> b) & 1u) (void)mbar_wait_bounded(mb0 + 8u * (unsigned)b, (phase >> b) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS) : "memory");
  }
}

template <int CIN, int N, int EPI>
static cudaError_t launch_tc(const bf16* X, const bf16* Wt, int coutp, const float* bias, const bf16* mask, void* Y,
                             int B, int H, int W, int* err, int num_sms, cudaStream_t st) {
  using G = TcGeom<CIN, N>;
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_conv3x3_tc<CIN, N, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
    // resident blocks per SM: shared memory (plus the 1 KB the runtime
    // reserves per block), 64 registers x 128 threads, and the SM's 512
    // tensor-memory columns, TMEM_COLS per block
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int by_smem = smem_sm / (int)(G::smem + 1024);
    int n = 512 / G::TMEM_COLS;
    if (by_smem < n) n = by_smem;
    if (65536 / (64 * TC_NT) < n) n = 65536 / (64 * TC_NT);
    per_sm = n < 1 ? 1 : n;
  }
  const long long tiles = (long long)cdiv(W, TC_TX) * cdiv(H, TC_TY) * B;
  const long long cap = (long long)per_sm * num_sms;
  const int grid = (int)(tiles < cap ? tiles : cap);
  if (grid == 0) return cudaSuccess;
  k_conv3x3_tc<CIN, N, EPI><<<grid, TC_NT, G::smem, st>>>(X, Wt, coutp, bias, mask, Y, B, H, W, err);
  iga_count_launch();
  return cudaGetLastError();
}

// The layers of the network (cnn.cu): forward 16 -> 32, 32 -> 32, 32 -> 2
// (N = 16: the two real outputs and zero columns), input gradients 16 -> 32
// and 32 -> 32 with the ReLU mask.
cudaError_t conv_tc_launch(int cin, int n, int epi, const bf16* X, const bf16* Wt, int coutp, const float* bias,
                           const bf16* mask, void* Y, int B, int H, int W, int* err, int num_sms, cudaStream_t st) {
  if (cin == 16 && n == 32 && epi == 0) return launch_tc<16, 32, 0>(X, Wt, coutp, bias, mask, Y, B, H, W, err, num_sms, st);
  if (cin == 32 && n == 32 && epi == 0) return launch_tc<32, 32, 0>(X, Wt, coutp, bias, mask, Y, B, H, W, err, num_sms, st);
  if (cin == 32 && n == 16 && epi == 1) return launch_tc<32, 16, 1>(X, Wt, coutp, bias, mask, Y, B, H, W, err, num_sms, st);
  if (cin == 16 && n == 32 && epi == 2) return launch_tc<16, 32, 2>(X, Wt, coutp, bias, mask, Y, B, H, W, err, num_sms, st);
  if (cin == 32 && n == 32 && epi == 2) return launch_tc<32, 32, 2>(X, Wt, coutp, bias, mask, Y, B, H, W, err, num_sms, st);
  return cudaErrorInvalidValue;
}
