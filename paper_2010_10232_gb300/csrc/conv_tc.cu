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
//     cb * 2944 + (hy * 10 + hx) * 16, cb = channel block of 8 (a block is
//     18 * 10 * 16 = 2880 bytes, padded to a 128-byte multiple for the tensor
//     copy).  For tap (dy, dx) the A core matrix of output row py is the 8
//     pixels (hy = py + dy, hx = dx .. dx + 7): SBO (next 8 rows = next pixel
//     row) = 160 B, LBO (next 8 channels) = 2944 B, start offset
//     cb * 2944 + (dy * 10 + dx) * 16.
//   B (weights, all taps, loaded once per block): byte (t, cb, n) at
//     ((t * CB + cb) * N + n) * 16: SBO (next 8 output channels) = 128 B,
//     LBO (next 8 input channels) = N * 16 B.
//
// Warp roles of a persistent block (192 threads) over tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...:
//   warp 0   the halo tile of each channel block by one tensor copy
//            (cp.async.bulk.tensor, 4D box 8 channels x 10 x 18 x 1 image;
//            outside the image the copy fills zeros) into a ring of three or
//            four stages, completion counted in bytes on the stage's mbarrier;
//   warp 1   the MMAs of a tile into one of two TMEM accumulators; its
//            commits release the stage and mark the accumulator full;
//   warps 2-5  read the accumulator (warp w: TMEM lanes 32 (w % 4) ..),
//            release it, and write the tile's outputs.
// Every wait is bounded: a role that gives up records the error and leaves
// its loop, the others then give up too; in-flight copies and MMAs are
// waited for (bounded) before the tensor memory is freed.
#include "common.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

typedef __nv_bfloat16 bf16;

namespace {

constexpr int TC_TX = 8, TC_TY = 16, TC_HX = TC_TX + 2, TC_HY = TC_TY + 2;
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

constexpr int WS_NA = 2, WS_NT = 192;              // TMEM accumulators, threads
constexpr int CB_STRIDE = 2944;                     // one channel block of the halo tile (2880 used)

template <int CIN, int N> struct TcGeom {
  static constexpr int CB = CIN / 8;
  static constexpr int NS = CIN <= 16 ? 4 : 3;      // A stages (three keep four 32-channel blocks per SM)
  static constexpr size_t a_stage = (size_t)CB * CB_STRIDE;
  static constexpr size_t b_bytes = (size_t)9 * CB * N * 16;
  static constexpr size_t bar_off = NS * a_stage + b_bytes;
  static constexpr int n_bar = 2 * NS + 2 * WS_NA;
  static constexpr size_t smem = bar_off + 8 * n_bar + 16 + 4 * N + 128;   // + TMEM slot, bias, alignment slack
  static constexpr unsigned tx_bytes = (unsigned)CB * TC_HY * TC_HX * 16;
  static constexpr int ACC_COLS = 32;                // one accumulator (>= N FP32 columns)
  static constexpr int TMEM_COLS = WS_NA * ACC_COLS;
  static_assert(N == 16 || N == 32, "accumulator width");
  static_assert(CIN % 16 == 0, "K chunks of 16 channels");
  static_assert(bar_off % 16 == 0 && CB_STRIDE % 128 == 0, "alignment");
};

__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
      : "memory");
}

// bounded wait on an mbarrier phase; false if the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(unsigned a, unsigned parity) {
  unsigned polls = 0;
  while (!mbar_try_wait(a, parity)) {
    if (++polls > TC_WAIT_LIMIT) return false;
    if (polls > 64) __nanosleep(32);          // spin first: most waits end within a few polls
  }
  return true;
}

}  // namespace

// bounded wait by lane 0 of a warp, the result for the whole warp
__device__ __forceinline__ bool warp_wait(unsigned a, unsigned parity, int lane) {
  bool ok = true;
  if (lane == 0) ok = mbar_wait_bounded(a, parity);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// X (through the tensor map tmx): NHWC bf16 [B][H][W][CIN]; Wt: [COUTP][9][CIN]
// bf16 (COUTP >= COUT real output channels, rows beyond COUTP read as zero up
// to N); EPI as in cnn.cu: 0 + bias, ReLU, bf16 [px][N]; 1 + bias, FP32
// [px][2]; 2 times (mask > 0), bf16 [px][N].  err: set to 1 if a wait gave up.
template <int CIN, int N, int EPI>
__global__ void __launch_bounds__(WS_NT) k_conv3x3_tc(const __grid_constant__ CUtensorMap tmx,
                                                      const bf16* __restrict__ Wt, int coutp,
                                                      const float* __restrict__ bias, const bf16* __restrict__ mask,
                                                      void* Yout, int B, int H, int W, int* err) {
  using G = TcGeom<CIN, N>;
  constexpr int CB = G::CB, WS_NS = G::NS;
  extern __shared__ unsigned char tc_raw[];
  const unsigned raw_s = smem_u32(tc_raw);
  const unsigned base = (raw_s + 127u) & ~127u;
  unsigned char* gbase = tc_raw + (base - raw_s);
  unsigned char* Bs = gbase + WS_NS * G::a_stage;
  const unsigned a_s0 = base, b_base = base + (unsigned)(WS_NS * G::a_stage);
  const unsigned bar = base + (unsigned)G::bar_off;
  auto full = [&](int q) { return bar + 8u * (unsigned)q; };
  auto empty = [&](int q) { return bar + 8u * (unsigned)(WS_NS + q); };
  auto accf = [&](int a) { return bar + 8u * (unsigned)(2 * WS_NS + a); };
  auto acce = [&](int a) { return bar + 8u * (unsigned)(2 * WS_NS + WS_NA + a); };
  unsigned* tslot = reinterpret_cast<unsigned*>(gbase + G::bar_off + 8 * G::n_bar);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < WS_NS; ++q) { mbar_init(full(q), 1); mbar_init(empty(q), 1); }
    for (int a = 0; a < WS_NA; ++a) { mbar_init(accf(a), 1); mbar_init(acce(a), 4); }   // acce: one arrival per epilogue warp
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // bias into shared memory (read by the epilogue as broadcasts)
  float* sbias = reinterpret_cast<float*>(gbase + G::bar_off + 8 * G::n_bar + 16);
  if (tid < N) sbias[tid] = (EPI == 0 || (EPI == 1 && tid < 2)) ? bias[tid] : 0.f;
  // weights into the B layout: chunk (t, cb, n) = Wt[n][t][8 cb .. 8 cb + 7]
  for (int i = tid; i < 9 * CB * N; i += WS_NT) {
    const int n = i % N, tcb = i / N, cb = tcb % CB, t = tcb / CB;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (n < coutp) v = *reinterpret_cast<const uint4*>(Wt + ((size_t)n * 9 + t) * CIN + cb * 8);
    *reinterpret_cast<uint4*>(Bs + (size_t)((t * CB + cb) * N + n) * 16) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy weights -> tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tslot;

  const int tiles_x = (W + TC_TX - 1) / TC_TX, tiles_y = (H + TC_TY - 1) / TC_TY;
  const int per_img = tiles_x * tiles_y, ntiles = per_img * B;
  const int nk = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto tile_xy = [&](int k, int& b, int& x0, int& y0) {
    const int tile = (int)blockIdx.x + k * (int)gridDim.x;
    b = tile / per_img;
    const int rem = tile - b * per_img, ty = rem / tiles_x;
    x0 = (rem - ty * tiles_x) * TC_TX;
    y0 = ty * TC_TY;
  };
  bool failed = false;

  if (warp == 0) {
    // ---- producer: tensor copies of the halo tiles
    int issued = 0;
    for (int k = 0; k < nk; ++k) {
      const int q = k % WS_NS;
      if (k >= WS_NS && !warp_wait(empty(q), ((k / WS_NS) - 1) & 1, lane)) { failed = true; break; }
      if (lane == 0) {
        int b, x0, y0;
        tile_xy(k, b, x0, y0);
        mbar_expect_tx(full(q), G::tx_bytes);
        const unsigned dst = a_s0 + (unsigned)(q * G::a_stage);
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) tma_load_4d(dst + cb * CB_STRIDE, &tmx, cb * 8, x0 - 1, y0 - 1, b, full(q));
      }
      __syncwarp();
      issued = k + 1;
    }
    // the last copies have landed before the block can end (the consumer saw
    // them already unless something failed)
    for (int k = max(0, issued - WS_NS); k < issued; ++k)
      if (!warp_wait(full(k % WS_NS), (k / WS_NS) & 1, lane)) failed = true;
  } else if (warp == 1) {
    // ---- MMA issue
    constexpr unsigned idesc = umma_idesc_bf16(128, N);
    constexpr unsigned A_LBO = CB_STRIDE, A_SBO = TC_HX * 16, B_LBO = N * 16, B_SBO = 8 * 16;
    int committed = 0;
    for (int k = 0; k < nk; ++k) {
      const int q = k % WS_NS, a = k % WS_NA;
      if (!warp_wait(full(q), (k / WS_NS) & 1, lane)) { failed = true; break; }
      if (k >= WS_NA && !warp_wait(acce(a), ((k / WS_NA) - 1) & 1, lane)) { failed = true; break; }
      if (lane == 0) {
        tc_fence_after();
        const unsigned a_base = a_s0 + (unsigned)(q * G::a_stage);
        const unsigned d_tmem = tmem + (unsigned)(a * G::ACC_COLS);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int dy = t / 3, dx = t % 3;
#pragma unroll
          for (int kc = 0; kc < CIN / 16; ++kc) {
            const unsigned a_off = (unsigned)((2 * kc) * CB_STRIDE + (dy * TC_HX + dx) * 16);
            const unsigned b_off = (unsigned)((t * CB + 2 * kc) * N * 16);
            tc_mma(d_tmem, umma_desc(a_base + a_off, A_LBO, A_SBO), umma_desc(b_base + b_off, B_LBO, B_SBO),
                   idesc, (t | kc) != 0 ? 1u : 0u);
          }
        }
        tc_commit(empty(q));
        tc_commit(accf(a));
      }
      __syncwarp();
      committed = k + 1;
    }
    // every MMA of this block has completed before the tensor memory is freed
    if (committed > 0 && !warp_wait(accf((committed - 1) % WS_NA), ((committed - 1) / WS_NA) & 1, lane)) failed = true;
  } else {
    // ---- epilogue: thread <-> TMEM lane 32 (warp % 4) + lane <-> pixel (m % 8, m / 8)
    const int qw = warp & 3;
    const int m = 32 * qw + lane;
    const float* bv = sbias;
    for (int k = 0; k < nk; ++k) {
      const int a = k % WS_NA;
      if (!warp_wait(accf(a), (k / WS_NA) & 1, lane)) { failed = true; break; }
      tc_fence_after();
      float acc[N];
      const unsigned trow = tmem + (unsigned)(a * G::ACC_COLS) + ((unsigned)(32 * qw) << 16);
      tc_ld16(trow, acc);
      if constexpr (N == 32) tc_ld16(trow + 16, acc + 16);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce(a));
      int b, x0, y0;
      tile_xy(k, b, x0, y0);
      const int gx = x0 + (m & 7), gy = y0 + (m >> 3);
      if (gx < W && gy < H) {
        const size_t p = (size_t)b * H * W + (size_t)gy * W + gx;
        if (EPI == 0) {
          __nv_bfloat162 o[N / 2];
#pragma unroll
          for (int c = 0; c < N; c += 2)
            o[c / 2] = __floats2bfloat162_rn(fmaxf(acc[c] + bv[c], 0.f), fmaxf(acc[c + 1] + bv[c + 1], 0.f));
#pragma unroll
          for (int v = 0; v < N / 8; ++v)
            reinterpret_cast<uint4*>((bf16*)Yout + p * N)[v] = reinterpret_cast<const uint4*>(o)[v];
        } else if (EPI == 1) {
          *reinterpret_cast<float2*>((float*)Yout + p * 2) = make_float2(acc[0] + bv[0], acc[1] + bv[1]);
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
  }
  if (failed && lane == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS) : "memory");
  }
}

// cuTensorMapEncodeTiled from the driver (no link against the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

template <int CIN, int N, int EPI>
static cudaError_t launch_tc(const bf16* X, const bf16* Wt, int coutp, const float* bias, const bf16* mask, void* Y,
                             int B, int H, int W, int* err, int num_sms, cudaStream_t st) {
  using G = TcGeom<CIN, N>;
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_conv3x3_tc<CIN, N, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
    // resident blocks per SM: shared memory (plus the 1 KB the runtime
    // reserves per block) and the SM's 512 tensor-memory columns
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int n = smem_sm / (int)(G::smem + 1024);
    if (512 / G::TMEM_COLS < n) n = 512 / G::TMEM_COLS;
    per_sm = n < 1 ? 1 : n;
  }
  const long long tiles = (long long)cdiv(W, TC_TX) * cdiv(H, TC_TY) * B;
  const long long cap = (long long)per_sm * num_sms;
  const int grid = (int)(tiles < cap ? tiles : cap);
  if (grid == 0) return cudaSuccess;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  if (!enc || ((uintptr_t)X & 15u)) return cudaErrorInvalidValue;
  // X as a 4D tensor (channels, x, y, image); the box is one channel block of
  // the 10 x 18 halo tile of one image
  CUtensorMap map;
  const cuuint64_t dims[4] = {(cuuint64_t)CIN, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)CIN * 2, (cuuint64_t)W * CIN * 2, (cuuint64_t)H * W * CIN * 2};
  const cuuint32_t box[4] = {8, (cuuint32_t)TC_HX, (cuuint32_t)TC_HY, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)X, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  k_conv3x3_tc<CIN, N, EPI><<<grid, WS_NT, G::smem, st>>>(map, Wt, coutp, bias, mask, Y, B, H, W, err);
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
