// Learned correction network for the FP32 CSLP V-cycle inside FGMRES (not in
// the paper): four 3x3 convolutions on the control-point grid, channels
// 3 -> 32 -> 32 -> 32 -> 2, ReLU after the first three, BF16 weights and
// activations with FP32 accumulation.
//
// The convolutions (forward, and the input gradient as the same convolution
// with flipped, channel-transposed weights and the ReLU mask of the forward
// activation) run on the tcgen05 tensor cores, conv_tc.cu.  The weight
// gradient is an FP32 reduction over pixels; Adam keeps FP32 master weights.
//
// Layouts: activations NHWC bf16 [B][H][W][C] with C padded to 16 (network
// input: Re r, Im r, kappa) or 32; network output FP32 [B][H][W][2];
// parameters flat FP32, layer by layer W[co][3][3][ci] then bias[co].
#include "common.cuh"
#include <cuda_bf16.h>
#include <cmath>
#include <new>

typedef __nv_bfloat16 bf16;

static const int NET_CH[5] = {3, 32, 32, 32, 2};
static const int NET_CP[5] = {16, 32, 32, 32, 16};   // padded channel counts of the stored tensors

struct iga_net {
  int nparam = 0;
  int off_w[4], off_b[4];
  float* master = nullptr;    // FP32 parameters
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  bf16* wf[4] = {};           // forward weights [COUTP][9][CINP]
  bf16* wb[4] = {};           // input-gradient weights [CINP][9][COUTP] (flipped taps)
  int step = 0;
  // activation workspace (grown on demand)
  size_t cap_px = 0;
  bf16* act[4] = {};          // layer inputs: act[0] = network input (16 ch), act[1..3] hidden (32 ch)
  float* out = nullptr;       // [px][2]
  bf16* g16 = nullptr;        // output gradient, 16 ch
  bf16* ga = nullptr;         // hidden gradients (32 ch), ping
  bf16* gb = nullptr;         // pong
  float* part = nullptr;      // wgrad partial sums
  size_t cap_part = 0;
  float* lossbuf = nullptr;   // per-sample (num, den) and the loss
  int cap_b = 0;
  int* tc_err = nullptr;      // set by a tensor-core convolution whose bounded wait gave up
  int num_sms = 148;
  DevBuf bufs;
  std::string err;
};

// ------------------------------------------------------------------ parameter packing
// Forward weights wf [coutf][9][cinp]; input-gradient weights wb [cinp][9][coutb]
// (out and in channels swapped, tap flipped to 8 - t).  Padding entries are 0.
__global__ void k_pack_weights(const float* master, int off_w, int cin, int cout, int cinp, int coutf, int coutb,
                               bf16* wf, bf16* wb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int tot = coutf * 9 * cinp;
  if (idx >= tot) return;
  int co = idx / (9 * cinp), rest = idx - co * 9 * cinp, t = rest / cinp, ci = rest - t * cinp;
  float w = (co < cout && ci < cin) ? master[off_w + (co * 9 + t) * cin + ci] : 0.f;
  wf[idx] = __float2bfloat16_rn(w);
  if (co < coutb) wb[((size_t)ci * 9 + (8 - t)) * coutb + co] = __float2bfloat16_rn(w);
}

__global__ void k_init_params(float* p, int n, unsigned long long seed, int off_w0, int n0, float s0, int off_w1,
                              int n1, float s1, int off_w2, int n2, float s2, int off_w3, int n3, float s3) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // counter-based normal sample (splitmix64 + Box-Muller)
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  double u1 = ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  unsigned long long z2 = z * 0xD1B54A32D192ED03ull + 0x8CB92BA72F3D8DD7ull;
  z2 ^= z2 >> 29;
  double u2 = ((z2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  float s = 0.f;
  if (i >= off_w0 && i < off_w0 + n0) s = s0;
  else if (i >= off_w1 && i < off_w1 + n1) s = s1;
  else if (i >= off_w2 && i < off_w2 + n2) s = s2;
  else if (i >= off_w3 && i < off_w3 + n3) s = s3;
  p[i] = (float)(g * s);          // biases start at zero
}

// ------------------------------------------------------------------ weight gradient (FP32)
// Block: 8 x 8 pixel tile of one image; partial dW[co][t][ci] and db[co] for the
// true channel counts, written to part[block][...]; reduced by k_reduce_part.
template <int CINP, int COUTP>
__global__ void __launch_bounds__(256) k_wgrad(const bf16* __restrict__ X, const bf16* __restrict__ dY, int cin,
                                               int cout, int H, int W, float* part, int nper) {
  constexpr int T = 8, HX = T + 2;
  __shared__ float Xs[HX * HX][CINP + 1];
  __shared__ float Ds[T * T][COUTP + 1];
  const int b = blockIdx.z, x0 = blockIdx.x * T, y0 = blockIdx.y * T;
  const size_t img = (size_t)b * H * W;
  for (int idx = threadIdx.x; idx < HX * HX * CINP; idx += 256) {
    int c = idx % CINP, pix = idx / CINP, hx = pix % HX, hy = pix / HX;
    int gy = y0 - 1 + hy, gx = x0 - 1 + hx;
    Xs[pix][c] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? __bfloat162float(X[(img + (size_t)gy * W + gx) * CINP + c]) : 0.f;
  }
  for (int idx = threadIdx.x; idx < T * T * COUTP; idx += 256) {
    int c = idx % COUTP, pix = idx / COUTP, px = pix % T, py = pix / T;
    int gy = y0 + py, gx = x0 + px;
    Ds[pix][c] = (gy < H && gx < W) ? __bfloat162float(dY[(img + (size_t)gy * W + gx) * COUTP + c]) : 0.f;
  }
  __syncthreads();
  const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  float* out = part + blk * nper;
  const int nw = cout * 9 * cin;
  for (int e = threadIdx.x; e < nw + cout; e += 256) {
    float s = 0.f;
    if (e < nw) {
      int co = e / (9 * cin), rest = e - co * 9 * cin, t = rest / cin, ci = rest - t * cin;
      int dy = t / 3, dx = t % 3;
      for (int py = 0; py < T; ++py)
        for (int px = 0; px < T; ++px) s += Ds[py * T + px][co] * Xs[(py + dy) * HX + px + dx][ci];
    } else {
      int co = e - nw;
      for (int pix = 0; pix < T * T; ++pix) s += Ds[pix][co];
    }
    out[e] = s;
  }
}

// grad[off + e] = sum over blocks of part[blk][e] (fixed order)
__global__ void k_reduce_part(const float* part, int nblk, int nper, float* grad, int off) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nper) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * nper + e];
  grad[off + e] = s;
}

// ------------------------------------------------------------------ loss, Adam
// per sample (num, den) = (sum (y - t)^2, sum t^2); one block per sample
__global__ void k_loss_sums(const float* Y, const float* T, size_t px, float* sums) {
  const int b = blockIdx.x;
  const float* y = Y + (size_t)b * px * 2;
  const float* t = T + (size_t)b * px * 2;
  float num = 0.f, den = 0.f;
  for (size_t i = threadIdx.x; i < px * 2; i += blockDim.x) {
    float d = y[i] - t[i];
    num += d * d;
    den += t[i] * t[i];
  }
  __shared__ float sn[256], sd[256];
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) { sn[threadIdx.x] += sn[threadIdx.x + s]; sd[threadIdx.x] += sd[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { sums[2 * b] = sn[0]; sums[2 * b + 1] = sd[0]; }
}
// dY (bf16, 16 channels) = 2 (y - t) / (den_b * B); loss = mean num/den
__global__ void k_loss_grad(const float* Y, const float* T, size_t px, int B, const float* sums, bf16* g16,
                            float* loss) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i == 0) {
    float L = 0.f;
    for (int b = 0; b < B; ++b) L += sums[2 * b] / fmaxf(sums[2 * b + 1], 1e-30f);
    *loss = L / B;
  }
  if (i >= px * B) return;
  int b = (int)(i / px);
  float sc = 2.f / (fmaxf(sums[2 * b + 1], 1e-30f) * B);
  __nv_bfloat162 d = __floats2bfloat162_rn(sc * (Y[2 * i] - T[2 * i]), sc * (Y[2 * i + 1] - T[2 * i + 1]));
  __nv_bfloat162* o = (__nv_bfloat162*)(g16 + i * 16);
  o[0] = d;
  __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
  for (int k = 1; k < 8; ++k) o[k] = z;
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------ host helpers
static iga_status net_err(iga_net* n, iga_status s, const char* msg) {
  if (n) n->err = msg;
  return s;
}

template <typename T> static T* nalloc(iga_net* n, size_t count) {
  void* p = nullptr;
  if (cudaMalloc(&p, (count ? count : 1) * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  n->bufs.ptrs.push_back(p);
  return (T*)p;
}

static iga_status net_pack(iga_net* n, cudaStream_t st) {
  for (int l = 0; l < 4; ++l) {
    // output layer: 8 padded output channels in the forward kernel, 16 in the
    // gradient tensor that feeds its input-gradient kernel
    int coutf = l == 3 ? 8 : NET_CP[l + 1];
    int coutb = NET_CP[l + 1];
    int tot = coutf * 9 * NET_CP[l];
    k_pack_weights<<<cdiv(tot, 256), 256, 0, st>>>(n->master, n->off_w[l], NET_CH[l], NET_CH[l + 1], NET_CP[l], coutf,
                                                   coutb, n->wf[l], n->wb[l]); iga_count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? IGA_OK : IGA_E_CUDA;
}

static iga_status net_workspace(iga_net* n, int B, int H, int W) {
  size_t px = (size_t)B * H * W;
  if (px > n->cap_px) {
    for (int l = 0; l < 4; ++l) n->act[l] = nalloc<bf16>(n, px * (l == 0 ? 16 : 32));
    n->out = nalloc<float>(n, px * 2);
    n->g16 = nalloc<bf16>(n, px * 16);
    n->ga = nalloc<bf16>(n, px * 32);
    n->gb = nalloc<bf16>(n, px * 32);
    if (!n->act[0] || !n->act[1] || !n->act[2] || !n->act[3] || !n->out || !n->g16 || !n->ga || !n->gb)
      return net_err(n, IGA_E_OOM, "net activations");
    n->cap_px = px;
  }
  size_t nblk = (size_t)B * cdiv(H, 8) * cdiv(W, 8);
  size_t need = nblk * (32 * 9 * 32 + 32);
  if (need > n->cap_part) {
    n->part = nalloc<float>(n, need);
    if (!n->part) return net_err(n, IGA_E_OOM, "net partials");
    n->cap_part = need;
  }
  if (B > n->cap_b) {
    n->lossbuf = nalloc<float>(n, 2 * (size_t)B + 2);
    if (!n->lossbuf) return net_err(n, IGA_E_OOM, "net loss");
    n->cap_b = B;
  }
  return IGA_OK;
}

cudaError_t conv_tc_launch(int cin, int n, int epi, const bf16* X, const bf16* Wt, int coutp, const float* bias,
                           const bf16* mask, void* Y, int B, int H, int W, int* err, int num_sms, cudaStream_t st);

// one convolution layer on the tensor cores (conv_tc.cu): CIN input channels,
// N accumulator columns, Wt with coutp rows
static void conv(iga_net* n, int cin, int N, int epi, const bf16* X, const bf16* Wt, int coutp, const float* bias,
                 const bf16* mask, void* Y, int B, int H, int W, cudaStream_t st) {
  conv_tc_launch(cin, N, epi, X, Wt, coutp, bias, mask, Y, B, H, W, n->tc_err, n->num_sms, st);
}

// forward: act[0] already holds the input; result in n->out (the output
// layer runs with 16 accumulator columns: its 8 stored weight rows and zeros)
static void net_forward(iga_net* n, int B, int H, int W, cudaStream_t st) {
  conv(n, 16, 32, 0, n->act[0], n->wf[0], 32, n->master + n->off_b[0], nullptr, n->act[1], B, H, W, st);
  conv(n, 32, 32, 0, n->act[1], n->wf[1], 32, n->master + n->off_b[1], nullptr, n->act[2], B, H, W, st);
  conv(n, 32, 32, 0, n->act[2], n->wf[2], 32, n->master + n->off_b[2], nullptr, n->act[3], B, H, W, st);
  conv(n, 32, 16, 1, n->act[3], n->wf[3], 8, n->master + n->off_b[3], nullptr, n->out, B, H, W, st);
}

// status of the tensor-core waits since the last check (synchronises)
static iga_status net_check_tc(iga_net* n, cudaStream_t st) {
  int h = 0;
  if (cudaMemcpyAsync(&h, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return net_err(n, IGA_E_CUDA, "net: stream error");
  if (h) {
    cudaMemsetAsync(n->tc_err, 0, sizeof(int), st);
    return net_err(n, IGA_E_TIMEOUT, "net: a tensor-core accumulator wait gave up");
  }
  return IGA_OK;
}

template <int CINP, int COUTP>
static void net_wgrad(iga_net* n, int l, const bf16* X, const bf16* dY, int B, int H, int W, cudaStream_t st) {
  dim3 grid(cdiv(W, 8), cdiv(H, 8), B);
  int nblk = grid.x * grid.y * grid.z;
  int nper = NET_CH[l + 1] * 9 * NET_CH[l] + NET_CH[l + 1];
  k_wgrad<CINP, COUTP><<<grid, 256, 0, st>>>(X, dY, NET_CH[l], NET_CH[l + 1], H, W, n->part, nper); iga_count_launch();
  k_reduce_part<<<cdiv(nper, 256), 256, 0, st>>>(n->part, nblk, nper, n->grad, n->off_w[l]); iga_count_launch();
}

// loss and gradient for (act[0], T); gradient into n->grad, loss into lossbuf[2B]
static void net_backward(iga_net* n, const float* T, int B, int H, int W, cudaStream_t st) {
  size_t px = (size_t)H * W;
  net_forward(n, B, H, W, st);
  k_loss_sums<<<B, 256, 0, st>>>(n->out, T, px, n->lossbuf); iga_count_launch();
  k_loss_grad<<<cdiv(px * B, 256), 256, 0, st>>>(n->out, T, px, B, n->lossbuf, n->g16, n->lossbuf + 2 * B); iga_count_launch();
  // layer 4 (32 -> 2): weight gradient, then input gradient through the ReLU of act[3]
  net_wgrad<32, 16>(n, 3, n->act[3], n->g16, B, H, W, st);
  conv(n, 16, 32, 2, n->g16, n->wb[3], 32, nullptr, n->act[3], n->ga, B, H, W, st);
  net_wgrad<32, 32>(n, 2, n->act[2], n->ga, B, H, W, st);
  conv(n, 32, 32, 2, n->ga, n->wb[2], 32, nullptr, n->act[2], n->gb, B, H, W, st);
  net_wgrad<32, 32>(n, 1, n->act[1], n->gb, B, H, W, st);
  conv(n, 32, 32, 2, n->gb, n->wb[1], 32, nullptr, n->act[1], n->ga, B, H, W, st);
  net_wgrad<16, 32>(n, 0, n->act[0], n->ga, B, H, W, st);
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int iga_net_num_params(void) {
  int n = 0;
  for (int l = 0; l < 4; ++l) n += NET_CH[l + 1] * 9 * NET_CH[l] + NET_CH[l + 1];
  return n;
}

iga_status iga_net_create(unsigned long long seed, iga_net** out) {
  if (!out) return IGA_E_INVALID;
  *out = nullptr;
  iga_net* n = new (std::nothrow) iga_net();
  if (!n) return IGA_E_OOM;
  int k = 0;
  for (int l = 0; l < 4; ++l) {
    n->off_w[l] = k;
    k += NET_CH[l + 1] * 9 * NET_CH[l];
    n->off_b[l] = k;
    k += NET_CH[l + 1];
  }
  n->nparam = k;
  n->master = nalloc<float>(n, k);
  n->grad = nalloc<float>(n, k);
  n->m = nalloc<float>(n, k);
  n->v = nalloc<float>(n, k);
  n->tc_err = nalloc<int>(n, 1);
  bool ok = n->master && n->grad && n->m && n->v && n->tc_err;
  for (int l = 0; l < 4 && ok; ++l) {
    size_t sz = (size_t)(l == 3 ? 16 : NET_CP[l + 1]) * 9 * 32;
    n->wf[l] = nalloc<bf16>(n, sz);
    n->wb[l] = nalloc<bf16>(n, sz);
    ok = n->wf[l] && n->wb[l];
  }
  if (!ok) { delete n; return IGA_E_OOM; }
  cudaMemset(n->tc_err, 0, sizeof(int));
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  cudaMemset(n->m, 0, sizeof(float) * k);
  cudaMemset(n->v, 0, sizeof(float) * k);
  cudaMemset(n->grad, 0, sizeof(float) * k);
  for (int l = 0; l < 4; ++l) {
    size_t sz = (size_t)(l == 3 ? 16 : NET_CP[l + 1]) * 9 * 32;
    cudaMemset(n->wf[l], 0, sizeof(bf16) * sz);
    cudaMemset(n->wb[l], 0, sizeof(bf16) * sz);
  }
  // He initialisation for the ReLU layers, small output layer
  float s[4];
  for (int l = 0; l < 4; ++l) s[l] = sqrtf(2.f / (9.f * NET_CH[l])) * (l == 3 ? 0.1f : 1.f);
  k_init_params<<<cdiv(k, 256), 256>>>(n->master, k, seed, n->off_w[0], n->off_b[0] - n->off_w[0], s[0], n->off_w[1],
                                      n->off_b[1] - n->off_w[1], s[1], n->off_w[2], n->off_b[2] - n->off_w[2], s[2],
                                      n->off_w[3], n->off_b[3] - n->off_w[3], s[3]); iga_count_launch();
  if (net_pack(n, 0) != IGA_OK || cudaDeviceSynchronize() != cudaSuccess) { delete n; return IGA_E_CUDA; }
  *out = n;
  return IGA_OK;
}

void iga_net_destroy(iga_net* n) {
  if (!n) return;
  cudaDeviceSynchronize();
  delete n;
}

const char* iga_net_last_error(const iga_net* n) { return n ? n->err.c_str() : "null network"; }

iga_status iga_net_get_params(iga_net* n, float* host, int cap) {
  if (!n || !host || cap < n->nparam) return IGA_E_INVALID;
  return cudaMemcpy(host, n->master, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost) == cudaSuccess ? IGA_OK : IGA_E_CUDA;
}

iga_status iga_net_set_params(iga_net* n, const float* host, int count) {
  if (!n || !host || count != n->nparam) return IGA_E_INVALID;
  if (cudaMemcpy(n->master, host, sizeof(float) * n->nparam, cudaMemcpyHostToDevice) != cudaSuccess) return IGA_E_CUDA;
  cudaMemset(n->m, 0, sizeof(float) * n->nparam);
  cudaMemset(n->v, 0, sizeof(float) * n->nparam);
  n->step = 0;
  TRY(net_pack(n, 0));
  return cudaDeviceSynchronize() == cudaSuccess ? IGA_OK : IGA_E_CUDA;
}

iga_status iga_net_forward(iga_net* n, const void* x, float* y, int B, int H, int W, void* stream) {
  if (!n || !x || !y || B < 1 || H < 1 || W < 1) return IGA_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(net_workspace(n, B, H, W));
  if (cudaMemcpyAsync(n->act[0], x, sizeof(bf16) * (size_t)B * H * W * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return IGA_E_CUDA;
  net_forward(n, B, H, W, st);
  if (cudaMemcpyAsync(y, n->out, sizeof(float) * (size_t)B * H * W * 2, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return IGA_E_CUDA;
  return cudaGetLastError() == cudaSuccess ? IGA_OK : IGA_E_CUDA;
}

// Loss and gradient without an update; grad_host (nparam floats) and loss_host
// are HOST pointers (either may be NULL).  Synchronises.
iga_status iga_net_grad(iga_net* n, const void* x, const float* t, int B, int H, int W, float* grad_host,
                        float* loss_host, void* stream) {
  if (!n || !x || !t || B < 1 || H < 1 || W < 1) return IGA_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(net_workspace(n, B, H, W));
  if (cudaMemcpyAsync(n->act[0], x, sizeof(bf16) * (size_t)B * H * W * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return IGA_E_CUDA;
  net_backward(n, t, B, H, W, st);
  if (grad_host && cudaMemcpyAsync(grad_host, n->grad, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return IGA_E_CUDA;
  if (loss_host && cudaMemcpyAsync(loss_host, n->lossbuf + 2 * B, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return IGA_E_CUDA;
  return net_check_tc(n, st);
}

// One Adam step (FP32 master weights) on the batch; loss_host (HOST, may be
// NULL) receives the batch loss before the update.  Asynchronous unless
// loss_host is given.
iga_status iga_net_train_step(iga_net* n, const void* x, const float* t, int B, int H, int W, float lr,
                              float* loss_host, void* stream) {
  if (!n || !x || !t || B < 1 || H < 1 || W < 1 || !(lr > 0.f)) return IGA_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(net_workspace(n, B, H, W));
  if (cudaMemcpyAsync(n->act[0], x, sizeof(bf16) * (size_t)B * H * W * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return IGA_E_CUDA;
  net_backward(n, t, B, H, W, st);
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
  k_adam<<<cdiv(n->nparam, 256), 256, 0, st>>>(n->master, n->grad, n->m, n->v, n->nparam, lr, b1, b2, 1e-8f, c1, c2); iga_count_launch();
  TRY(net_pack(n, st));
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, n->lossbuf + 2 * B, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return IGA_E_CUDA;
    return net_check_tc(n, st);
  }
  return cudaGetLastError() == cudaSuccess ? IGA_OK : IGA_E_CUDA;
}

}  // extern "C"

// ------------------------------------------------------------------ solver integration
// Pack a complex grid vector r (FP32 or FP64) into the network input:
// channels (Re r / s, Im r / s, kappa) in bf16, kappa = (k h)^2 at the dof's
// Greville point, s = RMS of r (device scalar).
template <typename C>
__global__ void k_net_pack(const C* r, int nx, int ny, int x0, int y0, int Hc, int Wc, const double* knots, int p,
                           int n_el, KFieldDev kf, const double* rms, bf16* X) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)Hc * Wc) return;
  int cy = (int)(i / Wc), cx = (int)(i - (size_t)cy * Wc);
  int iy = y0 + cy, ix = x0 + cx;
  float re = 0.f, im = 0.f, kap = 0.f;
  if (iy < ny && ix < nx) {
    double inv = *rms > 0.0 ? 1.0 / *rms : 0.0;
    C v = r[(size_t)iy * nx + ix];
    re = (float)(v.x * inv);
    im = (float)(v.y * inv);
    // Greville abscissae of full basis functions ix+1, iy+1
    double gx = 0.0, gy = 0.0;
    for (int a = 1; a <= p; ++a) { gx += knots[ix + 1 + a]; gy += knots[iy + 1 + a]; }
    gx /= p;
    gy /= p;
    double h = 1.0 / n_el;
    kap = (float)(kfield_k2(kf, gx, gy) * h * h);
  }
  __nv_bfloat162* o = (__nv_bfloat162*)(X + i * 16);
  o[0] = __floats2bfloat162_rn(re, im);
  o[1] = __floats2bfloat162_rn(kap, 0.f);
  __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
  for (int k = 2; k < 8; ++k) o[k] = z;
}

// target e / (s * gamma) as FP32 pairs for training crops
__global__ void k_net_target(const double2* e, int nx, int ny, int x0, int y0, int Hc, int Wc, const double* rms,
                             double gamma, float* T) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)Hc * Wc) return;
  int cy = (int)(i / Wc), cx = (int)(i - (size_t)cy * Wc);
  int iy = y0 + cy, ix = x0 + cx;
  float a = 0.f, b = 0.f;
  if (iy < ny && ix < nx && *rms > 0.0) {
    double sc = 1.0 / (*rms * gamma);
    double2 v = e[(size_t)iy * nx + ix];
    a = (float)(v.x * sc);
    b = (float)(v.y * sc);
  }
  T[2 * i] = a;
  T[2 * i + 1] = b;
}

__global__ void k_sub_f2(float2* a, const float2* b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = a[i] - b[i];
}

// RMS of a complex vector: per-block partial sums of |r_i|^2 into out[2 + b],
// then one block adds them in a fixed order into out[0].  out holds
// 2 + IGA_RMS_BLOCKS doubles.
constexpr int IGA_RMS_BLOCKS = 256;
template <typename C>
__global__ void k_rms_part(const C* r, size_t n, double* out) {
  __shared__ double s[256];
  double a = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a += (double)r[i].x * r[i].x + (double)r[i].y * r[i].y;
  s[threadIdx.x] = a;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[2 + blockIdx.x] = s[0];
}
__global__ void k_rms_finish(size_t n, int nb, double* out) {
  __shared__ double s[256];
  s[threadIdx.x] = threadIdx.x < nb ? out[2 + threadIdx.x] : 0.0;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(s[0] / (double)n);
}
template <typename C>
static void launch_rms(const C* r, size_t n, double* out, cudaStream_t st) {
  int nb = (int)std::max<size_t>(1, std::min<size_t>(IGA_RMS_BLOCKS, cdiv(n, 2048)));
  k_rms_part<C><<<nb, 256, 0, st>>>(r, n, out); iga_count_launch();
  k_rms_finish<<<1, 256, 0, st>>>(n, nb, out); iga_count_launch();
}

// z += gamma * s * y  if every output is finite (else z stays the plain V-cycle result)
__global__ void k_net_flag(const float* y, size_t n, int* bad) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n && !(isfinite(y[2 * i]) && isfinite(y[2 * i + 1]))) atomicExch(bad, 1);
}
__global__ void k_net_correct(float2* z, const float* y, size_t n, const double* rms, float gamma, const int* bad) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n || *bad) return;
  float sc = (float)(*rms) * gamma;
  z[i] = make_float2(z[i].x + sc * y[2 * i], z[i].y + sc * y[2 * i + 1]);
}

// Learned correction of the FP32 V-cycle: z += gamma s NN(r~ / s), r~ = r - M_beta z.
iga_status net_correct(iga_ctx* ctx, const float2* r, float2* z) {
  iga_net* n = ctx->net;
  LevelData& L = ctx->lv[0];
  cudaStream_t st = ctx->st;
  const int H = L.ny, W = L.nx;
  TRY(net_workspace(n, 1, H, W));
  float2* rt = L.fr;
  TRY(op_apply<float>(ctx, 0, OP_MB, z, rt, r, EPI_ZMINUS, nullptr, 0.0));
  launch_rms<float2>(rt, L.n, ctx->net_rms, st);
  k_net_pack<float2><<<cdiv(L.n, 256), 256, 0, st>>>(rt, W, H, 0, 0, H, W, L.knots, ctx->p, L.n_el, ctx->kf,
                                                      ctx->net_rms, n->act[0]); iga_count_launch();
  net_forward(n, 1, H, W, st);
  CK(cudaMemsetAsync(ctx->net_bad, 0, sizeof(int), st));
  k_net_flag<<<cdiv(L.n, 256), 256, 0, st>>>(n->out, L.n, ctx->net_bad); iga_count_launch();
  k_net_correct<<<cdiv(L.n, 256), 256, 0, st>>>(z, n->out, L.n, ctx->net_rms, (float)ctx->net_gamma, ctx->net_bad); iga_count_launch();
  CKL();
  return IGA_OK;
}

extern "C" {

// Attach a trained network: in precision 1 every preconditioner application
// becomes z = V(v) + gamma s NN(r~ / s) (NULL detaches).
iga_status iga_attach_net(iga_ctx* ctx, iga_net* net, double gamma) {
  if (!ctx) return IGA_E_INVALID;
  if (net && (ctx->prm.precision != 1 || ctx->dim != 2))
    return set_err(ctx, IGA_E_INVALID, "the learned correction needs a 2D context in precision 1");
  if (!ctx->net_rms) {
    ctx->net_rms = dalloc<double>(ctx, 2 + IGA_RMS_BLOCKS);
    ctx->net_bad = dalloc<int>(ctx, 1);
    if (!ctx->net_rms || !ctx->net_bad) return set_err(ctx, IGA_E_OOM, "net scalars");
  }
  if (net) {
    iga_status s = net_workspace(net, 1, ctx->lv[0].ny, ctx->lv[0].nx);
    if (s != IGA_OK) return set_err(ctx, s, "net workspace");
  }
  ctx->net = net;
  ctx->net_gamma = gamma;
  // the cached loop graph captured the previous preconditioner
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->gexec = nullptr;
  ctx->graph = nullptr;
  return IGA_OK;
}

// Training pair from a preconditioner input v (DEVICE, n complex128), built
// from the error propagation of the FP32 V-cycle V (no inverse needed):
// e_0 = V(v), then `cycles` times e <- e - V(M_beta e); rt = M_beta e.  The
// network's task NN(rt) ~ e is then exactly the inference-time task (the error
// M_beta^{-1} rt left by a V-cycle).  rt, e: DEVICE complex128.
iga_status iga_precond_pair(iga_ctx* ctx, const iga_c128* v, iga_c128* rt, iga_c128* e, int cycles) {
  if (!ctx || !v || !rt || !e || cycles < 1) return IGA_E_INVALID;
  LevelData& L = ctx->lv[0];
  size_t n = L.n;
  cudaStream_t st = ctx->st;
  launch_convert_d2f((const double2*)v, ctx->fin, n, st);
  TRY(mg_vcycle<float>(ctx, ctx->fin, ctx->fout));            // e_0 in fout
  float2* ecur = ctx->fout;
  float2* r = ctx->fin;
  float2* z = L.fr;
  for (int c = 0; c < cycles; ++c) {
    TRY(op_apply<float>(ctx, 0, OP_MB, ecur, r, nullptr, EPI_Y, nullptr, 0.0));   // r = M e
    TRY(mg_vcycle<float>(ctx, r, z));                                              // z = V(r)
    k_sub_f2<<<cdiv(n, 256), 256, 0, st>>>(ecur, z, n); iga_count_launch();        // e -= z
  }
  TRY(op_apply<float>(ctx, 0, OP_MB, ecur, r, nullptr, EPI_Y, nullptr, 0.0));     // rt = M e
  launch_convert_f2d(r, (double2*)rt, n, st);
  launch_convert_f2d(ecur, (double2*)e, n, st);
  CKL();
  return IGA_OK;
}

// Crop [y0, y0+Hc) x [x0, x0+Wc) of (rt, e) into a training sample: X (DEVICE
// bf16 [Hc][Wc][16]) and, if e and T are given, T (DEVICE FP32 [Hc][Wc][2]) =
// e / (rms(rt) * gamma).  Out-of-grid pixels are zero.
iga_status iga_net_pack(iga_ctx* ctx, const iga_c128* rt, const iga_c128* e, int x0, int y0, int Hc, int Wc,
                        void* X, float* T, double gamma) {
  if (!ctx || !rt || !X || Hc < 1 || Wc < 1 || x0 < 0 || y0 < 0 || ctx->dim != 2) return IGA_E_INVALID;
  LevelData& L = ctx->lv[0];
  if (!ctx->net_rms) {
    ctx->net_rms = dalloc<double>(ctx, 2 + IGA_RMS_BLOCKS);
    ctx->net_bad = dalloc<int>(ctx, 1);
    if (!ctx->net_rms || !ctx->net_bad) return set_err(ctx, IGA_E_OOM, "net scalars");
  }
  launch_rms<double2>((const double2*)rt, L.n, ctx->net_rms, ctx->st);
  size_t px = (size_t)Hc * Wc;
  k_net_pack<double2><<<cdiv(px, 256), 256, 0, ctx->st>>>((const double2*)rt, L.nx, L.ny, x0, y0, Hc, Wc, L.knots,
                                                          ctx->p, L.n_el, ctx->kf, ctx->net_rms, (bf16*)X); iga_count_launch();
  if (e && T) {
    k_net_target<<<cdiv(px, 256), 256, 0, ctx->st>>>((const double2*)e, L.nx, L.ny, x0, y0, Hc, Wc, ctx->net_rms,
                                                     gamma, T); iga_count_launch();
  }
  CKL();
  return IGA_OK;
}

}  // extern "C"
