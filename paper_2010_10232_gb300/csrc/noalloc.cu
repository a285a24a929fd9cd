// Allocation-free modified Gram-Schmidt sweep.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework whose
// caching allocator owns all device memory, or a latency-critical loop that
// must not pay cudaMalloc's implicit device synchronisation.  For them this
// file offers iga_mgs_noalloc: the same MGS sweep as iga_mgs, but with no
// context and no allocation.  Its only scratch (the per-block partial sums of
// the deterministic reductions) lives in the file-scope device array below,
// which every GPU that loads this library holds until the process exits.
#include "common.cuh"
#include <mutex>

// Largest reduction grid the static scratch can serve: two buffers of
// (re, im) partial sums per block, 1024 blocks -> 4096 doubles = 32 KiB.
#define IGA_NOALLOC_MAX_BLOCKS 1024
#define IGA_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_mgs_scratch[4 * IGA_NOALLOC_MAX_BLOCKS];

// MGS kernels (defined with the Krylov solver).
__global__ void k_mgs_step(const double2* V, size_t ldv, size_t n, int i, int j, double2* w,
                           const double* part_in, double* part_out, double2* h);
__global__ void k_finish_h(const double* part, int nb, double2* h);

// Device address of g_mgs_scratch, looked up once per device.  In host code the
// array's name only stands in for the device symbol, so the kernels are given
// this address instead.  The cache lives for the process: after a
// cudaDeviceReset the address would be stale (the header says so).
static double* g_scratch_addr[IGA_NOALLOC_MAX_DEVICES];
static int g_sms[IGA_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

static iga_status scratch_for_current_device(double** out, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= IGA_NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return IGA_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_mgs_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return IGA_E_CUDA;
    }
    int n_sms = 0;
    if (cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return IGA_E_CUDA;
    }
    g_sms[dev] = n_sms;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  *sms = g_sms[dev];
  return IGA_OK;
}

extern "C" iga_status iga_mgs_noalloc(const iga_c128* V, size_t ldv, size_t n, int j, iga_c128* w, iga_c128* h,
                                      void* stream) {
  if (!V || !w || !h || ((uintptr_t)V & 15u) || ((uintptr_t)w & 15u) || ((uintptr_t)h & 15u)) return IGA_E_INVALID;
  if (n == 0 || ldv < n || j < 0) return IGA_E_INVALID;
  double* scratch = nullptr;
  int sms = 0;
  iga_status s = scratch_for_current_device(&scratch, &sms);
  if (s != IGA_OK) return s;
  // same grid rule as the context path: two blocks per SM
  size_t nb = (size_t)2 * sms;
  if (nb > IGA_NOALLOC_MAX_BLOCKS) return IGA_E_INVALID;   // more SMs than the static scratch serves
  cudaStream_t st = (cudaStream_t)stream;
  double* pa = scratch;
  double* pb = scratch + 2 * nb;
  const double2* Vd = (const double2*)V;
  double2* wd = (double2*)w;
  double2* hd = (double2*)h;
  // Every partial sum is written before it is read, so the scratch needs no
  // clearing between calls.
  for (int i = 0; i <= j + 1; ++i) {
    const double* pin = (i & 1) ? pa : pb;
    double* pout = (i & 1) ? pb : pa;
    k_mgs_step<<<(unsigned)nb, IGA_RED_THREADS, 0, st>>>(Vd, ldv, n, i, j, wd, pin, pout, hd); iga_count_launch();
  }
  const double* plast = ((j + 1) & 1) ? pb : pa;
  k_finish_h<<<1, IGA_RED_THREADS, 0, st>>>(plast, (int)nb, hd + j + 1); iga_count_launch();
  return cudaGetLastError() == cudaSuccess ? IGA_OK : IGA_E_CUDA;
}
