// FMA-throughput probe (a measurement tool, not part of the solver library):
// it states the ALU ceiling of the FP64 operators beside the nominal figure.
// Every thread runs 8 independent FMA chains.  Built into
// measure/lib/libiga_measure.so by measure/build.py.
#include <cuda_runtime.h>

template <typename T>
__global__ void k_fma_probe(int iters, T* sink) {
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  const T m = (T)0.999999, c = (T)1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = a[k] * m + c;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == (T)12345.678) sink[0] = s;   // practically never: keeps the chains live
}

// Launches 8 x SM-count blocks of 256 threads in FP64 (precision 0) or FP32
// (1) on `stream`; *flops (host) receives the flop count of the launch so the
// caller can time it.  Returns 0, -1 for a bad argument, -2 for a CUDA error.
extern "C" int measure_probe_fma(int precision, int iters, void* sink, void* stream, double* flops) {
  if (!sink || iters < 1 || !flops) return -1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = sms * 8, threads = 256;
  if (precision == 0) k_fma_probe<double><<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, (double*)sink);
  else k_fma_probe<float><<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, (float*)sink);
  *flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
