// Measured peak rates of the plain ALUs (no tensor cores), the denominators
// of the root stage's roofline.  Each thread runs independent chains of fused
// multiply-adds, enough of them per SM to hide the pipeline latency:
//   kind 0  FP32        fma.rn.f32      (1 FMA = 2 flops per instruction)
//   kind 1  FP32 pairs  fma.rn.f32x2    (2 FMAs = 4 flops per instruction)
//   kind 2  FP64        fma.rn.f64
// The chains multiply by a factor just below 1 and add a small constant, so
// the values stay finite and normal; the result is stored only under a
// condition the compiler cannot decide, which keeps every FMA.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ftp.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a,
                                                        unsigned long long b,
                                                        unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__global__ void __launch_bounds__(kThreads) fma_f32_kernel(int iters, float a, float b,
                                                            float* out) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == -1.0f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_f32x2_kernel(int iters, float a, float b,
                                                              float* out) {
  unsigned long long x[8];
  const unsigned long long A = pack2(a, a), B = pack2(b, b);
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = pack2((float)(threadIdx.x + i), (float)(i - threadIdx.x));
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fma_f32x2(x[i], A, B);
  }
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s ^= x[i];
  if (s == 1ull) out[blockIdx.x] = 1.0f;
}

__global__ void __launch_bounds__(kThreads) fma_f64_kernel(int iters, double a, double b,
                                                            float* out) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (double)(threadIdx.x + i);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == -1.0) out[blockIdx.x] = (float)s;
}

}  // namespace

extern "C" ftp_status ftp_alu_peak(int device, int kind, int iters, double* flops, float* ms) {
  if (kind < 0 || kind > 2 || iters < 1 || iters > (1 << 26) || !flops || !ms)
    return FTP_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return FTP_ERR_INVALID_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return FTP_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * kBlocksPerSm;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ftp_status st = FTP_OK;
  if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = FTP_ERR_CUDA;
  } else {
    const float af = 0.99999994f, bf = 1e-3f;
    const double ad = 0.9999999999999999, bd = 1e-3;
    auto launch = [&](int n) {
      if (kind == 0) fma_f32_kernel<<<blocks, kThreads>>>(n, af, bf, out);
      else if (kind == 1) fma_f32x2_kernel<<<blocks, kThreads>>>(n, af, bf, out);
      else fma_f64_kernel<<<blocks, kThreads>>>(n, ad, bd, out);
    };
    launch(iters < 16 ? iters : 16);  // warm-up
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      st = FTP_ERR_CUDA;
    } else {
      cudaEventElapsedTime(ms, e0, e1);
      // flops per thread and outer iteration: 16 x 8 FMAs (FP32), 16 x 8 pairs
      // (FP32 pairs), 4 x 8 FMAs (FP64)
      const double per_iter = kind == 0 ? 256.0 : kind == 1 ? 512.0 : 64.0;
      *flops = per_iter * (double)iters * (double)blocks * kThreads;
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaSetDevice(prev);
  return st;
}
