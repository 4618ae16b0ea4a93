// fp32_peak.cu -- measured FP32 (and FP64) FMA throughput of the device, the denominators
// of the ALU rooflines that bench.py reports for the solve kernels. Every thread runs eight
// independent chains of fused multiply-adds (scalar fma.rn.f32, packed fma.rn.f32x2, which
// issues two FMAs per instruction, and fma.rn.f64) on a grid of 8 CTAs of 256 threads per
// SM; the best of five CUDA-event timed launches is printed as one JSON line:
//   {"ffma_tflops": ..., "ffma2_tflops": ..., "dfma_tflops": ..., "sms": ..., "clock_mhz": ...}
// Built beside libmts.so by build_lib.py; run by bench.py.
#include <cstdio>

#include <cuda_runtime.h>

typedef unsigned long long u64;

__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__global__ void chains_f32(float* out, int iters, float x) {
  float a[8];
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], x, 1e-7f);
  }
  float s = 0.0f;
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void chains_f32x2(float* out, int iters, float x) {
  u64 a[8], xx, cc;
  asm("mov.b64 %0, {%1,%2};" : "=l"(xx) : "f"(x), "f"(x));
  asm("mov.b64 %0, {%1,%2};" : "=l"(cc) : "f"(1e-7f), "f"(1e-7f));
  for (int i = 0; i < 8; ++i) {
    const float v = threadIdx.x * 1e-3f + i;
    asm("mov.b64 %0, {%1,%2};" : "=l"(a[i]) : "f"(v), "f"(v));
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = ffma2(a[i], xx, cc);
  }
  float s = 0.0f;
  for (int i = 0; i < 8; ++i) {
    float lo, hi;
    asm("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i]));
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void chains_f64(float* out, int iters, double x) {
  double a[8];
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fma(a[i], x, 1e-7);
  }
  double s = 0.0;
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

int main() {
  int dev = 0, sms = 0, clk_khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double tf[3] = {0.0, 0.0, 0.0};
  for (int kind = 0; kind < 3; ++kind) {
    const int n_it = kind == 2 ? iters / 64 : iters;  // FP64 runs at a small fraction of FP32
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
      cudaEventRecord(e0);
      if (kind == 0) chains_f32<<<blocks, threads>>>(out, n_it, 0.999f);
      else if (kind == 1) chains_f32x2<<<blocks, threads>>>(out, n_it, 0.999f);
      else chains_f64<<<blocks, threads>>>(out, n_it, 0.999);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    const double flops = 2.0 * 64.0 * n_it * (double)blocks * threads * (kind == 1 ? 2 : 1);
    tf[kind] = flops / (best * 1e-3) / 1e12;
  }
  const cudaError_t e = cudaGetLastError();
  cudaFree(out);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "%s\n", cudaGetErrorString(e));
    return 1;
  }
  std::printf("{\"ffma_tflops\": %.3f, \"ffma2_tflops\": %.3f, \"dfma_tflops\": %.4f, "
              "\"sms\": %d, \"clock_mhz\": %.1f}\n",
              tf[0], tf[1], tf[2], sms, clk_khz / 1000.0);
  return 0;
}
