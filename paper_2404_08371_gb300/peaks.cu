// Throughput probes for the roofline denominators of ALU-bound kernels: FP64 and FP32 FMA chains
// (16 independent chains per thread, enough warps to hide the pipeline latency) and a
// read + write streaming copy.  Prints one JSON object.
#include <cstdio>
#include <cuda_runtime.h>

template <typename T>
__global__ void fma_chains(T* out, T a, T b, int iters) {
  T r[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) r[c] = threadIdx.x * T(1e-9) + T(c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < 16; ++c) r[c] = r[c] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 16; ++c) s += r[c];
  if (s == T(12345.678)) out[threadIdx.x] = s;   // keeps the chains alive; never true
}

__global__ void stream_copy(const float4* __restrict__ a, float4* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}

template <typename T>
static double fma_tflops(int sms, int blocks_per_sm, int threads, int iters) {
  T* out;
  cudaMalloc(&out, threads * sizeof(T));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<sms * blocks_per_sm, threads>>>(out, T(0.999999), T(1e-7), 8);
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    fma_chains<T><<<sms * blocks_per_sm, threads>>>(out, T(0.999999), T(1e-7), iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 64.0 * iters * (double)sms * blocks_per_sm * threads;
    if (flops / ms / 1e9 > best) best = flops / ms / 1e9;
  }
  cudaFree(out);
  return best;
}

int main() {
  int sms = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  double f64 = 0, f32 = 0;
  for (int bps : {4, 8})
    for (int th : {256, 512}) {
      double v = fma_tflops<double>(sms, bps, th, 400);
      if (v > f64) f64 = v;
      v = fma_tflops<float>(sms, bps, th, 8000);
      if (v > f32) f32 = v;
    }
  const size_t n = (size_t)1 << 28;   // 4 GiB per buffer of float4
  float4 *a, *b;
  double gbs = 0.0;
  if (cudaMalloc(&a, n * sizeof(float4)) == cudaSuccess && cudaMalloc(&b, n * sizeof(float4)) == cudaSuccess) {
    cudaMemset(a, 0, n * sizeof(float4));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    stream_copy<<<sms * 8, 512>>>(a, b, n);
    for (int rep = 0; rep < 5; ++rep) {
      cudaEventRecord(e0);
      stream_copy<<<sms * 8, 512>>>(a, b, n);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double v = 2.0 * n * sizeof(float4) / ms / 1e6;
      if (v > gbs) gbs = v;
    }
    cudaFree(a);
    cudaFree(b);
  }
  printf("{\"sms\": %d, \"clock_khz\": %d, \"fp64_fma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, "
         "\"copy_gbs\": %.1f, \"error\": \"%s\"}\n",
         sms, clk, f64, f32, gbs, cudaGetErrorString(cudaGetLastError()));
  return 0;
}
