// Throughput probes for the roofline denominators of ALU-bound kernels: FP64 and FP32 FMA chains
// and a read + write streaming copy.  Prints one JSON object.
//
// The FMA probe measures the SM clock it ran at: thread 0 of block 0 reads clock64() and the
// global nanosecond timer at its start and end, so the result is reported both as TFLOP/s and as
// FMA per clock per SM (independent of the clock the GPU chose under this load).  A kernel timed
// at another clock then has the peak  FMA/clock/SM x 2 FLOP x SMs x its own SM clock.
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
__global__ void fma_chains(T* out, unsigned long long* clk, T a, T b, int iters) {
  unsigned long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    t0 = global_ns();
    c0 = clock64();
  }
  T r[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) r[c] = threadIdx.x * T(1e-9) + T(c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < 16; ++c) r[c] = fma(r[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 16; ++c) s += r[c];
  if (s == T(12345.678)) out[threadIdx.x] = s;   // keeps the chains alive; never true
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long c1 = clock64(), t1 = global_ns();
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
}

__global__ void stream_copy(const float4* __restrict__ a, float4* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}

struct FmaResult {
  double tflops = 0.0;        // best of the repetitions
  double mhz = 0.0;           // SM clock of that repetition
  double fma_per_clk_sm = 0.0;
};

template <typename T>
static FmaResult fma_probe(int sms, int blocks_per_sm, int threads, int iters) {
  T* out;
  unsigned long long* clk;
  cudaMalloc(&out, threads * sizeof(T));
  cudaMalloc(&clk, 2 * sizeof(unsigned long long));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<sms * blocks_per_sm, threads>>>(out, clk, T(0.999999), T(1e-7), 8);
  FmaResult best;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0);
    fma_chains<T><<<sms * blocks_per_sm, threads>>>(out, clk, T(0.999999), T(1e-7), iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long h[2] = {0, 0};
    cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost);
    const double fmas = 128.0 * iters * (double)sms * blocks_per_sm * threads;
    const double tf = 2.0 * fmas / ms / 1e9;
    if (tf > best.tflops) {
      best.tflops = tf;
      best.mhz = h[1] ? 1e3 * (double)h[0] / (double)h[1] : 0.0;
      // cycles of the whole kernel at the measured clock
      best.fma_per_clk_sm = best.mhz > 0 ? fmas / (ms * 1e3 * best.mhz) / sms : 0.0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  cudaFree(clk);
  return best;
}

int main() {
  int sms = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  FmaResult f64, f32;
  for (int bps : {4, 8})
    for (int th : {256, 512}) {
      if (bps * th > 2048) continue;   // every CTA resident at once
      FmaResult v = fma_probe<double>(sms, bps, th, 200);
      if (v.tflops > f64.tflops) f64 = v;
      v = fma_probe<float>(sms, bps, th, 4000);
      if (v.tflops > f32.tflops) f32 = v;
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
  printf("{\"sms\": %d, \"clock_attr_khz\": %d, \"fp64_fma_tflops\": %.4f, \"fp64_sm_mhz\": %.0f, "
         "\"fp64_fma_per_clk_sm\": %.3f, \"fp32_fma_tflops\": %.3f, \"fp32_sm_mhz\": %.0f, "
         "\"fp32_fma_per_clk_sm\": %.2f, \"copy_gbs\": %.1f, \"error\": \"%s\"}\n",
         sms, clk, f64.tflops, f64.mhz, f64.fma_per_clk_sm, f32.tflops, f32.mhz, f32.fma_per_clk_sm, gbs,
         cudaGetErrorString(cudaGetLastError()));
  return 0;
}
