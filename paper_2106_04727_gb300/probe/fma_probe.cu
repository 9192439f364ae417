// FP32 multiply-add throughput of this GPU, measured: the denominator of the
// roofline fraction the benchmark reports for its arithmetic-bound kernels.
//
// Every thread runs 8 independent chains of fused multiply-adds (scalar
// fmaf, or packed fma.rn.f32x2, two per instruction) for `iters` steps;
// enough warps per SM hide the pipeline latency, so the rate is the FMA
// pipe's issue rate at the clock the GPU holds under this load.  A flop is
// counted as in the benchmark: a multiply-add is 2.  Not part of the
// clustering library's interface; the benchmark loads it on its own.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int CHAINS = 8;
constexpr int TPB = 256;

__device__ __forceinline__ unsigned long long pk(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

__global__ void __launch_bounds__(TPB) k_fma(int iters, float m, float k, float *out) {
  float v[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) v[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) v[c] = fmaf(v[c], m, k);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += v[c];
  if (s == 1.2345f) out[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(TPB) k_fma2(int iters, float m, float k, float *out) {
  unsigned long long v[CHAINS];
  const unsigned long long mm = pk(m, m), kk = pk(k, k);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) v[c] = pk((float)threadIdx.x, (float)c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) v[c] = fma2(v[c], mm, kk);
  }
  unsigned long long s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s ^= v[c];
  if (s == 12345ull) out[blockIdx.x] = 1.f;
}

}  // namespace

// Runs the probe `reps` times on the current device and returns the best
// rate in TFLOP/s (multiply-add = 2 flops) and that run's milliseconds.
// packed = 1 uses fma.rn.f32x2.  Returns 0, or a CUDA error code.
extern "C" int hac_probe_fma(int packed, int reps, double *tflops, float *ms_out) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = sms * 8, iters = 1 << 16;
  float *out = nullptr;
  cudaEvent_t a, b;
  if ((e = cudaMalloc(&out, blocks * sizeof(float))) != cudaSuccess) return (int)e;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double best = 0.0;
  float best_ms = 0.f;
  for (int r = 0; r < reps + 1; ++r) {  // the first run warms up
    cudaEventRecord(a);
    if (packed)
      k_fma2<<<blocks, TPB>>>(iters, 0.999999f, 1e-7f, out);
    else
      k_fma<<<blocks, TPB>>>(iters, 0.999999f, 1e-7f, out);
    cudaEventRecord(b);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double fl = 2.0 * (packed ? 2.0 : 1.0) * CHAINS * (double)iters * blocks * TPB;
    const double t = fl / (ms * 1e-3) / 1e12;
    if (r > 0 && t > best) {
      best = t;
      best_ms = ms;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return (int)e;
  *tflops = best;
  *ms_out = best_ms;
  return 0;
}
