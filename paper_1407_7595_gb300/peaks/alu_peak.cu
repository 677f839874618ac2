// ALU throughput microbenchmarks: the denominators of the integrand kernels' roofline.
//
// Each kernel runs C independent dependent chains per thread of one operation
// (FP32 FFMA, FP64 DFMA, MUFU EX2, MUFU RSQ) over a full-occupancy grid, so
// the issue of that operation's pipe, not its latency, bounds the time. The
// host entry point times K launches with CUDA events on its own stream and
// returns the best rate. Nothing here changes a clock or power setting.
//
// Not part of the integrator: bench.py loads this library to state the FP32,
// FP64 and MUFU peaks of the GPU it runs on beside its roofline fractions.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;   // independent chains per thread
constexpr int kUnroll = 16;  // operations per chain per loop trip

__global__ void __launch_bounds__(256) k_ffma(float* sink, int iters, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3f * c + 1e-7f * threadIdx.x;
  const float m = 0.9999999f, k = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never taken
}

__global__ void __launch_bounds__(256) k_dfma(double* sink, int iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * c + 1e-9 * threadIdx.x;
  const double m = 0.99999999, k = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.2345) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never taken
}

// MUFU: a <- 2^(-a) (fixed point ~0.64) and a <- 1/sqrt(a) (fixed point 1), as
// PTX ex2.approx / rsqrt.approx; the negation is an operand modifier.
template <int OP>
__global__ void __launch_bounds__(256) k_mufu(float* sink, int iters, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3f * c + 1e-7f * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        float r;
        if (OP == 0)
          asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-a[c]));
        else
          asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c]));
        a[c] = r;
      }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never taken
}

}  // namespace

extern "C" {

// op: 0 FP32 FFMA, 1 FP64 DFMA, 2 MUFU EX2, 3 MUFU RSQ.
// Runs `reps` timed launches of `blocks_per_sm` x SMs blocks of 256 threads,
// each thread doing iters x 16 x 8 operations, after one untimed launch.
// Writes the best launch's operations per second (an FFMA or DFMA counts as one
// operation; the caller doubles it for flops) and its duration in ms.
// Returns 0, or the CUDA error code.
int alu_peak_run(int op, int blocks_per_sm, int iters, int reps, double* ops_per_s,
                 double* best_ms) {
  if (op < 0 || op > 3 || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || reps < 1 ||
      !ops_per_s || !best_ms)
    return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int threads = 256, blocks = sms * blocks_per_sm;
  void* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&sink, (size_t)blocks * threads * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 1e30f;
  for (int r = 0; e == cudaSuccess && r <= reps; ++r) {
    cudaEventRecord(t0, st);
    switch (op) {
      case 0: k_ffma<<<blocks, threads, 0, st>>>((float*)sink, iters, 1.0f); break;
      case 1: k_dfma<<<blocks, threads, 0, st>>>((double*)sink, iters, 1.0); break;
      case 2: k_mufu<0><<<blocks, threads, 0, st>>>((float*)sink, iters, 0.5f); break;
      default: k_mufu<1><<<blocks, threads, 0, st>>>((float*)sink, iters, 0.5f); break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && r > 0 && ms < best) best = ms;  // launch 0 is the warm-up
  }
  if (e == cudaSuccess) {
    const double ops = (double)blocks * threads * iters * kUnroll * kChains;
    *ops_per_s = ops / (best * 1e-3);
    *best_ms = best;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  return (int)e;
}

}  // extern "C"
