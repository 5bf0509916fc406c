// pt_peaks.cu — the measured peaks the benchmark's rooflines divide by (thesis Art. 1, Eqs. 28-29:
// T_eff is compared with the memory copy throughput T_peak measured on the same device).
//
//   copy     y = x over a caller buffer with 16-byte vector loads and stores (two FP64 values
//            per access), grid-stride, read + write bytes counted, best of `reps` launches;
//   fp64     a mix of the three FP64 instructions a PT iteration issues (DFMA, DADD, DMUL, one of
//            each per chain and step, 8 independent chains per thread so the pipe, not the
//            dependency latency, is the limit): FP64 thread-instructions per second;
//   fp32     FP32 FMA chains the same way: FP32 thread-instructions (2 flops each) per second.
// Each launch is timed with CUDA events on the caller's stream; the best (shortest) of `reps`
// launches is returned, after one untimed warm-up launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/porowave_pt.h"

namespace {

__global__ void k_peak_copy(const double2* __restrict__ x, double2* __restrict__ y, long long n2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2; e += (long long)gridDim.x * blockDim.x)
    y[e] = x[e];
}

constexpr int kChains = 8;

__global__ void k_peak_fp64(double* __restrict__ sink, int steps, double s) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = s * (threadIdx.x + c + 1);
  const double m = 1.0 - 1e-9 * s, d = 1e-12 * s;
  for (int t = 0; t < steps; ++t) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      a[c] = fma(a[c], m, d);     // DFMA
      a[c] = a[c] + d;            // DADD
      a[c] = a[c] * m;            // DMUL
    }
  }
  double r = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r += a[c];
  if (r == 12345.678) sink[blockIdx.x] = r;   // keeps the loop; never true for these inputs
}

__global__ void k_peak_fp32(float* __restrict__ sink, int steps, float s) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = s * (threadIdx.x + c + 1);
  const float m = 1.0f - 1e-6f * s, d = 1e-7f * s;
  for (int t = 0; t < steps; ++t) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, d);
  }
  float r = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r += a[c];
  if (r == 12345.678f) sink[blockIdx.x] = r;
}

int sms_of_current_device() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

template <class Launch>
int best_of(cudaStream_t st, int reps, Launch launch, double* best_ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return PT_ECUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return PT_ECUDA;
  }
  launch();   // warm-up
  double best = 1e300;
  cudaError_t e = cudaGetLastError();
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) best = std::min(best, (double)ms);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return PT_ECUDA;
  *best_ms = best;
  return PT_OK;
}

}  // namespace

extern "C" {

int pt_peak_copy(const void* src, void* dst, size_t bytes, int32_t reps, void* stream, double* best_ms,
                 double* gbs) {
  if (!src || !dst || !best_ms || bytes < 32 || reps < 1 || ((uintptr_t)src & 15u) || ((uintptr_t)dst & 15u))
    return PT_EINVAL;
  const int sms = sms_of_current_device();
  if (sms <= 0) return PT_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n2 = (long long)(bytes / 16);
  const int rc = best_of(st, reps, [&] {
    k_peak_copy<<<sms * 8, 256, 0, st>>>((const double2*)src, (double2*)dst, n2);
  }, best_ms);
  if (rc == PT_OK && gbs) *gbs = 2.0 * 16.0 * (double)n2 / (*best_ms * 1e-3) / 1e9;
  return rc;
}

int pt_peak_arith(int32_t kind, void* sink, int32_t steps, int32_t reps, void* stream, double* best_ms,
                  double* ginst) {
  if ((kind != 0 && kind != 1) || !sink || steps < 1 || reps < 1 || !best_ms) return PT_EINVAL;
  const int sms = sms_of_current_device();
  if (sms <= 0) return PT_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = sms * 8, threads = 256;   // 2048 threads per SM
  int rc;
  double per_thread;
  if (kind == 0) {
    rc = best_of(st, reps, [&] { k_peak_fp64<<<blocks, threads, 0, st>>>((double*)sink, steps, 1.0); }, best_ms);
    per_thread = 3.0 * kChains * steps;
  } else {
    rc = best_of(st, reps, [&] { k_peak_fp32<<<blocks, threads, 0, st>>>((float*)sink, steps, 1.0f); }, best_ms);
    per_thread = 1.0 * kChains * steps;
  }
  if (rc == PT_OK && ginst) *ginst = per_thread * blocks * threads / (*best_ms * 1e-3) / 1e9;
  return rc;
}

}  // extern "C"
