// Arithmetic peak probe: s2_fma_rate (declared in s2.h).
//
// The double-precision path of this library is bound by the FP64 unit, so
// its roofline needs that unit's rate on the GPU at hand and at the clock
// it runs at.  This probe measures it with a loop of independent fused
// multiply-adds (8 chains per thread, enough to cover the FMA latency, no
// memory traffic), in double or single precision, on every SM.  The
// result is the issue-limited FMA rate, counted as 2 flops per FMA.
#include <cuda_runtime.h>

#include "../../include/s2.h"

namespace {

constexpr int NT = 256;
constexpr int CHAINS = 8;
constexpr int ITERS = 4096;

// Written only when a result takes an impossible value, which keeps the
// compiler from removing the loop without any memory traffic.
__device__ double g_sink;

template <typename T>
__global__ void __launch_bounds__(NT) k_fma(T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == (T)-12345.678) g_sink = (double)s;
}

}  // namespace

extern "C" int s2_fma_rate(int precision, int device, double *gflops) {
  if (!gflops || (precision != S2_FP64 && precision != S2_MIXED)) return S2_EINVAL;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return S2_ECUDA;
  if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return S2_ECUDA;
  int dev = 0, sms = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = S2_ECUDA;
  float ms = 0.0f;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) || cudaEventCreate(&e0) || cudaEventCreate(&e1))
    goto done;
  {
    // 8 CTAs per SM of 256 threads: 64 warps, full occupancy
    const unsigned grid = (unsigned)sms * 8u;
    // a = 1 - 2^-20, b = 2^-30: the chains stay finite and normal
    for (int rep = 0; rep < 3; ++rep) {  // warm-up: clocks ramp up
      if (precision == S2_FP64) k_fma<double><<<grid, NT, 0, st>>>(1.0 - 0x1p-20, 0x1p-30);
      else k_fma<float><<<grid, NT, 0, st>>>(1.0f - 0x1p-20f, 0x1p-30f);
    }
    const int reps = precision == S2_FP64 ? 10 : 100;
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < reps; ++rep) {
      if (precision == S2_FP64) k_fma<double><<<grid, NT, 0, st>>>(1.0 - 0x1p-20, 0x1p-30);
      else k_fma<float><<<grid, NT, 0, st>>>(1.0f - 0x1p-20f, 0x1p-30f);
    }
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f))
      goto done;
    const double flops = 2.0 * CHAINS * ITERS * (double)NT * grid * reps;
    *gflops = flops / (ms * 1e-3) / 1e9;
    rc = S2_OK;
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaGetLastError();
  cudaSetDevice(prev);
  return rc;
}
