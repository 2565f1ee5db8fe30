// Test harness for the solver's hand-written numeric helpers (compiled by
// tests/test_gpu_helpers.py; not part of the library).  Each entry runs one
// helper over an array on the GPU and returns the results to the host.
#include <cuda_runtime.h>
#include <string.h>

#include "../paper_2304_05494_gb300/csrc/s2_internal.cuh"

using namespace s2;

namespace {

__global__ void k_helpers(int which, const double *in, double *out, int n, Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = in[i];
  switch (which) {
    case 0: out[i] = rcp_pos(x); break;                    // 1/x for x > 0
    case 1: out[i] = (double)d2f_int(x); break;             // double -> float on the integer pipe
    case 2: out[i] = (double)__double2float_rn(x); break;   // the hardware conversion
    case 3: out[i] = f2d_int(__double2float_rn(x)); break;  // float -> double on the integer pipe
    case 4: out[i] = viscosity(d, x); break;                // power law by the Halley step
    case 5: out[i] = pow(x * d.inv_t_ref, d.visc_exp) * d.inv_re; break;
  }
}

}  // namespace

// which: see k_helpers; omega = p/q the power-law exponent of cases 4, 5.
extern "C" int helpers_run(int which, const double *in, double *out, int n, int p, int q) {
  Dev d;
  memset(&d, 0, sizeof(d));
  d.inv_t_ref = 1.0;
  d.inv_re = 1.0;
  d.visc_exp = (double)p / q;
  d.visc_exp_f = (float)d.visc_exp;
  d.mu_p = p;
  d.mu_q = q;
  d.mu_qm1 = q - 1.0;
  d.mu_qp1 = q + 1.0;
  double *din = nullptr, *dout = nullptr;
  if (cudaMalloc(&din, n * sizeof(double)) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, n * sizeof(double)) != cudaSuccess) return 1;
  cudaMemcpy(din, in, n * sizeof(double), cudaMemcpyHostToDevice);
  k_helpers<<<(n + 255) / 256, 256>>>(which, din, dout, n, d);
  cudaError_t e = cudaMemcpy(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(din);
  cudaFree(dout);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : 2;
}
