// Allocation-free CFL time step: s2_cfl_dt_noalloc (declared in s2.h).
//
// Some callers cannot allocate device memory at the moment they need a
// time step: a serving loop that has handed all of the GPU's memory to a
// pooling allocator it does not control, code that runs while another
// framework holds the device's memory pool, or a real-time loop whose
// latency budget rules out cudaMalloc's implicit synchronisation.  This
// entry point computes the same quantity as the dt recomputation inside
// s2_step, but keeps its only scratch (one partial maximum per CTA) in a
// fixed array compiled into the library, so a call allocates nothing.
//
// The array lives in every GPU that loads the library, until the process
// exits.  Host code only sees a stand-in for it, so its device address is
// looked up (cudaGetSymbolAddress) once per device and context, on the
// first call with that device current, and cached with the identifier of
// the context it belongs to; a call that finds another context current
// (the device was reset since) looks it up again.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "s2_internal.cuh"

using namespace s2;

namespace {

constexpr int NT = 256;
constexpr int PTS_PER_THREAD = 16;
// Scratch: one partial maximum per CTA, 64 Ki doubles = 512 KiB per GPU.
constexpr int MAX_PARTS = 65536;
static __device__ __align__(256) double g_dt_parts[MAX_PARTS];

// Largest grid: one partial per CTA of NT * PTS_PER_THREAD points.
constexpr long long MAX_POINTS = (long long)MAX_PARTS * NT * PTS_PER_THREAD;

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
struct ScratchAddr {
  unsigned long long ctx_id;  // process-unique context identifier (cuCtxGetId)
  double *ptr;
};
ScratchAddr g_parts_addr[MAX_DEVICES] = {};

__device__ __forceinline__ double wmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ double block_max(double v) {
  __shared__ double red[NT / 32];
  v = wmax(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) r = wmax(r);
  return r;  // valid in thread 0
}

// Each CTA covers NT * PTS_PER_THREAD consecutive points and writes its
// maximum spectral radius (same per-point arithmetic as the solver's
// primitive kernel) to parts[blockIdx.x].
__global__ void __launch_bounds__(NT) k_cfl_parts(Dev d, const double *__restrict__ w, const double *__restrict__ eta_y,
                                                  double ey_uniform, double *parts) {
  double m = 0.0;
  long long base = (long long)blockIdx.x * NT * PTS_PER_THREAD;
  for (int t = 0; t < PTS_PER_THREAD; ++t) {
    long long q = base + (long long)t * NT + threadIdx.x;
    if (q >= d.n) break;
    int j = row_of(d, q);
    double rho = w[q];
    double ri = 1.0 / rho;
    double u = w[d.n + q] * ri, v = w[2 * d.n + q] * ri, ww = w[3 * d.n + q] * ri;
    double q2 = u * u + v * v + ww * ww;
    const double e = w[4 * d.n + q] * ri - 0.5 * q2;
    double T = e * d.icv;
    bool ok = true;
    if (d.kd.tp && positive_finite(rho) && finite_bits(e)) T = tp_temperature(d.kd, e, tp_guess(d.kd, e), 0.0, ok);
    // the solver's validity test (rho and T positive and finite, |u|^2
    // finite): an invalid point has no spectral radius, and dt = 0
    // reports it
    if (!ok || !positive_finite(rho) || !positive_finite(T) || !finite_bits(q2)) {
      m = INFINITY;
      continue;
    }
    double mu = d.viscous ? viscosity(d, T) : 0.0;
    double ey = eta_y ? eta_y[j] : ey_uniform;
    m = fmax(m, spectral_radius(d, rho, u, v, ww, T, mu, ey));
  }
  m = block_max(m);
  if (threadIdx.x == 0) parts[blockIdx.x] = m;
}

__global__ void __launch_bounds__(NT) k_cfl_final(const double *parts, int nparts, double cfl, double *dt) {
  double m = 0.0;
  for (int b = threadIdx.x; b < nparts; b += NT) m = fmax(m, parts[b]);
  m = block_max(m);
  if (threadIdx.x == 0) dt[0] = cfl / m;
}

// The driver's cuCtxGetCurrent and cuCtxGetId, reached through the
// runtime (no link against the driver library).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
void *driver_fn(const char *name) {
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return p;
}

// Identifier of the calling thread's current context; 0 if none is
// current yet (the runtime creates it at its first device call).
cudaError_t current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get = (CtxGetCurrentFn)driver_fn("cuCtxGetCurrent");
  static CtxGetIdFn get_id = (CtxGetIdFn)driver_fn("cuCtxGetId");
  *id = 0;
  if (!get || !get_id) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Device address of the scratch array on the current device, looked up
// once per device and context.
cudaError_t scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  unsigned long long id = 0;
  if ((e = current_context_id(&id)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!id || !g_parts_addr[dev].ptr || g_parts_addr[dev].ctx_id != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dt_parts);  // creates the context if none was current
    if (e != cudaSuccess) return e;
    if (!id && ((e = current_context_id(&id)) != cudaSuccess || !id)) return cudaErrorDeviceUninitialized;
    g_parts_addr[dev].ctx_id = id;
    g_parts_addr[dev].ptr = (double *)p;
  }
  *out = g_parts_addr[dev].ptr;
  return cudaSuccess;
}

}  // namespace

extern "C" int s2_cfl_dt_noalloc(const s2_grid *grid, const s2_gas *gas, const double *w, const double *eta_y,
                                 double cfl, double *dt, void *stream) {
  if (!grid || !gas || !w || !dt || !(cfl > 0)) return S2_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->lx > 0) || !(grid->ly > 0) || !(grid->lz > 0))
    return S2_EINVAL;
  if (check_gas(gas, 0.0) != S2_OK) return S2_EINVAL;
  // size checked factor by factor: every partial product stays below
  // MAX_POINTS before the next multiplication, so nothing overflows
  long long n = grid->nx;
  if (n > MAX_POINTS) return S2_ETOOBIG;
  n *= grid->ny;
  if (n > MAX_POINTS) return S2_ETOOBIG;
  n *= grid->nz;
  if (n > MAX_POINTS) return S2_ETOOBIG;
  const long long per_cta = (long long)NT * PTS_PER_THREAD;
  const long long nparts = (n + per_cta - 1) / per_cta;
  Dev d;
  memset(&d, 0, sizeof(d));
  d.nx = grid->nx;
  d.ny = grid->ny;
  d.nz = grid->nz;
  d.n = n;
  d.fnx.init((unsigned)grid->nx);
  d.fny.init((unsigned)grid->ny);
  d.dx = grid->lx / grid->nx;
  d.dz = grid->lz / grid->nz;
  set_gas(d, gas);
  double *parts = nullptr;
  if (scratch_address(&parts) != cudaSuccess) {
    cudaGetLastError();
    return S2_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double ey_uniform = grid->ny / grid->ly;
  k_cfl_parts<<<(unsigned)nparts, NT, 0, st>>>(d, w, eta_y, ey_uniform, parts);
  if (cudaGetLastError() != cudaSuccess) return S2_ECUDA;
  k_cfl_final<<<1, NT, 0, st>>>(parts, (int)nparts, cfl, dt);
  if (cudaGetLastError() != cudaSuccess) return S2_ECUDA;
  return S2_OK;
}
