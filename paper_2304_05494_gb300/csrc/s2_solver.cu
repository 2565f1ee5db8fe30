// libs2.so host runtime and the point-wise kernels of one RK3 stage.
//
// Stage sequence (paper Sec. 2 method; kernels of Table 2):
//   k_prims      w -> rho, u, v, w, T, p, H, c, mu   (+ CFL partials, compute_dt)
//   k_ghost_prim ghost faces: periodic copy / isothermal no-slip mirror
//   k_grad       velocity gradients, div u, shock sensor          (s2_visc.cu)
//   k_ghost_aux  ghost faces of div u and the sensor
//   k_flux x,y,z hybrid central/WENO convective fluxes (euler_*) (s2_flux.cu)
//   k_visc       viscous and heat-flux terms (visflx)            (s2_visc.cu)
//   k_force_*    bulk forcing reduction (force_rhs_1)
//   k_update     low-storage RK3 update w += dt gamma_k R + fln,
//                fln = dt rho_{k+1} R (update_flux, Sec. 3.2 Listing 4)
// One step (3 stages) is captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/s2.h"
#include "s2_internal.cuh"

using namespace s2;

namespace {

constexpr int NT = 256;
constexpr int NRED = 1024;  // blocks of the grid-stride reductions

// 6th-order central coefficients (first derivative a_l, second b_l).
const double A1[4] = {0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0};
const double B2[4] = {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};
// Wray's low-storage RK3 coefficients.
const double RK_G[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
const double RK_R[4] = {0.0, -17.0 / 60.0, -5.0 / 12.0, 0.0};

__device__ __forceinline__ void point_of(const Dev &d, long long q, int &i, int &j, int &k) {
  long long t = q / d.nx;
  i = (int)(q - t * d.nx);
  k = (int)(t / d.ny);
  j = (int)(t - (long long)k * d.ny);
}

__device__ __forceinline__ int imod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of NV values (deterministic order); result valid in thread 0.
template <int NVAL>
__device__ void block_sum(double *v) {
  __shared__ double red[NVAL][NT / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NVAL; ++m) {
    double s = warp_sum(v[m]);
    if (lane == 0) red[m][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int m = 0; m < NVAL; ++m) {
      double s = lane < NT / 32 ? red[m][lane] : 0.0;
      v[m] = warp_sum(s);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- metrics
// y metric from the node ordinates extended into the ghosts (periodic
// shift or mirror about the walls at -ly/2, ly/2): y_eta by the 6th-order
// stencil, eta_y = 1/y_eta, eta_yy = -y_etaeta/y_eta^3.  Also the
// pre-scaled coefficient tables used by the stencil kernels.
__global__ void k_metric(const double *yn, int ny, double ly, int wall, double *eta_y, double *ay,
                         double *by, double *ry, double *dvy) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ny) return;
  const double a[4] = {0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0};
  const double b[4] = {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};
  auto ext = [&](int jj) -> double {
    if (jj >= 0 && jj < ny) return yn[jj];
    if (!wall) {
      int m = ((jj % ny) + ny) % ny;
      int shift = (jj - m) / ny;
      return yn[m] + shift * ly;
    }
    if (jj < 0) return -ly - yn[-1 - jj];
    return ly - yn[2 * ny - 1 - jj];
  };
  double d1 = 0.0, d2 = b[0] * ext(j);
  for (int l = 1; l <= 3; ++l) {
    d1 += a[l] * (ext(j + l) - ext(j - l));
    d2 += b[l] * (ext(j + l) + ext(j - l));
  }
  double ey = 1.0 / d1;
  double eyy = -d2 / (d1 * d1 * d1);
  eta_y[j] = ey;
  for (int l = 1; l <= 3; ++l) ay[3 * j + l - 1] = a[l] * ey;
  for (int l = 0; l <= 3; ++l) by[4 * j + l] = b[l] * ey * ey;
  ry[j] = eyy / ey;
  dvy[j] = d1;
}

// ------------------------------------------------------------- primitives
// rho, u = (rho u)/rho, ..., T = (E - |u|^2/2)/c_v, p = rho R T,
// H = c_p T + |u|^2/2, mu = (T/T_ref)^omega/Re.  With want_dt, also the
// CFL spectral radius max into part[block] (c = sqrt(gamma R T)).
__global__ void __launch_bounds__(NT) k_prims(Dev d, int want_dt) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  double sr = 0.0;
  if (q < d.n) {
    int i, j, k;
    point_of(d, q, i, j, k);
    long long p = pidx(d, i, j, k);
    const double *w = d.w;
    double rho = w[q];
    double ri = 1.0 / rho;
    double u = w[d.n + q] * ri, v = w[2 * d.n + q] * ri, ww = w[3 * d.n + q] * ri;
    double q2 = u * u + v * v + ww * ww;
    double T = (w[4 * d.n + q] * ri - 0.5 * q2) * d.icv;
    double pr = rho * d.R * T;
    d.rho[p] = rho;
    d.u[p] = u;
    d.v[p] = v;
    d.ww[p] = ww;
    d.T[p] = T;
    d.p[p] = pr;
    d.H[p] = d.cp * T + 0.5 * q2;
    double mu = 0.0;
    if (d.viscous) {
      mu = viscosity(d, T);
      d.mu[q] = mu;
    }
    if (!(rho > 0.0) || !(T > 0.0) || !isfinite(rho) || !isfinite(T) || !isfinite(q2))
      atomicOr(&d.scal->status, ERR_NONFINITE);
    if (want_dt) sr = spectral_radius(d, rho, u, v, ww, T, mu, d.eta_y[j]);
  }
  if (want_dt) {
    __shared__ double red[NT / 32];
    double m = warp_max(sr);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
      s = warp_max(s);
      if (threadIdx.x == 0) d.part[blockIdx.x] = s;
    }
  }
}

// dt = cfl / max(spectral radius) over the partials of k_prims.
__global__ void k_dt_final(Dev d, int nparts) {
  double m = 0.0;
  for (int b = threadIdx.x; b < nparts; b += NT) m = fmax(m, d.part[b]);
  __shared__ double red[NT / 32];
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    s = warp_max(s);
    if (threadIdx.x == 0) {
      d.scal->dt_max_rate = s;
      d.scal->dt = d.cfl / s;
    }
  }
}

// ----------------------------------------------------------------- ghosts
// Face ghosts (GH deep) of the primitive fields.  x and z periodic; y
// periodic or isothermal no-slip wall mirrored about the face between the
// outermost node and its ghost: u -> -u, T -> 2 T_w - T, p -> p,
// rho = p/(R T), H from T and |u|.
__global__ void __launch_bounds__(NT) k_ghost_prim(Dev d) {
  long long nxf = 2LL * GH * d.ny * d.nz, nyf = 2LL * GH * d.nx * d.nz, nzf = 2LL * GH * d.nx * d.ny;
  long long t = (long long)blockIdx.x * NT + threadIdx.x;
  if (t >= nxf + nyf + nzf) return;
  int di, dj, dk, si, sj, sk;
  bool wall = false;
  if (t < nxf) {
    int g = (int)(t % (2 * GH));
    long long r = t / (2 * GH);
    dj = (int)(r % d.ny);
    dk = (int)(r / d.ny);
    di = g < GH ? -1 - g : d.nx + (g - GH);
    si = imod(di, d.nx); sj = dj; sk = dk;
  } else if (t < nxf + nyf) {
    t -= nxf;
    di = (int)(t % d.nx);
    long long r = t / d.nx;
    int g = (int)(r % (2 * GH));
    dk = (int)(r / (2 * GH));
    dj = g < GH ? -1 - g : d.ny + (g - GH);
    si = di; sk = dk;
    if (d.wall_y) {
      wall = true;
      sj = dj < 0 ? -1 - dj : 2 * d.ny - 1 - dj;
    } else {
      sj = imod(dj, d.ny);
    }
  } else {
    t -= nxf + nyf;
    di = (int)(t % d.nx);
    long long r = t / d.nx;
    int g = (int)(r % (2 * GH));
    dj = (int)(r / (2 * GH));
    dk = g < GH ? -1 - g : d.nz + (g - GH);
    si = di; sj = dj;
    sk = imod(dk, d.nz);
  }
  long long dp = pidx(d, di, dj, dk), sp = pidx(d, si, sj, sk);
  if (!wall) {
    d.rho[dp] = d.rho[sp];
    d.u[dp] = d.u[sp];
    d.v[dp] = d.v[sp];
    d.ww[dp] = d.ww[sp];
    d.T[dp] = d.T[sp];
    d.p[dp] = d.p[sp];
    d.H[dp] = d.H[sp];
  } else {
    double u = -d.u[sp], v = -d.v[sp], ww = -d.ww[sp];
    double T = 2.0 * d.t_wall - d.T[sp];
    double pr = d.p[sp];
    d.u[dp] = u;
    d.v[dp] = v;
    d.ww[dp] = ww;
    d.T[dp] = T;
    d.p[dp] = pr;
    d.rho[dp] = pr / (d.R * T);
    d.H[dp] = d.cp * T + 0.5 * (u * u + v * v + ww * ww);
    if (!(T > 0.0)) atomicOr(&d.scal->status, ERR_NONFINITE);
  }
}

// Face ghosts of div u and of the sensor.  At a wall the sensor is
// mirrored and the divergence of the mirrored velocity field is
// -u_x + v_y - w_z at the mirror node.
__global__ void __launch_bounds__(NT) k_ghost_aux(Dev d) {
  long long nxf = 2LL * GH * d.ny * d.nz, nyf = 2LL * GH * d.nx * d.nz, nzf = 2LL * GH * d.nx * d.ny;
  long long t = (long long)blockIdx.x * NT + threadIdx.x;
  if (t >= nxf + nyf + nzf) return;
  int di, dj, dk, si, sj, sk;
  bool wall = false;
  if (t < nxf) {
    int g = (int)(t % (2 * GH));
    long long r = t / (2 * GH);
    dj = (int)(r % d.ny);
    dk = (int)(r / d.ny);
    di = g < GH ? -1 - g : d.nx + (g - GH);
    si = imod(di, d.nx); sj = dj; sk = dk;
  } else if (t < nxf + nyf) {
    t -= nxf;
    di = (int)(t % d.nx);
    long long r = t / d.nx;
    int g = (int)(r % (2 * GH));
    dk = (int)(r / (2 * GH));
    dj = g < GH ? -1 - g : d.ny + (g - GH);
    si = di; sk = dk;
    if (d.wall_y) {
      wall = true;
      sj = dj < 0 ? -1 - dj : 2 * d.ny - 1 - dj;
    } else {
      sj = imod(dj, d.ny);
    }
  } else {
    t -= nxf + nyf;
    di = (int)(t % d.nx);
    long long r = t / d.nx;
    int g = (int)(r % (2 * GH));
    dj = (int)(r / (2 * GH));
    dk = g < GH ? -1 - g : d.nz + (g - GH);
    si = di; sj = dj;
    sk = imod(dk, d.nz);
  }
  long long dp = pidx(d, di, dj, dk), sp = pidx(d, si, sj, sk);
  d.sens[dp] = d.sens[sp];
  if (!wall) {
    d.div[dp] = d.div[sp];
  } else {
    long long q = ((long long)sk * d.ny + sj) * d.nx + si;
    double ux = d.g[0 * d.n + q], vy = d.g[4 * d.n + q], wz = d.g[8 * d.n + q];
    d.div[dp] = -ux + vy - wz;
  }
}

// ---------------------------------------------------------------- forcing
// force_rhs_1: partial sums of R_rhou dV (dV ~ 1/eta_y), deterministic.
__global__ void __launch_bounds__(NT) k_force_partial(Dev d) {
  double s = 0.0;
  for (long long q = (long long)blockIdx.x * NT + threadIdx.x; q < d.n; q += (long long)gridDim.x * NT) {
    int j = (int)((q / d.nx) % d.ny);
    s += d.fl[d.n + q] * d.dvy[j];
  }
  double v[1] = {s};
  block_sum<1>(v);
  if (threadIdx.x == 0) d.part[blockIdx.x] = v[0];
}

__global__ void k_force_final(Dev d, int nparts) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += NT) s += d.part[b];
  double v[1] = {s};
  block_sum<1>(v);
  if (threadIdx.x == 0) d.scal->force = -v[0] * d.vol_inv;
}

// ----------------------------------------------------------------- update
// w <- w + dt gamma_k R + fln ; fln <- dt rho_{k+1} R, with R = fl + the
// forcing (f on rho u, f u on rho E).  Stage 0 reads no fln; the last
// stage writes none and advances the clock.
__global__ void __launch_bounds__(NT) k_update(Dev d, double gk, double rk1, int stage) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  const double dt = d.scal->dt;
  if (q < d.n) {
    double f = d.force ? d.scal->force : 0.0;
    double fu = 0.0;
    if (d.force) {
      int i, j, k;
      point_of(d, q, i, j, k);
      fu = f * d.u[pidx(d, i, j, k)];
    }
    const double a = dt * gk, b = dt * rk1;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      long long o = v * d.n + q;
      double R = d.fl[o];
      if (v == 1) R += f;
      if (v == 4) R += fu;
      double wn = fma(a, R, d.w[o]);
      if (stage > 0) wn += d.fln[o];
      d.w[o] = wn;
      if (stage < 2) d.fln[o] = b * R;
    }
  }
  if (stage == 2 && q == 0) d.scal->t += dt;
}

// R = fl + forcing into out (diagnostics).
__global__ void __launch_bounds__(NT) k_rhs_out(Dev d, double *out) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  double f = d.force ? d.scal->force : 0.0;
  double fu = 0.0;
  if (d.force) {
    int i, j, k;
    point_of(d, q, i, j, k);
    fu = f * d.u[pidx(d, i, j, k)];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double R = d.fl[v * d.n + q];
    if (v == 1) R += f;
    if (v == 4) R += fu;
    out[v * d.n + q] = R;
  }
}

// ------------------------------------------------------------------ stats
// Integrals of rho, rho u_a, rho E, rho|u|^2/2 (dV = dx dz / eta_y) and
// the sum of (R_rhou)^2 of the last RHS evaluation.
constexpr int NSTAT = 7;
__global__ void __launch_bounds__(NT) k_stats_partial(Dev d) {
  double v[NSTAT] = {0, 0, 0, 0, 0, 0, 0};
  double f = d.force ? d.scal->force : 0.0;
  for (long long q = (long long)blockIdx.x * NT + threadIdx.x; q < d.n; q += (long long)gridDim.x * NT) {
    int j = (int)((q / d.nx) % d.ny);
    double dv = d.dvy[j] * d.dx * d.dz;
    double rho = d.w[q], mx = d.w[d.n + q], my = d.w[2 * d.n + q], mz = d.w[3 * d.n + q];
    v[0] += rho * dv;
    v[1] += mx * dv;
    v[2] += my * dv;
    v[3] += mz * dv;
    v[4] += d.w[4 * d.n + q] * dv;
    v[5] += 0.5 * (mx * mx + my * my + mz * mz) / rho * dv;
    double r = d.fl[d.n + q] + f;
    v[6] += r * r;
  }
  block_sum<NSTAT>(v);
  if (threadIdx.x == 0)
    for (int m = 0; m < NSTAT; ++m) d.part[m * NRED + blockIdx.x] = v[m];
}

__global__ void k_stats_final(Dev d, int nparts) {
  double v[NSTAT];
  for (int m = 0; m < NSTAT; ++m) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += NT) s += d.part[m * NRED + b];
    v[m] = s;
  }
  block_sum<NSTAT>(v);
  if (threadIdx.x == 0)
    for (int m = 0; m < NSTAT; ++m) d.scal->red[m] = v[m];
}

}  // namespace

// ======================================================================
// Host runtime
// ======================================================================
struct s2_solver {
  Dev d;
  s2_grid grid;
  s2_gas gas;
  s2_bcs bcs;
  s2_scheme sch;
  s2_device dev;
  int device;
  cudaStream_t stream;
  bool own_stream;
  std::vector<void *> blocks;
  long long step;
  int nparts_prims;
  cudaGraphExec_t graph[2];
  bool graph_ready[2];
  bool graph_disabled;
  int last_status;
  size_t flag_bytes[3];
  long long launches_per_step[2];
  long long launches;
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? S2_OK : S2_ECUDA; }

void *dalloc(s2_solver *s, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (s->dev.alloc) {
    p = s->dev.alloc(bytes, s->dev.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) s->blocks.push_back(p);
  return p;
}

void release(s2_solver *s) {
  for (int g = 0; g < 2; ++g)
    if (s->graph_ready[g]) cudaGraphExecDestroy(s->graph[g]);
  for (void *p : s->blocks) {
    if (s->dev.free) s->dev.free(p, s->dev.ctx);
    else cudaFree(p);
  }
  s->blocks.clear();
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

// Launch bookkeeping: per-class kernel counts and, when profiling, CUDA
// events around every class on the solver's stream.
struct Trace {
  long long count[S2_PROF_KINDS] = {0};
  bool timed = false;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
};

template <class F>
cudaError_t run(Trace *tr, cudaStream_t st, int kind, int nkernels, F f) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (tr && tr->timed) {
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return cudaErrorMemoryAllocation;
    cudaEventRecord(a, st);
  }
  cudaError_t e = f();
  if (tr) {
    tr->count[kind] += nkernels;
    if (tr->timed) {
      cudaEventRecord(b, st);
      tr->recs.push_back({kind, a, b});
    }
  }
  return e;
}

// One RHS evaluation (all terms up to the forcing reduction).
cudaError_t enqueue_rhs(s2_solver *s, int want_dt, Trace *tr) {
  const Dev &d = s->d;
  cudaStream_t st = s->stream;
  cudaError_t e;
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  long long nghost = 2LL * GH * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
  unsigned ngb = (unsigned)((nghost + NT - 1) / NT);
  e = run(tr, st, S2_PROF_PRIMS, 1, [&] {
    k_prims<<<nb, NT, 0, st>>>(d, want_dt);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  if (want_dt) {
    e = run(tr, st, S2_PROF_DT, 1, [&] {
      k_dt_final<<<1, NT, 0, st>>>(d, (int)nb);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  e = run(tr, st, S2_PROF_GHOST, 1, [&] {
    k_ghost_prim<<<ngb, NT, 0, st>>>(d);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  if (d.viscous || d.weno) {
    e = run(tr, st, S2_PROF_GRAD, 1, [&] { return launch_grad(d, st); });
    if (e != cudaSuccess) return e;
    e = run(tr, st, S2_PROF_GHOST_AUX, 1, [&] {
      k_ghost_aux<<<ngb, NT, 0, st>>>(d);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  if (d.weno) {
    // wcount and the three list lengths are adjacent
    if ((e = cudaMemsetAsync(&d.scal->wcount, 0, sizeof(unsigned long long) + 4 * sizeof(unsigned), st)) !=
        cudaSuccess)
      return e;
  }
  for (int dir = 0; dir < 3; ++dir) {
    e = run(tr, st, S2_PROF_FLUX_X + dir, 1, [&] { return launch_flux(d, dir, dir > 0, st); });
    if (e != cudaSuccess) return e;
  }
  if (d.weno) {
    e = run(tr, st, S2_PROF_WENO, 3, [&] {
      cudaError_t r = cudaSuccess;
      for (int dir = 0; dir < 3 && r == cudaSuccess; ++dir) r = launch_weno(d, dir, st);
      return r;
    });
    if (e != cudaSuccess) return e;
  }
  if (d.viscous) {
    e = run(tr, st, S2_PROF_VISC, 1, [&] { return launch_visc(d, st); });
    if (e != cudaSuccess) return e;
  } else if (d.weno) {
    e = run(tr, st, S2_PROF_APPLY, 1, [&] { return launch_apply(d, st); });
    if (e != cudaSuccess) return e;
  }
  if (d.force) {
    e = run(tr, st, S2_PROF_FORCE, 2, [&] {
      k_force_partial<<<NRED, NT, 0, st>>>(d);
      k_force_final<<<1, NT, 0, st>>>(d, NRED);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t enqueue_step(s2_solver *s, int want_dt, Trace *tr) {
  const Dev &d = s->d;
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  cudaError_t e;
  for (int st = 0; st < 3; ++st) {
    if ((e = enqueue_rhs(s, st == 0 ? want_dt : 0, tr)) != cudaSuccess) return e;
    e = run(tr, s->stream, S2_PROF_UPDATE, 1, [&] {
      k_update<<<nb, NT, 0, s->stream>>>(d, RK_G[st], RK_R[st + 1], st);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

long long total(const Trace &t) {
  long long c = 0;
  for (int k = 0; k < S2_PROF_KINDS; ++k) c += t.count[k];
  return c;
}

int build_graph(s2_solver *s, int variant) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  Trace tr;
  cudaError_t e = enqueue_step(s, variant, &tr);
  cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return -1;
  }
  cudaGraphExec_t ex;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return -1;
  }
  cudaGraphDestroy(g);
  s->graph[variant] = ex;
  s->graph_ready[variant] = true;
  s->launches_per_step[variant] = total(tr);
  return 0;
}

int read_status(s2_solver *s) {
  int st = 0;
  if (cudaMemcpyAsync(&st, &s->d.scal->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return S2_ECUDA;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return S2_ECUDA;
  if (st & ERR_NONFINITE) return S2_ENONFINITE;
  return S2_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

// Gas constants of a Dev from the public description (reference units).
void s2::set_gas(Dev &d, const s2_gas *gas) {
  d.gamma = gas->gamma;
  d.R = 1.0 / (gas->gamma * gas->mach_ref * gas->mach_ref);
  d.gR = gas->gamma * d.R;
  // viscosity exponent as a ratio of small integers when it is one
  d.mu_p = 0;
  d.mu_q = 0;
  for (int q = 1; q <= 64 && gas->visc_exp >= 0.0; ++q) {
    double pq = gas->visc_exp * q;
    double r = floor(pq + 0.5);
    if (fabs(pq - r) <= 1e-12 * q && r <= 64.0) {
      d.mu_p = (int)r;
      d.mu_q = q;
      break;
    }
  }
  d.cv = d.R / (gas->gamma - 1.0);
  d.icv = 1.0 / d.cv;
  d.cp = gas->gamma * d.cv;
  d.prandtl = gas->prandtl;
  d.re = gas->re_ref;
  d.visc_exp = gas->visc_exp;
  d.inv_t_ref = 1.0 / gas->t_ref;
  d.cp_over_pr = d.cp / gas->prandtl;
  d.viscous = gas->re_ref > 0.0;
}

extern "C" {

const char *s2_strerror(int code) {
  switch (code) {
    case S2_OK: return "ok";
    case S2_EINVAL: return "invalid argument or unsupported configuration";
    case S2_ENOMEM: return "out of memory";
    case S2_ECUDA: return "CUDA runtime error";
    case S2_ENONFINITE: return "non-positive density/temperature or non-finite value";
    case S2_ETIMEOUT: return "device wait timed out";
    case S2_EBUSY: return "solver busy";
    case S2_ETOOBIG: return "grid larger than the fixed scratch of the allocation-free entry point";
  }
  return "unknown error";
}

int s2_create(const s2_grid *grid, const s2_metrics *metrics, const s2_gas *gas, const s2_bcs *bcs,
              const s2_scheme *scheme, const s2_device *dev, s2_solver **out) {
  if (!out || !grid || !gas || !bcs || !scheme) return S2_EINVAL;
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return S2_EINVAL;
  if (!(grid->lx > 0) || !(grid->ly > 0) || !(grid->lz > 0)) return S2_EINVAL;
  if (bcs->x != S2_BC_PERIODIC || bcs->z != S2_BC_PERIODIC) return S2_EINVAL;
  if (bcs->y != S2_BC_PERIODIC && bcs->y != S2_BC_ISOTHERMAL_WALL) return S2_EINVAL;
  if (bcs->y == S2_BC_ISOTHERMAL_WALL && (grid->ny < GH || !(bcs->t_wall > 0))) return S2_EINVAL;
  if (scheme->central_order != 6 || scheme->visc_order != 6) return S2_EINVAL;
  if (scheme->weno_order != 0 && scheme->weno_order != 5 && scheme->weno_order != 7) return S2_EINVAL;
  if (scheme->precision != S2_FP64) return S2_EINVAL;
  if (!(scheme->cfl > 0) && !(scheme->dt_fixed > 0)) return S2_EINVAL;
  if (!(gas->gamma > 1.0) || !(gas->mach_ref > 0) || !(gas->prandtl > 0) || !(gas->t_ref > 0)) return S2_EINVAL;
  long long n = (long long)grid->nx * grid->ny * grid->nz;
  if (n > (1LL << 40)) return S2_EINVAL;
  // interface slots of a direction are listed as 32-bit indices
  if (scheme->weno_order && (long long)(grid->nx + 1) * (grid->ny + 1) * (long long)(grid->nz + 1) > 0xffffffffLL)
    return S2_EINVAL;
  if (metrics && metrics->y) {
    for (int j = 1; j < grid->ny; ++j)
      if (!(metrics->y[j] > metrics->y[j - 1])) return S2_EINVAL;
    if (bcs->y == S2_BC_ISOTHERMAL_WALL &&
        !(metrics->y[0] > -0.5 * grid->ly && metrics->y[grid->ny - 1] < 0.5 * grid->ly))
      return S2_EINVAL;
  }

  s2_solver *s = new (std::nothrow) s2_solver();
  if (!s) return S2_ENOMEM;
  s->grid = *grid;
  s->gas = *gas;
  s->bcs = *bcs;
  s->sch = *scheme;
  if (s->sch.dt_every < 1) s->sch.dt_every = 1;
  if (dev) s->dev = *dev;
  else {
    memset(&s->dev, 0, sizeof(s->dev));
    s->dev.device = -1;
  }
  if ((s->dev.alloc == nullptr) != (s->dev.free == nullptr)) {
    delete s;
    return S2_EINVAL;
  }
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return S2_ECUDA;
  }
  s->device = s->dev.device >= 0 ? s->dev.device : cur;
  DeviceGuard guard(s->device);
  if (s->dev.stream) {
    s->stream = (cudaStream_t)s->dev.stream;
    s->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return S2_ECUDA;
    }
    s->own_stream = true;
  }
  if (flux_set_attributes() != cudaSuccess) {
    cudaGetLastError();
    release(s);
    delete s;
    return S2_ECUDA;
  }

  Dev &d = s->d;
  memset(&d, 0, sizeof(d));
  d.nx = grid->nx;
  d.ny = grid->ny;
  d.nz = grid->nz;
  d.px = ((grid->nx + 2 * GH) + 3) / 4 * 4;
  d.py = grid->ny + 2 * GH;
  d.pz = grid->nz + 2 * GH;
  d.sy = d.px;
  d.sz = (long long)d.px * d.py;
  d.off0 = GH * d.sz + GH * d.sy + GH;
  d.n = n;
  d.dx = grid->lx / grid->nx;
  d.dz = grid->lz / grid->nz;
  d.idx = 1.0 / d.dx;
  d.idz = 1.0 / d.dz;
  for (int l = 1; l <= 3; ++l) {
    d.ax[l] = A1[l] / d.dx;
    d.az[l] = A1[l] / d.dz;
  }
  for (int l = 0; l <= 3; ++l) {
    d.bx[l] = B2[l] / (d.dx * d.dx);
    d.bz[l] = B2[l] / (d.dz * d.dz);
  }
  set_gas(d, gas);
  d.t_wall = bcs->t_wall;
  d.thr = scheme->sensor_threshold;
  d.cfl = scheme->cfl;
  d.wall_y = bcs->y == S2_BC_ISOTHERMAL_WALL;
  d.weno = scheme->weno_order;
  d.force = bcs->force_mass_flow ? 1 : 0;

  size_t np = (size_t)d.px * d.py * d.pz;
  size_t nn = (size_t)n;
  bool ok = true;
  auto A = [&](size_t count) -> double * {
    double *p = (double *)dalloc(s, count * sizeof(double));
    if (!p) ok = false;
    return p;
  };
  d.w = A(NV * nn);
  d.fl = A(NV * nn);
  d.fln = A(NV * nn);
  d.rho = A(np); d.u = A(np); d.v = A(np); d.ww = A(np);
  d.T = A(np); d.p = A(np); d.H = A(np);
  d.div = A(np); d.sens = A(np);
  d.mu = A(nn);
  d.g = A(9 * nn);
  double *eta = A(grid->ny), *ay = A(3 * grid->ny), *by = A(4 * grid->ny), *ry = A(grid->ny), *dvy = A(grid->ny);
  size_t nparts = (size_t)((n + NT - 1) / NT);
  if (nparts < (size_t)NRED * NSTAT) nparts = (size_t)NRED * NSTAT;
  d.part = A(nparts);
  d.scal = (Scal *)dalloc(s, sizeof(Scal));
  if (!d.scal) ok = false;
  s->flag_bytes[0] = (size_t)grid->nz * grid->ny * (grid->nx + 1);
  s->flag_bytes[1] = (size_t)grid->nz * (grid->ny + 1) * grid->nx;
  s->flag_bytes[2] = (size_t)(grid->nz + 1) * grid->ny * grid->nx;
  for (int a = 0; a < 3; ++a) {
    d.nslot[a] = (long long)s->flag_bytes[a];
    d.flag[a] = (unsigned char *)dalloc(s, s->flag_bytes[a]);
    size_t nl = scheme->weno_order ? s->flag_bytes[a] : 1;
    d.wlist[a] = (unsigned *)dalloc(s, nl * sizeof(unsigned));
    d.dF[a] = (double *)dalloc(s, NV * nl * sizeof(double));
    if (!d.flag[a] || !d.wlist[a] || !d.dF[a]) ok = false;
  }
  if (!ok) {
    release(s);
    delete s;
    return S2_ENOMEM;
  }
  d.eta_y = eta;
  d.ay = ay;
  d.by = by;
  d.ry = ry;
  d.dvy = dvy;

  cudaError_t e = cudaSuccess;
  double *pads[] = {d.rho, d.u, d.v, d.ww, d.T, d.p, d.H, d.div, d.sens};
  for (double *p : pads)
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, np * sizeof(double), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.w, 0, NV * nn * sizeof(double), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.fl, 0, NV * nn * sizeof(double), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.fln, 0, NV * nn * sizeof(double), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.scal, 0, sizeof(Scal), s->stream);
  for (int a = 0; a < 3 && e == cudaSuccess; ++a)
    e = cudaMemsetAsync(d.flag[a], 0, s->flag_bytes[a], s->stream);
  // y nodes -> device, metric kernel
  std::vector<double> yn(grid->ny);
  for (int j = 0; j < grid->ny; ++j)
    yn[j] = (metrics && metrics->y) ? metrics->y[j] : -0.5 * grid->ly + (j + 0.5) * grid->ly / grid->ny;
  double *ynd = A(grid->ny);
  if (!ok) {
    release(s);
    delete s;
    return S2_ENOMEM;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ynd, yn.data(), sizeof(double) * grid->ny, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) {
    k_metric<<<(grid->ny + 127) / 128, 128, 0, s->stream>>>(ynd, grid->ny, grid->ly, d.wall_y, eta, ay, by, ry,
                                                             dvy);
    e = cudaGetLastError();
  }
  std::vector<double> dv(grid->ny);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dv.data(), dvy, sizeof(double) * grid->ny, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(s);
    delete s;
    return S2_ECUDA;
  }
  // forcing normalisation: 1 / sum_j (nx nz / eta_y)  (constant of the grid)
  double den = 0.0;
  for (int j = 0; j < grid->ny; ++j) den += dv[j] * (double)grid->nx * grid->nz;
  d.vol_inv = 1.0 / den;
  // initial dt
  double dt0 = scheme->cfl > 0 ? 0.0 : scheme->dt_fixed;
  cudaMemcpyAsync(&d.scal->dt, &dt0, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
    release(s);
    delete s;
    return S2_ECUDA;
  }
  s->step = 0;
  s->nparts_prims = (int)((n + NT - 1) / NT);
  s->graph_disabled = getenv("S2_NO_GRAPH") != nullptr;
  *out = s;
  return S2_OK;
}

int s2_set_state(s2_solver *s, const double *w, int where) {
  if (!s || !w || (where != S2_HOST && where != S2_DEVICE)) return S2_EINVAL;
  DeviceGuard guard(s->device);
  size_t bytes = NV * (size_t)s->d.n * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(s->d.w, w, bytes, where == S2_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d.fln, 0, bytes, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&s->d.scal->status, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_err(e);
}

int s2_get_state(s2_solver *s, double *w, int where) {
  if (!s || !w || (where != S2_HOST && where != S2_DEVICE)) return S2_EINVAL;
  DeviceGuard guard(s->device);
  size_t bytes = NV * (size_t)s->d.n * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(w, s->d.w, bytes, where == S2_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                  s->stream);
  if (e != cudaSuccess) return S2_ECUDA;
  return read_status(s);
}

int s2_step(s2_solver *s, int n) {
  if (!s || n < 0) return S2_EINVAL;
  DeviceGuard guard(s->device);
  for (int it = 0; it < n; ++it) {
    int want_dt = (s->sch.cfl > 0 && (s->step % s->sch.dt_every) == 0) ? 1 : 0;
    if (!s->graph_disabled && !s->graph_ready[want_dt] && build_graph(s, want_dt) != 0) s->graph_disabled = true;
    cudaError_t e;
    if (!s->graph_disabled) {
      e = cudaGraphLaunch(s->graph[want_dt], s->stream);
      s->launches += s->launches_per_step[want_dt];
    } else {
      Trace tr;
      e = enqueue_step(s, want_dt, &tr);
      s->launches += total(tr);
    }
    if (e != cudaSuccess) return S2_ECUDA;
    s->step++;
  }
  return S2_OK;
}

int s2_sync(s2_solver *s) {
  if (!s) return S2_EINVAL;
  DeviceGuard guard(s->device);
  return read_status(s);
}

int s2_set_clock(s2_solver *s, double t, long long step, double dt) {
  if (!s || step < 0) return S2_EINVAL;
  DeviceGuard guard(s->device);
  cudaError_t e = cudaMemcpyAsync(&s->d.scal->t, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && dt > 0)
    e = cudaMemcpyAsync(&s->d.scal->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return S2_ECUDA;
  s->step = step;
  return S2_OK;
}

int s2_rhs(s2_solver *s, double *rhs, int where) {
  if (!s || !rhs || (where != S2_HOST && where != S2_DEVICE)) return S2_EINVAL;
  DeviceGuard guard(s->device);
  cudaError_t e = enqueue_rhs(s, 0, nullptr);
  if (e != cudaSuccess) return S2_ECUDA;
  unsigned nb = (unsigned)((s->d.n + NT - 1) / NT);
  size_t bytes = NV * (size_t)s->d.n * sizeof(double);
  // fln is zero between steps and rewritten before it is read: use it as
  // the staging buffer, then clear it again.
  double *dst = where == S2_DEVICE ? rhs : s->d.fln;
  k_rhs_out<<<nb, NT, 0, s->stream>>>(s->d, dst);
  if ((e = cudaGetLastError()) != cudaSuccess) return S2_ECUDA;
  if (where == S2_HOST) {
    e = cudaMemcpyAsync(rhs, s->d.fln, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d.fln, 0, bytes, s->stream);
    if (e != cudaSuccess) return S2_ECUDA;
  }
  return read_status(s);
}

int s2_get_flags(s2_solver *s, unsigned char *fx, unsigned char *fy, unsigned char *fz) {
  if (!s) return S2_EINVAL;
  DeviceGuard guard(s->device);
  unsigned char *o[3] = {fx, fy, fz};
  for (int a = 0; a < 3; ++a)
    if (o[a] &&
        cudaMemcpyAsync(o[a], s->d.flag[a], s->flag_bytes[a], cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
      return S2_ECUDA;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return S2_ECUDA;
  return S2_OK;
}

int s2_stats(s2_solver *s, s2_stats_t *out) {
  if (!s || !out) return S2_EINVAL;
  DeviceGuard guard(s->device);
  k_stats_partial<<<NRED, NT, 0, s->stream>>>(s->d);
  if (cudaGetLastError() != cudaSuccess) return S2_ECUDA;
  k_stats_final<<<1, NT, 0, s->stream>>>(s->d, NRED);
  if (cudaGetLastError() != cudaSuccess) return S2_ECUDA;
  Scal h;
  if (cudaMemcpyAsync(&h, s->d.scal, sizeof(Scal), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) return S2_ECUDA;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return S2_ECUDA;
  memset(out, 0, sizeof(*out));
  out->t = h.t;
  out->step = s->step;
  out->dt = h.dt;
  out->mass = h.red[0];
  out->mom[0] = h.red[1];
  out->mom[1] = h.red[2];
  out->mom[2] = h.red[3];
  out->energy = h.red[4];
  out->kinetic = h.red[5];
  out->residual_rhou = sqrt(h.red[6] / (double)s->d.n);
  out->weno_frac = s->d.weno ? (double)h.wcount / (3.0 * (double)s->d.n) : 0.0;
  out->forcing = h.force;
  out->launches = s->launches;
  out->status = (h.status & ERR_NONFINITE) ? S2_ENONFINITE : S2_OK;
  return out->status;
}

int s2_profile(s2_solver *s, int n, double *ms, long long *launches) {
  if (!s || n < 0) return S2_EINVAL;
  DeviceGuard guard(s->device);
  Trace tr;
  tr.timed = true;
  int rc = S2_OK;
  for (int it = 0; it < n && rc == S2_OK; ++it) {
    int want_dt = (s->sch.cfl > 0 && (s->step % s->sch.dt_every) == 0) ? 1 : 0;
    if (enqueue_step(s, want_dt, &tr) != cudaSuccess) rc = S2_ECUDA;
    else s->step++;
  }
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) rc = S2_ECUDA;
  double acc[S2_PROF_KINDS] = {0};
  for (auto &r : tr.recs) {
    float t = 0.f;
    if (rc == S2_OK && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) acc[r.kind] += t;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  s->launches += total(tr);
  for (int k = 0; k < S2_PROF_KINDS; ++k) {
    if (ms) ms[k] = acc[k];
    if (launches) launches[k] = tr.count[k];
  }
  if (rc != S2_OK) return rc;
  return read_status(s);
}

const char *s2_profile_name(int kind) {
  static const char *names[S2_PROF_KINDS] = {"prims", "dt", "ghost", "grad", "ghost_aux", "flux_x", "flux_y",
                                             "flux_z", "visc", "force", "update", "weno", "apply"};
  return (kind >= 0 && kind < S2_PROF_KINDS) ? names[kind] : nullptr;
}

void s2_destroy(s2_solver *s) {
  if (!s) return;
  {
    DeviceGuard guard(s->device);
    cudaStreamSynchronize(s->stream);
    release(s);
  }
  delete s;
}

}  // extern "C"
