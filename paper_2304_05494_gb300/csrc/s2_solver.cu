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

#include <cmath>
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

// Central coefficients of order 2L (L = 1..4): first derivative a_l,
// second derivative b_l (b_0 the centre weight).
const double A1_ORD[5][5] = {{0.0, 0.0, 0.0, 0.0, 0.0},
                             {0.0, 1.0 / 2.0, 0.0, 0.0, 0.0},
                             {0.0, 2.0 / 3.0, -1.0 / 12.0, 0.0, 0.0},
                             {0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0, 0.0},
                             {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0}};
const double B2_ORD[5][5] = {{0.0, 0.0, 0.0, 0.0, 0.0},
                             {-2.0, 1.0, 0.0, 0.0, 0.0},
                             {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0, 0.0, 0.0},
                             {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0, 0.0},
                             {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0}};

// Stencil tables passed to the metric kernel.
struct MetricCoef {
  double am[5], bm[5];  // metric order (the higher of the two)
  double av[5], bv[5];  // viscous order
  int lm, lv;
};
// Wray's low-storage RK3 coefficients.
const double RK_G[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
const double RK_R[4] = {0.0, -17.0 / 60.0, -5.0 / 12.0, 0.0};


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
// pre-scaled coefficient tables used by the stencil kernels, in double and
// in single precision.
__global__ void k_metric(const double *yn, int ny, double ly, int wall, MetricCoef mc, double *eta_y, double *ay,
                         double *by, double *ry, double *dvy, float *eta_yf, float *ayf, float *byf, float *ryf) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ny) return;
  const double *a = mc.am, *b = mc.bm;
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
  for (int l = 1; l <= mc.lm; ++l) {
    d1 += a[l] * (ext(j + l) - ext(j - l));
    d2 += b[l] * (ext(j + l) + ext(j - l));
  }
  double ey = 1.0 / d1;
  double eyy = -d2 / (d1 * d1 * d1);
  eta_y[j] = ey;
  eta_yf[j] = (float)ey;
  for (int l = 1; l <= 4; ++l) {
    ay[4 * j + l - 1] = mc.av[l] * ey;
    ayf[4 * j + l - 1] = (float)(mc.av[l] * ey);
  }
  for (int l = 0; l <= 4; ++l) {
    by[5 * j + l] = mc.bv[l] * ey * ey;
    byf[5 * j + l] = (float)(mc.bv[l] * ey * ey);
  }
  ry[j] = eyy / ey;
  ryf[j] = (float)(eyy / ey);
  dvy[j] = d1;
}

__device__ __forceinline__ void dt_block_max(const Dev &d, double sr, int want_dt, unsigned bx) {
  if (want_dt) {
    __shared__ double red[NT / 32];
    double m = warp_max(sr);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
      s = warp_max(s);
      if (threadIdx.x == 0 && S2_OK_IDX(d, bx, d.nparts)) d.part[bx] = s;
    }
  }
}

// Whether this launch computes the CFL partials: decided once per CTA (the
// step counter is 64-bit, and a 64-bit remainder per thread would go
// through the double-precision unit).
__device__ __forceinline__ int block_want_dt(const Dev &d, int stage0) {
  __shared__ int want;
  if (threadIdx.x == 0) want = stage0 && dt_due(d);
  __syncthreads();
  return want;
}

// ------------------------------------------------------------- primitives
// rho, u = (rho u)/rho, ..., T from e = E - |u|^2/2 (e/c_v, or the
// inverse of e(T) of a thermally perfect gas), p = rho R T, H = e + R T +
// |u|^2/2, mu = (T/T_ref)^omega/Re.  With want_dt, also the CFL spectral
// radius max into part[block] (c = sqrt(gamma R T)).
// TP: thermally perfect gas (a separate instantiation keeps the
// calorically perfect kernel free of the Newton iteration's code).
template <bool TP>
__device__ __forceinline__ void prims_body(const Dev &__restrict__ d, const Blk &B, int stage0) {
  long long q = (long long)B.x * NT + threadIdx.x;
  const View<double> V = view<double>(d);
  const int want_dt = block_want_dt(d, stage0);
  double sr = 0.0;
  if (q < d.n) {
    int i, j, k;
    point_of(d, q, i, j, k);
    long long p = pidx(d, i, j, k);
    const double *w = d.w;
    double rho = w[q];
    double ri = rcp_pos(rho);
    double u = w[d.n + q] * ri, v = w[2 * d.n + q] * ri, ww = w[3 * d.n + q] * ri;
    double q2 = u * u + v * v + ww * ww;
    const double e = w[4 * d.n + q] * ri - 0.5 * q2;
    double T = e * d.icv;
    double h = d.cp * T;  // enthalpy
    const bool okp = S2_OK_IDX(d, p, d.np);
    if (TP) {
      // T from e by Newton's method, from the point's previous temperature
      double T0 = 0.0;
      S2_GUARD(okp) T0 = V.T[p];
      if (!positive_finite(T0)) T0 = tp_guess(d.kd, e);
      bool ok = true;
      T = tp_temperature(d.kd, e, T0, 0.0, ok);
      if (!ok) atomicOr(&d.scal->status, ERR_NONFINITE);
      h = fma(d.R, T, e);
    }
    double pr = rho * d.R * T;
    S2_GUARD(okp) {
      V.rho[p] = rho;
      V.u[p] = u;
      V.v[p] = v;
      V.ww[p] = ww;
      V.T[p] = T;
      V.p[p] = pr;
      V.H[p] = h + 0.5 * q2;
    }
    double mu = 0.0;
    if (d.viscous) {
      mu = viscosity(d, T);
      V.mu[q] = mu;
    }
    if (!positive_finite(rho) || !positive_finite(T) || !finite_bits(q2))
      atomicOr(&d.scal->status, ERR_NONFINITE);
    if (want_dt) sr = spectral_radius<TP>(d, rho, u, v, ww, T, mu, d.eta_y[j]);
  }
  dt_block_max(d, sr, want_dt, B.x);
}

template <bool TP>
__global__ void __launch_bounds__(NT) k_prims(Dev d, int stage0) {
  prims_body<TP>(d, grid_blk(), stage0);
}

template <bool TP>
__global__ void __launch_bounds__(NT) kb_prims(BatchArgs ba, int stage0) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  prims_body<TP>(sd, B, stage0);
}

// Mixed path: the internal energy per volume rho e = E - rho |u|^2 / 2 is
// formed by a double-precision subtraction (E and the kinetic energy nearly
// cancel at high speed), the kinetic part itself to single-precision
// relative accuracy: the relative error of rho e is then about
// 2^-24 (1 + KE / (rho e)), KE/(rho e) = gamma (gamma-1) M^2 / 2.  Everything
// else, and everything stored, is single precision; the one double
// operation per point leaves the kernel bound by memory traffic.
__device__ __forceinline__ void prims_mixed_body(const Dev &__restrict__ d, const Blk &B, int stage0) {
  long long q = (long long)B.x * NT + threadIdx.x;
  const View<float> V = view<float>(d);
  const int want_dt = block_want_dt(d, stage0);
  const Consts<float> &K = d.kf;
  double sr = 0.0;
  if (q < d.n) {
    int i, j, k;
    point_of(d, q, i, j, k);
    long long p = pidx(d, i, j, k);
    const double *w = d.w;
    const float rf = d2f_int(w[q]);
    const float rif = 1.0f / rf;
    float u = d2f_int(w[d.n + q]) * rif, v = d2f_int(w[2 * d.n + q]) * rif, ww = d2f_int(w[3 * d.n + q]) * rif;
    float q2 = u * u + v * v + ww * ww;
    const float rhoe = d2f_int(w[4 * d.n + q] - f2d_int(0.5f * rf * q2));
    float T = rhoe * rif * K.icv;
    float h = K.cp * T;  // enthalpy
    bool ok = true;
    const bool okp = S2_OK_IDX(d, p, d.np);
    if (K.tp) {
      // T from e by Newton's method, from the point's previous temperature
      const float e = rhoe * rif;
      float T0 = 0.0f;
      S2_GUARD(okp) T0 = V.T[p];
      if (!(T0 > 0.0f && T0 < 3.0e38f)) T0 = tp_guess(K, e);
      T = tp_temperature(K, e, T0, 0.0f, ok);
      h = fmaf(K.R_gas, T, e);
    }
    S2_GUARD(okp) {
      V.rho[p] = rf;
      V.u[p] = u;
      V.v[p] = v;
      V.ww[p] = ww;
      V.T[p] = T;
      V.p[p] = rf * K.R_gas * T;
      V.H[p] = h + 0.5f * q2;
    }
    float mu = 0.0f;
    if (d.viscous) {
      mu = viscosity(d, T);
      V.mu[q] = mu;
    }
    if (!ok || !(rf > 0.0f) || !(T > 0.0f) || !isfinite(rf) || !isfinite(T) || !isfinite(q2))
      atomicOr(&d.scal->status, ERR_NONFINITE);
    if (want_dt) {
      float gam = K.gamma, c2 = K.gR * T;
      if (K.tp) {
        const float cp = tp_cp(K, T, 1.0f / T);
        gam = cp / (cp - K.R_gas);
        c2 = gam * K.R_gas * T;
      }
      float cs = sqrtf(c2);
      float ey = d.eta_yf[j];
      float srf = (fabsf(u) + cs) * K.idx + (fabsf(v) + cs) * ey + (fabsf(ww) + cs) * K.idz;
      if (d.viscous)
        srf += gam * mu / ((float)d.prandtl * rf) * (K.idx * K.idx + ey * ey + K.idz * K.idz);
      sr = srf;
    }
  }
  dt_block_max(d, sr, want_dt, B.x);
}

__global__ void __launch_bounds__(NT) k_prims_mixed(Dev d, int stage0) { prims_mixed_body(d, grid_blk(), stage0); }

__global__ void __launch_bounds__(NT) kb_prims_mixed(BatchArgs ba, int stage0) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  prims_mixed_body(sd, B, stage0);
}

// dt = cfl / max(spectral radius) over the partials of k_prims, at the
// steps where it is due (no-op otherwise).
__device__ __forceinline__ void dt_final_body(const Dev &__restrict__ d, int nparts) {
  if (!dt_due(d)) return;
  double m = 0.0;
  if (!S2_OK_IDX(d, nparts - 1, d.nparts)) nparts = 0;
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

__global__ void k_dt_final(Dev d, int nparts) { dt_final_body(d, nparts); }

// one CTA per box; nparts[b]: box b's CFL partials
__global__ void __launch_bounds__(NT) kb_dt_final(BatchArgs ba, const int *nparts) {
  S2_BATCH_ENTER(ba, sd, B, b);
  dt_final_body(sd, nparts[b]);
}

// ----------------------------------------------------------------- ghosts
// Face ghost (GH deep) t of the three face sets -> destination and source.
__device__ __forceinline__ bool ghost_map(const Dev &d, long long t, int &di, int &dj, int &dk, int &si, int &sj,
                                          int &sk) {
  const unsigned nxf = 2u * GH * d.ny * d.nz, nyf = 2u * GH * d.nx * d.nz;
  unsigned u = (unsigned)t;
  bool wall = false;
  if (u < nxf) {
    int g = (int)(u % (2 * GH));
    unsigned r = u / (2 * GH), kk = d.fny.div(r);
    dj = (int)(r - kk * (unsigned)d.ny);
    dk = (int)kk;
    di = g < GH ? -1 - g : d.nx + (g - GH);
    si = imod(di, d.nx); sj = dj; sk = dk;
  } else if (u < nxf + nyf) {
    u -= nxf;
    unsigned r = d.fnx.div(u);
    di = (int)(u - r * (unsigned)d.nx);
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
    u -= nxf + nyf;
    unsigned r = d.fnx.div(u);
    di = (int)(u - r * (unsigned)d.nx);
    int g = (int)(r % (2 * GH));
    dj = (int)(r / (2 * GH));
    dk = g < GH ? -1 - g : d.nz + (g - GH);
    si = di; sj = dj;
    sk = imod(dk, d.nz);
  }
  return wall;
}

// Face ghosts of the primitive fields.  x and z periodic; y periodic or
// isothermal no-slip wall mirrored about the face between the outermost
// node and its ghost: u -> -u, T -> 2 T_w - T, p -> p, rho = p/(R T), H =
// h(T) + |u|^2/2.
template <class R>
__device__ __forceinline__ void ghost_prim_body(const Dev &__restrict__ d, const Blk &B) {
  long long total = 2LL * GH * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
  long long t = (long long)B.x * NT + threadIdx.x;
  if (t >= total) return;
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  int di, dj, dk, si, sj, sk;
  bool wall = ghost_map(d, t, di, dj, dk, si, sj, sk);
  long long dp = pidx(d, di, dj, dk), sp = pidx(d, si, sj, sk);
  if (!(S2_OK_IDX(d, dp, d.np) && S2_OK_IDX(d, sp, d.np))) return;
  if (!wall) {
    // all loads first (the stores could alias them as far as the compiler
    // knows; interleaving would serialise the round trips)
    const R r = V.rho[sp], u = V.u[sp], v = V.v[sp], ww = V.ww[sp], T = V.T[sp], pr = V.p[sp], H = V.H[sp];
    V.rho[dp] = r;
    V.u[dp] = u;
    V.v[dp] = v;
    V.ww[dp] = ww;
    V.T[dp] = T;
    V.p[dp] = pr;
    V.H[dp] = H;
  } else {
    R u = -V.u[sp], v = -V.v[sp], ww = -V.ww[sp];
    R T = R(2) * K.t_wall - V.T[sp];
    R pr = V.p[sp];
    V.u[dp] = u;
    V.v[dp] = v;
    V.ww[dp] = ww;
    V.T[dp] = T;
    V.p[dp] = pr;
    V.rho[dp] = pr / (K.R_gas * T);
    const R h = K.tp ? fma(K.R_gas, T, tp_e(K, T, rcp_pos(T))) : K.cp * T;
    V.H[dp] = h + R(0.5) * (u * u + v * v + ww * ww);
    if (!(T > R(0))) atomicOr(&d.scal->status, ERR_NONFINITE);
  }
}

template <class R>
__global__ void __launch_bounds__(NT) k_ghost_prim(Dev d) {
  ghost_prim_body<R>(d, grid_blk());
}

template <class R>
__global__ void __launch_bounds__(NT) kb_ghost_prim(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  ghost_prim_body<R>(sd, B);
}

// Face ghosts of div u and of the sensor.  At a wall the sensor is
// mirrored and the divergence of the mirrored velocity field is
// -u_x + v_y - w_z at the mirror node.
template <class R>
__device__ __forceinline__ void ghost_aux_body(const Dev &__restrict__ d, const Blk &B) {
  long long total = 2LL * GH * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
  long long t = (long long)B.x * NT + threadIdx.x;
  if (t >= total) return;
  const View<R> V = view<R>(d);
  int di, dj, dk, si, sj, sk;
  bool wall = ghost_map(d, t, di, dj, dk, si, sj, sk);
  long long dp = pidx(d, di, dj, dk), sp = pidx(d, si, sj, sk);
  if (!(S2_OK_IDX(d, dp, d.np) && S2_OK_IDX(d, sp, d.np))) return;
  const R sv = V.sens[sp];
  if (!wall) {
    const R dv = V.div[sp];
    V.sens[dp] = sv;
    V.div[dp] = dv;
    return;
  }
  V.sens[dp] = sv;
  if (!d.mixed) {  // the mixed path's gradient pass writes these itself
    long long q = ((long long)sk * d.ny + sj) * d.nx + si;
    if (!S2_OK_IDX(d, q, d.n)) return;
    R ux = V.g[0 * d.n + q], vy = V.g[4 * d.n + q], wz = V.g[8 * d.n + q];
    V.div[dp] = -ux + vy - wz;
  }
}

template <class R>
__global__ void __launch_bounds__(NT) k_ghost_aux(Dev d) {
  ghost_aux_body<R>(d, grid_blk());
}

template <class R>
__global__ void __launch_bounds__(NT) kb_ghost_aux(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  ghost_aux_body<R>(sd, B);
}

// ---------------------------------------------------------------- forcing
// force_rhs_1: partial sums of R_rhou dV (dV ~ 1/eta_y), deterministic.
// One warp per x-row (fixed j, k): the row is summed in the path's
// precision and weighted by dy/deta once, so the loop carries no index
// division.
template <class R>
__device__ __forceinline__ void force_partial_body(const Dev &__restrict__ d, const Blk &B) {
  const View<R> V = view<R>(d);
  const int lane = threadIdx.x & 31;
  const long long rows = (long long)d.ny * d.nz;
  double s = 0.0;
  for (long long r = (long long)B.x * (NT / 32) + (threadIdx.x >> 5); r < rows;
       r += (long long)B.nx * (NT / 32)) {
    const R *row = V.fl + d.n + r * d.nx;
    R sr = 0;
    for (int i = lane; i < d.nx; i += 32) sr += row[i];
    const unsigned ru = (unsigned)r;
    s += (double)sr * d.dvy[(int)(ru - d.fny.div(ru) * (unsigned)d.ny)];
  }
  double v[1] = {s};
  block_sum<1>(v);
  if (threadIdx.x == 0 && S2_OK_IDX(d, B.x, d.nparts)) d.part[B.x] = v[0];
}

template <class R>
__global__ void __launch_bounds__(NT) k_force_partial(Dev d) {
  force_partial_body<R>(d, grid_blk());
}

template <class R>
__global__ void __launch_bounds__(NT) kb_force_partial(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  force_partial_body<R>(sd, B);
}

__device__ __forceinline__ void force_final_body(const Dev &__restrict__ d, int nparts) {
  double s = 0.0;
  if (!S2_OK_IDX(d, nparts - 1, d.nparts)) nparts = 0;
  for (int b = threadIdx.x; b < nparts; b += NT) s += d.part[b];
  double v[1] = {s};
  block_sum<1>(v);
  if (threadIdx.x == 0) d.scal->force = -v[0] * d.vol_inv;
}

__global__ void k_force_final(Dev d, int nparts) { force_final_body(d, nparts); }

// one CTA per box; nparts[b]: box b's forcing partials
__global__ void __launch_bounds__(NT) kb_force_final(BatchArgs ba, const int *nparts) {
  S2_BATCH_ENTER(ba, sd, B, b);
  force_final_body(sd, nparts[b]);
}

// The per-RHS counters of the hybrid scheme (flagged interfaces and the
// three list lengths), zeroed for every box of a batch in one launch.
__global__ void __launch_bounds__(NT) kb_reset_counts(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  if (threadIdx.x == 0) {
    sd.scal->wcount = 0;
    for (int a = 0; a < 4; ++a) sd.scal->nlist[a] = 0;
  }
}

// ----------------------------------------------------------------- update
// w <- w + dt gamma_k R + fln ; fln <- dt rho_{k+1} R, with R = fl + the
// forcing (f on rho u, f u on rho E).  Stage 0 reads no fln; the last
// stage writes none and advances the clock.
__device__ __forceinline__ void update_body(const Dev &__restrict__ d, const Blk &B, double gk, double rk1, int stage) {
  long long q = (long long)B.x * NT + threadIdx.x;
  const View<double> V = view<double>(d);
  const double dt = d.scal->dt;
  if (q < d.n) {
    double f = d.force ? d.scal->force : 0.0;
    double fu = 0.0;
    if (d.force) {
      int i, j, k;
      point_of(d, q, i, j, k);
      const long long pu = pidx(d, i, j, k);
      if (S2_OK_IDX(d, pu, d.np)) fu = f * V.u[pu];
    }
    const double a = dt * gk, b = dt * rk1;
    // every load before the first store: the arrays could alias as far as
    // the compiler knows, so interleaving would serialise the round trips
    double R[NV], wo[NV], ro[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long o = v * d.n + q;
      R[v] = V.fl[o];
      wo[v] = d.w[o];
      ro[v] = stage > 0 ? V.fln[o] : 0.0;
    }
    R[1] += f;
    R[4] += fu;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long o = v * d.n + q;
      double wn = fma(a, R[v], wo[v]);
      if (stage > 0) wn += ro[v];
      d.w[o] = wn;
      if (stage < 2) V.fln[o] = b * R[v];
    }
  }
  if (stage == 2 && q == 0) {
    d.scal->t += dt;
    d.scal->nstep += 1;
  }
}

__global__ void __launch_bounds__(NT) k_update(Dev d, double gk, double rk1, int stage) {
  update_body(d, grid_blk(), gk, rk1, stage);
}

__global__ void __launch_bounds__(NT) kb_update(BatchArgs ba, double gk, double rk1, int stage) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  update_body(sd, B, gk, rk1, stage);
}

// Mixed path: the increment dt gamma_k R + fln is formed in single
// precision (R and the register are single precision) and accumulated
// into the double-precision state.
__device__ __forceinline__ void update_mixed_body(const Dev &__restrict__ d, const Blk &B, double gk, double rk1, int stage) {
  long long q = (long long)B.x * NT + threadIdx.x;
  const View<float> V = view<float>(d);
  // dt gamma_k, dt rho_{k+1} and the forcing in single precision, once per
  // CTA: the per-point path then needs the double-precision unit only for
  // the five additions to the state (float -> double on the integer pipe)
  __shared__ float coef[3];
  const double dt = d.scal->dt;
  if (threadIdx.x == 0) {
    coef[0] = (float)(dt * gk);
    coef[1] = (float)(dt * rk1);
    coef[2] = d.force ? (float)d.scal->force : 0.0f;
  }
  __syncthreads();
  if (q < d.n) {
    const float a = coef[0], b = coef[1], f = coef[2];
    float fu = 0.0f;
    if (d.force) {
      int i, j, k;
      point_of(d, q, i, j, k);
      const long long pu = pidx(d, i, j, k);
      if (S2_OK_IDX(d, pu, d.np)) fu = f * V.u[pu];
    }
    // every load before the first store (see k_update)
    float R[NV], ro[NV];
    double wo[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long o = v * d.n + q;
      R[v] = V.fl[o];
      wo[v] = d.w[o];
      ro[v] = stage > 0 ? V.fln[o] : 0.0f;
    }
    R[1] += f;
    R[4] += fu;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long o = v * d.n + q;
      const float inc = stage > 0 ? fmaf(a, R[v], ro[v]) : a * R[v];
      d.w[o] = wo[v] + f2d_int(inc);
      if (stage < 2) V.fln[o] = b * R[v];
    }
  }
  if (stage == 2 && q == 0) {
    d.scal->t += dt;
    d.scal->nstep += 1;
  }
}

__global__ void __launch_bounds__(NT) k_update_mixed(Dev d, double gk, double rk1, int stage) {
  update_mixed_body(d, grid_blk(), gk, rk1, stage);
}

__global__ void __launch_bounds__(NT) kb_update_mixed(BatchArgs ba, double gk, double rk1, int stage) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  update_mixed_body(sd, B, gk, rk1, stage);
}

// Primitive fields prim[v][k][j][i] = (rho, u, v, w, T) -> conserved
// state w with the solver's gas, E = e(T) + |u|^2/2 (e = c_v T, or the
// thermally perfect e(T)).  prim and w may be the same array: each thread
// reads its point's five values before writing them.
__global__ void __launch_bounds__(NT) k_from_prims(Dev d, const double *prim, double *w) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const double rho = prim[q], u = prim[d.n + q], v = prim[2 * d.n + q], ww = prim[3 * d.n + q];
  const double T = prim[4 * d.n + q];
  if (!positive_finite(rho) || !positive_finite(T)) atomicOr(&d.scal->status, ERR_NONFINITE);
  const double e = d.kd.tp ? tp_e(d.kd, T, rcp_pos(T)) : d.cv * T;
  w[q] = rho;
  w[d.n + q] = rho * u;
  w[2 * d.n + q] = rho * v;
  w[3 * d.n + q] = rho * ww;
  w[4 * d.n + q] = rho * (e + 0.5 * (u * u + v * v + ww * ww));
}

// Conserved state -> primitive fields (rho, u, v, w, T), T in double
// precision in both modes (the thermally perfect inversion from the
// linearisation of e(T) about T = 1).
__global__ void __launch_bounds__(NT) k_to_prims(Dev d, const double *w, double *prim) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const double rho = w[q], ri = 1.0 / rho;
  const double u = w[d.n + q] * ri, v = w[2 * d.n + q] * ri, ww = w[3 * d.n + q] * ri;
  const double e = w[4 * d.n + q] * ri - 0.5 * (u * u + v * v + ww * ww);
  double T = e * d.icv;
  bool ok = true;
  if (d.kd.tp) T = tp_temperature(d.kd, e, tp_guess(d.kd, e), 0.0, ok);
  if (!ok || !positive_finite(rho) || !positive_finite(T)) atomicOr(&d.scal->status, ERR_NONFINITE);
  prim[q] = rho;
  prim[d.n + q] = u;
  prim[2 * d.n + q] = v;
  prim[3 * d.n + q] = ww;
  prim[4 * d.n + q] = T;
}

// R = fl + forcing into out (diagnostics, double).
template <class R>
__global__ void __launch_bounds__(NT) k_rhs_out(Dev d, double *out) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const View<R> V = view<R>(d);
  double f = d.force ? d.scal->force : 0.0;
  double fu = 0.0;
  if (d.force) {
    int i, j, k;
    point_of(d, q, i, j, k);
    fu = f * (double)V.u[pidx(d, i, j, k)];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double Rv = (double)V.fl[v * d.n + q];
    if (v == 1) Rv += f;
    if (v == 4) Rv += fu;
    out[v * d.n + q] = Rv;
  }
}

// ------------------------------------------------------------------ stats
// Integrals of rho, rho u_a, rho E, rho|u|^2/2 (dV = dx dz / eta_y) and
// the sum of (R_rhou)^2 of the last RHS evaluation.
constexpr int NSTAT = 7;
template <class R>
__global__ void __launch_bounds__(NT) k_stats_partial(Dev d) {
  const View<R> V = view<R>(d);
  double v[NSTAT] = {0, 0, 0, 0, 0, 0, 0};
  double f = d.force ? d.scal->force : 0.0;
  for (long long q = (long long)blockIdx.x * NT + threadIdx.x; q < d.n; q += (long long)gridDim.x * NT) {
    int j = row_of(d, q);
    double dv = d.dvy[j] * d.dx * d.dz;
    double rho = d.w[q], mx = d.w[d.n + q], my = d.w[2 * d.n + q], mz = d.w[3 * d.n + q];
    v[0] += rho * dv;
    v[1] += mx * dv;
    v[2] += my * dv;
    v[3] += mz * dv;
    v[4] += d.w[4 * d.n + q] * dv;
    v[5] += 0.5 * (mx * mx + my * my + mz * mz) / rho * dv;
    double r = (double)V.fl[d.n + q] + f;
    v[6] += r * r;
  }
  block_sum<NSTAT>(v);
  if (threadIdx.x == 0)
    for (int m = 0; m < NSTAT; ++m)
      if (S2_OK_IDX(d, m * NRED + blockIdx.x, d.nparts)) d.part[m * NRED + blockIdx.x] = v[m];
}

__global__ void k_stats_final(Dev d, int nparts) {
  double v[NSTAT];
  for (int m = 0; m < NSTAT; ++m) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += NT)
      if (S2_OK_IDX(d, m * NRED + b, d.nparts)) s += d.part[m * NRED + b];
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
  cudaGraphExec_t graph;
  bool graph_ready;
  bool graph_disabled;
  int last_status;
  size_t flag_bytes[3];
  long long launches_per_step;
  long long launches;
  size_t rsize;         // bytes of the arithmetic type (8 FP64, 4 mixed)
  double *rhs_stage;    // staging of s2_rhs output
  FluxMaps fmaps[3][2];  // tensor maps of the staged fields, per direction and tile variant
  // second stream for the WENO corrections of a direction, which run while
  // the flux kernels of the next directions do (fork after each flux
  // kernel, join before the viscous pass)
  cudaStream_t side;
  cudaEvent_t ev_flux[3], ev_join;
  // s2_stream_states (set up at its first call): one device staging buffer
  // per direction, the copy-in and copy-out streams and their events
  double *stage_in, *stage_out;
  cudaStream_t cin, cout;
  cudaEvent_t ev_in_ready, ev_in_free, ev_out_ready, ev_out_free;
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
  if (s->graph_ready) cudaGraphExecDestroy(s->graph);
  for (int a = 0; a < 3; ++a)
    if (s->ev_flux[a]) cudaEventDestroy(s->ev_flux[a]);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->side) cudaStreamDestroy(s->side);
  for (cudaEvent_t ev : {s->ev_in_ready, s->ev_in_free, s->ev_out_ready, s->ev_out_free})
    if (ev) cudaEventDestroy(ev);
  if (s->cin) cudaStreamDestroy(s->cin);
  if (s->cout) cudaStreamDestroy(s->cout);
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
cudaError_t enqueue_rhs(s2_solver *s, int stage0, Trace *tr) {
  const Dev &d = s->d;
  cudaStream_t st = s->stream;
  cudaError_t e;
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  long long nghost = 2LL * GH * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
  unsigned ngb = (unsigned)((nghost + NT - 1) / NT);
  e = run(tr, st, S2_PROF_PRIMS, 1, [&] {
    if (d.mixed) k_prims_mixed<<<nb, NT, 0, st>>>(d, stage0);
    else if (d.kd.tp) k_prims<true><<<nb, NT, 0, st>>>(d, stage0);
    else k_prims<false><<<nb, NT, 0, st>>>(d, stage0);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  if (stage0 && d.cfl > 0.0) {
    e = run(tr, st, S2_PROF_DT, 1, [&] {
      k_dt_final<<<1, NT, 0, st>>>(d, (int)nb);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  e = run(tr, st, S2_PROF_GHOST, 1, [&] {
    if (d.mixed) k_ghost_prim<float><<<ngb, NT, 0, st>>>(d);
    else k_ghost_prim<double><<<ngb, NT, 0, st>>>(d);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  if (d.viscous || d.weno) {
    e = run(tr, st, S2_PROF_GRAD, 1, [&] { return launch_grad(d, st); });
    if (e != cudaSuccess) return e;
    e = run(tr, st, S2_PROF_GHOST_AUX, 1, [&] {
      if (d.mixed) k_ghost_aux<float><<<ngb, NT, 0, st>>>(d);
      else k_ghost_aux<double><<<ngb, NT, 0, st>>>(d);
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
  // Outside the per-kernel profile, each direction's WENO corrections run
  // on the side stream as soon as its flux kernel has listed the flagged
  // interfaces, beside the flux kernels of the next directions (they share
  // no output: dF of the direction against the RHS and the other lists).
  // Double precision only: there both are bound by the double-precision
  // unit and the WENO kernels fill its idle slots (1 % per step); the
  // single-precision flux kernels occupy every SM with a persistent grid
  // and measured slower with the extra branch.
  const bool overlap = d.weno && !d.mixed && !(tr && tr->timed);
  for (int dir = 0; dir < 3; ++dir) {
    e = run(tr, st, S2_PROF_FLUX_X + dir, 1, [&] { return launch_flux(d, s->fmaps[dir], dir, dir > 0, st); });
    if (e != cudaSuccess) return e;
    if (overlap) {
      if ((e = cudaEventRecord(s->ev_flux[dir], st)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(s->side, s->ev_flux[dir], 0)) != cudaSuccess) return e;
      if ((e = launch_weno(d, dir, s->side)) != cudaSuccess) return e;
      if (tr) tr->count[S2_PROF_WENO] += 1;
    }
  }
  if (overlap) {
    if ((e = cudaEventRecord(s->ev_join, s->side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, s->ev_join, 0)) != cudaSuccess) return e;
  } else if (d.weno) {
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
    const int fused = visc_force_partials(d);  // partials already written by the viscous pass
    e = run(tr, st, S2_PROF_FORCE, fused ? 1 : 2, [&] {
      if (fused) {
        k_force_final<<<1, NT, 0, st>>>(d, fused);
        return cudaGetLastError();
      }
      if (d.mixed) k_force_partial<float><<<NRED, NT, 0, st>>>(d);
      else k_force_partial<double><<<NRED, NT, 0, st>>>(d);
      k_force_final<<<1, NT, 0, st>>>(d, NRED);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t enqueue_step(s2_solver *s, Trace *tr) {
  const Dev &d = s->d;
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  cudaError_t e;
  for (int st = 0; st < 3; ++st) {
    if ((e = enqueue_rhs(s, st == 0, tr)) != cudaSuccess) return e;
    e = run(tr, s->stream, S2_PROF_UPDATE, 1, [&] {
      if (d.mixed) k_update_mixed<<<nb, NT, 0, s->stream>>>(d, RK_G[st], RK_R[st + 1], st);
      else k_update<<<nb, NT, 0, s->stream>>>(d, RK_G[st], RK_R[st + 1], st);
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

int build_graph(s2_solver *s) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  Trace tr;
  cudaError_t e = enqueue_step(s, &tr);
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
  s->graph = ex;
  s->graph_ready = true;
  s->launches_per_step = total(tr);
  return 0;
}

int read_status(s2_solver *s) {
  int st = 0;
  if (cudaMemcpyAsync(&st, &s->d.scal->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return S2_ECUDA;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return S2_ECUDA;
  if (st & ERR_BOUNDS) return S2_EBOUNDS;
  if (st & ERR_NONFINITE) return S2_ENONFINITE;
  if (st & ERR_TIMEOUT) return S2_ETIMEOUT;
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
      d.mu_qm1 = q - 1.0;
      d.mu_qp1 = q + 1.0;
      break;
    }
  }
  d.cv = d.R / (gas->gamma - 1.0);
  d.icv = 1.0 / d.cv;
  d.cp = gas->gamma * d.cv;
  d.prandtl = gas->prandtl;
  d.re = gas->re_ref;
  d.inv_re = 1.0 / gas->re_ref;
  d.visc_exp_f = (float)gas->visc_exp;
  d.visc_exp = gas->visc_exp;
  d.inv_t_ref = 1.0 / gas->t_ref;
  d.cp_over_pr = d.cp / gas->prandtl;
  d.viscous = gas->re_ref > 0.0;
  // thermally perfect gas: coefficients of c_p, dc_p/dT and e(T) in both
  // precisions (kernels of both paths read them from the constants)
  d.kd.R_gas = d.R;
  d.kf.R_gas = (float)d.R;
  d.kd.inv_pr = 1.0 / gas->prandtl;
  d.kf.inv_pr = (float)d.kd.inv_pr;
  d.kd.tp = d.kf.tp = gas->cp_coeffs ? 1 : 0;
  if (gas->cp_coeffs) {
    double c[7];
    for (int l = 0; l < 7; ++l) c[l] = d.R * gas->cp_coeffs[l];
    const double dcc[6] = {-2.0 * c[0], -c[1], c[3], 2.0 * c[4], 3.0 * c[5], 4.0 * c[6]};
    const double ecf[7] = {-c[0], c[1], c[2] - d.R, c[3] / 2.0, c[4] / 3.0, c[5] / 4.0, c[6] / 5.0};
    for (int l = 0; l < 7; ++l) {
      d.kd.cpc[l] = c[l];
      d.kf.cpc[l] = (float)c[l];
      d.kd.ecf[l] = ecf[l];
      d.kf.ecf[l] = (float)ecf[l];
    }
    for (int l = 0; l < 6; ++l) {
      d.kd.dcc[l] = dcc[l];
      d.kf.dcc[l] = (float)dcc[l];
    }
    double e1 = 0.0, cv1 = -d.R;
    for (int l = 0; l < 7; ++l) {
      if (l != 1) e1 += ecf[l];
      cv1 += c[l];
    }
    d.kd.e1 = e1;
    d.kf.e1 = (float)e1;
    d.kd.icv1 = 1.0 / cv1;
    d.kf.icv1 = (float)d.kd.icv1;
  }
}

// S2_OK if the gas is usable: gamma > 1, positive reference values and,
// for a thermally perfect gas, finite coefficients with c_v > 0 at T = 1,
// T = t_ref and T = t_extra (the wall temperature; ignored if <= 0).
int s2::check_gas(const s2_gas *gas, double t_extra) {
  if (!(gas->gamma > 1.0) || !(gas->mach_ref > 0) || !(gas->prandtl > 0) || !(gas->t_ref > 0)) return S2_EINVAL;
  if (!gas->cp_coeffs) return S2_OK;
  for (int l = 0; l < 7; ++l)
    if (!std::isfinite(gas->cp_coeffs[l])) return S2_EINVAL;
  const double Ts[3] = {1.0, gas->t_ref, t_extra};
  for (double T : Ts) {
    if (!(T > 0)) continue;
    double cpr = 0.0;  // c_p / R
    for (int l = -2; l <= 4; ++l) cpr += gas->cp_coeffs[l + 2] * std::pow(T, l);
    if (!(cpr > 1.0)) return S2_EINVAL;
  }
  return S2_OK;
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
    case S2_EBOUNDS: return "index out of its array's bounds (checked build)";
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
  auto valid_order = [](int o) { return o == 2 || o == 4 || o == 6 || o == 8; };
  if (!valid_order(scheme->central_order) || !valid_order(scheme->visc_order)) return S2_EINVAL;
  if (scheme->weno_order != 0 && scheme->weno_order != 1 && scheme->weno_order != 3 && scheme->weno_order != 5 &&
      scheme->weno_order != 7)
    return S2_EINVAL;
  if (scheme->precision != S2_FP64 && scheme->precision != S2_MIXED) return S2_EINVAL;
  if (scheme->keep < -1 || scheme->keep > 16 || (scheme->keep != 0 && gas->cp_coeffs)) return S2_EINVAL;
  if (!(scheme->cfl > 0) && !(scheme->dt_fixed > 0)) return S2_EINVAL;
  if (check_gas(gas, bcs->y == S2_BC_ISOTHERMAL_WALL ? bcs->t_wall : 0.0) != S2_OK) return S2_EINVAL;
  long long n = (long long)grid->nx * grid->ny * grid->nz;
  // point and interface-slot indices are split in 32-bit unsigned arithmetic
  if ((long long)(grid->nx + 1) * (grid->ny + 1) * (long long)(grid->nz + 1) > 0x7fffffffLL) return S2_EINVAL;
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
  {
    bool ok = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) == cudaSuccess;
    for (int a = 0; a < 3 && ok; ++a) ok = cudaEventCreateWithFlags(&s->ev_flux[a], cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      release(s);
      delete s;
      return S2_ECUDA;
    }
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
  d.fnx.init((unsigned)grid->nx);
  d.fny.init((unsigned)grid->ny);
  d.fnx1.init((unsigned)grid->nx + 1u);
  d.fny1.init((unsigned)grid->ny + 1u);
  if (cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess || d.nsm < 1) d.nsm = 1;
  // bounded waits for asynchronous copies: 2 s.  S2_TEST_STALL_COPIES=1 in
  // the environment makes every staging barrier expect 16 bytes more than
  // its copies deliver, with a 20 ms limit: the waits run out, the kernels
  // return and the step reports S2_ETIMEOUT (failure-detection test; no
  // fault, the copies themselves complete).
  d.wait_ns = 2000000000ull;
  d.tx_extra = 0;
  if (const char *ev = getenv("S2_TEST_STALL_COPIES")) {
    if (atoi(ev) > 0) {
      d.tx_extra = 16;
      d.wait_ns = 20000000ull;
    }
  }
  d.dx = grid->lx / grid->nx;
  d.dz = grid->lz / grid->nz;
  d.idx = 1.0 / d.dx;
  d.idz = 1.0 / d.dz;
  d.npc = scheme->central_order / 2;
  d.keep = scheme->keep;
  d.npv = scheme->visc_order / 2;
  for (int l = 0; l <= 4; ++l) {
    d.ax[l] = l ? A1_ORD[d.npv][l] / d.dx : 0.0;
    d.az[l] = l ? A1_ORD[d.npv][l] / d.dz : 0.0;
    d.bx[l] = B2_ORD[d.npv][l] / (d.dx * d.dx);
    d.bz[l] = B2_ORD[d.npv][l] / (d.dz * d.dz);
  }
  set_gas(d, gas);
  d.t_wall = bcs->t_wall;
  d.thr = scheme->sensor_threshold;
  d.cfl = scheme->cfl;
  d.dt_every = s->sch.dt_every;
  d.wall_y = bcs->y == S2_BC_ISOTHERMAL_WALL;
  d.weno = scheme->weno_order;
  d.force = bcs->force_mass_flow ? 1 : 0;
  d.mixed = scheme->precision == S2_MIXED ? 1 : 0;
  // default flux tiles: the wide ones everywhere in double precision; in
  // single precision the narrow y and z tiles (measured ~5 % faster on a
  // 256 x 128 x 128 channel)
  d.tile[0] = 0;
  d.tile[1] = d.tile[2] = d.mixed;
  for (int a = 0; a < 3; ++a) d.flux_cps[a] = 0;
  d.zs = ZS_DEFAULT;
  d.weno_cps = 16;
  // scheme constants in both arithmetic types
  {
    Consts<double> &k = d.kd;
    for (int l = 0; l < 5; ++l) {
      k.ax[l] = d.ax[l];
      k.az[l] = d.az[l];
      k.bx[l] = d.bx[l];
      k.bz[l] = d.bz[l];
      k.acen[l] = A1_ORD[d.npc][l];
    }
    k.idx = d.idx;
    k.idz = d.idz;
    k.idx2 = 2.0 * d.idx;
    k.idz2 = 2.0 * d.idz;
    k.R_gas = d.R;
    k.cp = d.cp;
    k.gamma = d.gamma;
    k.gR = d.gR;
    k.icv = d.icv;
    k.visc_exp = d.visc_exp;
    k.inv_t_ref = d.inv_t_ref;
    k.t_wall = d.t_wall;
    k.cp_over_pr = d.cp_over_pr;
    k.re = d.re;
    k.inv_re = d.inv_re;
    k.thr = d.thr;
    k.thr2 = d.thr * d.thr;
    k.b0xz = d.bx[0] + d.bz[0];
    Consts<float> &f = d.kf;
    for (int l = 0; l < 5; ++l) {
      f.ax[l] = (float)k.ax[l];
      f.az[l] = (float)k.az[l];
      f.bx[l] = (float)k.bx[l];
      f.bz[l] = (float)k.bz[l];
      f.acen[l] = (float)k.acen[l];
    }
    f.idx = (float)k.idx;
    f.idz = (float)k.idz;
    f.idx2 = 2.0f * f.idx;
    f.idz2 = 2.0f * f.idz;
    f.R_gas = (float)k.R_gas;
    f.cp = (float)k.cp;
    f.gamma = (float)k.gamma;
    f.gR = (float)k.gR;
    f.icv = (float)k.icv;
    f.visc_exp = (float)k.visc_exp;
    f.inv_t_ref = (float)k.inv_t_ref;
    f.t_wall = (float)k.t_wall;
    f.cp_over_pr = (float)k.cp_over_pr;
    f.re = (float)k.re;
    f.inv_re = (float)k.inv_re;
    f.thr = (float)k.thr;
    f.thr2 = f.thr * f.thr;
    f.b0xz = (float)k.b0xz;
  }

  size_t np = (size_t)d.px * d.py * d.pz;
  d.np = (long long)np;
  size_t nn = (size_t)n;
  const size_t rs = d.mixed ? sizeof(float) : sizeof(double);  // bytes of the arithmetic type
  s->rsize = rs;
  bool ok = true;
  auto A = [&](size_t count) -> double * {
    double *p = (double *)dalloc(s, count * sizeof(double));
    if (!p) ok = false;
    return p;
  };
  auto AR = [&](size_t count) -> void * {
    void *p = dalloc(s, count * rs);
    if (!p) ok = false;
    return p;
  };
  d.w = A(NV * nn);
  d.fl = AR(NV * nn);
  d.fln = AR(NV * nn);
  d.rho = AR(np); d.u = AR(np); d.v = AR(np); d.ww = AR(np);
  d.T = AR(np); d.p = AR(np); d.H = AR(np);
  d.div = AR(np); d.sens = AR(np);
  d.mu = AR(nn);
  d.g = d.mixed ? nullptr : AR(9 * nn);  // the mixed viscous pass recomputes the gradients
  // s2_rhs stages its double output in fln when that is double, else here
  s->rhs_stage = d.mixed ? A(NV * nn) : (double *)d.fln;
  double *eta = A(grid->ny), *ay = A(4 * grid->ny), *by = A(5 * grid->ny), *ry = A(grid->ny), *dvy = A(grid->ny);
  float *etaf = (float *)dalloc(s, sizeof(float) * grid->ny), *ayf = (float *)dalloc(s, sizeof(float) * 4 * grid->ny);
  float *byf = (float *)dalloc(s, sizeof(float) * 5 * grid->ny), *ryf = (float *)dalloc(s, sizeof(float) * grid->ny);
  if (!etaf || !ayf || !byf || !ryf) ok = false;
  size_t nparts = (size_t)((n + NT - 1) / NT);
  if (nparts < (size_t)NRED * NSTAT) nparts = (size_t)NRED * NSTAT;
  {  // forcing partials of k_visc_z, for the smallest tunable plane count
    Dev dz = d;
    dz.zs = ZS_MIN;
    if (nparts < (size_t)z_pass_blocks(dz)) nparts = (size_t)z_pass_blocks(dz);
  }
  d.part = A(nparts);
  d.nparts = (long long)nparts;
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
    d.dF[a] = dalloc(s, NV * nl * rs);
    if (!d.flag[a] || !d.wlist[a] || !d.dF[a]) ok = false;
  }
  if (!ok) {
    release(s);
    delete s;
    return S2_ENOMEM;
  }
  // tile boxes of the convective kernels (fields 16-byte aligned, as the
  // tensor memory accelerator requires)
  if (flux_make_maps(d, s->fmaps) != cudaSuccess) {
    cudaGetLastError();
    release(s);
    delete s;
    return S2_EINVAL;
  }
  d.eta_y = eta;
  d.ay = ay;
  d.by = by;
  d.ry = ry;
  d.dvy = dvy;
  d.eta_yf = etaf;
  d.ayf = ayf;
  d.byf = byf;
  d.ryf = ryf;

  cudaError_t e = cudaSuccess;
  void *pads[] = {d.rho, d.u, d.v, d.ww, d.T, d.p, d.H, d.div, d.sens};
  for (void *p : pads)
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, np * rs, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.w, 0, NV * nn * sizeof(double), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.fl, 0, NV * nn * rs, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.fln, 0, NV * nn * rs, s->stream);
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
    MetricCoef mc;
    mc.lv = d.npv;
    mc.lm = d.npc > d.npv ? d.npc : d.npv;
    for (int l = 0; l < 5; ++l) {
      mc.am[l] = A1_ORD[mc.lm][l];
      mc.bm[l] = B2_ORD[mc.lm][l];
      mc.av[l] = A1_ORD[mc.lv][l];
      mc.bv[l] = B2_ORD[mc.lv][l];
    }
    k_metric<<<(grid->ny + 127) / 128, 128, 0, s->stream>>>(ynd, grid->ny, grid->ly, d.wall_y, mc, eta, ay, by, ry,
                                                             dvy, etaf, ayf, byf, ryf);
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
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d.fln, 0, NV * (size_t)s->d.n * s->rsize, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&s->d.scal->status, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_err(e);
}

int s2_set_primitives(s2_solver *s, const double *prim, int where) {
  if (!s || !prim || (where != S2_HOST && where != S2_DEVICE)) return S2_EINVAL;
  DeviceGuard guard(s->device);
  size_t bytes = NV * (size_t)s->d.n * sizeof(double);
  unsigned nb = (unsigned)((s->d.n + NT - 1) / NT);
  cudaError_t e = cudaMemsetAsync(&s->d.scal->status, 0, sizeof(int), s->stream);
  if (where == S2_HOST) {
    // stage the primitives in the state array and convert in place
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d.w, prim, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) k_from_prims<<<nb, NT, 0, s->stream>>>(s->d, s->d.w, s->d.w);
  } else if (e == cudaSuccess) {
    k_from_prims<<<nb, NT, 0, s->stream>>>(s->d, prim, s->d.w);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d.fln, 0, NV * (size_t)s->d.n * s->rsize, s->stream);
  if (e != cudaSuccess) return S2_ECUDA;
  return read_status(s);
}

int s2_get_primitives(s2_solver *s, double *prim, int where) {
  if (!s || !prim || (where != S2_HOST && where != S2_DEVICE)) return S2_EINVAL;
  DeviceGuard guard(s->device);
  size_t bytes = NV * (size_t)s->d.n * sizeof(double);
  unsigned nb = (unsigned)((s->d.n + NT - 1) / NT);
  // FP64: fln is zero between steps; it stages the result and is cleared
  // again afterwards (as in s2_rhs)
  double *dst = where == S2_DEVICE ? prim : s->rhs_stage;
  k_to_prims<<<nb, NT, 0, s->stream>>>(s->d, s->d.w, dst);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && where == S2_HOST) {
    e = cudaMemcpyAsync(prim, s->rhs_stage, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && !s->d.mixed) e = cudaMemsetAsync(s->d.fln, 0, bytes, s->stream);
  }
  if (e != cudaSuccess) return S2_ECUDA;
  return read_status(s);
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
    if (!s->graph_disabled && !s->graph_ready && build_graph(s) != 0) s->graph_disabled = true;
    cudaError_t e;
    if (!s->graph_disabled) {
      e = cudaGraphLaunch(s->graph, s->stream);
      s->launches += s->launches_per_step;
    } else {
      Trace tr;
      e = enqueue_step(s, &tr);
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

namespace {

// Staging buffers (one allocation), streams and events of s2_stream_states.
int stream_setup(s2_solver *s) {
  if (s->stage_in) return S2_OK;
  const size_t n5 = NV * (size_t)s->d.n;
  // each handle is created once (a failed call leaves the others for s2_destroy)
  for (cudaStream_t *q : {&s->cin, &s->cout})
    if (!*q && cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) != cudaSuccess) {
      *q = nullptr;
      return S2_ECUDA;
    }
  for (cudaEvent_t *ev : {&s->ev_in_ready, &s->ev_in_free, &s->ev_out_ready, &s->ev_out_free})
    if (!*ev && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) {
      *ev = nullptr;
      return S2_ECUDA;
    }
  double *p = (double *)dalloc(s, 2 * n5 * sizeof(double));
  if (!p) return S2_ENOMEM;
  s->stage_in = p;
  s->stage_out = p + n5;
  return S2_OK;
}

}  // namespace

int s2_stream_states(s2_solver *s, const double *w_in, long long in_stride, double *w_out, long long out_stride,
                     int count, int nsteps) {
  if (!s || !w_in || !w_out || count < 0 || nsteps < 0 || in_stride < 0 || out_stride < 0) return S2_EINVAL;
  if (count == 0) return S2_OK;
  DeviceGuard guard(s->device);
  int rc = stream_setup(s);
  if (rc != S2_OK) return rc;
  const size_t n5 = NV * (size_t)s->d.n, bytes = n5 * sizeof(double);
  cudaStream_t st = s->stream;
  // copy-in of state j+1 and copy-out of result j-1 overlap the steps of
  // state j; each staging buffer is handed between its copy stream and the
  // solver's stream by a pair of events
  cudaError_t e = cudaMemsetAsync(&s->d.scal->status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->stage_in, w_in, bytes, cudaMemcpyDefault, s->cin);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_in_ready, s->cin);
  for (int j = 0; j < count && e == cudaSuccess && rc == S2_OK; ++j) {
    e = cudaStreamWaitEvent(st, s->ev_in_ready, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d.w, s->stage_in, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d.fln, 0, n5 * s->rsize, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_in_free, st);
    if (e == cudaSuccess && j + 1 < count) {
      e = cudaStreamWaitEvent(s->cin, s->ev_in_free, 0);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->stage_in, w_in + (j + 1) * in_stride, bytes, cudaMemcpyDefault, s->cin);
      if (e == cudaSuccess) e = cudaEventRecord(s->ev_in_ready, s->cin);
    }
    if (e == cudaSuccess) rc = s2_step(s, nsteps);
    if (e == cudaSuccess && rc == S2_OK) {
      e = cudaStreamWaitEvent(st, s->ev_out_free, 0);
      if (e == cudaSuccess) e = cudaMemcpyAsync(s->stage_out, s->d.w, bytes, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = cudaEventRecord(s->ev_out_ready, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cout, s->ev_out_ready, 0);
      if (e == cudaSuccess) e = cudaMemcpyAsync(w_out + j * out_stride, s->stage_out, bytes, cudaMemcpyDefault, s->cout);
      if (e == cudaSuccess) e = cudaEventRecord(s->ev_out_free, s->cout);
    }
  }
  // no copy outlives the call, also after an error
  const cudaError_t e1 = cudaStreamSynchronize(s->cin), e2 = cudaStreamSynchronize(s->cout);
  if (e != cudaSuccess || e1 != cudaSuccess || e2 != cudaSuccess) {
    cudaStreamSynchronize(st);
    return S2_ECUDA;
  }
  if (rc != S2_OK) {
    cudaStreamSynchronize(st);
    return rc;
  }
  return read_status(s);
}

int s2_set_tuning(s2_solver *s, const s2_tuning *t) {
  if (!s || !t) return S2_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (t->tiles[a] != 0 && t->tiles[a] != 1) return S2_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (t->flux_ctas_per_sm[a] < 0 || t->flux_ctas_per_sm[a] > 16) return S2_EINVAL;
  if (t->z_planes != 0 && t->z_planes != 4 && t->z_planes != 8 && t->z_planes != 12 && t->z_planes != 16 &&
      t->z_planes != 24)
    return S2_EINVAL;
  if (t->weno_ctas_per_sm < 0 || t->weno_ctas_per_sm > 64) return S2_EINVAL;
  DeviceGuard guard(s->device);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return S2_ECUDA;
  for (int a = 0; a < 3; ++a) s->d.tile[a] = t->tiles[a];
  for (int a = 0; a < 3; ++a) s->d.flux_cps[a] = t->flux_ctas_per_sm[a];
  s->d.zs = t->z_planes ? t->z_planes : ZS_DEFAULT;
  s->d.weno_cps = t->weno_ctas_per_sm ? t->weno_ctas_per_sm : 16;
  if (s->graph_ready) {
    cudaGraphExecDestroy(s->graph);
    s->graph_ready = false;
  }
  return S2_OK;
}

int s2_get_tuning(const s2_solver *s, s2_tuning *t) {
  if (!s || !t) return S2_EINVAL;
  for (int a = 0; a < 3; ++a) t->tiles[a] = s->d.tile[a];
  for (int a = 0; a < 3; ++a) t->flux_ctas_per_sm[a] = s->d.flux_cps[a];
  t->z_planes = s->d.zs;
  t->weno_ctas_per_sm = s->d.weno_cps;
  return S2_OK;
}

int s2_set_tiles(s2_solver *s, const int *tiles) {
  if (!s || !tiles) return S2_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (tiles[a] != 0 && tiles[a] != 1) return S2_EINVAL;
  DeviceGuard guard(s->device);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return S2_ECUDA;
  for (int a = 0; a < 3; ++a) s->d.tile[a] = tiles[a];
  if (s->graph_ready) {
    cudaGraphExecDestroy(s->graph);
    s->graph_ready = false;
  }
  return S2_OK;
}

int s2_set_clock(s2_solver *s, double t, long long step, double dt) {
  if (!s || step < 0) return S2_EINVAL;
  DeviceGuard guard(s->device);
  cudaError_t e = cudaMemcpyAsync(&s->d.scal->t, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->d.scal->nstep, &step, sizeof(long long), cudaMemcpyHostToDevice, s->stream);
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
  // FP64: fln is zero between steps and rewritten before it is read, so it
  // serves as the staging buffer and is cleared again afterwards.
  double *dst = where == S2_DEVICE ? rhs : s->rhs_stage;
  if (s->d.mixed) k_rhs_out<float><<<nb, NT, 0, s->stream>>>(s->d, dst);
  else k_rhs_out<double><<<nb, NT, 0, s->stream>>>(s->d, dst);
  if ((e = cudaGetLastError()) != cudaSuccess) return S2_ECUDA;
  if (where == S2_HOST) {
    e = cudaMemcpyAsync(rhs, s->rhs_stage, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && !s->d.mixed) e = cudaMemsetAsync(s->d.fln, 0, bytes, s->stream);
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
  if (s->d.mixed) k_stats_partial<float><<<NRED, NT, 0, s->stream>>>(s->d);
  else k_stats_partial<double><<<NRED, NT, 0, s->stream>>>(s->d);
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
  out->status = (h.status & ERR_BOUNDS)      ? S2_EBOUNDS
                : (h.status & ERR_NONFINITE) ? S2_ENONFINITE
                : (h.status & ERR_TIMEOUT)   ? S2_ETIMEOUT
                                             : S2_OK;
  return out->status;
}

int s2_profile(s2_solver *s, int n, double *ms, long long *launches) {
  if (!s || n < 0) return S2_EINVAL;
  DeviceGuard guard(s->device);
  Trace tr;
  tr.timed = true;
  int rc = S2_OK;
  for (int it = 0; it < n && rc == S2_OK; ++it) {
    if (enqueue_step(s, &tr) != cudaSuccess) rc = S2_ECUDA;
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

}  // extern "C"

// ======================================================================
// Batched stepping
// ======================================================================
// Work-list mode (default): members whose kernels are the same
// instantiations (precision, orders, WENO order, tile shapes, gas model,
// and the viscous / WENO / forcing / CFL switches) form a group, and every
// kernel of a stage is ONE launch over the whole group: a table in device
// memory lists, per box, the box's parameters and the CTAs of the launch
// that work on it (BoxGrid); each CTA finds its box, copies the box's
// parameters to shared memory and runs the same kernel body as a solo
// launch on its box-local tile.  Persistent single-precision flux grids
// are shared out over the boxes in proportion to their tiles.  Groups are
// concurrent branches of the batch's step graph.  Branch mode: the
// members' own step sequences as concurrent branches.
enum BatchClass {
  BC_PRIMS,  // one thread per interior point (prims, update, WENO apply)
  BC_GHOST,  // one thread per face-ghost point
  BC_GRAD,
  BC_VISC,
  BC_FLUX0,
  BC_FLUX1,
  BC_FLUX2,
  BC_WENO0,
  BC_WENO1,
  BC_WENO2,
  BC_FORCE,  // grid-stride forcing partials (NRED CTAs per box)
  BC_ONE,    // one CTA per box
  BC_COUNT
};

struct BatchGroup {
  std::vector<s2_solver *> members;
  cudaStream_t stream;  // the first member's: this group's branch of the step graph
  void *mem;            // the device tables, one block
  Dev *dev;             // [n] parameters of the boxes
  BoxGrid *grid[BC_COUNT];
  unsigned total[BC_COUNT];
  int *nparts_dt, *nparts_force;  // [n]
  FluxMaps *maps[3];              // [n] tensor maps of the group's tile variant
  void *tgs[3];                   // [n] flux tile-grid records
  long long launches;             // kernels per step
};

struct s2_batch {
  std::vector<s2_solver *> members;
  cudaStream_t stream;
  bool own_stream;
  int device;
  int mode;
  cudaGraphExec_t graph;
  bool ready;
  long long launches_per_step;
  std::vector<long long> member_launches;  // kernels per step that work on each member
  std::vector<cudaEvent_t> events;         // fork + one join per branch
  std::vector<BatchGroup> groups;
  std::vector<s2_solver *> solo;           // work-list mode: members large enough to run their own launches
};

namespace {

bool same_kernels(const Dev &a, const Dev &b) {
  return a.mixed == b.mixed && a.npc == b.npc && a.npv == b.npv && a.weno == b.weno && a.kd.tp == b.kd.tp &&
         a.tile[0] == b.tile[0] && a.tile[1] == b.tile[1] && a.tile[2] == b.tile[2] && a.viscous == b.viscous &&
         a.force == b.force && (a.cfl > 0.0) == (b.cfl > 0.0) && a.zs == b.zs;
}

void *batch_alloc(s2_solver *s, size_t bytes) {
  void *p = nullptr;
  if (s->dev.alloc) return s->dev.alloc(bytes, s->dev.ctx);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void batch_free(s2_solver *s, void *p) {
  if (!p) return;
  if (s->dev.free) s->dev.free(p, s->dev.ctx);
  else cudaFree(p);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The group's work lists and tables, built on the host and copied once.
int group_setup(BatchGroup &g) {
  const int n = (int)g.members.size();
  const Dev &d0 = g.members[0]->d;
  std::vector<Dev> devs(n);
  for (int b = 0; b < n; ++b) devs[b] = g.members[b]->d;
  std::vector<std::vector<BoxGrid>> grids(BC_COUNT, std::vector<BoxGrid>(n + 1));
  std::vector<int> ndt(n), nforce(n);
  FluxBoxPlan fp[3];
  std::vector<FluxBoxPlan> plans(3 * (size_t)n);
  long long tiles_sum[3] = {0, 0, 0}, slots_sum[3] = {0, 0, 0};
  for (int b = 0; b < n; ++b)
    for (int dir = 0; dir < 3; ++dir) {
      if (flux_batch_plan(devs[b], dir, &plans[3 * b + dir]) != cudaSuccess) return S2_ECUDA;
      tiles_sum[dir] += plans[3 * b + dir].tiles;
      slots_sum[dir] += devs[b].nslot[dir];
    }
  for (int dir = 0; dir < 3; ++dir) fp[dir] = plans[dir];
  auto set = [&](int c, int b, unsigned gx, unsigned gy, unsigned gz) {
    BoxGrid &e = grids[c][b];
    e.gx = gx ? gx : 1;
    e.gy = gy ? gy : 1;
    e.gz = gz ? gz : 1;
  };
  for (int b = 0; b < n; ++b) {
    const Dev &d = devs[b];
    const unsigned nb = (unsigned)((d.n + NT - 1) / NT);
    const long long nghost = 2LL * GH * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
    const unsigned ngb = (unsigned)((nghost + NT - 1) / NT);
    set(BC_PRIMS, b, nb, 1, 1);
    set(BC_GHOST, b, ngb, 1, 1);
    if (d.mixed) {
      unsigned zg[3];
      z_pass_grid(d, zg);
      set(BC_GRAD, b, zg[0], zg[1], zg[2]);
      set(BC_VISC, b, zg[0], zg[1], zg[2]);
    } else {
      set(BC_GRAD, b, nb, 1, 1);
      set(BC_VISC, b, nb, 1, 1);
    }
    for (int dir = 0; dir < 3; ++dir) {
      const FluxBoxPlan &pl = plans[3 * b + dir];
      unsigned c = (unsigned)pl.tiles;
      if (pl.persistent) {
        // the resident CTAs of a full device, shared out by tiles
        const double share = (double)pl.per_sm * d.nsm * pl.tiles / (double)tiles_sum[dir];
        unsigned k = (unsigned)share;
        if (k < 1) k = 1;
        if (k < c) c = k;
      }
      set(BC_FLUX0 + dir, b, c, 1, 1);
      // WENO: the solo launch's CTAs shared out by interface slots
      const unsigned solo = weno_batch_blocks(d, dir);
      unsigned w = (unsigned)(16.0 * d.nsm * (double)d.nslot[dir] / (double)slots_sum[dir]) + 1;
      set(BC_WENO0 + dir, b, w < solo ? w : solo, 1, 1);
    }
    set(BC_FORCE, b, NRED, 1, 1);
    set(BC_ONE, b, 1, 1, 1);
    ndt[b] = (int)nb;
    const int fused = visc_force_partials(d);
    nforce[b] = fused ? fused : NRED;
  }
  for (int c = 0; c < BC_COUNT; ++c) {
    unsigned long long acc = 0;
    for (int b = 0; b < n; ++b) {
      grids[c][b].start = (unsigned)acc;
      acc += (unsigned long long)grids[c][b].gx * grids[c][b].gy * grids[c][b].gz;
    }
    if (acc >= (1ull << 31)) return S2_EINVAL;
    grids[c][n] = BoxGrid{(unsigned)acc, 1, 1, 1};
    g.total[c] = (unsigned)acc;
  }
  // one block: tensor maps (64-byte aligned), parameters, tile grids, work lists
  size_t off = 0;
  size_t o_maps[3], o_dev, o_tg[3], o_grid[BC_COUNT], o_ndt, o_nf;
  for (int dir = 0; dir < 3; ++dir) {
    o_maps[dir] = off;
    off = align_up(off + sizeof(FluxMaps) * n, 128);
  }
  o_dev = off;
  off = align_up(off + sizeof(Dev) * n, 128);
  for (int dir = 0; dir < 3; ++dir) {
    o_tg[dir] = off;
    off = align_up(off + (size_t)fp[dir].tg_size * n, 128);
  }
  for (int c = 0; c < BC_COUNT; ++c) {
    o_grid[c] = off;
    off = align_up(off + sizeof(BoxGrid) * (n + 1), 128);
  }
  o_ndt = off;
  off = align_up(off + sizeof(int) * n, 128);
  o_nf = off;
  off = align_up(off + sizeof(int) * n, 128);
  std::vector<unsigned char> host(off, 0);
  for (int b = 0; b < n; ++b)
    for (int dir = 0; dir < 3; ++dir) {
      const s2_solver *m = g.members[b];
      memcpy(host.data() + o_maps[dir] + sizeof(FluxMaps) * b, &m->fmaps[dir][d0.tile[dir] && !d0.keep ? 1 : 0],
             sizeof(FluxMaps));
      memcpy(host.data() + o_tg[dir] + (size_t)fp[dir].tg_size * b, plans[3 * b + dir].tg, fp[dir].tg_size);
    }
  memcpy(host.data() + o_dev, devs.data(), sizeof(Dev) * n);
  for (int c = 0; c < BC_COUNT; ++c) memcpy(host.data() + o_grid[c], grids[c].data(), sizeof(BoxGrid) * (n + 1));
  memcpy(host.data() + o_ndt, ndt.data(), sizeof(int) * n);
  memcpy(host.data() + o_nf, nforce.data(), sizeof(int) * n);
  g.mem = batch_alloc(g.members[0], off);
  if (!g.mem) return S2_ENOMEM;
  // on the group's (idle) stream: a legacy-stream copy would wait for
  // unrelated work on blocking streams
  if (cudaMemcpyAsync(g.mem, host.data(), off, cudaMemcpyHostToDevice, g.stream) != cudaSuccess ||
      cudaStreamSynchronize(g.stream) != cudaSuccess)
    return S2_ECUDA;
  unsigned char *base = (unsigned char *)g.mem;
  for (int dir = 0; dir < 3; ++dir) {
    g.maps[dir] = (FluxMaps *)(base + o_maps[dir]);
    g.tgs[dir] = base + o_tg[dir];
  }
  g.dev = (Dev *)(base + o_dev);
  for (int c = 0; c < BC_COUNT; ++c) g.grid[c] = (BoxGrid *)(base + o_grid[c]);
  g.nparts_dt = (int *)(base + o_ndt);
  g.nparts_force = (int *)(base + o_nf);
  return S2_OK;
}

// One RK3 step of every box of a group: the stage sequence of
// enqueue_step, each kernel launched once for all boxes.
cudaError_t enqueue_group_step(BatchGroup &g) {
  const Dev &d0 = g.members[0]->d;
  const int n = (int)g.members.size();
  cudaStream_t st = g.stream;
  auto ba = [&](int c) { return BatchArgs{g.dev, g.grid[c], n}; };
  long long cnt = 0;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    ++cnt;
    if (e == cudaSuccess) e = r;
  };
  for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
    const int stage0 = stage == 0;
    if (d0.mixed) kb_prims_mixed<<<g.total[BC_PRIMS], NT, 0, st>>>(ba(BC_PRIMS), stage0);
    else if (d0.kd.tp) kb_prims<true><<<g.total[BC_PRIMS], NT, 0, st>>>(ba(BC_PRIMS), stage0);
    else kb_prims<false><<<g.total[BC_PRIMS], NT, 0, st>>>(ba(BC_PRIMS), stage0);
    chk(cudaGetLastError());
    if (stage0 && d0.cfl > 0.0) {
      kb_dt_final<<<g.total[BC_ONE], NT, 0, st>>>(ba(BC_ONE), g.nparts_dt);
      chk(cudaGetLastError());
    }
    if (d0.mixed) kb_ghost_prim<float><<<g.total[BC_GHOST], NT, 0, st>>>(ba(BC_GHOST));
    else kb_ghost_prim<double><<<g.total[BC_GHOST], NT, 0, st>>>(ba(BC_GHOST));
    chk(cudaGetLastError());
    if (d0.viscous || d0.weno) {
      chk(launch_grad_batch(d0, ba(BC_GRAD), g.total[BC_GRAD], st));
      if (d0.mixed) kb_ghost_aux<float><<<g.total[BC_GHOST], NT, 0, st>>>(ba(BC_GHOST));
      else kb_ghost_aux<double><<<g.total[BC_GHOST], NT, 0, st>>>(ba(BC_GHOST));
      chk(cudaGetLastError());
    }
    if (d0.weno) {
      kb_reset_counts<<<g.total[BC_ONE], NT, 0, st>>>(ba(BC_ONE));
      chk(cudaGetLastError());
    }
    for (int dir = 0; dir < 3; ++dir)
      chk(launch_flux_batch(d0, ba(BC_FLUX0 + dir), g.total[BC_FLUX0 + dir], g.maps[dir], g.tgs[dir], dir, dir > 0,
                            st));
    if (d0.weno)
      for (int dir = 0; dir < 3; ++dir) chk(launch_weno_batch(d0, ba(BC_WENO0 + dir), g.total[BC_WENO0 + dir], dir, st));
    if (d0.viscous) chk(launch_visc_batch(d0, ba(BC_VISC), g.total[BC_VISC], st));
    else if (d0.weno) chk(launch_apply_batch(d0, ba(BC_PRIMS), g.total[BC_PRIMS], st));
    if (d0.force) {
      if (!visc_force_partials(d0)) {
        if (d0.mixed) kb_force_partial<float><<<g.total[BC_FORCE], NT, 0, st>>>(ba(BC_FORCE));
        else kb_force_partial<double><<<g.total[BC_FORCE], NT, 0, st>>>(ba(BC_FORCE));
        chk(cudaGetLastError());
      }
      kb_force_final<<<g.total[BC_ONE], NT, 0, st>>>(ba(BC_ONE), g.nparts_force);
      chk(cudaGetLastError());
    }
    if (d0.mixed) kb_update_mixed<<<g.total[BC_PRIMS], NT, 0, st>>>(ba(BC_PRIMS), RK_G[stage], RK_R[stage + 1], stage);
    else kb_update<<<g.total[BC_PRIMS], NT, 0, st>>>(ba(BC_PRIMS), RK_G[stage], RK_R[stage + 1], stage);
    chk(cudaGetLastError());
  }
  g.launches = cnt;
  return e;
}

int batch_build(s2_batch *b) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return S2_ECUDA;
  }
  cudaError_t e = cudaEventRecord(b->events[0], b->stream);
  long long total_launches = 0;
  b->member_launches.assign(b->members.size(), 0);
  if (b->mode == S2_BATCH_BRANCHES) {
    for (size_t m = 0; m < b->members.size() && e == cudaSuccess; ++m) {
      s2_solver *s = b->members[m];
      e = cudaStreamWaitEvent(s->stream, b->events[0], 0);
      Trace tr;
      if (e == cudaSuccess) e = enqueue_step(s, &tr);
      total_launches += total(tr);
      b->member_launches[m] = total(tr);
      if (e == cudaSuccess) e = cudaEventRecord(b->events[1 + m], s->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->events[1 + m], 0);
    }
  } else {
    size_t ev = 1;
    for (size_t k = 0; k < b->groups.size() && e == cudaSuccess; ++k, ++ev) {
      BatchGroup &grp = b->groups[k];
      e = cudaStreamWaitEvent(grp.stream, b->events[0], 0);
      if (e == cudaSuccess) e = enqueue_group_step(grp);
      total_launches += grp.launches;
      for (size_t m = 0; m < b->members.size(); ++m)
        for (s2_solver *s : grp.members)
          if (s == b->members[m]) b->member_launches[m] = grp.launches;
      if (e == cudaSuccess) e = cudaEventRecord(b->events[ev], grp.stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->events[ev], 0);
    }
    for (size_t k = 0; k < b->solo.size() && e == cudaSuccess; ++k, ++ev) {
      s2_solver *s = b->solo[k];
      e = cudaStreamWaitEvent(s->stream, b->events[0], 0);
      Trace tr;
      if (e == cudaSuccess) e = enqueue_step(s, &tr);
      total_launches += total(tr);
      for (size_t m = 0; m < b->members.size(); ++m)
        if (b->members[m] == s) b->member_launches[m] = total(tr);
      if (e == cudaSuccess) e = cudaEventRecord(b->events[ev], s->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->events[ev], 0);
    }
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return S2_ECUDA;
  }
  cudaGraphExec_t ex;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return S2_ECUDA;
  }
  b->graph = ex;
  b->ready = true;
  b->launches_per_step = total_launches;
  return S2_OK;
}

void batch_release(s2_batch *b) {
  if (b->ready) cudaGraphExecDestroy(b->graph);
  for (cudaEvent_t ev : b->events)
    if (ev) cudaEventDestroy(ev);
  for (BatchGroup &g : b->groups) batch_free(g.members[0], g.mem);
  b->groups.clear();
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

}  // namespace

extern "C" {

int s2_batch_create_ex(s2_solver *const *members, int count, void *stream, int mode, s2_batch **out) {
  if (!out || !members || count < 1 ||
      (mode != S2_BATCH_WORKLIST && mode != S2_BATCH_BRANCHES && mode != S2_BATCH_WORKLIST_ALL))
    return S2_EINVAL;
  *out = nullptr;
  int device = members[0] ? members[0]->device : -1;
  for (int m = 0; m < count; ++m) {
    if (!members[m] || members[m]->device != device) return S2_EINVAL;
    for (int k = 0; k < m; ++k)
      if (members[k] == members[m]) return S2_EINVAL;
  }
  s2_batch *b = new (std::nothrow) s2_batch();
  if (!b) return S2_ENOMEM;
  DeviceGuard guard(device);
  b->members.assign(members, members + count);
  b->device = device;
  b->mode = mode;
  if (stream) {
    b->stream = (cudaStream_t)stream;
    b->own_stream = false;
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return S2_ECUDA;
  } else {
    b->own_stream = true;
  }
  int rc = S2_OK;
  if (mode != S2_BATCH_BRANCHES) {
    for (s2_solver *s : b->members) {
      if (mode == S2_BATCH_WORKLIST && s->d.n >= S2_BATCH_SOLO_POINTS) {  // fills enough of the GPU on its own
        b->solo.push_back(s);
        continue;
      }
      BatchGroup *g = nullptr;
      for (BatchGroup &x : b->groups)
        if (same_kernels(x.members[0]->d, s->d)) g = &x;
      if (!g) {
        b->groups.emplace_back();
        g = &b->groups.back();
        g->stream = s->stream;
        g->mem = nullptr;
      }
      g->members.push_back(s);
    }
    if (mode == S2_BATCH_WORKLIST) {
      // a group of a few boxes saves few launches: its members keep their own
      std::vector<BatchGroup> kept;
      for (BatchGroup &g : b->groups) {
        if ((int)g.members.size() >= S2_BATCH_MIN_GROUP) kept.push_back(g);
        else b->solo.insert(b->solo.end(), g.members.begin(), g.members.end());
      }
      b->groups.swap(kept);
    }
    for (BatchGroup &g : b->groups)
      if (rc == S2_OK) rc = group_setup(g);
  }
  const size_t branches = mode != S2_BATCH_BRANCHES ? b->groups.size() + b->solo.size() : (size_t)count;
  b->events.assign(branches + 1, nullptr);
  for (auto &ev : b->events)
    if (rc == S2_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = S2_ECUDA;
  // the members' own pending work is ordered before the batch's first step
  for (s2_solver *s : b->members)
    if (rc == S2_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = S2_ECUDA;
  if (rc == S2_OK) rc = batch_build(b);
  if (rc != S2_OK) {
    batch_release(b);
    delete b;
    return rc;
  }
  *out = b;
  return S2_OK;
}

int s2_batch_create(s2_solver *const *members, int count, void *stream, s2_batch **out) {
  return s2_batch_create_ex(members, count, stream, S2_BATCH_WORKLIST, out);
}

long long s2_batch_launches(const s2_batch *b) { return b ? b->launches_per_step : -1; }

int s2_batch_step(s2_batch *b, int n) {
  if (!b || n < 0) return S2_EINVAL;
  DeviceGuard guard(b->device);
  for (int it = 0; it < n; ++it) {
    if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return S2_ECUDA;
    for (size_t m = 0; m < b->members.size(); ++m) {
      b->members[m]->step++;
      b->members[m]->launches += b->member_launches[m];
    }
  }
  return S2_OK;
}

int s2_batch_sync(s2_batch *b) {
  if (!b) return S2_EINVAL;
  DeviceGuard guard(b->device);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return S2_ECUDA;
  int rc = S2_OK;
  for (s2_solver *s : b->members) {
    int r = read_status(s);
    if (r != S2_OK && rc == S2_OK) rc = r;
  }
  return rc;
}

void s2_batch_destroy(s2_batch *b) {
  if (!b) return;
  {
    DeviceGuard guard(b->device);
    cudaStreamSynchronize(b->stream);
    batch_release(b);
  }
  delete b;
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
