// Velocity gradients + shock sensor, and the viscous/heat-flux terms.
//
// Paper Sec. 2: the switch between central and WENO fluxes is a modified
// Ducros sensor; the viscous terms are expanded in Laplacian form and
// discretised with 6th-order central formulae (visflx_nosensor of Table 2).
//
// k_grad, one thread per interior point: the nine velocity gradients
// d u_a / d x_b (stored, the viscous kernel reuses them), theta = div u
// (stored with ghosts: the viscous terms differentiate it again) and the
// sensor  max(-theta / sqrt(theta^2 + |curl u|^2 + (U0/L0)^2), 0).
//
// k_visc, one thread per interior point, adds to the RHS
//   momentum_a: mu (lap u_a + d_a theta / 3) + d_b mu (d_b u_a + d_a u_b)
//               - (2/3) theta d_a mu
//   energy:     u_a momentum_a + tau_ab d_b u_a + k lap T + grad k . grad T
// with grad mu = (omega mu / T) grad T (power law), k = mu c_p / Pr,
// d2/dy2 = eta_y^2 d2/deta2 + eta_yy d/deta.  The same pass adds the WENO
// corrections of the hybrid convective flux (k_apply does it alone for
// inviscid runs): per direction -scale (dF_{i+1/2} - dF_{i-1/2}) over the
// flagged interfaces, in a fixed order.
#include "s2_internal.cuh"

namespace s2 {
namespace {

constexpr int NT = 256;

__device__ __forceinline__ void point_of(const Dev &d, long long q, int &i, int &j, int &k) {
  long long t = q / d.nx;
  i = (int)(q - t * d.nx);
  k = (int)(t / d.ny);
  j = (int)(t - (long long)k * d.ny);
}

// Pre-scaled stencil coefficients of one direction at one point.
struct C4 {
  double c0, c1, c2, c3;
};

// first derivative: c1 (f+1 - f-1) + c2 (f+2 - f-2) + c3 (f+3 - f-3)
__device__ __forceinline__ double d1(const double *__restrict__ f, long long p, long long s, const C4 &c) {
  return c.c1 * (__ldg(f + p + s) - __ldg(f + p - s)) + c.c2 * (__ldg(f + p + 2 * s) - __ldg(f + p - 2 * s)) +
         c.c3 * (__ldg(f + p + 3 * s) - __ldg(f + p - 3 * s));
}

// second derivative: c0 f + c1 (f+1 + f-1) + c2 (f+2 + f-2) + c3 (f+3 + f-3)
__device__ __forceinline__ double d2(const double *__restrict__ f, long long p, long long s, const C4 &c) {
  return c.c0 * __ldg(f + p) + c.c1 * (__ldg(f + p + s) + __ldg(f + p - s)) +
         c.c2 * (__ldg(f + p + 2 * s) + __ldg(f + p - 2 * s)) + c.c3 * (__ldg(f + p + 3 * s) + __ldg(f + p - 3 * s));
}

// Hybrid-scheme correction of point (i, j, k): R -= scale_d (dF_hi - dF_lo)
// summed over the directions whose interfaces around the point are flagged.
__device__ __forceinline__ void weno_correction(const Dev &d, int i, int j, int k, double *R) {
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    int pos = dir == 0 ? i : (dir == 1 ? j : k);
    long long lo = islot(d, dir, pos - 1, i, j, k), hi = islot(d, dir, pos, i, j, k);
    bool fl = d.flag[dir][lo], fh = d.flag[dir][hi];
    if (fl || fh) {
      double scale = dir == 0 ? d.idx : (dir == 1 ? __ldg(d.eta_y + j) : d.idz);
      const long long ns = d.nslot[dir];
      const double *dF = d.dF[dir];
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        double c = (fh ? dF[f * ns + hi] : 0.0) - (fl ? dF[f * ns + lo] : 0.0);
        R[f] = fma(-scale, c, R[f]);
      }
    }
  }
}

__global__ void __launch_bounds__(NT) k_apply(Dev d) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  int i, j, k;
  point_of(d, q, i, j, k);
  double R[NV];
#pragma unroll
  for (int f = 0; f < NV; ++f) R[f] = d.fl[f * d.n + q];
  weno_correction(d, i, j, k, R);
#pragma unroll
  for (int f = 0; f < NV; ++f) d.fl[f * d.n + q] = R[f];
}

__global__ void __launch_bounds__(NT) k_grad(Dev d) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  int i, j, k;
  point_of(d, q, i, j, k);
  long long p = pidx(d, i, j, k);
  const C4 cx = {0.0, d.ax[1], d.ax[2], d.ax[3]}, cz = {0.0, d.az[1], d.az[2], d.az[3]};
  const C4 cy = {0.0, __ldg(d.ay + 3 * j), __ldg(d.ay + 3 * j + 1), __ldg(d.ay + 3 * j + 2)};
  const double *vel[3] = {d.u, d.v, d.ww};
  double g[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g[a][0] = d1(vel[a], p, 1, cx);
    g[a][1] = d1(vel[a], p, d.sy, cy);
    g[a][2] = d1(vel[a], p, d.sz, cz);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) d.g[(3 * a + b) * d.n + q] = g[a][b];
  double th = g[0][0] + g[1][1] + g[2][2];
  d.div[p] = th;
  if (d.weno) {
    double o1 = g[2][1] - g[1][2], o2 = g[0][2] - g[2][0], o3 = g[1][0] - g[0][1];
    double om2 = o1 * o1 + o2 * o2 + o3 * o3;
    double sv = -th / sqrt(th * th + om2 + 1.0);
    d.sens[p] = sv > 0.0 ? sv : 0.0;
  }
}

__global__ void __launch_bounds__(NT) k_visc(Dev d) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  int i, j, k;
  point_of(d, q, i, j, k);
  long long p = pidx(d, i, j, k);
  const C4 cx = {0.0, d.ax[1], d.ax[2], d.ax[3]}, cz = {0.0, d.az[1], d.az[2], d.az[3]};
  const C4 cy = {0.0, __ldg(d.ay + 3 * j), __ldg(d.ay + 3 * j + 1), __ldg(d.ay + 3 * j + 2)};
  const C4 bx = {d.bx[0], d.bx[1], d.bx[2], d.bx[3]}, bz = {d.bz[0], d.bz[1], d.bz[2], d.bz[3]};
  const C4 by = {__ldg(d.by + 4 * j), __ldg(d.by + 4 * j + 1), __ldg(d.by + 4 * j + 2), __ldg(d.by + 4 * j + 3)};
  const double ry = __ldg(d.ry + j);  // eta_yy / eta_y
  double g[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) g[a][b] = __ldg(d.g + (3 * a + b) * d.n + q);
  const double *vel[3] = {d.u, d.v, d.ww};
  double lap[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    lap[a] = d2(vel[a], p, 1, bx) + (d2(vel[a], p, d.sy, by) + ry * g[a][1]) + d2(vel[a], p, d.sz, bz);
  double gT[3], gth[3];
  gT[0] = d1(d.T, p, 1, cx);
  gT[1] = d1(d.T, p, d.sy, cy);
  gT[2] = d1(d.T, p, d.sz, cz);
  double lapT = d2(d.T, p, 1, bx) + (d2(d.T, p, d.sy, by) + ry * gT[1]) + d2(d.T, p, d.sz, bz);
  gth[0] = d1(d.div, p, 1, cx);
  gth[1] = d1(d.div, p, d.sy, cy);
  gth[2] = d1(d.div, p, d.sz, cz);
  const double T = __ldg(d.T + p);
  const double mu = __ldg(d.mu + q);
  const double mut = d.visc_exp * mu / T;
  const double kc = mu * d.cp_over_pr;
  double gmu[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) gmu[b] = mut * gT[b];
  const double th = __ldg(d.div + p);
  const double uv[3] = {__ldg(d.u + p), __ldg(d.v + p), __ldg(d.ww + p)};
  double mom[3], en = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double m = mu * (lap[a] + gth[a] * (1.0 / 3.0));
#pragma unroll
    for (int b = 0; b < 3; ++b) m += gmu[b] * (g[a][b] + g[b][a]);
    m -= (2.0 / 3.0) * th * gmu[a];
    mom[a] = m;
    en += uv[a] * m;
  }
  // tau : grad u
  double tg = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) tg += (g[a][b] + g[b][a]) * g[a][b];
  tg -= (2.0 / 3.0) * th * th;
  en += mu * tg;
  en += kc * lapT;
  en += d.cp_over_pr * (gmu[0] * gT[0] + gmu[1] * gT[1] + gmu[2] * gT[2]);
  double R[NV];
  R[0] = d.fl[q];
#pragma unroll
  for (int a = 0; a < 3; ++a) R[1 + a] = d.fl[(1 + a) * d.n + q] + mom[a];
  R[4] = d.fl[4 * d.n + q] + en;
  if (d.weno) weno_correction(d, i, j, k, R);
  if (d.weno) d.fl[q] = R[0];
#pragma unroll
  for (int f = 1; f < NV; ++f) d.fl[f * d.n + q] = R[f];
}

}  // namespace

cudaError_t launch_grad(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  k_grad<<<nb, NT, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_apply(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  k_apply<<<nb, NT, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_visc(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  k_visc<<<nb, NT, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace s2
