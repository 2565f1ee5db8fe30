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
//
// Every kernel is instantiated for R = double (FP64 path) and R = float
// (arithmetic of the mixed path).
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
template <class R>
struct C4 {
  R c0, c1, c2, c3;
};

// first derivative: c1 (f+1 - f-1) + c2 (f+2 - f-2) + c3 (f+3 - f-3)
template <class R>
__device__ __forceinline__ R d1(const R *__restrict__ f, long long p, long long s, const C4<R> &c) {
  return c.c1 * (__ldg(f + p + s) - __ldg(f + p - s)) + c.c2 * (__ldg(f + p + 2 * s) - __ldg(f + p - 2 * s)) +
         c.c3 * (__ldg(f + p + 3 * s) - __ldg(f + p - 3 * s));
}

// second derivative: c0 f + c1 (f+1 + f-1) + c2 (f+2 + f-2) + c3 (f+3 + f-3)
template <class R>
__device__ __forceinline__ R d2(const R *__restrict__ f, long long p, long long s, const C4<R> &c) {
  return c.c0 * __ldg(f + p) + c.c1 * (__ldg(f + p + s) + __ldg(f + p - s)) +
         c.c2 * (__ldg(f + p + 2 * s) + __ldg(f + p - 2 * s)) + c.c3 * (__ldg(f + p + 3 * s) + __ldg(f + p - 3 * s));
}

// Hybrid-scheme correction of point (i, j, k): R -= scale_d (dF_hi - dF_lo)
// summed over the directions whose interfaces around the point are flagged.
template <class R>
__device__ __forceinline__ void weno_correction(const Dev &d, const View<R> &V, int i, int j, int k, R *Rv) {
  const Consts<R> &K = consts<R>(d);
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    int pos = dir == 0 ? i : (dir == 1 ? j : k);
    long long lo = islot(d, dir, pos - 1, i, j, k), hi = islot(d, dir, pos, i, j, k);
    bool fl = d.flag[dir][lo], fh = d.flag[dir][hi];
    if (fl || fh) {
      R scale = dir == 0 ? K.idx : (dir == 1 ? __ldg(V.eta_y + j) : K.idz);
      const long long ns = d.nslot[dir];
      const R *dF = V.dF[dir];
#pragma unroll
      for (int f = 0; f < NV; ++f) {
        R c = (fh ? dF[f * ns + hi] : R(0)) - (fl ? dF[f * ns + lo] : R(0));
        Rv[f] = fma(-scale, c, Rv[f]);
      }
    }
  }
}

template <class R>
__global__ void __launch_bounds__(NT) k_apply(Dev d) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const View<R> V = view<R>(d);
  int i, j, k;
  point_of(d, q, i, j, k);
  R Rv[NV];
#pragma unroll
  for (int f = 0; f < NV; ++f) Rv[f] = V.fl[f * d.n + q];
  weno_correction(d, V, i, j, k, Rv);
#pragma unroll
  for (int f = 0; f < NV; ++f) V.fl[f * d.n + q] = Rv[f];
}

template <class R>
__global__ void __launch_bounds__(NT) k_grad(Dev d) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  int i, j, k;
  point_of(d, q, i, j, k);
  long long p = pidx(d, i, j, k);
  const C4<R> cx = {R(0), K.ax[1], K.ax[2], K.ax[3]}, cz = {R(0), K.az[1], K.az[2], K.az[3]};
  const C4<R> cy = {R(0), __ldg(V.ay + 3 * j), __ldg(V.ay + 3 * j + 1), __ldg(V.ay + 3 * j + 2)};
  const R *vel[3] = {V.u, V.v, V.ww};
  R g[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g[a][0] = d1(vel[a], p, 1, cx);
    g[a][1] = d1(vel[a], p, d.sy, cy);
    g[a][2] = d1(vel[a], p, d.sz, cz);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) V.g[(3 * a + b) * d.n + q] = g[a][b];
  R th = g[0][0] + g[1][1] + g[2][2];
  V.div[p] = th;
  if (d.weno) {
    R o1 = g[2][1] - g[1][2], o2 = g[0][2] - g[2][0], o3 = g[1][0] - g[0][1];
    R om2 = o1 * o1 + o2 * o2 + o3 * o3;
    R sv = -th / sqrt(th * th + om2 + R(1));
    V.sens[p] = sv > R(0) ? sv : R(0);
  }
}

template <class R>
__global__ void __launch_bounds__(NT) k_visc(Dev d) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  int i, j, k;
  point_of(d, q, i, j, k);
  long long p = pidx(d, i, j, k);
  const C4<R> cx = {R(0), K.ax[1], K.ax[2], K.ax[3]}, cz = {R(0), K.az[1], K.az[2], K.az[3]};
  const C4<R> cy = {R(0), __ldg(V.ay + 3 * j), __ldg(V.ay + 3 * j + 1), __ldg(V.ay + 3 * j + 2)};
  const C4<R> bx = {K.bx[0], K.bx[1], K.bx[2], K.bx[3]}, bz = {K.bz[0], K.bz[1], K.bz[2], K.bz[3]};
  const C4<R> by = {__ldg(V.by + 4 * j), __ldg(V.by + 4 * j + 1), __ldg(V.by + 4 * j + 2), __ldg(V.by + 4 * j + 3)};
  const R ry = __ldg(V.ry + j);  // eta_yy / eta_y
  R g[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) g[a][b] = __ldg(V.g + (3 * a + b) * d.n + q);
  const R *vel[3] = {V.u, V.v, V.ww};
  R lap[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    lap[a] = d2(vel[a], p, 1, bx) + (d2(vel[a], p, d.sy, by) + ry * g[a][1]) + d2(vel[a], p, d.sz, bz);
  R gT[3], gth[3];
  gT[0] = d1(V.T, p, 1, cx);
  gT[1] = d1(V.T, p, d.sy, cy);
  gT[2] = d1(V.T, p, d.sz, cz);
  R lapT = d2(V.T, p, 1, bx) + (d2(V.T, p, d.sy, by) + ry * gT[1]) + d2(V.T, p, d.sz, bz);
  gth[0] = d1(V.div, p, 1, cx);
  gth[1] = d1(V.div, p, d.sy, cy);
  gth[2] = d1(V.div, p, d.sz, cz);
  const R T = __ldg(V.T + p);
  const R mu = __ldg(V.mu + q);
  const R mut = K.visc_exp * mu / T;
  const R kc = mu * K.cp_over_pr;
  R gmu[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) gmu[b] = mut * gT[b];
  const R th = __ldg(V.div + p);
  const R uv[3] = {__ldg(V.u + p), __ldg(V.v + p), __ldg(V.ww + p)};
  R mom[3], en = R(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R m = mu * (lap[a] + gth[a] * R(1.0 / 3.0));
#pragma unroll
    for (int b = 0; b < 3; ++b) m += gmu[b] * (g[a][b] + g[b][a]);
    m -= R(2.0 / 3.0) * th * gmu[a];
    mom[a] = m;
    en += uv[a] * m;
  }
  // tau : grad u
  R tg = R(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) tg += (g[a][b] + g[b][a]) * g[a][b];
  tg -= R(2.0 / 3.0) * th * th;
  en += mu * tg;
  en += kc * lapT;
  en += K.cp_over_pr * (gmu[0] * gT[0] + gmu[1] * gT[1] + gmu[2] * gT[2]);
  R Rv[NV];
  Rv[0] = V.fl[q];
#pragma unroll
  for (int a = 0; a < 3; ++a) Rv[1 + a] = V.fl[(1 + a) * d.n + q] + mom[a];
  Rv[4] = V.fl[4 * d.n + q] + en;
  if (d.weno) weno_correction(d, V, i, j, k, Rv);
  if (d.weno) V.fl[q] = Rv[0];
#pragma unroll
  for (int f = 1; f < NV; ++f) V.fl[f * d.n + q] = Rv[f];
}

}  // namespace

cudaError_t launch_grad(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  if (d.mixed) k_grad<float><<<nb, NT, 0, st>>>(d);
  else k_grad<double><<<nb, NT, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_apply(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  if (d.mixed) k_apply<float><<<nb, NT, 0, st>>>(d);
  else k_apply<double><<<nb, NT, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_visc(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  if (d.mixed) k_visc<float><<<nb, NT, 0, st>>>(d);
  else k_visc<double><<<nb, NT, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace s2
