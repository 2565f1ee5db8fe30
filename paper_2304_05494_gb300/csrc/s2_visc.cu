// Velocity gradients + shock sensor, and the viscous/heat-flux terms.
//
// Paper Sec. 2: the switch between central and WENO fluxes is a modified
// Ducros sensor; the viscous terms are expanded in Laplacian form and
// discretised with central formulae of order 2, 4, 6 or 8 (visflx_nosensor
// of Table 2; the sensor's derivatives use the same order).
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

// Pre-scaled stencil coefficients of one direction at one point (c[0] is
// the centre weight of a second derivative; c[1..NP] the pair weights).
template <class R>
struct C5 {
  R c[5];
};

// first derivative: sum_{l=1..NP} c_l (f_{+l} - f_{-l})
template <int NP, class R>
__device__ __forceinline__ R d1(const R *__restrict__ f, long long p, long long s, const C5<R> &c) {
  R r = c.c[1] * (__ldg(f + p + s) - __ldg(f + p - s));
#pragma unroll
  for (int l = 2; l <= NP; ++l) r += c.c[l] * (__ldg(f + p + l * s) - __ldg(f + p - l * s));
  return r;
}

// Laplacian of f in the computational coordinates, centre weight c0 of
// all three directions together: c0 f + sum_d sum_l b_{d,l} (f_{+l} + f_{-l})
template <int NP, class R>
__device__ __forceinline__ R lap3(const R *__restrict__ f, long long p, long long sy, long long sz, R c0,
                                  const C5<R> &bx, const C5<R> &by, const C5<R> &bz) {
  R r = c0 * __ldg(f + p);
#pragma unroll
  for (int l = 1; l <= NP; ++l) r = fma(bx.c[l], __ldg(f + p + l) + __ldg(f + p - l), r);
#pragma unroll
  for (int l = 1; l <= NP; ++l) r = fma(by.c[l], __ldg(f + p + l * sy) + __ldg(f + p - l * sy), r);
#pragma unroll
  for (int l = 1; l <= NP; ++l) r = fma(bz.c[l], __ldg(f + p + l * sz) + __ldg(f + p - l * sz), r);
  return r;
}

template <int NP, class R>
__device__ __forceinline__ void coeffs(const Dev &d, const View<R> &V, int j, C5<R> &cx, C5<R> &cy, C5<R> &cz) {
  const Consts<R> &K = consts<R>(d);
#pragma unroll
  for (int l = 0; l <= 4; ++l) {
    cx.c[l] = l ? K.ax[l] : R(0);
    cz.c[l] = l ? K.az[l] : R(0);
    cy.c[l] = (l && l <= NP) ? __ldg(V.ay + 4 * j + l - 1) : R(0);
  }
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

template <class R, int NP>
__global__ void __launch_bounds__(NT) k_grad(Dev d) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const View<R> V = view<R>(d);
  int i, j, k;
  point_of(d, q, i, j, k);
  long long p = pidx(d, i, j, k);
  C5<R> cx, cy, cz;
  coeffs<NP>(d, V, j, cx, cy, cz);
  const R *vel[3] = {V.u, V.v, V.ww};
  R g[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g[a][0] = d1<NP>(vel[a], p, 1, cx);
    g[a][1] = d1<NP>(vel[a], p, d.sy, cy);
    g[a][2] = d1<NP>(vel[a], p, d.sz, cz);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) V.g[(3 * a + b) * d.n + q] = g[a][b];
  R th = g[0][0] + g[1][1] + g[2][2];
  V.div[p] = th;
  if (d.weno) {
    // The Ducros sensor theta = max(-div / sqrt(div^2 + |omega|^2 + 1), 0)
    // enters the scheme only through theta > thr; that test is stored
    // (1 or 0), evaluated without a root or a division: for thr >= 0,
    // theta > thr <=> div < 0 and div^2 > thr^2 (div^2 + |omega|^2 + 1).
    const Consts<R> &K = consts<R>(d);
    R o1 = g[2][1] - g[1][2], o2 = g[0][2] - g[2][0], o3 = g[1][0] - g[0][1];
    R om2 = o1 * o1 + o2 * o2 + o3 * o3;
    R th2 = th * th;
    bool on = K.thr < R(0) || (th < R(0) && th2 > K.thr2 * (th2 + om2 + R(1)));
    V.sens[p] = on ? R(1) : R(0);
  }
}

template <class R, int NP>
__global__ void __launch_bounds__(NT) k_visc(Dev d) {
  long long q = (long long)blockIdx.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  int i, j, k;
  point_of(d, q, i, j, k);
  long long p = pidx(d, i, j, k);
  C5<R> cx, cy, cz, bx, by, bz;
  coeffs<NP>(d, V, j, cx, cy, cz);
#pragma unroll
  for (int l = 0; l <= 4; ++l) {
    bx.c[l] = K.bx[l];
    bz.c[l] = K.bz[l];
    by.c[l] = l <= NP ? __ldg(V.by + 5 * j + l) : R(0);
  }
  const R ry = __ldg(V.ry + j);  // eta_yy / eta_y
  const R c0 = by.c[0] + K.b0xz;
  R g[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) g[a][b] = __ldg(V.g + (3 * a + b) * d.n + q);
  const R *vel[3] = {V.u, V.v, V.ww};
  // Laplacians in physical coordinates: d2/dy2 = eta_y^2 d2/deta2 + eta_yy d/deta
  R lap[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) lap[a] = fma(ry, g[a][1], lap3<NP>(vel[a], p, d.sy, d.sz, c0, bx, by, bz));
  R gT[3], gth[3];
  gT[0] = d1<NP>(V.T, p, 1, cx);
  gT[1] = d1<NP>(V.T, p, d.sy, cy);
  gT[2] = d1<NP>(V.T, p, d.sz, cz);
  const R lapT = fma(ry, gT[1], lap3<NP>(V.T, p, d.sy, d.sz, c0, bx, by, bz));
  gth[0] = d1<NP>(V.div, p, 1, cx);
  gth[1] = d1<NP>(V.div, p, d.sy, cy);
  gth[2] = d1<NP>(V.div, p, d.sz, cz);
  const R T = __ldg(V.T + p);
  const R mu = __ldg(V.mu + q);
  const R mut = K.visc_exp * mu * rcp_pos(T);  // d mu / d T of the power law
  R gmu[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) gmu[b] = mut * gT[b];
  const R th = __ldg(V.div + p);
  const R uv[3] = {__ldg(V.u + p), __ldg(V.v + p), __ldg(V.ww + p)};
  // tau / mu = S - (2/3) theta I with S_ab = g_ab + g_ba: its diagonal
  // dg_a = 2 g_aa - (2/3) theta and the off-diagonal S_01, S_02, S_12.
  const R tq = R(2.0 / 3.0) * th;
  R dg[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) dg[a] = fma(R(2), g[a][a], -tq);
  const R s01 = g[0][1] + g[1][0], s02 = g[0][2] + g[2][0], s12 = g[1][2] + g[2][1];
  const R so[3][3] = {{R(0), s01, s02}, {s01, R(0), s12}, {s02, s12, R(0)}};
  // d_b tau_ab = mu (lap u_a + (1/3) d_a theta) + sum_b (d_b mu) tau_ab / mu
  R mom[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R m = mu * fma(gth[a], R(1.0 / 3.0), lap[a]);
    m = fma(gmu[a], dg[a], m);
#pragma unroll
    for (int b = 0; b < 3; ++b)
      if (b != a) m = fma(gmu[b], so[a][b], m);
    mom[a] = m;
  }
  // energy: u . div tau + tau : grad u + div(k grad T), k = mu cp / Pr;
  // tau : grad u / mu = sum_a dg_a g_aa + S_01^2 + S_02^2 + S_12^2, and
  // grad k . grad T = (cp/Pr) (d mu/dT) |grad T|^2
  R en = uv[0] * mom[0];
  en = fma(uv[1], mom[1], en);
  en = fma(uv[2], mom[2], en);
  R tg = dg[0] * g[0][0];
  tg = fma(dg[1], g[1][1], tg);
  tg = fma(dg[2], g[2][2], tg);
  tg = fma(s01, s01, tg);
  tg = fma(s02, s02, tg);
  tg = fma(s12, s12, tg);
  en = fma(mu, tg, en);
  R gT2 = gT[0] * gT[0];
  gT2 = fma(gT[1], gT[1], gT2);
  gT2 = fma(gT[2], gT[2], gT2);
  en = fma(K.cp_over_pr, fma(mut, gT2, mu * lapT), en);
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

template <class R>
void grad_np(const Dev &d, unsigned nb, cudaStream_t st) {
  switch (d.npv) {
    case 1: k_grad<R, 1><<<nb, NT, 0, st>>>(d); break;
    case 2: k_grad<R, 2><<<nb, NT, 0, st>>>(d); break;
    case 3: k_grad<R, 3><<<nb, NT, 0, st>>>(d); break;
    default: k_grad<R, 4><<<nb, NT, 0, st>>>(d); break;
  }
}

template <class R>
void visc_np(const Dev &d, unsigned nb, cudaStream_t st) {
  switch (d.npv) {
    case 1: k_visc<R, 1><<<nb, NT, 0, st>>>(d); break;
    case 2: k_visc<R, 2><<<nb, NT, 0, st>>>(d); break;
    case 3: k_visc<R, 3><<<nb, NT, 0, st>>>(d); break;
    default: k_visc<R, 4><<<nb, NT, 0, st>>>(d); break;
  }
}

}  // namespace

cudaError_t launch_grad(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  if (d.mixed) grad_np<float>(d, nb, st);
  else grad_np<double>(d, nb, st);
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
  if (d.mixed) visc_np<float>(d, nb, st);
  else visc_np<double>(d, nb, st);
  return cudaGetLastError();
}

}  // namespace s2
