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
#include <type_traits>

#include "s2_internal.cuh"

namespace s2 {
namespace {

constexpr int NT = 256;


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
    const long long lo = islot32(d, dir, pos - 1, i, j, k), hi = islot32(d, dir, pos, i, j, k);
    if (!(S2_OK_IDX(d, lo, d.nslot[dir]) && S2_OK_IDX(d, hi, d.nslot[dir]))) continue;
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

// The Ducros sensor theta = max(-div / sqrt(div^2 + |omega|^2 + 1), 0)
// enters the scheme only through theta > thr; that test is stored (1 or
// 0), evaluated without a root or a division: for thr >= 0,
// theta > thr <=> div < 0 and div^2 > thr^2 (div^2 + |omega|^2 + 1).
template <class R>
__device__ __forceinline__ R sensor_test(const Consts<R> &K, const R (&g)[3][3], R th) {
  R o1 = g[2][1] - g[1][2], o2 = g[0][2] - g[2][0], o3 = g[1][0] - g[0][1];
  R om2 = o1 * o1 + o2 * o2 + o3 * o3;
  R th2 = th * th;
  bool on = K.thr < R(0) || (th < R(0) && th2 > K.thr2 * (th2 + om2 + R(1)));
  return on ? R(1) : R(0);
}

// Double precision: the margin m = theta^2 - thr^2 (theta^2 + |omega|^2 + 1)
// is first formed in single precision from the gradients converted on the
// integer pipe.  With u = 2^-24 and A_k = |a_k| + |b_k| for the two
// gradients of omega_k, its rounding error is below ~12.1 u (theta^2 +
// thr^2 (theta^2 + sum A_k^2 + 1)) (conversion, differences, squares,
// sums, products); when |m| exceeds 2^-19 = 32 u times that scale the sign
// of m is the exact one, and so the double-precision test's (which is
// exact outside ~1e-15 of the scale).  Otherwise -- within ~1e-6 of the
// threshold, or for values outside the single-precision range (the margin
// is then not finite) -- the double-precision test decides.  The
// decisions are identical; the double-precision unit skips ~12
// operations per point.
template <>
__device__ __forceinline__ double sensor_test<double>(const Consts<double> &K, const double (&g)[3][3], double th) {
  if (K.thr < 0.0) return 1.0;
  const float a1 = d2f_int(g[2][1]), b1 = d2f_int(g[1][2]);
  const float a2 = d2f_int(g[0][2]), b2 = d2f_int(g[2][0]);
  const float a3 = d2f_int(g[1][0]), b3 = d2f_int(g[0][1]);
  const float thf = d2f_int(th), t2 = d2f_int(K.thr2);
  const float o1 = a1 - b1, o2 = a2 - b2, o3 = a3 - b3;
  const float om2 = o1 * o1 + o2 * o2 + o3 * o3;
  const float th2 = thf * thf;
  const float m = th2 - t2 * (th2 + om2 + 1.0f);
  const float s1 = fabsf(a1) + fabsf(b1), s2 = fabsf(a2) + fabsf(b2), s3 = fabsf(a3) + fabsf(b3);
  const float scale = th2 + t2 * (th2 + (s1 * s1 + s2 * s2 + s3 * s3) + 1.0f);
  if (fabsf(m) > 0x1p-19f * scale) return (thf < 0.0f && m > 0.0f) ? 1.0 : 0.0;
  const double od1 = g[2][1] - g[1][2], od2 = g[0][2] - g[2][0], od3 = g[1][0] - g[0][1];
  const double dom2 = od1 * od1 + od2 * od2 + od3 * od3;
  const double dth2 = th * th;
  return (th < 0.0 && dth2 > K.thr2 * (dth2 + dom2 + 1.0)) ? 1.0 : 0.0;
}

// Viscous momentum and energy terms of one point from its derivatives:
// velocity gradient g[a][b] = d u_a / d x_b, Laplacians lap[a] and lapT,
// grad T, grad theta; T, mu, theta and u at the point.
template <class R>
__device__ __forceinline__ void visc_terms(const Consts<R> &K, const R (&g)[3][3], const R (&lap)[3], const R (&gT)[3],
                                           R lapT, const R (&gth)[3], R T, R mu, R th, const R (&uv)[3], R (&mom)[3],
                                           R &en) {
  const R mut = K.visc_exp * mu * rcp_pos(T);  // d mu / d T of the power law
  R gmu[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) gmu[b] = mut * gT[b];
  // tau / mu = S - (2/3) theta I with S_ab = g_ab + g_ba: its diagonal
  // dg_a = 2 g_aa - (2/3) theta and the off-diagonal S_01, S_02, S_12.
  const R tq = R(2.0 / 3.0) * th;
  R dg[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) dg[a] = fma(R(2), g[a][a], -tq);
  const R s01 = g[0][1] + g[1][0], s02 = g[0][2] + g[2][0], s12 = g[1][2] + g[2][1];
  const R so[3][3] = {{R(0), s01, s02}, {s01, R(0), s12}, {s02, s12, R(0)}};
  // d_b tau_ab = mu (lap u_a + (1/3) d_a theta) + sum_b (d_b mu) tau_ab / mu
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
  // grad k . grad T = (cp/Pr) (d mu/dT) |grad T|^2 (plus the c_p'(T) term
  // of a thermally perfect gas)
  R e = uv[0] * mom[0];
  e = fma(uv[1], mom[1], e);
  e = fma(uv[2], mom[2], e);
  R tg = dg[0] * g[0][0];
  tg = fma(dg[1], g[1][1], tg);
  tg = fma(dg[2], g[2][2], tg);
  tg = fma(s01, s01, tg);
  tg = fma(s02, s02, tg);
  tg = fma(s12, s12, tg);
  e = fma(mu, tg, e);
  R gT2 = gT[0] * gT[0];
  gT2 = fma(gT[1], gT[1], gT2);
  gT2 = fma(gT[2], gT[2], gT2);
  R cpr = K.cp_over_pr;
  if (K.tp) {
    // k = mu c_p(T)/Pr: grad k . grad T gains mu (c_p'(T)/Pr) |grad T|^2
    const R rT = rcp_pos(T);
    cpr = tp_cp(K, T, rT) * K.inv_pr;
    e = fma(mu * tp_dcp(K, T, rT) * K.inv_pr, gT2, e);
  }
  en = fma(cpr, fma(mut, gT2, mu * lapT), e);
}

template <class R>
__device__ __forceinline__ void apply_body(const Dev &__restrict__ d, const Blk &B) {
  long long q = (long long)B.x * NT + threadIdx.x;
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
__global__ void __launch_bounds__(NT) k_apply(Dev d) {
  apply_body<R>(d, grid_blk());
}

template <class R>
__global__ void __launch_bounds__(NT) kb_apply(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  apply_body<R>(sd, B);
}

template <class R, int NP>
__device__ __forceinline__ void grad_body(const Dev &__restrict__ d, const Blk &B) {
  long long q = (long long)B.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const View<R> V = view<R>(d);
  int i, j, k;
  point_of(d, q, i, j, k);
  long long p = pidx(d, i, j, k);
  // the stencils reach p -+ NP sz (z is the largest stride)
  if (!(S2_OK_IDX(d, p - NP * d.sz, d.np) && S2_OK_IDX(d, p + NP * d.sz, d.np))) return;
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
  if (d.weno) V.sens[p] = sensor_test(consts<R>(d), g, th);
}

template <class R, int NP>
__global__ void __launch_bounds__(NT) k_grad(Dev d) {
  grad_body<R, NP>(d, grid_blk());
}

template <class R, int NP>
__global__ void __launch_bounds__(NT) kb_grad(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  grad_body<R, NP>(sd, B);
}

template <class R, int NP>
__device__ __forceinline__ void visc_body(const Dev &__restrict__ d, const Blk &B) {
  long long q = (long long)B.x * NT + threadIdx.x;
  if (q >= d.n) return;
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  int i, j, k;
  point_of(d, q, i, j, k);
  long long p = pidx(d, i, j, k);
  if (!(S2_OK_IDX(d, p - NP * d.sz, d.np) && S2_OK_IDX(d, p + NP * d.sz, d.np))) return;
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
  const R uv[3] = {__ldg(V.u + p), __ldg(V.v + p), __ldg(V.ww + p)};
  R mom[3], en;
  visc_terms(K, g, lap, gT, lapT, gth, __ldg(V.T + p), __ldg(V.mu + q), __ldg(V.div + p), uv, mom, en);
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

template <class R, int NP>
__global__ void __launch_bounds__(NT) k_visc(Dev d) {
  visc_body<R, NP>(d, grid_blk());
}

template <class R, int NP>
__global__ void __launch_bounds__(NT) kb_visc(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  visc_body<R, NP>(sd, B);
}

// ------------------------------------------------ z-marching (mixed path)
// The single-precision path is bound by memory traffic, not arithmetic, so
// its gradient and viscous kernels march through z instead of giving each
// point its own 3-D stencil gathers.  A CTA owns a ZTX x ZTY tile of x-y
// columns over d.zs consecutive z-planes.  Per plane, the fields are staged
// once in shared memory with an NP-point x-y halo (x and y derivatives);
// along z each thread keeps its column's 2 NP + 1 values in registers
// (z derivatives).  The next plane's column values and halo values are
// loaded while the current plane is computed, and the staging buffer is
// double-buffered, so one barrier per plane suffices.  The viscous pass
// recomputes the velocity gradients from the staged values rather than
// reading nine stored ones.
constexpr int ZTX = 32, ZTY = 8;  // x-y tile; d.zs planes per CTA (tunable)

template <int NP>
struct ZGeom {
  static constexpr int SX = ZTX + 2 * NP, SY = ZTY + 2 * NP, SIZE = SX * SY;
  static constexpr int NH = SIZE - ZTX * ZTY;          // halo positions per plane
  static constexpr int HPT = (NH + NT - 1) / NT;        // halo slots per thread
};

// Shared-memory position (hx, hy) of halo slot h: NP full rows above the
// tile, NP columns each side of its ZTY rows, NP full rows below.
template <int NP>
__device__ __forceinline__ void zhalo_pos(int h, int &hx, int &hy) {
  constexpr int SX = ZGeom<NP>::SX;
  constexpr int TOP = NP * SX, MID = ZTY * 2 * NP;
  if (h < TOP) {
    hy = h / SX;
    hx = h - hy * SX;
  } else if (h < TOP + MID) {
    h -= TOP;
    hy = NP + h / (2 * NP);
    int r = h - (hy - NP) * 2 * NP;
    hx = r < NP ? r : ZTX + r;
  } else {
    h -= TOP + MID;
    hy = NP + ZTY + h / SX;
    hx = h - (hy - NP - ZTY) * SX;
  }
}

// Per-thread addressing of a z-marching tile: the thread's own column and
// its halo slots, as padded offsets without the z term (valid when inside
// the padded box; out-of-box slots are never read by an active point).
template <int NP, int ZS>
struct ZTile {
  int i, j, x0, y0, z0, z1;
  bool active, cvalid;
  long long cbase;                      // padded offset of (i, j, 0)
  long long hbase[ZGeom<NP>::HPT];
  int hoff[ZGeom<NP>::HPT];             // shared offset, -1 when unused
  __device__ __forceinline__ ZTile(const Dev &d, const Blk &B) {
    constexpr int SX = ZGeom<NP>::SX;
    const int tid = threadIdx.x;
    x0 = B.x * ZTX;
    y0 = B.y * ZTY;
    z0 = B.z * ZS;
    z1 = min(z0 + ZS, d.nz);
    i = x0 + tid % ZTX;
    j = y0 + tid / ZTX;
    active = i < d.nx && j < d.ny;
    cvalid = i < d.nx + GH && j < d.ny + GH;
    cbase = cvalid ? pidx(d, i, j, 0) : 0;
    // loads reach planes z0 - NP .. z1 - 1 + NP of the column and its halo
    if (cvalid && !(S2_OK_IDX(d, cbase + (z0 - NP) * d.sz, d.np) && S2_OK_IDX(d, cbase + (z1 - 1 + NP) * d.sz, d.np)))
      cvalid = active = false;
#pragma unroll
    for (int s = 0; s < ZGeom<NP>::HPT; ++s) {
      int h = tid + s * NT, hx = 0, hy = 0;
      hoff[s] = -1;
      hbase[s] = 0;
      if (h < ZGeom<NP>::NH) {
        zhalo_pos<NP>(h, hx, hy);
        int ii = x0 - NP + hx, jj = y0 - NP + hy;
        if (ii < d.nx + GH && jj < d.ny + GH) {
          hoff[s] = hy * SX + hx;
          hbase[s] = pidx(d, ii, jj, 0);
          if (!(S2_OK_IDX(d, hbase[s] + (z0 - NP) * d.sz, d.np) &&
                S2_OK_IDX(d, hbase[s] + (z1 - 1 + NP) * d.sz, d.np)))
            hoff[s] = -1;
        }
      }
    }
  }
  __device__ __forceinline__ int centre() const {
    return (threadIdx.x / ZTX + NP) * ZGeom<NP>::SX + threadIdx.x % ZTX + NP;
  }
};

// z-marching gradient pass: theta = div u (with ghosts at walls) and the
// sensor test.  NF = 3 staged fields (u, v, w).
template <int NP, int ZS>
__device__ __forceinline__ void grad_z_body(const Dev &__restrict__ d, const Blk &B) {
  using R = float;
  constexpr int NF = 3, NQ = 2 * NP + 1, SZ = ZGeom<NP>::SIZE, SX = ZGeom<NP>::SX, HPT = ZGeom<NP>::HPT;
  __shared__ R sm[2][NF][SZ];
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  const ZTile<NP, ZS> t(d, B);
  const R *src[NF] = {V.u, V.v, V.ww};
  const long long sz = d.sz;
  C5<R> cx, cy, cz;
  coeffs<NP>(d, V, t.active ? t.j : 0, cx, cy, cz);
  R q[NF][NQ], pf[NF], hr[NF][HPT];
  // prologue: the column's planes z0-NP .. z0+NP, the halo of plane z0
#pragma unroll
  for (int f = 0; f < NF; ++f) {
#pragma unroll
    for (int m = 0; m < NQ - 1; ++m) q[f][m] = t.cvalid ? __ldg(src[f] + t.cbase + (t.z0 - NP + m) * sz) : R(0);
    pf[f] = t.cvalid ? __ldg(src[f] + t.cbase + (t.z0 + NP) * sz) : R(0);
#pragma unroll
    for (int s = 0; s < HPT; ++s) hr[f][s] = t.hoff[s] >= 0 ? __ldg(src[f] + t.hbase[s] + t.z0 * sz) : R(0);
  }
  const int c = t.centre();
  for (int k = t.z0; k < t.z1; ++k) {
    const int b = (k - t.z0) & 1;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      q[f][NQ - 1] = pf[f];
      sm[b][f][c] = q[f][NP];
#pragma unroll
      for (int s = 0; s < HPT; ++s)
        if (t.hoff[s] >= 0) sm[b][f][t.hoff[s]] = hr[f][s];
    }
    if (k + 1 < t.z1) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        pf[f] = t.cvalid ? __ldg(src[f] + t.cbase + (k + 1 + NP) * sz) : R(0);
#pragma unroll
        for (int s = 0; s < HPT; ++s) hr[f][s] = t.hoff[s] >= 0 ? __ldg(src[f] + t.hbase[s] + (k + 1) * sz) : R(0);
      }
    }
    __syncthreads();
    if (t.active) {
      R g[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R *S = sm[b][a];
        R gx = cx.c[1] * (S[c + 1] - S[c - 1]);
        R gy = cy.c[1] * (S[c + SX] - S[c - SX]);
        R gz = cz.c[1] * (q[a][NP + 1] - q[a][NP - 1]);
#pragma unroll
        for (int l = 2; l <= NP; ++l) {
          gx = fma(cx.c[l], S[c + l] - S[c - l], gx);
          gy = fma(cy.c[l], S[c + l * SX] - S[c - l * SX], gy);
          gz = fma(cz.c[l], q[a][NP + l] - q[a][NP - l], gz);
        }
        g[a][0] = gx;
        g[a][1] = gy;
        g[a][2] = gz;
      }
      const R th = g[0][0] + g[1][1] + g[2][2];
      const long long p = t.cbase + k * sz;
      V.div[p] = th;
      // wall ghosts of theta: the divergence of the mirrored velocity
      // field at the mirror node is -u_x + v_y - w_z
      if (d.wall_y) {
        const long long plo = pidx(d, t.i, -1 - t.j, k), phi = pidx(d, t.i, 2 * d.ny - 1 - t.j, k);
        if (t.j < GH && S2_OK_IDX(d, plo, d.np)) V.div[plo] = -g[0][0] + g[1][1] - g[2][2];
        if (t.j >= d.ny - GH && S2_OK_IDX(d, phi, d.np)) V.div[phi] = -g[0][0] + g[1][1] - g[2][2];
      }
      if (d.weno) V.sens[p] = sensor_test(K, g, th);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int m = 0; m < NQ - 1; ++m) q[f][m] = q[f][m + 1];
  }
}

template <int NP, int ZS>
__global__ void __launch_bounds__(NT, 3) k_grad_z(Dev d) {
  grad_z_body<NP, ZS>(d, grid_blk());
}

template <int NP, int ZS>
__global__ void __launch_bounds__(NT, 3) kb_grad_z(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  grad_z_body<NP, ZS>(sd, B);
}

// z-marching viscous pass (velocity gradients recomputed), plus the WENO
// corrections.  NF = 5 staged fields (u, v, w, T, theta).  The next
// plane's halo and the point's RHS and viscosity arrive by cp.async while
// the current plane is computed (the plane's centre values come from the
// column queue in registers).
template <int NP, int ZS>
__device__ __forceinline__ void visc_z_body(const Dev &__restrict__ d, const Blk &B) {
  using R = float;
  constexpr int NF = 5, NQ = 2 * NP + 1, SZ = ZGeom<NP>::SIZE, SX = ZGeom<NP>::SX, HPT = ZGeom<NP>::HPT;
  __shared__ R sm[2][NF][SZ];
  __shared__ R pre[2][NV + 1][NT];  // the thread's RHS (NV) and mu, by plane parity
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  const ZTile<NP, ZS> t(d, B);
  const R *src[NF] = {V.u, V.v, V.ww, V.T, V.div};
  const long long sz = d.sz;
  const int jc = t.active ? t.j : 0;
  C5<R> cx, cy, cz, bx, by, bz;
  coeffs<NP>(d, V, jc, cx, cy, cz);
#pragma unroll
  for (int l = 0; l <= 4; ++l) {
    bx.c[l] = K.bx[l];
    bz.c[l] = K.bz[l];
    by.c[l] = l <= NP ? __ldg(V.by + 5 * jc + l) : R(0);
  }
  const R ry = __ldg(V.ry + jc);
  const R c0 = by.c[0] + K.b0xz;
  const int tid = threadIdx.x;
  // asynchronous part of plane kk into buffer bb: its halo, the point's RHS and mu
  auto fetch = [&](int kk, int bb) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int s = 0; s < HPT; ++s)
        if (t.hoff[s] >= 0) cp_async4(&sm[bb][f][t.hoff[s]], src[f] + t.hbase[s] + kk * sz);
    if (t.active) {
      const long long qk = ((long long)kk * d.ny + t.j) * d.nx + t.i;
#pragma unroll
      for (int f = 0; f < NV; ++f) cp_async4(&pre[bb][f][tid], V.fl + f * d.n + qk);
      cp_async4(&pre[bb][NV][tid], V.mu + qk);
    }
    cp_async_commit();
  };
  R q[NF][NQ], pf[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
#pragma unroll
    for (int m = 0; m < NQ - 1; ++m) q[f][m] = t.cvalid ? __ldg(src[f] + t.cbase + (t.z0 - NP + m) * sz) : R(0);
    pf[f] = t.cvalid ? __ldg(src[f] + t.cbase + (t.z0 + NP) * sz) : R(0);
  }
  fetch(t.z0, 0);
  const int c = t.centre();
  R fsum = R(0);  // the column's R_rho u, for the bulk forcing
  for (int k = t.z0; k < t.z1; ++k) {
    const int b = (k - t.z0) & 1;
    const long long qi = ((long long)k * d.ny + t.j) * d.nx + t.i;  // interior index
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      q[f][NQ - 1] = pf[f];
      sm[b][f][c] = q[f][NP];
    }
    cp_async_wait_all();
    // every thread has finished the previous plane (whose buffer the next
    // fetch overwrites) and this plane's halo is in place
    __syncthreads();
    if (k + 1 < t.z1) {
#pragma unroll
      for (int f = 0; f < NF; ++f) pf[f] = t.cvalid ? __ldg(src[f] + t.cbase + (k + 1 + NP) * sz) : R(0);
      fetch(k + 1, b ^ 1);
    }
    if (t.active) {
      R Rv[NV];
#pragma unroll
      for (int f = 0; f < NV; ++f) Rv[f] = pre[b][f][tid];
      const R mu = pre[b][NV][tid];
      // first derivatives (x, y from shared memory, z from the column)
      R gd[NF][3];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const R *S = sm[b][f];
        R gx = cx.c[1] * (S[c + 1] - S[c - 1]);
        R gy = cy.c[1] * (S[c + SX] - S[c - SX]);
        R gz = cz.c[1] * (q[f][NP + 1] - q[f][NP - 1]);
#pragma unroll
        for (int l = 2; l <= NP; ++l) {
          gx = fma(cx.c[l], S[c + l] - S[c - l], gx);
          gy = fma(cy.c[l], S[c + l * SX] - S[c - l * SX], gy);
          gz = fma(cz.c[l], q[f][NP + l] - q[f][NP - l], gz);
        }
        gd[f][0] = gx;
        gd[f][1] = gy;
        gd[f][2] = gz;
      }
      // Laplacians of u, v, w, T: d2/dy2 = eta_y^2 d2/deta2 + eta_yy d/deta
      R lp[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const R *S = sm[b][f];
        R r = c0 * q[f][NP];
#pragma unroll
        for (int l = 1; l <= NP; ++l) r = fma(bx.c[l], S[c + l] + S[c - l], r);
#pragma unroll
        for (int l = 1; l <= NP; ++l) r = fma(by.c[l], S[c + l * SX] + S[c - l * SX], r);
#pragma unroll
        for (int l = 1; l <= NP; ++l) r = fma(bz.c[l], q[f][NP + l] + q[f][NP - l], r);
        lp[f] = fma(ry, gd[f][1], r);
      }
      const R g[3][3] = {{gd[0][0], gd[0][1], gd[0][2]}, {gd[1][0], gd[1][1], gd[1][2]}, {gd[2][0], gd[2][1], gd[2][2]}};
      const R lap[3] = {lp[0], lp[1], lp[2]};
      const R gT[3] = {gd[3][0], gd[3][1], gd[3][2]};
      const R gth[3] = {gd[4][0], gd[4][1], gd[4][2]};
      const R uv[3] = {q[0][NP], q[1][NP], q[2][NP]};
      R mom[3], en;
      visc_terms(K, g, lap, gT, lp[3], gth, q[3][NP], mu, q[4][NP], uv, mom, en);
#pragma unroll
      for (int a = 0; a < 3; ++a) Rv[1 + a] += mom[a];
      Rv[4] += en;
      if (d.weno) weno_correction(d, V, t.i, t.j, k, Rv);
      if (d.weno) V.fl[qi] = Rv[0];
#pragma unroll
      for (int f = 1; f < NV; ++f) V.fl[f * d.n + qi] = Rv[f];
      fsum += Rv[1];
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int m = 0; m < NQ - 1; ++m) q[f][m] = q[f][m + 1];
  }
  // forcing: this CTA's share of sum R_rho u dV (dV ~ dy/deta), summed in
  // double in a fixed order into part[CTA]
  if (d.force) {
    double v = t.active ? (double)fsum * d.dvy[t.j] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double wsum[NT / 32];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < NT / 32; ++w) tot += wsum[w];
      d.part[((long long)B.z * B.ny + B.y) * B.nx + B.x] = tot;
    }
  }
}

template <int NP, int ZS>
__global__ void __launch_bounds__(NT, 2) k_visc_z(Dev d) {
  visc_z_body<NP, ZS>(d, grid_blk());
}

template <int NP, int ZS>
__global__ void __launch_bounds__(NT, 2) kb_visc_z(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  visc_z_body<NP, ZS>(sd, B);
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

// Planes per CTA of the z-marching passes, compiled as template arguments
// (a loop of compile-time length keeps the z queue in fixed registers).
template <int NPV, class F>
void z_launch(F f, int zs) {
  switch (zs) {
    case 4: f(std::integral_constant<int, 4>()); break;
    case 8: f(std::integral_constant<int, 8>()); break;
    case 16: f(std::integral_constant<int, 16>()); break;
    case 24: f(std::integral_constant<int, 24>()); break;
    default: f(std::integral_constant<int, 12>()); break;
  }
}

static dim3 zgrid(const Dev &d) {
  return dim3((d.nx + ZTX - 1) / ZTX, (d.ny + ZTY - 1) / ZTY, (d.nz + d.zs - 1) / d.zs);
}

cudaError_t launch_grad(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  if (d.mixed) {
    switch (d.npv) {
      case 1: z_launch<1>([&](auto zs) { k_grad_z<1, decltype(zs)::value><<<zgrid(d), NT, 0, st>>>(d); }, d.zs); break;
      case 2: z_launch<2>([&](auto zs) { k_grad_z<2, decltype(zs)::value><<<zgrid(d), NT, 0, st>>>(d); }, d.zs); break;
      case 3: z_launch<3>([&](auto zs) { k_grad_z<3, decltype(zs)::value><<<zgrid(d), NT, 0, st>>>(d); }, d.zs); break;
      default: z_launch<4>([&](auto zs) { k_grad_z<4, decltype(zs)::value><<<zgrid(d), NT, 0, st>>>(d); }, d.zs); break;
    }
  } else {
    grad_np<double>(d, nb, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  if (d.mixed) k_apply<float><<<nb, NT, 0, st>>>(d);
  else k_apply<double><<<nb, NT, 0, st>>>(d);
  return cudaGetLastError();
}

long long z_pass_blocks(const Dev &d) {
  dim3 g = zgrid(d);
  return (long long)g.x * g.y * g.z;
}

int visc_force_partials(const Dev &d) {
  if (!(d.mixed && d.force && d.viscous)) return 0;
  return (int)z_pass_blocks(d);
}

void z_pass_grid(const Dev &d, unsigned g[3]) {
  const dim3 z = zgrid(d);
  g[0] = z.x;
  g[1] = z.y;
  g[2] = z.z;
}

// Batched: every box of a batch group in one launch (instantiation of d0).
cudaError_t launch_grad_batch(const Dev &d0, const BatchArgs &ba, unsigned total, cudaStream_t st) {
  if (d0.mixed) {
    switch (d0.npv) {
      case 1: z_launch<1>([&](auto zs) { kb_grad_z<1, decltype(zs)::value><<<total, NT, 0, st>>>(ba); }, d0.zs); break;
      case 2: z_launch<2>([&](auto zs) { kb_grad_z<2, decltype(zs)::value><<<total, NT, 0, st>>>(ba); }, d0.zs); break;
      case 3: z_launch<3>([&](auto zs) { kb_grad_z<3, decltype(zs)::value><<<total, NT, 0, st>>>(ba); }, d0.zs); break;
      default: z_launch<4>([&](auto zs) { kb_grad_z<4, decltype(zs)::value><<<total, NT, 0, st>>>(ba); }, d0.zs); break;
    }
  } else {
    switch (d0.npv) {
      case 1: kb_grad<double, 1><<<total, NT, 0, st>>>(ba); break;
      case 2: kb_grad<double, 2><<<total, NT, 0, st>>>(ba); break;
      case 3: kb_grad<double, 3><<<total, NT, 0, st>>>(ba); break;
      default: kb_grad<double, 4><<<total, NT, 0, st>>>(ba); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_visc_batch(const Dev &d0, const BatchArgs &ba, unsigned total, cudaStream_t st) {
  if (d0.mixed) {
    switch (d0.npv) {
      case 1: z_launch<1>([&](auto zs) { kb_visc_z<1, decltype(zs)::value><<<total, NT, 0, st>>>(ba); }, d0.zs); break;
      case 2: z_launch<2>([&](auto zs) { kb_visc_z<2, decltype(zs)::value><<<total, NT, 0, st>>>(ba); }, d0.zs); break;
      case 3: z_launch<3>([&](auto zs) { kb_visc_z<3, decltype(zs)::value><<<total, NT, 0, st>>>(ba); }, d0.zs); break;
      default: z_launch<4>([&](auto zs) { kb_visc_z<4, decltype(zs)::value><<<total, NT, 0, st>>>(ba); }, d0.zs); break;
    }
  } else {
    switch (d0.npv) {
      case 1: kb_visc<double, 1><<<total, NT, 0, st>>>(ba); break;
      case 2: kb_visc<double, 2><<<total, NT, 0, st>>>(ba); break;
      case 3: kb_visc<double, 3><<<total, NT, 0, st>>>(ba); break;
      default: kb_visc<double, 4><<<total, NT, 0, st>>>(ba); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_batch(const Dev &d0, const BatchArgs &ba, unsigned total, cudaStream_t st) {
  if (d0.mixed) kb_apply<float><<<total, NT, 0, st>>>(ba);
  else kb_apply<double><<<total, NT, 0, st>>>(ba);
  return cudaGetLastError();
}

cudaError_t launch_visc(const Dev &d, cudaStream_t st) {
  unsigned nb = (unsigned)((d.n + NT - 1) / NT);
  if (d.mixed) {
    switch (d.npv) {
      case 1: z_launch<1>([&](auto zs) { k_visc_z<1, decltype(zs)::value><<<zgrid(d), NT, 0, st>>>(d); }, d.zs); break;
      case 2: z_launch<2>([&](auto zs) { k_visc_z<2, decltype(zs)::value><<<zgrid(d), NT, 0, st>>>(d); }, d.zs); break;
      case 3: z_launch<3>([&](auto zs) { k_visc_z<3, decltype(zs)::value><<<zgrid(d), NT, 0, st>>>(d); }, d.zs); break;
      default: z_launch<4>([&](auto zs) { k_visc_z<4, decltype(zs)::value><<<zgrid(d), NT, 0, st>>>(d); }, d.zs); break;
    }
  } else {
    visc_np<double>(d, nb, st);
  }
  return cudaGetLastError();
}

}  // namespace s2
