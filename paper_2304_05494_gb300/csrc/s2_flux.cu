// Convective flux kernels: hybrid central / WENO, one direction at a time.
//
// Paper Sec. 2: the convective terms use the energy-preserving split
// (skew-symmetric) form written as numerical fluxes (Pirozzoli, JCP 2010)
// in smooth regions and, at interfaces flagged by the Ducros-type sensor, a
// WENO reconstruction of characteristic fluxes (Lax-Friedrichs splitting)
// projected back on the right eigenvectors.  These are the euler_{x,y,z}
// kernels of Table 2.  The paper's transposition kernel for x is not needed:
// every direction stages its pencils through shared memory.
//
// k_flux<DIR>  one CTA per tile of L points along DIR times W pencils:
//   1. stage the primitives of the tile plus GH ghost points each side
//      (coalesced: the x-contiguous index runs fastest);
//   2. per position a the pair fluxes T_l(a) of the pairs (a, a+l), l=1..3:
//      m = (rho_a+rho_b)(un_a+un_b), T = m (1, su, sv, sw, sH), s. = pair sums;
//   3. the central flux difference D(a) = sum_l c_l [T_l(a) - T_l(a-l)]
//      + sum_l a_l (p_{a+l} - p_{a-l}) equals F_{a+1/2} - F_{a-1/2} of the
//      split-form interface flux; -scale D goes into the RHS;
//   4. interface flags (max sensor over the WENO stencil > threshold) are
//      stored and the flagged interfaces appended to a global list.
// k_weno<DIR>  one thread per listed interface (globally compacted, so
//   shocks cause no divergence in the central kernel and no idle lanes
//   here): F_weno - F_central at the interface.
// The corrections are added per point, in a fixed order, by the viscous
// kernel (or k_apply when inviscid): deterministic, no atomics on the RHS.
#include "s2_internal.cuh"

namespace s2 {
namespace {

// 6th-order central coefficients a_l (first derivative).
__device__ __constant__ double kA[4] = {0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0};

template <int DIR>
struct Tile;
template <>
struct Tile<0> {  // x: 64 along x, 4 rows (y)
  static constexpr int L = 64, W = 4;
};
template <>
struct Tile<1> {  // y: 32 along y, 8 columns (x)
  static constexpr int L = 32, W = 8;
};
template <>
struct Tile<2> {  // z: 32 along z, 8 columns (x)
  static constexpr int L = 32, W = 8;
};

constexpr int NTHREADS = 256;
enum { F_RHO = 0, F_U, F_V, F_W, F_H, F_P, F_S, NF };

template <int DIR, int WR>
__global__ void __launch_bounds__(NTHREADS, 3) k_flux(Dev d, int accumulate) {
  constexpr int L = Tile<DIR>::L, W = Tile<DIR>::W;
  constexpr int LE = L + 2 * GH;       // extended positions per pencil
  constexpr int SF = LE * W;           // doubles per shared field
  constexpr int LT = L + 3;            // pair-flux positions a = -3 .. L-1
  constexpr int ST = LT * W;           // doubles per pair-flux slot
  constexpr int NFLD = WR > 0 ? NF : F_S;  // the sensor is staged only for WENO
  extern __shared__ double smem[];
  double *S = smem;                    // [NF][LE][W]
  double *TP = smem + NF * SF;         // [3][5][LT][W]

  const int tid = threadIdx.x;
  const int n = DIR == 0 ? d.nx : (DIR == 1 ? d.ny : d.nz);
  int x0 = 0, y0 = 0, z0 = 0;
  if (DIR == 0) { x0 = blockIdx.x * L; y0 = blockIdx.y * W; z0 = blockIdx.z; }
  if (DIR == 1) { x0 = blockIdx.x * W; y0 = blockIdx.y * L; z0 = blockIdx.z; }
  if (DIR == 2) { x0 = blockIdx.x * W; z0 = blockIdx.y * L; y0 = blockIdx.z; }
  const int s0 = DIR == 0 ? x0 : (DIR == 1 ? y0 : z0);
  const int nac = DIR == 0 ? d.ny : d.nx;   // extent across
  const int c0 = DIR == 0 ? y0 : x0;

  const double *src[NF] = {d.rho, d.u, d.v, d.ww, d.H, d.p, d.sens};

  // ---- 1. stage the tile (positions s0-GH .. s0+L+GH-1) ----
  for (int idx = tid; idx < SF; idx += NTHREADS) {
    int a, cc;
    if (DIR == 0) { a = idx % LE; cc = idx / LE; }
    else { cc = idx % W; a = idx / W; }
    int s = s0 + a - GH;
    bool ok = (c0 + cc < nac) && (s < n + GH);
    long long g = 0;
    if (ok) {
      if (DIR == 0) g = pidx(d, s, y0 + cc, z0);
      else if (DIR == 1) g = pidx(d, x0 + cc, s, z0);
      else g = pidx(d, x0 + cc, y0, s);
    }
#pragma unroll
    for (int f = 0; f < NFLD; ++f) S[f * SF + a * W + cc] = ok ? __ldg(src[f] + g) : 1.0;
  }
  __syncthreads();

  // ---- 2. pair fluxes T_l(a), a = -3 .. L-1 ----
  for (int idx = tid; idx < ST; idx += NTHREADS) {
    int a = idx / W, cc = idx % W;        // a in 0..LT-1 <-> position a-3
    int ae = a - 3 + GH;                  // extended index of the position
    const double *Sr = S + F_RHO * SF, *Su = S + F_U * SF, *Sv = S + F_V * SF, *Sw = S + F_W * SF,
                 *Sh = S + F_H * SF;
    int q0 = ae * W + cc;
    double r0 = Sr[q0], u0 = Su[q0], v0 = Sv[q0], w0 = Sw[q0], h0 = Sh[q0];
#pragma unroll
    for (int l = 1; l <= 3; ++l) {
      int q1 = q0 + l * W;
      double su = u0 + Su[q1], sv = v0 + Sv[q1], sw = w0 + Sw[q1];
      double sun = DIR == 0 ? su : (DIR == 1 ? sv : sw);
      double m = (r0 + Sr[q1]) * sun;
      double *T = TP + ((l - 1) * 5) * ST + idx;
      T[0] = m;
      T[ST] = m * su;
      T[2 * ST] = m * sv;
      T[3 * ST] = m * sw;
      T[4 * ST] = m * (h0 + Sh[q1]);
    }
  }

  // ---- 4. flags of the interfaces this tile owns, global list ----
  // A tile owns the interfaces a+1/2 with a in 0..L-1, the first tile of a
  // pencil also the one before its first point (a = -1): every interface
  // slot 0..n of a pencil is owned exactly once.
  if constexpr (WR > 0) {
    const double *Ss = S + F_S * SF;
    const long long thr_bits = __double_as_longlong(d.thr);
    constexpr int NI = (L + 1) * W;
    unsigned long long mycount = 0;
    for (int base = 0; base < NI; base += NTHREADS) {
      int idx = base + tid;
      bool flag = false;
      long long slot = 0;
      if (idx < NI) {
        int a = idx / W - 1, cc = idx % W;
        int s = s0 + a;
        bool own = (c0 + cc < nac) && s <= n - 1 && (a >= 0 || s == -1);
        if (own) {
          // the sensor is >= 0, so its IEEE bit patterns order like the
          // values: max and comparison run on the integer pipe
          long long mx = 0;
#pragma unroll
          for (int m = -WR + 1; m <= WR; ++m) {
            long long b = __double_as_longlong(Ss[(a + m + GH) * W + cc]);
            mx = b > mx ? b : mx;
          }
          flag = d.thr < 0.0 || mx > thr_bits;
          if (flag && a >= 0) mycount++;
          int i = DIR == 0 ? 0 : x0 + cc, j = DIR == 0 ? y0 + cc : (DIR == 1 ? 0 : y0), k = DIR == 2 ? 0 : z0;
          slot = islot(d, DIR, s, i, j, k);
          d.flag[DIR][slot] = flag;
        }
      }
      unsigned bal = __ballot_sync(0xffffffffu, flag);
      if (bal) {
        int lane = tid & 31;
        int leader = __ffs(bal) - 1;
        unsigned off = 0;
        if (lane == leader) off = atomicAdd(&d.scal->nlist[DIR], (unsigned)__popc(bal));
        off = __shfl_sync(0xffffffffu, off, leader);
        if (flag) d.wlist[DIR][off + __popc(bal & ((1u << lane) - 1u))] = (unsigned)slot;
      }
    }
    for (int o = 16; o > 0; o >>= 1) mycount += __shfl_xor_sync(0xffffffffu, mycount, o);
    if ((tid & 31) == 0 && mycount) atomicAdd(&d.scal->wcount, mycount);
  }
  __syncthreads();

  // ---- 3. central flux difference of the thread's point -> RHS ----
  int a, cc;
  if (DIR == 0) { a = tid % L; cc = tid / L; }
  else { cc = tid % W; a = tid / W; }
  if ((c0 + cc < nac) && (s0 + a < n)) {
    const double c1[4] = {0.0, 0.5 * 0.75, 0.5 * -0.15, 0.5 * (1.0 / 60.0)};
    const double c2[4] = {0.0, 0.25 * 0.75, 0.25 * -0.15, 0.25 * (1.0 / 60.0)};
    double D[5];
    int at = (a + 3) * W + cc;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      double acc = 0.0;
#pragma unroll
      for (int l = 1; l <= 3; ++l) {
        const double *T = TP + ((l - 1) * 5 + f) * ST;
        acc = fma(f == 0 ? c1[l] : c2[l], T[at] - T[at - l * W], acc);
      }
      D[f] = acc;
    }
    const double *Sp = S + F_P * SF;
    int ap = (a + GH) * W + cc;
    double dp = 0.0;
#pragma unroll
    for (int l = 1; l <= 3; ++l) dp = fma(kA[l], Sp[ap + l * W] - Sp[ap - l * W], dp);
    D[1 + DIR] += dp;
    int i = DIR == 0 ? x0 + a : x0 + cc;
    int j = DIR == 0 ? y0 + cc : (DIR == 1 ? y0 + a : y0);
    int k = DIR == 2 ? z0 + a : z0;
    double scale = DIR == 0 ? d.idx : (DIR == 1 ? __ldg(d.eta_y + j) : d.idz);
    long long q = ((long long)k * d.ny + j) * d.nx + i;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      double *o = d.fl + f * d.n + q;
      double prev = accumulate ? *o : 0.0;
      *o = fma(-scale, D[f], prev);
    }
  }
}

// ------------------------------------------------------------------ WENO
// Reconstruction at i+1/2 from 2r-1 values g[0..2r-2] centred on g[r-1]:
// Jiang & Shu (r=3), Balsara & Shu (r=4), alpha_k = d_k/(eps+beta_k)^2;
// the normalisation sum alpha_k q_k / sum alpha_k is evaluated with one
// division by multiplying through by prod_k (eps+beta_k)^2.
__device__ __forceinline__ double weno5(const double *g) {
  const double eps = 1e-6;
  double q0 = (2.0 * g[0] - 7.0 * g[1] + 11.0 * g[2]) * (1.0 / 6.0);
  double q1 = (-g[1] + 5.0 * g[2] + 2.0 * g[3]) * (1.0 / 6.0);
  double q2 = (2.0 * g[2] + 5.0 * g[3] - g[4]) * (1.0 / 6.0);
  double t, b0, b1, b2;
  t = g[0] - 2.0 * g[1] + g[2]; b0 = (13.0 / 12.0) * t * t;
  t = g[0] - 4.0 * g[1] + 3.0 * g[2]; b0 += 0.25 * t * t;
  t = g[1] - 2.0 * g[2] + g[3]; b1 = (13.0 / 12.0) * t * t;
  t = g[1] - g[3]; b1 += 0.25 * t * t;
  t = g[2] - 2.0 * g[3] + g[4]; b2 = (13.0 / 12.0) * t * t;
  t = 3.0 * g[2] - 4.0 * g[3] + g[4]; b2 += 0.25 * t * t;
  double s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
  s0 *= s0; s1 *= s1; s2 *= s2;
  double a0 = 0.1 * s1 * s2, a1 = 0.6 * s0 * s2, a2 = 0.3 * s0 * s1;
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

__device__ __forceinline__ double weno7(const double *g) {
  const double eps = 1e-6;
  double q0 = (-3.0 * g[0] + 13.0 * g[1] - 23.0 * g[2] + 25.0 * g[3]) * (1.0 / 12.0);
  double q1 = (g[1] - 5.0 * g[2] + 13.0 * g[3] + 3.0 * g[4]) * (1.0 / 12.0);
  double q2 = (-g[2] + 7.0 * g[3] + 7.0 * g[4] - g[5]) * (1.0 / 12.0);
  double q3 = (3.0 * g[3] + 13.0 * g[4] - 5.0 * g[5] + g[6]) * (1.0 / 12.0);
  // smoothness indicators: 240 x the Jiang-Shu measure as sums of squares
  // of the undivided differences of each 4-point substencil
  double bk[4];
  const double c10[4] = {5.0 / 2.0, 3.0 / 2.0, 1.0 / 2.0, -1.0 / 2.0};
  const double c11[4] = {11.0 / 6.0, 1.0 / 3.0, -1.0 / 6.0, 1.0 / 3.0};
  const double c2[4] = {2.0, 1.0, 0.0, -1.0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double e1 = g[k + 1] - g[k];
    double e2 = g[k + 2] - 2.0 * g[k + 1] + g[k];
    double e3 = g[k + 3] - 3.0 * g[k + 2] + 3.0 * g[k + 1] - g[k];
    double t1 = e1 + c10[k] * e2 + c11[k] * e3;
    double t2 = e2 + c2[k] * e3;
    bk[k] = 240.0 * t1 * t1 + 260.0 * t2 * t2 + (781.0 / 3.0) * e3 * e3;
  }
  double s0 = eps + bk[0], s1 = eps + bk[1], s2 = eps + bk[2], s3 = eps + bk[3];
  s0 *= s0; s1 *= s1; s2 *= s2; s3 *= s3;
  double p01 = s0 * s1, p23 = s2 * s3;
  double a0 = (1.0 / 35.0) * s1 * p23, a1 = (12.0 / 35.0) * s0 * p23;
  double a2 = (18.0 / 35.0) * p01 * s3, a3 = (4.0 / 35.0) * p01 * s2;
  return (a0 * q0 + a1 * q1 + a2 * q2 + a3 * q3) / (a0 + a1 + a2 + a3);
}

template <int WR>
__device__ __forceinline__ double weno_rec(const double *g) {
  if constexpr (WR == 3) return weno5(g);
  else return weno7(g);
}

// F_weno - F_central at every listed interface of direction DIR.
//
// In the frame (normal n, tangents t1, t2) of the interface, with the Roe
// state (u_n, u_1, u_2, H~, c~), b = gamma-1, h2 = 1/(2 c~^2), the left
// eigenvector rows applied to W = (rho, m_n, m_1, m_2, E) are
//   l_0 W = A + B,  l_4 W = A - B,  l_1 W = rho - 2A,
//   l_2 W = m_1 - u_1 rho,  l_3 W = m_2 - u_2 rho,
//   A = h2 b (q~^2/2 rho - u_n m_n - u_1 m_1 - u_2 m_2 + E),
//   B = h2 c~ (u_n rho - m_n),
// and, with the point's flux F = u_n W + p (0, 1, 0, 0, u_n),
//   l_e F = u_n (l_e W) + p (l_e[1] + l_e[4] u_n),
// i.e. + PA - PB, + PA + PB, - 2 PA, 0, 0 for e = 0, 4, 1, 2, 3 with
// PA = p h2 b (u_n - u~_n), PB = p h2 c~.  Lax-Friedrichs: each field's
// dissipation is the largest |eigenvalue| (u_n - c, u_n, u_n + c) over the
// stencil points.  The result goes back with the right eigenvectors.
template <int DIR, int WR>
__global__ void __launch_bounds__(128) k_weno(Dev d) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int NP = 2 * WR;  // stencil points s-WR+1 .. s+WR
  const unsigned cnt = d.scal->nlist[DIR];
  const double *vel[3] = {d.u, d.v, d.ww};
  const double gam = d.gamma, bq = gam - 1.0;
  for (unsigned e0 = blockIdx.x * blockDim.x + threadIdx.x; e0 < cnt; e0 += gridDim.x * blockDim.x) {
    const long long slot = d.wlist[DIR][e0];
    int i = 0, j = 0, k = 0, s;
    if (DIR == 0) {
      long long t = slot / (d.nx + 1);
      s = (int)(slot - t * (d.nx + 1)) - 1;
      j = (int)(t % d.ny);
      k = (int)(t / d.ny);
      i = s;
    } else if (DIR == 1) {
      long long t = slot / d.nx;
      i = (int)(slot - t * d.nx);
      s = (int)(t % (d.ny + 1)) - 1;
      k = (int)(t / (d.ny + 1));
      j = s;
    } else {
      long long t = slot / d.nx;
      i = (int)(slot - t * d.nx);
      j = (int)(t % d.ny);
      s = (int)(t / d.ny) - 1;
      k = s;
    }
    const long long stride = DIR == 0 ? 1 : (DIR == 1 ? d.sy : d.sz);
    const long long p0 = pidx(d, i, j, k);  // point s of the interface s+1/2

    // --- central split-form flux at this interface
    double FC[5] = {0, 0, 0, 0, 0}, fp = 0.0;
#pragma unroll
    for (int l = 1; l <= 3; ++l) {
      double acc[5] = {0, 0, 0, 0, 0}, ps = 0.0;
#pragma unroll
      for (int m = 0; m < l; ++m) {
        long long a = p0 - m * stride, b = p0 + (l - m) * stride;
        double sr = __ldg(d.rho + a) + __ldg(d.rho + b);
        double su = __ldg(d.u + a) + __ldg(d.u + b), sv = __ldg(d.v + a) + __ldg(d.v + b);
        double sw = __ldg(d.ww + a) + __ldg(d.ww + b);
        double sh = __ldg(d.H + a) + __ldg(d.H + b);
        double sun = DIR == 0 ? su : (DIR == 1 ? sv : sw);
        double mm = sr * sun;
        acc[0] += mm;
        acc[1] += mm * su;
        acc[2] += mm * sv;
        acc[3] += mm * sw;
        acc[4] += mm * sh;
        ps += __ldg(d.p + a) + __ldg(d.p + b);
      }
      double al = kA[l];
      FC[0] += 0.5 * al * acc[0];
#pragma unroll
      for (int f = 1; f < 5; ++f) FC[f] += 0.25 * al * acc[f];
      fp += al * ps;
    }
    FC[1 + DIR] += fp;

    // --- Roe average of the two interface states
    const long long ia = p0, ib = p0 + stride;
    double ra = sqrt(__ldg(d.rho + ia)), rb = sqrt(__ldg(d.rho + ib));
    double inv = 1.0 / (ra + rb);
    double un = (ra * __ldg(vel[DIR] + ia) + rb * __ldg(vel[DIR] + ib)) * inv;
    double ut1 = (ra * __ldg(vel[T1] + ia) + rb * __ldg(vel[T1] + ib)) * inv;
    double ut2 = (ra * __ldg(vel[T2] + ia) + rb * __ldg(vel[T2] + ib)) * inv;
    double Ht = (ra * __ldg(d.H + ia) + rb * __ldg(d.H + ib)) * inv;
    double q2 = un * un + ut1 * ut1 + ut2 * ut2;
    double c2 = bq * (Ht - 0.5 * q2);
    double cs = sqrt(c2);
    double h2 = 0.5 / c2;
    double hb = h2 * bq, hc = h2 * cs;

    // --- per stencil point: l_e W and l_e F for the five fields
    double V[5][NP], G[5][NP];
    double al0 = 0.0, al1 = 0.0, al4 = 0.0;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      long long q = p0 + (m - WR + 1) * stride;
      double r = __ldg(d.rho + q), unm = __ldg(vel[DIR] + q);
      double u1 = __ldg(vel[T1] + q), u2 = __ldg(vel[T2] + q);
      double pm = __ldg(d.p + q), hm = __ldg(d.H + q);
      double cm = sqrt(d.gR * __ldg(d.T + q));
      double mn = r * unm, m1 = r * u1, m2 = r * u2, E = r * hm - pm;
      double A = hb * (0.5 * q2 * r - un * mn - ut1 * m1 - ut2 * m2 + E);
      double B = hc * (un * r - mn);
      double PA = pm * hb * (unm - un), PB = pm * hc;
      V[0][m] = A + B;
      V[1][m] = r - 2.0 * A;
      V[2][m] = m1 - ut1 * r;
      V[3][m] = m2 - ut2 * r;
      V[4][m] = A - B;
      G[0][m] = unm * V[0][m] + PA - PB;
      G[1][m] = unm * V[1][m] - 2.0 * PA;
      G[2][m] = unm * V[2][m];
      G[3][m] = unm * V[3][m];
      G[4][m] = unm * V[4][m] + PA + PB;
      al0 = fmax(al0, fabs(unm - cm));
      al1 = fmax(al1, fabs(unm));
      al4 = fmax(al4, fabs(unm + cm));
    }
    double gh[5];
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      double alpha = e == 0 ? al0 : (e == 4 ? al4 : al1);
      double gp[2 * WR - 1], gmn[2 * WR - 1];
#pragma unroll
      for (int m = 0; m < 2 * WR - 1; ++m) {
        gp[m] = 0.5 * (G[e][m] + alpha * V[e][m]);
        int mm = NP - 1 - m;
        gmn[m] = 0.5 * (G[e][mm] - alpha * V[e][mm]);
      }
      gh[e] = weno_rec<WR>(gp) + weno_rec<WR>(gmn);
    }
    // --- back to conserved fluxes with the right eigenvectors
    double s014 = gh[0] + gh[1] + gh[4];
    double dn = gh[4] - gh[0];
    double Fr[5];
    Fr[0] = s014;
    Fr[1 + DIR] = un * s014 + cs * dn;
    Fr[1 + T1] = ut1 * s014 + gh[2];
    Fr[1 + T2] = ut2 * s014 + gh[3];
    Fr[4] = Ht * (gh[0] + gh[4]) + un * cs * dn + 0.5 * q2 * gh[1] + ut1 * gh[2] + ut2 * gh[3];
    const long long ns = d.nslot[DIR];
#pragma unroll
    for (int f = 0; f < 5; ++f) d.dF[DIR][f * ns + slot] = Fr[f] - FC[f];
  }
}

template <int DIR>
constexpr size_t flux_smem() {
  constexpr int L = Tile<DIR>::L, W = Tile<DIR>::W;
  return sizeof(double) * ((size_t)NF * (L + 2 * GH) * W + (size_t)15 * (L + 3) * W);
}

template <int DIR, int WR>
cudaError_t launch_one(const Dev &d, int accumulate, cudaStream_t st) {
  constexpr int L = Tile<DIR>::L, W = Tile<DIR>::W;
  dim3 grid;
  if (DIR == 0) grid = dim3((d.nx + L - 1) / L, (d.ny + W - 1) / W, d.nz);
  if (DIR == 1) grid = dim3((d.nx + W - 1) / W, (d.ny + L - 1) / L, d.nz);
  if (DIR == 2) grid = dim3((d.nx + W - 1) / W, (d.nz + L - 1) / L, d.ny);
  k_flux<DIR, WR><<<grid, NTHREADS, flux_smem<DIR>(), st>>>(d, accumulate);
  return cudaGetLastError();
}

template <int DIR, int WR>
cudaError_t launch_weno_one(const Dev &d, cudaStream_t st) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long need = (d.nslot[DIR] + 127) / 128;
  long long cap = 8LL * sms;
  unsigned nb = (unsigned)(need < cap ? need : cap);
  if (nb == 0) nb = 1;
  k_weno<DIR, WR><<<nb, 128, 0, st>>>(d);
  return cudaGetLastError();
}

template <int DIR, int WR>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_flux<DIR, WR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)flux_smem<DIR>());
}

}  // namespace

cudaError_t flux_set_attributes() {
  cudaError_t e = cudaSuccess, r;
#define S2_ATTR(D, R) if ((r = set_attr<D, R>()) != cudaSuccess) e = r;
  S2_ATTR(0, 0) S2_ATTR(1, 0) S2_ATTR(2, 0)
  S2_ATTR(0, 3) S2_ATTR(1, 3) S2_ATTR(2, 3)
  S2_ATTR(0, 4) S2_ATTR(1, 4) S2_ATTR(2, 4)
#undef S2_ATTR
  return e;
}

cudaError_t launch_flux(const Dev &d, int dir, int accumulate, cudaStream_t st) {
  int wr = d.weno == 5 ? 3 : (d.weno == 7 ? 4 : 0);
  switch (dir * 10 + wr) {
    case 0: return launch_one<0, 0>(d, accumulate, st);
    case 3: return launch_one<0, 3>(d, accumulate, st);
    case 4: return launch_one<0, 4>(d, accumulate, st);
    case 10: return launch_one<1, 0>(d, accumulate, st);
    case 13: return launch_one<1, 3>(d, accumulate, st);
    case 14: return launch_one<1, 4>(d, accumulate, st);
    case 20: return launch_one<2, 0>(d, accumulate, st);
    case 23: return launch_one<2, 3>(d, accumulate, st);
    case 24: return launch_one<2, 4>(d, accumulate, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_weno(const Dev &d, int dir, cudaStream_t st) {
  int wr = d.weno == 5 ? 3 : (d.weno == 7 ? 4 : 0);
  switch (dir * 10 + wr) {
    case 3: return launch_weno_one<0, 3>(d, st);
    case 4: return launch_weno_one<0, 4>(d, st);
    case 13: return launch_weno_one<1, 3>(d, st);
    case 14: return launch_weno_one<1, 4>(d, st);
    case 23: return launch_weno_one<2, 3>(d, st);
    case 24: return launch_weno_one<2, 4>(d, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace s2
