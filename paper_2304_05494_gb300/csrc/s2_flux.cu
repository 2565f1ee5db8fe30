// Convective flux kernels: one per direction, hybrid central / WENO.
//
// Paper Sec. 2: the convective terms use the energy-preserving split
// (skew-symmetric) form written as numerical fluxes (Pirozzoli, JCP 2010)
// in smooth regions and, at interfaces flagged by the Ducros-type sensor, a
// WENO reconstruction of characteristic fluxes (Lax-Friedrichs splitting)
// projected back on the right eigenvectors.  These are the euler_{x,y,z}
// kernels of Table 2; the paper's transposition kernel for x is not needed
// because every direction stages its pencils through shared memory.
//
// One CTA owns a tile of L points along the flux direction times W pencils.
//  1. the primitives of the tile plus GH ghost points each side go to
//     shared memory (coalesced: the x-contiguous index runs fastest);
//  2. per point a the "pair fluxes" T_l(a) of the pairs (a, a+l), l=1..3,
//     are formed once: m = (rho_a+rho_b)(un_a+un_b), T = m (1, su, sv, sw,
//     sH) with s. the pair sums;
//  3. the central flux difference of point a is
//        D(a) = sum_l c_l [T_l(a) - T_l(a-l)] + sum_l a_l (p_{a+l} - p_{a-l}),
//     equal to F_{a+1/2} - F_{a-1/2} of the split-form interface flux;
//  4. flagged interfaces are compacted in shared memory; the whole CTA
//     then evaluates F_weno - F_central for the compacted list (no warp
//     divergence between central and WENO work) into shared slots;
//  5. every point adds its two interface corrections in a fixed order
//     (deterministic) and accumulates -scale * D into the RHS.
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
// shared field slots
enum { F_RHO = 0, F_U, F_V, F_W, F_H, F_P, F_C, F_S, NF };

// WENO reconstruction at i+1/2 from 2r-1 values g[0..2r-2] centred on g[r-1],
// Jiang-Shu (r=3) / Balsara-Shu (r=4) with alpha_k = d_k/(eps+beta_k)^2;
// the normalisation sum_k alpha_k q_k / sum_k alpha_k is evaluated with a
// single division by multiplying through by prod_k (eps+beta_k)^2.
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
  double b0 = bk[0], b1 = bk[1], b2 = bk[2], b3 = bk[3];
  double s0 = eps + b0, s1 = eps + b1, s2 = eps + b2, s3 = eps + b3;
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

// F_weno - F_central at the interface between tile positions ae and ae+1
// (indices into the shared arrays, stride W between positions).
// Output in the original component order.
template <int DIR, int WR, int STRIDE>
__device__ void weno_minus_central(const double *__restrict__ S, int sfield, int base, double gam,
                                   double *dF) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int NP = 2 * WR;  // stencil points base-WR+1 .. base+WR
  const double *rho = S + F_RHO * sfield;
  const double *vel[3] = {S + F_U * sfield, S + F_V * sfield, S + F_W * sfield};
  const double *Hh = S + F_H * sfield;
  const double *pp = S + F_P * sfield;
  const double *cc = S + F_C * sfield;
  // --- central split-form flux at this interface (same as the central pass)
  double FC[5] = {0, 0, 0, 0, 0};
  double fp = 0.0;
#pragma unroll
  for (int l = 1; l <= 3; ++l) {
    double acc[5] = {0, 0, 0, 0, 0}, ps = 0.0;
#pragma unroll
    for (int m = 0; m < l; ++m) {
      int a = base + (0 - m) * STRIDE, b = base + (l - m) * STRIDE;
      double sr = rho[a] + rho[b];
      double su = vel[0][a] + vel[0][b], sv = vel[1][a] + vel[1][b], sw = vel[2][a] + vel[2][b];
      double sh = Hh[a] + Hh[b];
      double sun = DIR == 0 ? su : (DIR == 1 ? sv : sw);
      double mm = sr * sun;
      acc[0] += mm;
      acc[1] += mm * su;
      acc[2] += mm * sv;
      acc[3] += mm * sw;
      acc[4] += mm * sh;
      ps += pp[a] + pp[b];
    }
    double al = kA[l];
    FC[0] += 0.5 * al * acc[0];
#pragma unroll
    for (int f = 1; f < 5; ++f) FC[f] += 0.25 * al * acc[f];
    fp += al * ps;
  }
  FC[1 + DIR] += fp;

  // --- Roe average of the two interface states
  const int ia = base, ib = base + STRIDE;
  double ra = sqrt(rho[ia]), rb = sqrt(rho[ib]);
  double inv = 1.0 / (ra + rb);
  double un = (ra * vel[DIR][ia] + rb * vel[DIR][ib]) * inv;
  double ut1 = (ra * vel[T1][ia] + rb * vel[T1][ib]) * inv;
  double ut2 = (ra * vel[T2][ia] + rb * vel[T2][ib]) * inv;
  double Ht = (ra * Hh[ia] + rb * Hh[ib]) * inv;
  double bq = gam - 1.0;
  double q2 = un * un + ut1 * ut1 + ut2 * ut2;
  double c2 = bq * (Ht - 0.5 * q2);
  double cs = sqrt(c2);
  double ic2 = 1.0 / c2;
  double h2 = 0.5 * ic2;

  // stencil states in the rotated frame (normal, t1, t2)
  double Wr[NP], Wn[NP], Wt1[NP], Wt2[NP], We[NP], unm[NP], pm[NP], cm[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    int q = base + (m - WR + 1) * STRIDE;
    double r = rho[q];
    unm[m] = vel[DIR][q];
    Wr[m] = r;
    Wn[m] = r * unm[m];
    Wt1[m] = r * vel[T1][q];
    Wt2[m] = r * vel[T2][q];
    pm[m] = pp[q];
    We[m] = r * Hh[q] - pm[m];
    cm[m] = cc[q];
  }

  double gh[5];
#pragma unroll
  for (int e = 0; e < 5; ++e) {
    // left eigenvector row e (rotated frame)
    double l0, l1, l2, l3, l4;
    if (e == 0) {
      l0 = h2 * (0.5 * bq * q2 + un * cs); l1 = h2 * (-bq * un - cs);
      l2 = h2 * (-bq * ut1); l3 = h2 * (-bq * ut2); l4 = h2 * bq;
    } else if (e == 1) {
      l0 = 1.0 - 0.5 * bq * q2 * ic2; l1 = bq * un * ic2; l2 = bq * ut1 * ic2;
      l3 = bq * ut2 * ic2; l4 = -bq * ic2;
    } else if (e == 2) {
      l0 = -ut1; l1 = 0.0; l2 = 1.0; l3 = 0.0; l4 = 0.0;
    } else if (e == 3) {
      l0 = -ut2; l1 = 0.0; l2 = 0.0; l3 = 1.0; l4 = 0.0;
    } else {
      l0 = h2 * (0.5 * bq * q2 - un * cs); l1 = h2 * (-bq * un + cs);
      l2 = h2 * (-bq * ut1); l3 = h2 * (-bq * ut2); l4 = h2 * bq;
    }
    double vv[NP], gg[NP], alpha = 0.0;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      double v;
      if (e == 2) v = Wt1[m] - ut1 * Wr[m];
      else if (e == 3) v = Wt2[m] - ut2 * Wr[m];
      else v = l0 * Wr[m] + l1 * Wn[m] + l2 * Wt1[m] + l3 * Wt2[m] + l4 * We[m];
      vv[m] = v;
      // physical flux F = u_n W + p (0, 1, 0, 0, u_n)  ->  L_e F
      if (e == 2 || e == 3) gg[m] = unm[m] * v;
      else gg[m] = unm[m] * v + pm[m] * (l1 + l4 * unm[m]);
      double lam = e == 0 ? unm[m] - cm[m] : (e == 4 ? unm[m] + cm[m] : unm[m]);
      alpha = fmax(alpha, fabs(lam));
    }
    double gp[2 * WR - 1], gmn[2 * WR - 1];
#pragma unroll
    for (int m = 0; m < 2 * WR - 1; ++m) {
      gp[m] = 0.5 * (gg[m] + alpha * vv[m]);
      int mm = NP - 1 - m;
      gmn[m] = 0.5 * (gg[mm] - alpha * vv[mm]);
    }
    gh[e] = weno_rec<WR>(gp) + weno_rec<WR>(gmn);
  }
  // back to conserved fluxes with the right eigenvectors
  double s014 = gh[0] + gh[1] + gh[4];
  double dn = gh[4] - gh[0];
  double Fr[5];
  Fr[0] = s014;
  Fr[1 + DIR] = un * s014 + cs * dn;
  Fr[1 + T1] = ut1 * s014 + gh[2];
  Fr[1 + T2] = ut2 * s014 + gh[3];
  Fr[4] = Ht * (gh[0] + gh[4]) + un * cs * dn + 0.5 * q2 * gh[1] + ut1 * gh[2] + ut2 * gh[3];
#pragma unroll
  for (int f = 0; f < 5; ++f) dF[f] = Fr[f] - FC[f];
}

template <int DIR, int WR>
__global__ void __launch_bounds__(NTHREADS, 1) k_flux(Dev d, int accumulate, int record) {
  constexpr int L = Tile<DIR>::L, W = Tile<DIR>::W;
  constexpr int LE = L + 2 * GH;       // extended positions per pencil
  constexpr int SF = LE * W;           // doubles per shared field
  constexpr int LT = L + 3;            // pair-flux positions a = -3 .. L-1
  constexpr int ST = LT * W;           // doubles per pair-flux slot
  constexpr int NFLD = WR > 0 ? NF : F_C;  // fields staged (c, sensor only for WENO)
  extern __shared__ double smem[];
  double *S = smem;                    // [NF][LE][W]
  double *TP = smem + NF * SF;         // [3][5][LT][W]; reused for WENO corrections
  __shared__ unsigned char fl[(L + 1) * W];
  __shared__ unsigned short list[(L + 1) * W];
  __shared__ int nlist;

  const int tid = threadIdx.x;
  const int n = DIR == 0 ? d.nx : (DIR == 1 ? d.ny : d.nz);
  int x0 = 0, y0 = 0, z0 = 0;
  if (DIR == 0) { x0 = blockIdx.x * L; y0 = blockIdx.y * W; z0 = blockIdx.z; }
  if (DIR == 1) { x0 = blockIdx.x * W; y0 = blockIdx.y * L; z0 = blockIdx.z; }
  if (DIR == 2) { x0 = blockIdx.x * W; z0 = blockIdx.y * L; y0 = blockIdx.z; }
  const int s0 = DIR == 0 ? x0 : (DIR == 1 ? y0 : z0);
  const int nac = DIR == 0 ? d.ny : d.nx;   // extent across
  const int c0 = DIR == 0 ? y0 : x0;
  if (tid == 0) nlist = 0;

  const double *src[NF] = {d.rho, d.u, d.v, d.ww, d.H, d.p, d.c, d.sens};

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

  // ---- 2. pair fluxes T_l(a), a = -3 .. L-1; flags of interfaces a+1/2 ----
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
  unsigned long long mycount = 0;
  if constexpr (WR > 0) {
    const double *Ss = S + F_S * SF;
    const int ni = (L + 1) * W;
    for (int base = 0; base < ni; base += NTHREADS) {
      int idx = base + tid;
      bool flag = false;
      int a = 0, cc = 0;
      if (idx < ni) {
        a = idx / W - 1;  // interface a+1/2, a in -1 .. L-1
        cc = idx % W;
        int s = s0 + a;
        if (c0 + cc < nac && s >= -1 && s <= n - 1) {
          double mx = 0.0;
#pragma unroll
          for (int m = -WR + 1; m <= WR; ++m) mx = fmax(mx, Ss[(a + m + GH) * W + cc]);
          flag = mx > d.thr;
          if (flag && a >= 0) mycount++;
        }
        fl[idx] = flag;
        if (record && c0 + cc < nac && s >= -1 && s <= n - 1) {
          long long slot;
          if (DIR == 0) slot = ((long long)z0 * d.ny + (y0 + cc)) * (d.nx + 1) + (s + 1);
          else if (DIR == 1) slot = ((long long)z0 * (d.ny + 1) + (s + 1)) * d.nx + (x0 + cc);
          else slot = ((long long)(s + 1) * d.ny + y0) * d.nx + (x0 + cc);
          d.flagrec[DIR][slot] = flag;
        }
      }
      unsigned bal = __ballot_sync(0xffffffffu, flag);
      if (bal) {
        int lane = tid & 31;
        int leader = __ffs(bal) - 1;
        int off = 0;
        if (lane == leader) off = atomicAdd(&nlist, __popc(bal));
        off = __shfl_sync(0xffffffffu, off, leader);
        if (flag) list[off + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)idx;
      }
    }
  }
  __syncthreads();

  // ---- 3. central flux difference of the thread's point ----
  int a, cc;
  if (DIR == 0) { a = tid % L; cc = tid / L; }
  else { cc = tid % W; a = tid / W; }
  const bool active = (c0 + cc < nac) && (s0 + a < n);
  double D[5];
  {
    const double c1[4] = {0.0, 0.5 * 0.75, 0.5 * -0.15, 0.5 * (1.0 / 60.0)};
    const double c2[4] = {0.0, 0.25 * 0.75, 0.25 * -0.15, 0.25 * (1.0 / 60.0)};
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
  }

  // ---- 4. WENO corrections for the compacted flagged interfaces ----
  if constexpr (WR > 0) {
    __syncthreads();  // everyone done reading TP; reuse it for corrections
    const int cnt = nlist;
    double *DF = TP;  // [5][(L+1)*W]
    constexpr int NI = (L + 1) * W;
    for (int e = tid; e < cnt; e += NTHREADS) {
      int idx = list[e];
      int ai = idx / W - 1, ci = idx % W;
      double dF[5];
      weno_minus_central<DIR, WR, W>(S, SF, (ai + GH) * W + ci, d.gamma, dF);
#pragma unroll
      for (int f = 0; f < 5; ++f) DF[f * NI + idx] = dF[f];
    }
    __syncthreads();
    if (active) {
      int ir = (a + 1) * W + cc, il = a * W + cc;  // interfaces a+1/2 and a-1/2
      if (fl[ir]) {
#pragma unroll
        for (int f = 0; f < 5; ++f) D[f] += DF[f * NI + ir];
      }
      if (fl[il]) {
#pragma unroll
        for (int f = 0; f < 5; ++f) D[f] -= DF[f * NI + il];
      }
    }
    // flagged-interface count for the monitoring fraction
    for (int o = 16; o > 0; o >>= 1) mycount += __shfl_xor_sync(0xffffffffu, mycount, o);
    if ((tid & 31) == 0 && mycount) atomicAdd(&d.scal->wcount, mycount);
  }

  // ---- 5. accumulate -scale * D into the RHS ----
  if (active) {
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

template <int DIR, int WR>
constexpr size_t flux_smem() {
  constexpr int L = Tile<DIR>::L, W = Tile<DIR>::W;
  return sizeof(double) * ((size_t)NF * (L + 2 * GH) * W + (size_t)15 * (L + 3) * W);
}

template <int DIR, int WR>
cudaError_t launch_one(const Dev &d, int accumulate, int record, cudaStream_t st) {
  constexpr int L = Tile<DIR>::L, W = Tile<DIR>::W;
  dim3 grid;
  if (DIR == 0) grid = dim3((d.nx + L - 1) / L, (d.ny + W - 1) / W, d.nz);
  if (DIR == 1) grid = dim3((d.nx + W - 1) / W, (d.ny + L - 1) / L, d.nz);
  if (DIR == 2) grid = dim3((d.nx + W - 1) / W, (d.nz + L - 1) / L, d.ny);
  k_flux<DIR, WR><<<grid, NTHREADS, flux_smem<DIR, WR>(), st>>>(d, accumulate, record);
  return cudaGetLastError();
}

template <int DIR, int WR>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_flux<DIR, WR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)flux_smem<DIR, WR>());
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

cudaError_t launch_flux(const Dev &d, int dir, int accumulate, int record, cudaStream_t st) {
  int wr = d.weno == 5 ? 3 : (d.weno == 7 ? 4 : 0);
  switch (dir * 10 + wr) {
    case 0: return launch_one<0, 0>(d, accumulate, record, st);
    case 3: return launch_one<0, 3>(d, accumulate, record, st);
    case 4: return launch_one<0, 4>(d, accumulate, record, st);
    case 10: return launch_one<1, 0>(d, accumulate, record, st);
    case 13: return launch_one<1, 3>(d, accumulate, record, st);
    case 14: return launch_one<1, 4>(d, accumulate, record, st);
    case 20: return launch_one<2, 0>(d, accumulate, record, st);
    case 23: return launch_one<2, 3>(d, accumulate, record, st);
    case 24: return launch_one<2, 4>(d, accumulate, record, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace s2
