// Internal declarations shared by the translation units of libs2.so.
// Not part of the public ABI (include/s2.h).
#pragma once
#include <cuda.h>  // CUtensorMap (the tensor-memory-access descriptor type)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/s2.h"

namespace s2 {

// Ghost width of every padded field (WENO7 needs 4; central-6, WENO5 and
// the 6th-order derivatives need 3).
constexpr int GH = 4;
constexpr int NV = 5;

// Device-side scalars of one solver.
struct Scal {
  double dt;              // current time step
  double t;               // simulated time
  double force;           // body force of the last RHS evaluation
  double dt_max_rate;     // last max spectral radius
  unsigned long long wcount;  // flagged interfaces of the last RHS evaluation
  unsigned int nlist[4];  // per-direction lengths of the flagged-interface lists
  int status;             // OR of the ERR_* bits met (0: none)
  int pad;
  long long nstep;        // completed RK3 steps (decides the dt recomputation on the device)
  double red[8];          // results of the last stats reduction
};

// Error bits kernels OR into Scal::status (mapped on the host to
// S2_ENONFINITE, S2_ETIMEOUT and S2_EBOUNDS).
constexpr int ERR_NONFINITE = 1;
constexpr int ERR_TIMEOUT = 2;  // a bounded wait on an asynchronous copy gave up
constexpr int ERR_BOUNDS = 4;   // an index left its array (checked build)

// Scheme constants in the arithmetic type R of a kernel (double for the
// FP64 path, float for the flux arithmetic of the mixed path).
template <class R>
struct Consts {
  R ax[5], az[5];          // a_l/dx, a_l/dz (first derivative of the viscous order, l = 1..4)
  R bx[5], bz[5];          // b_l/dx^2, b_l/dz^2 (second derivative, l = 0..4)
  R acen[5];               // a_l of the central (convective) order, l = 1..4
  R idx, idz;              // 1/dx, 1/dz
  R idx2, idz2;            // 2/dx, 2/dz
  R R_gas, cp, gamma, gR, icv, visc_exp, inv_t_ref, t_wall, cp_over_pr, re, inv_re, thr;
  R thr2;                  // thr^2 (sensor test without a root)
  R b0xz;                  // b_0/dx^2 + b_0/dz^2 (x and z centre weights of the Laplacian)
  // thermally perfect gas (tp = 1): c_p(T) = sum_{l=-2..4} cpc[l+2] T^l;
  // dcc = (-2 c_-2, -c_-1, c_1, 2 c_2, 3 c_3, 4 c_4) for dc_p/dT;
  // ecf = (-c_-2, c_-1, c_0 - R, c_1/2, c_2/3, c_3/4, c_4/5) for e(T);
  // e1 = e(1), icv1 = 1/c_v(1) (the first Newton guess); inv_pr = 1/Pr
  int tp;
  R cpc[7], dcc[6], ecf[7];
  R e1, icv1, inv_pr;
};

// Division of 32-bit unsigned integers by a run-time constant d >= 1 as a
// multiply-high and shifts (Granlund & Montgomery, PLDI 1994, round-up
// method): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, and
// n / d = (t + ((n - t) >> 1)) >> (l - 1) with t = mulhi(m, n), exact for
// every n < 2^32.  Point and slot indices are split with it: on GB300 a
// 64-bit integer division goes through the double-precision unit, which
// the mixed path otherwise leaves idle and the FP64 path needs for its
// arithmetic.
struct FastDiv {
  unsigned d, m, l;
  __host__ void init(unsigned dv) {
    d = dv;
    l = 0;
    while ((1ull << l) < dv) ++l;
    m = (unsigned)(((1ull << 32) * ((1ull << l) - dv)) / dv + 1);
  }
  __host__ __device__ __forceinline__ unsigned div(unsigned n) const {
    if (l == 0) return n;
#ifdef __CUDA_ARCH__
    const unsigned t = __umulhi(m, n);
#else
    const unsigned t = (unsigned)(((unsigned long long)m * n) >> 32);
#endif
    return (t + ((n - t) >> 1)) >> (l - 1);
  }
};

// Everything a kernel needs, passed by value.
struct Dev {
  int nx, ny, nz;
  int px, py, pz;          // padded extents (x pitch rounded up)
  long long sy, sz;        // padded strides
  long long off0;          // padded offset of interior point (0,0,0)
  long long n;             // nx*ny*nz (< 2^31; slot counts < 2^32)
  long long np;            // px*py*pz: elements of a padded field
  long long nparts;        // elements of the reduction partials
  FastDiv fnx, fny, fnx1, fny1;  // divisions by nx, ny, nx+1, ny+1
  double dx, dz, idx, idz;  // spacings and their inverses
  double ax[5], az[5];     // a_l/dx, a_l/dz (first derivative, viscous order, l = 1..4)
  double bx[5], bz[5];     // b_l/dx^2, b_l/dz^2 (second derivative, viscous order, l = 0..4)
  int npc, npv;            // stencil pairs of the central and the viscous order (order / 2)
  int keep;                // central flux: 0 split form; n >= 1 KEEP-n; -1 KEEP with exact log means
  double R, cv, icv, cp, gamma, prandtl, re, visc_exp, inv_t_ref, t_wall, cp_over_pr;
  double inv_re;           // 1 / Re
  float visc_exp_f;        // omega in single precision (seed of the viscosity law)
  double gR;               // gamma R (c^2 = gamma R T)
  int mu_p, mu_q;          // visc_exp = mu_p/mu_q when rational with small terms, else mu_q = 0
  double mu_qm1, mu_qp1;   // mu_q - 1, mu_q + 1
  double thr;              // sensor threshold
  double cfl;
  int dt_every;            // recompute dt at steps that are multiples of this (cfl > 0)
  double vol_inv;          // 1 / sum(dV) / (dx dz) for the forcing
  int viscous, wall_y, weno, force;
  int mixed;               // 0: FP64 everywhere; 1: FP32 primitives and flux arithmetic, FP64 state
  int tile[3];             // flux tile variant per direction (0 default, 1 narrow)
  int flux_cps[3];         // single-precision flux grids, per direction: resident CTAs per SM to use (0: all that fit)
  int zs;                  // planes per CTA of the z-marching passes (mixed path)
  int weno_cps;            // WENO grids: CTAs per SM
  int nsm;                 // multiprocessors of the device
  unsigned long long wait_ns;  // limit of a kernel's wait for an asynchronous copy
  unsigned tx_extra;       // bytes a staging barrier expects beyond its copies (0; test hook)
  Consts<double> kd;
  Consts<float> kf;
  // state (FP64 in both modes; interior layout [v][k][j][i])
  double *w;
  // RHS accumulator and RK register (R), same layout
  void *fl, *fln;
  // primitives with ghosts (R)
  void *rho, *u, *v, *ww, *T, *p, *H;
  // auxiliary fields (R)
  void *mu;                // interior
  void *g;                 // 9 velocity gradients, interior, g[(3a+b)*n + q] = d u_a / d x_b
  void *div, *sens;        // padded; sens holds the sensor test theta > thr as 1 / 0
  // metrics (length ny): eta_y; a_l eta_y (4/j); b_l eta_y^2 (5/j); eta_yy/eta_y; 1/eta_y
  // (a_l, b_l of the viscous order; the metric itself uses the higher order)
  const double *eta_y, *ay, *by, *ry, *dvy;
  const float *eta_yf, *ayf, *byf, *ryf;  // the same in single precision
  Scal *scal;
  double *part;            // reduction partials
  // hybrid scheme, per direction: interface flags (n_d + 1 slots per
  // pencil), the compacted list of flagged slots and F_weno - F_central at
  // every listed slot (5 values, slot-major per component)
  unsigned char *flag[3];
  unsigned int *wlist[3];
  void *dF[3];             // R
  long long nslot[3];
};

// Block coordinates of a kernel body.  A launch for one box uses the CUDA
// grid's own (grid_blk); a batched launch, whose CTAs work on many boxes,
// gives each CTA its box-local coordinates (batch_enter), so the same body
// computes the same tiles either way.
struct Blk {
  unsigned x, y, z;     // block index
  unsigned nx, ny, nz;  // grid extent
};

__device__ __forceinline__ Blk grid_blk() {
  return Blk{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z};
}

// Batched launches (one launch for all boxes of a batch group): CTAs
// start .. start + gx gy gz - 1 of the launch form box b's own grid.  The
// table holds nbox + 1 entries; the last start is the launch's CTA count.
struct BoxGrid {
  unsigned start, gx, gy, gz;
};

struct BatchArgs {
  const Dev *dev;       // [nbox] parameters of the boxes (device memory)
  const BoxGrid *grid;  // [nbox + 1] this launch's work list
  int nbox;
};

// The box of this CTA (binary search of the work list) and its box-local
// block coordinates.
__device__ __forceinline__ int batch_locate(const BatchArgs &ba, Blk &B) {
  __shared__ int sbox;
  if (threadIdx.x == 0) {
    int lo = 0, hi = ba.nbox - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ba.grid[mid].start <= blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    sbox = lo;
  }
  __syncthreads();
  const int b = sbox;
  const BoxGrid g = ba.grid[b];
  unsigned l = blockIdx.x - g.start;
  B.nx = g.gx;
  B.ny = g.gy;
  B.nz = g.gz;
  B.x = l % g.gx;
  l /= g.gx;
  B.y = l % g.gy;
  B.z = l / g.gy;
  return b;
}

// The same, and the box's parameters copied to shared memory (sd).
__device__ __forceinline__ int batch_enter(const BatchArgs &ba, Dev &sd, Blk &B) {
  const int b = batch_locate(ba, B);
  static_assert(sizeof(Dev) % 8 == 0, "Dev is copied in 8-byte words");
  const unsigned long long *src = (const unsigned long long *)(ba.dev + b);
  unsigned long long *dst = (unsigned long long *)&sd;
  for (int i = threadIdx.x; i < (int)(sizeof(Dev) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return b;
}

// Opening of a batched kernel: the CTA's box (int BOX), its block
// coordinates (Blk BL) and its parameters (const Dev &D, a shared-memory
// copy of the table entry).
#define S2_BATCH_ENTER(BA, D, BL, BOX)        \
  __shared__ Dev D##_s;                       \
  Blk BL;                                     \
  const int BOX = batch_enter(BA, D##_s, BL); \
  const Dev &D = D##_s;                       \
  (void)BOX

// Typed views of the fields of a Dev in the arithmetic type R.
template <class R>
struct View {
  R *fl, *fln, *rho, *u, *v, *ww, *T, *p, *H, *mu, *g, *div, *sens;
  R *dF[3];
  const R *eta_y, *ay, *by, *ry;
};

template <class R>
__host__ __device__ inline const Consts<R> &consts(const Dev &d);
template <>
__host__ __device__ inline const Consts<double> &consts<double>(const Dev &d) {
  return d.kd;
}
template <>
__host__ __device__ inline const Consts<float> &consts<float>(const Dev &d) {
  return d.kf;
}

template <class R>
__host__ __device__ inline View<R> view(const Dev &d) {
  View<R> v;
  v.fl = (R *)d.fl;
  v.fln = (R *)d.fln;
  v.rho = (R *)d.rho;
  v.u = (R *)d.u;
  v.v = (R *)d.v;
  v.ww = (R *)d.ww;
  v.T = (R *)d.T;
  v.p = (R *)d.p;
  v.H = (R *)d.H;
  v.mu = (R *)d.mu;
  v.g = (R *)d.g;
  v.div = (R *)d.div;
  v.sens = (R *)d.sens;
  for (int a = 0; a < 3; ++a) v.dF[a] = (R *)d.dF[a];
  if constexpr (sizeof(R) == 8) {
    v.eta_y = (const R *)d.eta_y;
    v.ay = (const R *)d.ay;
    v.by = (const R *)d.by;
    v.ry = (const R *)d.ry;
  } else {
    v.eta_y = (const R *)d.eta_yf;
    v.ay = (const R *)d.ayf;
    v.by = (const R *)d.byf;
    v.ry = (const R *)d.ryf;
  }
  return v;
}

// Bit pattern of a non-negative value as a signed integer that orders like
// the value (exact comparisons on the integer pipe).
__device__ __forceinline__ long long order_bits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ int order_bits(float x) { return __float_as_int(x); }

__host__ __device__ inline long long pidx(const Dev &d, int i, int j, int k) {
  return d.off0 + (long long)k * d.sz + (long long)j * d.sy + i;
}

// (i, j, k) of interior point q = (k ny + j) nx + i.
__device__ __forceinline__ void point_of(const Dev &d, long long q, int &i, int &j, int &k) {
  const unsigned u = (unsigned)q, t = d.fnx.div(u);
  i = (int)(u - t * (unsigned)d.nx);
  const unsigned kk = d.fny.div(t);
  j = (int)(t - kk * (unsigned)d.ny);
  k = (int)kk;
}

// Bounds checks of the checked build (-DS2_CHECKED): each index is tested
// against its array before the access it guards; a failure records
// ERR_BOUNDS and the access is skipped.  The release build compiles the
// tests away (S2_OK_IDX is then constant true).
#ifdef S2_CHECKED
__device__ __forceinline__ bool s2_idx_ok(const Dev &d, long long i, long long size) {
  if (i >= 0 && i < size) return true;
  atomicOr(&d.scal->status, ERR_BOUNDS);
  return false;
}
#define S2_OK_IDX(d, i, size) s2_idx_ok((d), (long long)(i), (long long)(size))
#define S2_GUARD(ok) if (ok)
#else
#define S2_OK_IDX(d, i, size) true
#define S2_GUARD(ok)
#endif

// j of interior point q.
__device__ __forceinline__ int row_of(const Dev &d, long long q) {
  const unsigned t = d.fnx.div((unsigned)q);
  return (int)(t - d.fny.div(t) * (unsigned)d.ny);
}

// Integer power by repeated squaring (e >= 0).
// IEEE-754 format conversions done with integer operations.  GB300 runs
// double-precision arithmetic (and the F2F conversions) on its narrow FP64
// pipe; these keep the mixed path's float<->double traffic on the integer
// pipe.  Normal numbers only: zero and subnormals map to signed zero,
// out-of-range magnitudes to infinity, NaN to NaN/infinity.
//   double -> float, rounded to nearest (ties away from zero)
__device__ __forceinline__ float d2f_int(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  b = (b & 0x7fffffffffffffffull) + (1ull << 28);  // round the 29 dropped bits
  int e = (int)(b >> 52) - 1023 + 127;
  unsigned mant = (unsigned)((b >> 29) & 0x7fffffu);
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | mant);
}
//   float -> double, exact
__device__ __forceinline__ double f2d_int(float x) {
  unsigned b = __float_as_uint(x);
  unsigned sign = b & 0x80000000u;
  unsigned e = (b >> 23) & 0xffu;
  unsigned mant = b & 0x7fffffu;
  if (e == 0) return __hiloint2double((int)sign, 0);
  unsigned ed = e == 255u ? 2047u : e - 127u + 1023u;
  return __hiloint2double((int)(sign | (ed << 20) | (mant >> 3)), (int)(mant << 29));
}

// 0 < x < infinity (false for NaN), tested on the bit pattern.
__device__ __forceinline__ bool positive_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7ff0000000000000LL;
}

// x finite (false for infinities and NaN), tested on the bit pattern.
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < 0x7ff0000000000000LL;
}

// 1/x for x > 0 in double precision by the Newton-Raphson iteration
// r <- r + r (1 - x r) from a single-precision approximate reciprocal: the
// relative error squares per step, ~2^-22 -> 2^-44 -> 2^-88, so two steps
// leave only the final rounding (within 1 ulp of the quotient 1/x).  Four
// FP64 fused multiply-adds; the seed and the conversions run on the
// single-precision and integer pipes.  Magnitudes outside [2^-100, 2^100]
// (where the single-precision seed could flush or overflow) take the
// library division.
__device__ __forceinline__ double rcp_pos(double x) {
  const int ex = (int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu) - 1023;
  if (ex < -100 || ex > 100) return 1.0 / x;
  float xf = d2f_int(x), rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
  double r = f2d_int(rf);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float rcp_pos(float x) { return 1.0f / x; }

// x^e for e >= 0 by binary powering, starting from the lowest set bit
// (no multiplications by 1, no square after the last bit).
__device__ __forceinline__ double ipow(double x, int e) {
  if (e <= 0) return 1.0;
  while (!(e & 1)) {
    x *= x;
    e >>= 1;
  }
  double r = x;
  e >>= 1;
  while (e) {
    x *= x;
    if (e & 1) r *= x;
    e >>= 1;
  }
  return r;
}

// mu = (T/T_ref)^omega / Re.  For omega = p/q with small p >= 0, q (0.76 =
// 19/25) the root y of y^q = x^p is found from a single-precision seed by
// one Halley step, y <- y ((q-1) y^q + (q+1) a) / ((q+1) y^q + (q-1) a),
// a = x^p, whose cubic convergence takes the ~1e-7 seed to double
// precision; otherwise the library pow.
__device__ __forceinline__ double viscosity(const Dev &d, double T) {
  double x = T * d.inv_t_ref;
  double y;
  if (d.mu_q > 0) {
    y = f2d_int(powf(d2f_int(x), d.visc_exp_f));
    double a = ipow(x, d.mu_p), yq = ipow(y, d.mu_q);
    y = y * (d.mu_qm1 * yq + d.mu_qp1 * a) * rcp_pos(d.mu_qp1 * yq + d.mu_qm1 * a);
  } else {
    y = pow(x, d.visc_exp);
  }
  return y * d.inv_re;
}

// ---------------------------------------------- thermally perfect gas
// Sec. 2: the specific heats may depend on T through NASA polynomials
// (McBride et al. 2002, 9-coefficient form): c_p(T) = sum_{l=-2..4} c_l T^l
// with c_l = R a_l, c_v = c_p - R, and the internal energy the c_v
// antiderivative with zero constant,
//   e(T) = -c_-2/T + c_-1 ln T + T (e_0 + T (e_1 + T (e_2 + T (e_3 + T e_4)))),
// e_0 = c_0 - R, e_m = c_m/(m+1).  rT = 1/T is passed in.
__device__ __forceinline__ double tp_log(double x) { return log(x); }
__device__ __forceinline__ float tp_log(float x) { return logf(x); }

template <class R>
__device__ __forceinline__ R tp_cp(const Consts<R> &K, R T, R rT) {
  const R pos = fma(T, fma(T, fma(T, fma(T, K.cpc[6], K.cpc[5]), K.cpc[4]), K.cpc[3]), K.cpc[2]);
  return fma(rT, fma(rT, K.cpc[0], K.cpc[1]), pos);
}

template <class R>
__device__ __forceinline__ R tp_dcp(const Consts<R> &K, R T, R rT) {
  const R pos = fma(T, fma(T, fma(T, K.dcc[5], K.dcc[4]), K.dcc[3]), K.dcc[2]);
  return fma(rT * rT, fma(rT, K.dcc[0], K.dcc[1]), pos);
}

template <class R>
__device__ __forceinline__ R tp_e(const Consts<R> &K, R T, R rT) {
  R e = fma(T, fma(T, fma(T, fma(T, fma(T, K.ecf[6], K.ecf[5]), K.ecf[4]), K.ecf[3]), K.ecf[2]), K.ecf[0] * rT);
  if (K.ecf[1] != R(0)) e = fma(K.ecf[1], tp_log(T), e);
  return e;
}

// c^2 = gamma(T) R T = c_p R T / (c_p - R)
template <class R>
__device__ __forceinline__ R tp_sound2(const Consts<R> &K, R T) {
  const R cp = tp_cp(K, T, rcp_pos(T));
  return cp * K.R_gas * T * rcp_pos(cp - K.R_gas);
}

// The temperature at which e(T) + sR T equals target (sR = 0: internal
// energy, sR = R: enthalpy) by Newton's method from T (> 0), whose
// derivative is c_p - R + sR.  It stops after a step below tol T: the
// iteration converges quadratically, so the error is then of order tol^2
// (1e-18 in double, 1e-7 in single precision).  ok is cleared if that
// does not happen within 24 steps or T leaves T > 0.
template <class R>
__device__ __forceinline__ R tp_temperature(const Consts<R> &K, R target, R T, R sR, bool &ok) {
  const R tol = sizeof(R) == 8 ? R(1e-9) : R(3e-4);
  const R dR = sR - K.R_gas;
  for (int it = 0; it < 24; ++it) {
    const R rT = rcp_pos(T);
    const R f = fma(sR, T, tp_e(K, T, rT)) - target;
    const R dT = f * rcp_pos(tp_cp(K, T, rT) + dR);
    T -= dT;
    if (!(T > R(0))) break;
    if (fabs(dT) <= tol * T) return T;
  }
  ok = false;
  return T;
}

// First guess of T from e: the linearisation of e(T) about T = 1.
template <class R>
__device__ __forceinline__ R tp_guess(const Consts<R> &K, R e) {
  const R T0 = fma(e - K.e1, K.icv1, R(1));
  return T0 > R(0) ? T0 : R(1);
}

// CFL spectral radius of one point (compute_dt of Table 2):
// (|u|+c)/dx + (|v|+c) eta_y + (|w|+c)/dz, plus for viscous runs
// gamma mu / (Pr rho) (1/dx^2 + eta_y^2 + 1/dz^2), c = sqrt(gamma R T),
// gamma = gamma(T) for a thermally perfect gas.
// MAYBE_TP = false: the caller knows the gas is calorically perfect.
template <bool MAYBE_TP = true>
__device__ __forceinline__ double spectral_radius(const Dev &d, double rho, double u, double v, double ww, double T,
                                                  double mu, double ey) {
  double gam = d.gamma;
  if (MAYBE_TP && d.kd.tp) {
    const double cp = tp_cp(d.kd, T, rcp_pos(T));
    gam = cp / (cp - d.R);
  }
  double cs = sqrt(gam * d.R * T);
  double sr = (fabs(u) + cs) / d.dx + (fabs(v) + cs) * ey + (fabs(ww) + cs) / d.dz;
  if (d.viscous) sr += gam * mu / (d.prandtl * rho) * (1.0 / (d.dx * d.dx) + ey * ey + 1.0 / (d.dz * d.dz));
  return sr;
}

// Logarithmic mean (a - b) / (ln a - ln b) of a, b > 0, the averages of
// the KEEP-n flux: from the first n terms of its series in z = (a-b)/(a+b),
// <a,b> = (a+b)/2 / sum_{k<n} z^2k/(2k+1); n < 0: exactly, as the
// quotient of logarithms unless z^2 is small, where the series is summed
// below rounding (6 terms in double, 4 in single precision).
template <class R>
__device__ __forceinline__ R log_mean(R a, R b, int n) {
  const R s = a + b, z = (a - b) / s, u = z * z;
  if (n < 0) {
    if (u > (sizeof(R) == 8 ? R(1e-4) : R(1e-2))) return (a - b) / tp_log(a / b);
    n = sizeof(R) == 8 ? 6 : 4;
  }
  R F = R(0), zk = R(1);
  for (int k = 0; k < n; ++k) {
    F += zk / R(2 * k + 1);
    zk *= u;
  }
  return R(0.5) * s / F;
}

// KEEP-n two-point flux of the points a and b along the direction with
// normal velocity un: <rho>{u_n} (1, {u}, e~ + (u_a . u_b)/2) + ({p} n,
// (p_a un_b + p_b un_a)/2), e~ = 1/((gamma-1) <rho/p>) (c_v/<1/T> of the
// ideal gas).  f[0..4].
template <int DIR, class R>
__device__ __forceinline__ void keep_pair(R ra, R ua, R va, R wa, R pa, R rb, R ub, R vb, R wb, R pb, R gm1, int n,
                                          R *f) {
  const R una = DIR == 0 ? ua : (DIR == 1 ? va : wa), unb = DIR == 0 ? ub : (DIR == 1 ? vb : wb);
  const R rl = log_mean(ra, rb, n), bl = log_mean(ra / pa, rb / pb, n);
  const R fr = rl * (R(0.5) * (una + unb));
  f[0] = fr;
  f[1] = fr * (R(0.5) * (ua + ub));
  f[2] = fr * (R(0.5) * (va + vb));
  f[3] = fr * (R(0.5) * (wa + wb));
  f[1 + DIR] += R(0.5) * (pa + pb);
  const R uab = ua * ub + va * vb + wa * wb;
  f[4] = fr * (R(1) / (gm1 * bl) + R(0.5) * uab) + R(0.5) * (pa * unb + pb * una);
}

// Slot of the interface between points s and s+1 (s = -1 .. n_d - 1) of
// the pencil through (i, j, k) along direction dir: n_d + 1 slots per pencil.
__host__ __device__ inline long long islot(const Dev &d, int dir, int s, int i, int j, int k) {
  if (dir == 0) return ((long long)k * d.ny + j) * (d.nx + 1) + (s + 1);
  if (dir == 1) return ((long long)k * (d.ny + 1) + (s + 1)) * d.nx + i;
  return ((long long)(s + 1) * d.ny + j) * d.nx + i;
}

// The same in 32-bit unsigned arithmetic, exact for every slot of a grid
// (s2_create keeps (nx+1)(ny+1)(nz+1) below 2^31).
__device__ __forceinline__ unsigned islot32(const Dev &d, int dir, int s, int i, int j, int k) {
  const unsigned nx = (unsigned)d.nx, ny = (unsigned)d.ny;
  if (dir == 0) return ((unsigned)k * ny + (unsigned)j) * (nx + 1u) + (unsigned)(s + 1);
  if (dir == 1) return ((unsigned)k * (ny + 1u) + (unsigned)(s + 1)) * nx + (unsigned)i;
  return ((unsigned)(s + 1) * ny + (unsigned)j) * nx + (unsigned)i;
}

// Single-precision power law mu = (T/T_ref)^omega / Re of the mixed path,
// as 2^(omega log2 x) from the hardware base-2 logarithm and exponential:
// for x = T/T_ref in the flow's range (0.1 .. 10) the logarithm's absolute
// error (~2^-22) and the exponential's 2 ulp give mu to ~3e-7 relative,
// the single-precision level of the rest of the path, in a handful of
// instructions instead of the general powf.
__device__ __forceinline__ float viscosity(const Dev &d, float T) {
  return exp2f(d.kf.visc_exp * __log2f(T * d.kf.inv_t_ref)) * d.kf.inv_re;
}

// Whether the CFL dt is recomputed at the step now starting (read on the
// device from the step counter, so one captured graph serves every step).
__device__ __forceinline__ bool dt_due(const Dev &d) {
  return d.cfl > 0.0 && (d.scal->nstep % d.dt_every) == 0;
}

// Asynchronous staging: tiles arrive in shared memory by the tensor memory
// accelerator (cp.async.bulk.tensor, one box per field), completing on an
// mbarrier.
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Per-thread asynchronous copies of single words into shared memory
// (cp.async, cached in L1): the z-marching passes fetch the next plane's
// halo, and the viscous pass its point's RHS and viscosity, while the
// current plane is computed, without holding the values in registers.
// A thread's own copies are complete after cp_async_wait_all; a barrier
// then makes them visible to the CTA.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity; gives up (false) once limit_ns
// of global time have passed, so a copy that never completes cannot hang
// the kernel.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_addr(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Tensor maps of the staged primitive fields (rho, u, v, w, H, p, sensor)
// for the tile box of one direction and tile variant.
struct FluxMaps {
  CUtensorMap m[7];
};

// Launch helpers (defined in the kernel translation units).
cudaError_t flux_make_maps(const Dev &d, FluxMaps (&maps)[3][2]);
cudaError_t launch_flux(const Dev &d, const FluxMaps (&maps)[2], int dir, int accumulate, cudaStream_t st);
cudaError_t launch_weno(const Dev &d, int dir, cudaStream_t st);
cudaError_t launch_grad(const Dev &d, cudaStream_t st);
cudaError_t launch_visc(const Dev &d, cudaStream_t st);
// Forcing partials the viscous launch writes itself (mixed path), else 0;
// CTAs of the mixed path's z-marching passes.
int visc_force_partials(const Dev &d);
long long z_pass_blocks(const Dev &d);
cudaError_t launch_apply(const Dev &d, cudaStream_t st);
cudaError_t flux_set_attributes();

// Batched launches (one launch for every box of a batch group; the boxes
// share the kernel instantiation of d0).  Planning, per box and direction:
// the flux kernel's tile count, its resident CTAs per multiprocessor, and
// its tile-grid record (tg_size bytes, stored per box in a device array
// that the launch reads); the WENO kernel's CTA count.
struct FluxBoxPlan {
  unsigned char tg[64];
  int tg_size, tiles, per_sm;
  bool persistent;  // single precision: CTAs walk several tiles
};
cudaError_t flux_batch_plan(const Dev &d, int dir, FluxBoxPlan *out);
unsigned weno_batch_blocks(const Dev &d, int dir);
cudaError_t launch_flux_batch(const Dev &d0, const BatchArgs &ba, unsigned total, const FluxMaps *maps,
                              const void *tgs, int dir, int accumulate, cudaStream_t st);
cudaError_t launch_weno_batch(const Dev &d0, const BatchArgs &ba, unsigned total, int dir, cudaStream_t st);
// z-marching passes of the mixed path: grid of one box (x, y, z blocks)
void z_pass_grid(const Dev &d, unsigned g[3]);
// Planes per CTA of the z-marching passes: compiled for 4, 8, 12, 16 and
// 24 (the forcing partials are sized for the smallest).
constexpr int ZS_MIN = 4, ZS_DEFAULT = 12;
cudaError_t launch_grad_batch(const Dev &d0, const BatchArgs &ba, unsigned total, cudaStream_t st);
cudaError_t launch_visc_batch(const Dev &d0, const BatchArgs &ba, unsigned total, cudaStream_t st);
cudaError_t launch_apply_batch(const Dev &d0, const BatchArgs &ba, unsigned total, cudaStream_t st);

// Gas constants (R, c_v, c_p, viscosity law) of a Dev from s2_gas.
void set_gas(Dev &d, const s2_gas *gas);
int check_gas(const s2_gas *gas, double t_extra);

}  // namespace s2
