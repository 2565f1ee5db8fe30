/*
 * Plain FP64 CPU oracle of the STREAmS-2 right-hand side and its
 * low-storage RK3 update.  TEST INFRASTRUCTURE ONLY: it is called by the
 * tests, by the smoke check and by the benchmark's CPU-baseline leg, never by
 * the product path, and it shares no code, header or table with the CUDA
 * library.
 *
 * What it computes (paper Sec. 2, "Numerical Methods"): the compressible
 * Navier-Stokes equations for an ideal gas, calorically perfect or
 * thermally perfect (specific heats from a NASA polynomial in T), on a
 * Cartesian grid (stretched in y), finite differences, with
 *   - a hybrid convective discretisation: the energy-preserving split
 *     ("skew-symmetric") form of the convective terms written as numerical
 *     fluxes (Pirozzoli, J. Comput. Phys. 2010), switched at interfaces
 *     flagged by a modified Ducros shock sensor to a WENO reconstruction of
 *     characteristic fluxes (Lax-Friedrichs splitting), projected back on
 *     the right eigenvectors of the Euler equations (Jiang & Shu 1996 WENO5,
 *     Balsara & Shu 2000 WENO7);
 *   - viscous terms expanded in Laplacian form, 6th-order central formulae;
 *   - a third-order low-storage Runge-Kutta scheme (Wray's coefficients);
 *   - the update "w += fln" of the flux register (Sec. 3.2, Listing 4), the
 *     forcing reduction force_rhs_1 and the CFL reduction compute_dt of
 *     Table 2.
 * The paper prints no formula; where it is silent the choices below are
 * readings of the cited published methods (listed as such in the design
 * notes).  Everything is written in the most direct form: interface fluxes
 * by their double sums, eigenvector matrices built explicitly, WENO weights
 * by their definition, derivatives by their stencils.  No blocking, fusion
 * or reordering.
 *
 * Layout of a state w: five fields (rho, rho u, rho v, rho w, rho E), each
 * nz*ny*nx doubles with i (x) fastest: w[f][k][j][i].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NV 5
#define GH 4 /* ghost width of the padded work arrays (WENO7 needs 4) */

/* Operation tally: the counting build (oracle/tally.py) defines OR_SECTION
 * to attribute the floating-point operations that follow a marker to one
 * part of the method; the plain build compiles the markers away. */
#ifndef OR_SECTION
#define OR_SECTION(sec) ((void)0)
#endif
enum {
  SEC_PRIMS,     /* primitive recovery, H and c */
  SEC_SENSOR,    /* velocity gradients, divergence, shock sensor */
  SEC_CENTRAL,   /* split-form central interface fluxes and the flux differences */
  SEC_WENO,      /* characteristic WENO interface fluxes */
  SEC_VISC_GRAD, /* the viscous terms' nine velocity gradients */
  SEC_VISC,      /* the rest of the viscous and heat-flux terms */
  SEC_FORCE,     /* channel forcing */
  SEC_UPDATE,    /* RK3 update */
  SEC_DT,        /* CFL time step */
  SEC_PRIMS_HC,  /* H and c on interior and ghost points */
  SEC_GHOST,     /* ghost values of the primitives, divergence and sensor */
  SEC_OTHER
};

/* Central first derivative of order 2L (L = 1..4, the paper's orders
 * 2/4/6/8, Sec. 2): f' = sum_{l=1..L} a_l (f_{i+l} - f_{i-l}). */
static const double A1_ORD[5][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {0.0, 1.0 / 2.0, 0.0, 0.0, 0.0},
    {0.0, 2.0 / 3.0, -1.0 / 12.0, 0.0, 0.0},
    {0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0, 0.0},
    {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0}};
/* Central second derivative of order 2L: f'' = b_0 f_i + sum_l b_l (f_{i+l} + f_{i-l}). */
static const double B2_ORD[5][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {-2.0, 1.0, 0.0, 0.0, 0.0},
    {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0, 0.0, 0.0},
    {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0, 0.0},
    {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0}};

/* Wray's low-storage RK3: w_k = w_{k-1} + dt (gamma_k R_{k-1} + rho_k R_{k-2}) */
static const double RK_GAMMA[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
static const double RK_RHO[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

/* Problem description.  x and z are periodic; y is periodic or bounded by
 * isothermal no-slip walls at y = -ly/2 and y = +ly/2 (nodes strictly
 * inside, the walls lying half way between the outermost node and its
 * mirror image). */
typedef struct {
  int nx, ny, nz;
  double lx, ly, lz;
  const double *y;      /* ny node ordinates, or NULL for uniform nodes */
  double gamma, prandtl, mach, re, visc_exp, t_ref;
  int bc_y;             /* 0 periodic, 1 isothermal no-slip walls */
  double t_wall;
  int force;            /* 1: uniform x body force keeping the bulk rho*u constant */
  int weno_order;       /* 0 (central everywhere), 1, 3, 5 or 7 */
  double threshold;     /* interface is WENO iff max sensor over its stencil > threshold */
  int central_order;    /* 2, 4, 6 or 8: split-form convective flux */
  int visc_order;       /* 2, 4, 6 or 8: viscous terms and the sensor's derivatives */
  const double *cp_coef; /* NULL: calorically perfect; else a_{-2..4} of c_p/R = sum a_l T^l */
  int keep;             /* central flux: 0 split form; n >= 1 KEEP-n (series of n terms); -1 KEEP, exact log mean */
} or_cfg;

/* Which terms or_rhs evaluates. */
#define OR_CONV 1
#define OR_VISC 2
#define OR_FORCE 4

typedef struct {
  const or_cfg *c;
  int lc, lv;               /* stencil half-widths: central flux, viscous/sensor */
  const double *ac, *av, *bv; /* their coefficients */
  int nx, ny, nz, px, py, pz;
  size_t np, n;
  double R, cv, cp, dx, dz, eps_sensor;
  int tp;                   /* thermally perfect gas: c_p/R = sum_{l=-2..4} a[l+2] T^l */
  double a[7];
  int viscous;
  double *eta_y, *eta_yy; /* ny */
  double *rho, *u, *v, *w, *T, *p, *H, *cs, *sens, *div;
} ws_t;

#define PI(s, i, j, k) \
  ((((size_t)((k) + GH)) * (size_t)(s)->py + (size_t)((j) + GH)) * (size_t)(s)->px + (size_t)((i) + GH))
#define WI(s, i, j, k) ((((size_t)(k)) * (size_t)(s)->ny + (size_t)(j)) * (size_t)(s)->nx + (size_t)(i))

static int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* ---------------------------------------------------------------- grid ---
 * Grid metrics of the stretched y direction (paper Sec. 3.1: the Grid
 * object evaluates the metrics).  The flux is computed in the uniform index
 * eta; d/dy = eta_y d/deta with y_eta from the 6th-order stencil applied to
 * the node ordinates extended into the ghosts (periodic shift, or mirror
 * about the walls), eta_yy = -y_etaeta / y_eta^3. */
static double node_y(const or_cfg *c, int j) {
  if (c->y) return c->y[j];
  return -0.5 * c->ly + (j + 0.5) * c->ly / c->ny;
}

static double ext_y(const or_cfg *c, int j) {
  int ny = c->ny;
  if (j >= 0 && j < ny) return node_y(c, j);
  if (c->bc_y == 0) {
    int jm = imod(j, ny);
    int shift = (j - jm) / ny;
    return node_y(c, jm) + shift * c->ly;
  }
  if (j < 0) return 2.0 * (-0.5 * c->ly) - node_y(c, -1 - j);
  return 2.0 * (0.5 * c->ly) - node_y(c, 2 * ny - 1 - j);
}

/* Metric stencils: the higher of the two orders in use. */
static int metric_half_width(const or_cfg *c) {
  int o = c->central_order > c->visc_order ? c->central_order : c->visc_order;
  return o / 2;
}

void or_metric(const or_cfg *c, double *eta_y, double *eta_yy) {
  int lm = metric_half_width(c);
  const double *A1 = A1_ORD[lm], *B2 = B2_ORD[lm];
  for (int j = 0; j < c->ny; ++j) {
    double d1 = 0.0, d2 = B2[0] * ext_y(c, j);
    for (int l = 1; l <= lm; ++l) {
      d1 += A1[l] * (ext_y(c, j + l) - ext_y(c, j - l));
      d2 += B2[l] * (ext_y(c, j + l) + ext_y(c, j - l));
    }
    eta_y[j] = 1.0 / d1;
    eta_yy[j] = -d2 / (d1 * d1 * d1);
  }
}

/* ------------------------------------------------------------ workspace --- */
static int valid_order(int o) { return o == 2 || o == 4 || o == 6 || o == 8; }

/* Non-dimensional gas (reference density, velocity, temperature, length
 * all 1): R = 1/(gamma M^2), so p = rho R T and, for a calorically perfect
 * gas, c = sqrt(gamma R T). */
static void gas_init(ws_t *s, const or_cfg *c) {
  s->c = c;
  s->R = 1.0 / (c->gamma * c->mach * c->mach);
  s->cv = s->R / (c->gamma - 1.0);
  s->cp = c->gamma * s->cv;
  s->tp = c->cp_coef != NULL;
  if (s->tp)
    for (int l = 0; l < 7; ++l) s->a[l] = c->cp_coef[l];
}

static int ws_init(ws_t *s, const or_cfg *c) {
  memset(s, 0, sizeof(*s));
  s->c = c;
  if (!valid_order(c->central_order) || !valid_order(c->visc_order)) return -1;
  if (c->keep < -1 || (c->keep != 0 && c->cp_coef)) return -1; /* KEEP: calorically perfect gas */
  s->lc = c->central_order / 2;
  s->lv = c->visc_order / 2;
  s->ac = A1_ORD[s->lc];
  s->av = A1_ORD[s->lv];
  s->bv = B2_ORD[s->lv];
  s->nx = c->nx; s->ny = c->ny; s->nz = c->nz;
  s->px = c->nx + 2 * GH; s->py = c->ny + 2 * GH; s->pz = c->nz + 2 * GH;
  s->np = (size_t)s->px * s->py * s->pz;
  s->n = (size_t)c->nx * c->ny * c->nz;
  gas_init(s, c);
  s->dx = c->lx / c->nx;
  s->dz = c->lz / c->nz;
  s->eps_sensor = 1.0; /* (U0/L0)^2 in reference units */
  s->viscous = c->re > 0.0;
  s->eta_y = (double *)malloc(sizeof(double) * c->ny);
  s->eta_yy = (double *)malloc(sizeof(double) * c->ny);
  double **f[] = {&s->rho, &s->u, &s->v, &s->w, &s->T, &s->p, &s->H, &s->cs, &s->sens, &s->div};
  for (size_t q = 0; q < sizeof(f) / sizeof(f[0]); ++q) {
    *f[q] = (double *)calloc(s->np, sizeof(double));
    if (!*f[q]) return -1;
  }
  if (!s->eta_y || !s->eta_yy) return -1;
  or_metric(c, s->eta_y, s->eta_yy);
  return 0;
}

static void ws_free(ws_t *s) {
  double *f[] = {s->rho, s->u, s->v, s->w, s->T, s->p, s->H, s->cs, s->sens, s->div};
  for (size_t q = 0; q < sizeof(f) / sizeof(f[0]); ++q) free(f[q]);
  free(s->eta_y); free(s->eta_yy);
}

/* ------------------------------------------------------- thermodynamics ---
 * Calorically perfect gas: c_p and c_v constant, e = c_v T.  Thermally
 * perfect gas (paper Sec. 2: the temperature dependence of the specific
 * heats through NASA polynomials, McBride et al. 2002): c_p/R is the
 * polynomial sum_{l=-2..4} a_l T^l of the NASA Glenn 9-coefficient form, in
 * reference units of T; c_v = c_p - R; the internal energy is the
 * antiderivative of c_v with zero integration constant,
 *   e/R = -a_{-2}/T + a_{-1} ln T + (a_0 - 1) T + a_1 T^2/2 + a_2 T^3/3
 *         + a_3 T^4/4 + a_4 T^5/5,
 * which is c_v T when only a_0 is non-zero; h = e + R T, and the speed of
 * sound is c = sqrt(gamma(T) R T), gamma(T) = c_p/c_v. */
static double cp_of(const ws_t *s, double T) {
  if (!s->tp) return s->cp;
  double r = 0.0;
  for (int l = -2; l <= 4; ++l) r += s->a[l + 2] * pow(T, l);
  return s->R * r;
}

/* d c_p / d T */
static double dcp_of(const ws_t *s, double T) {
  if (!s->tp) return 0.0;
  double r = 0.0;
  for (int l = -2; l <= 4; ++l)
    if (l != 0) r += l * s->a[l + 2] * pow(T, l - 1);
  return s->R * r;
}

static double e_of(const ws_t *s, double T) {
  if (!s->tp) return s->cv * T;
  double r = -T;
  for (int l = -2; l <= 4; ++l) {
    if (l == -1) r += s->a[1] * log(T);
    else r += s->a[l + 2] * pow(T, l + 1) / (l + 1);
  }
  return s->R * r;
}

static double gamma_of(const ws_t *s, double T) {
  if (!s->tp) return s->c->gamma;
  double cp = cp_of(s, T);
  return cp / (cp - s->R);
}

/* The temperature at which e(T) (enthalpy = 0) or h(T) = e(T) + R T
 * (enthalpy = 1) equals target: Newton's method on that increasing
 * function (its derivative c_v or c_p is positive) from T0, until a step
 * changes T by at most 1e-13 relative; NaN if that does not happen within
 * 100 steps. */
static double temperature_of(const ws_t *s, double target, int enthalpy, double T0) {
  if (!s->tp) return enthalpy ? target / s->cp : target / s->cv;
  double T = T0 > 0.0 ? T0 : 1.0;
  for (int it = 0; it < 100; ++it) {
    double f = e_of(s, T) + (enthalpy ? s->R * T : 0.0) - target;
    double df = cp_of(s, T) - (enthalpy ? 0.0 : s->R);
    double Tn = T - f / df;
    if (!(Tn > 0.0)) Tn = 0.5 * T; /* stay in the domain T > 0 */
    if (fabs(Tn - T) <= 1e-13 * Tn) return Tn;
    T = Tn;
  }
  return NAN;
}

/* T from e, starting from the linearisation of e(T) about T = 1. */
static double T_of_e(const ws_t *s, double e) {
  if (!s->tp) return e / s->cv;
  double T0 = 1.0 + (e - e_of(s, 1.0)) / (cp_of(s, 1.0) - s->R);
  return temperature_of(s, e, 0, T0);
}

/* ------------------------------------------------------------ primitives ---
 * Primitive recovery: rho, u = (rho u)/rho, ..., T from e = E - |u|^2/2
 * (e/c_v, or the inverse of e(T) for a thermally perfect gas), p = rho R T;
 * then the ghost faces; then H = h(T) + |u|^2/2 and c = sqrt(gamma(T) R T)
 * on interior and ghost faces. */
static void fill_ghost_prims(ws_t *s) {
  const or_cfg *c = s->c;
  OR_SECTION(SEC_GHOST);
  int nx = s->nx, ny = s->ny, nz = s->nz;
  double *fl[] = {s->rho, s->u, s->v, s->w, s->T, s->p};
  /* x faces (periodic) */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int g = 1; g <= GH; ++g)
        for (int q = 0; q < 6; ++q) {
          fl[q][PI(s, -g, j, k)] = fl[q][PI(s, nx - g, j, k)];
          fl[q][PI(s, nx - 1 + g, j, k)] = fl[q][PI(s, g - 1, j, k)];
        }
  /* z faces (periodic) */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int g = 1; g <= GH; ++g)
        for (int q = 0; q < 6; ++q) {
          fl[q][PI(s, i, j, -g)] = fl[q][PI(s, i, j, nz - g)];
          fl[q][PI(s, i, j, nz - 1 + g)] = fl[q][PI(s, i, j, g - 1)];
        }
  /* y faces */
  for (int k = 0; k < nz; ++k)
    for (int i = 0; i < nx; ++i)
      for (int g = 1; g <= GH; ++g) {
        if (c->bc_y == 0) {
          for (int q = 0; q < 6; ++q) {
            fl[q][PI(s, i, -g, k)] = fl[q][PI(s, i, ny - g, k)];
            fl[q][PI(s, i, ny - 1 + g, k)] = fl[q][PI(s, i, g - 1, k)];
          }
        } else {
          /* mirror about the wall: ghost -g <-> node g-1 (bottom),
           * ghost ny-1+g <-> node ny-g (top).  No slip: velocity odd;
           * isothermal: T_ghost = 2 T_wall - T; pressure even; density
           * from the equation of state. */
          int gj[2] = {-g, ny - 1 + g}, mj[2] = {g - 1, ny - g};
          for (int side = 0; side < 2; ++side) {
            size_t a = PI(s, i, gj[side], k), b = PI(s, i, mj[side], k);
            s->u[a] = -s->u[b];
            s->v[a] = -s->v[b];
            s->w[a] = -s->w[b];
            s->T[a] = 2.0 * c->t_wall - s->T[b];
            s->p[a] = s->p[b];
            s->rho[a] = s->p[a] / (s->R * s->T[a]);
          }
        }
      }
}

static void prims(ws_t *s, const double *w) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  size_t n = s->n;
  OR_SECTION(SEC_PRIMS);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t q = WI(s, i, j, k), a = PI(s, i, j, k);
        double rho = w[q];
        double u = w[n + q] / rho, v = w[2 * n + q] / rho, ww = w[3 * n + q] / rho;
        double e = w[4 * n + q] / rho - 0.5 * (u * u + v * v + ww * ww);
        double T = T_of_e(s, e);
        s->rho[a] = rho; s->u[a] = u; s->v[a] = v; s->w[a] = ww;
        s->T[a] = T; s->p[a] = rho * s->R * T;
      }
  fill_ghost_prims(s);
  /* H and c everywhere the primitives are defined (edges/corners stay 0) */
  OR_SECTION(SEC_PRIMS_HC);
#pragma omp parallel for schedule(static)
  for (int kk = 0; kk < s->pz; ++kk)
    for (int jj = 0; jj < s->py; ++jj)
      for (int ii = 0; ii < s->px; ++ii) {
        size_t a = ((size_t)kk * s->py + jj) * s->px + ii;
        double T = s->T[a];
        double q2 = s->u[a] * s->u[a] + s->v[a] * s->v[a] + s->w[a] * s->w[a];
        if (!s->tp) {
          s->H[a] = s->cp * T + 0.5 * q2;
          s->cs[a] = T > 0.0 ? sqrt(s->c->gamma * s->R * T) : 0.0;
        } else if (T > 0.0) {
          s->H[a] = e_of(s, T) + s->R * T + 0.5 * q2;
          s->cs[a] = sqrt(gamma_of(s, T) * s->R * T);
        } else { /* edges and corners of the work arrays */
          s->H[a] = 0.5 * q2;
          s->cs[a] = 0.0;
        }
      }
}

/* ---------------------------------------------------------- derivatives --- */
/* derivatives of the viscous order (viscous terms and sensor) */
static double d1(const ws_t *s, const double *f, int i, int j, int k, int dir) {
  const double *A1 = s->av;
  double r = 0.0;
  for (int l = 1; l <= s->lv; ++l) {
    if (dir == 0) r += A1[l] * (f[PI(s, i + l, j, k)] - f[PI(s, i - l, j, k)]);
    else if (dir == 1) r += A1[l] * (f[PI(s, i, j + l, k)] - f[PI(s, i, j - l, k)]);
    else r += A1[l] * (f[PI(s, i, j, k + l)] - f[PI(s, i, j, k - l)]);
  }
  if (dir == 0) return r / s->dx;
  if (dir == 1) return r * s->eta_y[j];
  return r / s->dz;
}

/* derivative in index space (no metric) */
static double d1_idx(const ws_t *s, const double *f, int i, int j, int k, int dir) {
  const double *A1 = s->av;
  double r = 0.0;
  for (int l = 1; l <= s->lv; ++l) {
    if (dir == 0) r += A1[l] * (f[PI(s, i + l, j, k)] - f[PI(s, i - l, j, k)]);
    else if (dir == 1) r += A1[l] * (f[PI(s, i, j + l, k)] - f[PI(s, i, j - l, k)]);
    else r += A1[l] * (f[PI(s, i, j, k + l)] - f[PI(s, i, j, k - l)]);
  }
  return r;
}

static double d2(const ws_t *s, const double *f, int i, int j, int k, int dir) {
  const double *B2 = s->bv;
  double r = B2[0] * f[PI(s, i, j, k)];
  for (int l = 1; l <= s->lv; ++l) {
    if (dir == 0) r += B2[l] * (f[PI(s, i + l, j, k)] + f[PI(s, i - l, j, k)]);
    else if (dir == 1) r += B2[l] * (f[PI(s, i, j + l, k)] + f[PI(s, i, j - l, k)]);
    else r += B2[l] * (f[PI(s, i, j, k + l)] + f[PI(s, i, j, k - l)]);
  }
  if (dir == 0) return r / (s->dx * s->dx);
  if (dir == 2) return r / (s->dz * s->dz);
  /* d2f/dy2 = eta_y^2 f_etaeta + eta_yy f_eta */
  double ey = s->eta_y[j];
  return ey * ey * r + s->eta_yy[j] * d1_idx(s, f, i, j, k, 1);
}

/* --------------------------------------------------------------- sensor ---
 * Modified Ducros sensor (paper Sec. 2): theta = div u, omega = curl u,
 * sensor = max(-theta / sqrt(theta^2 + |omega|^2 + eps), 0), eps = (U0/L0)^2.
 * It also stores theta, whose derivatives the viscous terms use.  Ghost
 * values: periodic copy, or at a wall the mirror value of the sensor and
 * the divergence of the mirrored velocity field (-u_x + v_y - w_z at the
 * mirror node, since u, w are odd in y with even x/z derivatives and v is
 * odd with an even y derivative). */
static void sensor(ws_t *s) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  OR_SECTION(SEC_SENSOR);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double ux = d1(s, s->u, i, j, k, 0), uy = d1(s, s->u, i, j, k, 1), uz = d1(s, s->u, i, j, k, 2);
        double vx = d1(s, s->v, i, j, k, 0), vy = d1(s, s->v, i, j, k, 1), vz = d1(s, s->v, i, j, k, 2);
        double wx = d1(s, s->w, i, j, k, 0), wy = d1(s, s->w, i, j, k, 1), wz = d1(s, s->w, i, j, k, 2);
        double th = ux + vy + wz;
        double o1 = wy - vz, o2 = uz - wx, o3 = vx - uy;
        double om2 = o1 * o1 + o2 * o2 + o3 * o3;
        double sv = -th / sqrt(th * th + om2 + s->eps_sensor);
        size_t a = PI(s, i, j, k);
        s->sens[a] = sv > 0.0 ? sv : 0.0;
        s->div[a] = th;
      }
  OR_SECTION(SEC_GHOST);
  double *fl[] = {s->sens, s->div};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int g = 1; g <= GH; ++g)
        for (int q = 0; q < 2; ++q) {
          fl[q][PI(s, -g, j, k)] = fl[q][PI(s, nx - g, j, k)];
          fl[q][PI(s, nx - 1 + g, j, k)] = fl[q][PI(s, g - 1, j, k)];
        }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int g = 1; g <= GH; ++g)
        for (int q = 0; q < 2; ++q) {
          fl[q][PI(s, i, j, -g)] = fl[q][PI(s, i, j, nz - g)];
          fl[q][PI(s, i, j, nz - 1 + g)] = fl[q][PI(s, i, j, g - 1)];
        }
  for (int k = 0; k < nz; ++k)
    for (int i = 0; i < nx; ++i)
      for (int g = 1; g <= GH; ++g) {
        if (s->c->bc_y == 0) {
          for (int q = 0; q < 2; ++q) {
            fl[q][PI(s, i, -g, k)] = fl[q][PI(s, i, ny - g, k)];
            fl[q][PI(s, i, ny - 1 + g, k)] = fl[q][PI(s, i, g - 1, k)];
          }
        } else {
          int gj[2] = {-g, ny - 1 + g}, mj[2] = {g - 1, ny - g};
          for (int side = 0; side < 2; ++side) {
            int m = mj[side];
            if (m < 0 || m >= ny) continue;
            double ux = d1(s, s->u, i, m, k, 0), vy = d1(s, s->v, i, m, k, 1), wz = d1(s, s->w, i, m, k, 2);
            s->sens[PI(s, i, gj[side], k)] = s->sens[PI(s, i, m, k)];
            s->div[PI(s, i, gj[side], k)] = -ux + vy - wz;
          }
        }
      }
}

/* ------------------------------------------------------------------ WENO ---
 * Left-biased WENO reconstruction at x_{i+1/2} from the 2r-1 values
 * f[0..2r-2] centred on f[r-1] = f_i.  r = 3: Jiang & Shu (1996) WENO5;
 * r = 4: Balsara & Shu (2000) WENO7.  Weights alpha_k = d_k/(eps+beta_k)^2,
 * eps = 1e-6. */
#define WENO_EPS 1e-6

/* Candidate values q_k and smoothness indicators beta_k of the r
 * substencils; returns r (0 for an unsupported order).  Order 1 is the
 * first-order upwind value, order 3 the two-stencil WENO3 (same Jiang-Shu
 * construction). */
int or_weno_parts(int order, const double *g, double *q, double *b) {
  if (order == 1) { /* g[0] = f_i */
    q[0] = g[0];
    b[0] = 0.0;
    return 1;
  }
  if (order == 3) { /* g[0..2] = f_{i-1} .. f_{i+1} */
    q[0] = (-g[0] + 3.0 * g[1]) / 2.0;
    q[1] = (g[1] + g[2]) / 2.0;
    b[0] = (g[1] - g[0]) * (g[1] - g[0]);
    b[1] = (g[2] - g[1]) * (g[2] - g[1]);
    return 2;
  }
  if (order == 5) { /* g[0..4] = f_{i-2} .. f_{i+2} */
    q[0] = (2.0 * g[0] - 7.0 * g[1] + 11.0 * g[2]) / 6.0;
    q[1] = (-g[1] + 5.0 * g[2] + 2.0 * g[3]) / 6.0;
    q[2] = (2.0 * g[2] + 5.0 * g[3] - g[4]) / 6.0;
    double t;
    t = g[0] - 2.0 * g[1] + g[2]; b[0] = 13.0 / 12.0 * t * t;
    t = g[0] - 4.0 * g[1] + 3.0 * g[2]; b[0] += 0.25 * t * t;
    t = g[1] - 2.0 * g[2] + g[3]; b[1] = 13.0 / 12.0 * t * t;
    t = g[1] - g[3]; b[1] += 0.25 * t * t;
    t = g[2] - 2.0 * g[3] + g[4]; b[2] = 13.0 / 12.0 * t * t;
    t = 3.0 * g[2] - 4.0 * g[3] + g[4]; b[2] += 0.25 * t * t;
    return 3;
  }
  if (order == 7) { /* g[0..6] = f_{i-3} .. f_{i+3} */
    q[0] = (-3.0 * g[0] + 13.0 * g[1] - 23.0 * g[2] + 25.0 * g[3]) / 12.0;
    q[1] = (g[1] - 5.0 * g[2] + 13.0 * g[3] + 3.0 * g[4]) / 12.0;
    q[2] = (-g[2] + 7.0 * g[3] + 7.0 * g[4] - g[5]) / 12.0;
    q[3] = (3.0 * g[3] + 13.0 * g[4] - 5.0 * g[5] + g[6]) / 12.0;
    /* Balsara & Shu's indicators (240 x the Jiang-Shu measure
     * sum_l int (d^l p_k/dx^l)^2) written as sums of squares of the
     * undivided differences e1, e2, e3 of each substencil, which keeps
     * them free of the cancellation of the expanded quadratic form. */
    static const double c1[4][2] = {{5.0 / 2.0, 11.0 / 6.0}, {3.0 / 2.0, 1.0 / 3.0},
                                    {1.0 / 2.0, -1.0 / 6.0}, {-1.0 / 2.0, 1.0 / 3.0}};
    static const double c2[4] = {2.0, 1.0, 0.0, -1.0};
    for (int k = 0; k < 4; ++k) {
      const double *h = g + k; /* substencil f_{i-3+k} .. f_{i+k} */
      double e1 = h[1] - h[0];
      double e2 = h[2] - 2.0 * h[1] + h[0];
      double e3 = h[3] - 3.0 * h[2] + 3.0 * h[1] - h[0];
      double s1 = e1 + c1[k][0] * e2 + c1[k][1] * e3;
      double s2 = e2 + c2[k] * e3;
      b[k] = 240.0 * s1 * s1 + 260.0 * s2 * s2 + 781.0 / 3.0 * e3 * e3;
    }
    return 4;
  }
  return 0;
}

/* Optimal (linear) weights d_k. */
static const double WENO1_D[1] = {1.0};
static const double WENO3_D[2] = {1.0 / 3.0, 2.0 / 3.0};
static const double WENO5_D[3] = {0.1, 0.6, 0.3};
static const double WENO7_D[4] = {1.0 / 35.0, 12.0 / 35.0, 18.0 / 35.0, 4.0 / 35.0};

double or_weno_rec(int order, const double *f) {
  double q[4], b[4];
  int r = or_weno_parts(order, f, q, b);
  if (!r) return NAN;
  const double *d = r == 1 ? WENO1_D : (r == 2 ? WENO3_D : (r == 3 ? WENO5_D : WENO7_D));
  double a[4], sa = 0.0;
  for (int k = 0; k < r; ++k) { a[k] = d[k] / ((WENO_EPS + b[k]) * (WENO_EPS + b[k])); sa += a[k]; }
  double res = 0.0;
  for (int k = 0; k < r; ++k) res += a[k] / sa * q[k];
  return res;
}

/* Eigenvector matrices of the Euler flux Jacobian along direction dir at
 * the state (velocity uv[3], total enthalpy H): columns of Rm are the right
 * eigenvectors for the eigenvalues (u_n - c, u_n, u_n, u_n, u_n + c), rows of
 * Lm the left eigenvectors, Lm = Rm^-1.  Row-major 5x5.  Returns c. */
double or_eigvec(double gamma, int dir, const double *uv, double H, double *Lm, double *Rm) {
  double b = gamma - 1.0;
  double q2 = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
  double c2 = b * (H - 0.5 * q2);
  double c = sqrt(c2);
  double n[3] = {0.0, 0.0, 0.0};
  n[dir] = 1.0;
  int t1 = (dir + 1) % 3, t2 = (dir + 2) % 3; /* tangential axes */
  double un = uv[dir];
  for (int q = 0; q < 25; ++q) { Lm[q] = 0.0; Rm[q] = 0.0; }
  /* right eigenvectors (columns) */
  Rm[0 * 5 + 0] = 1.0;
  for (int a = 0; a < 3; ++a) Rm[(1 + a) * 5 + 0] = uv[a] - c * n[a];
  Rm[4 * 5 + 0] = H - un * c;
  Rm[0 * 5 + 1] = 1.0;
  for (int a = 0; a < 3; ++a) Rm[(1 + a) * 5 + 1] = uv[a];
  Rm[4 * 5 + 1] = 0.5 * q2;
  Rm[(1 + t1) * 5 + 2] = 1.0;
  Rm[4 * 5 + 2] = uv[t1];
  Rm[(1 + t2) * 5 + 3] = 1.0;
  Rm[4 * 5 + 3] = uv[t2];
  Rm[0 * 5 + 4] = 1.0;
  for (int a = 0; a < 3; ++a) Rm[(1 + a) * 5 + 4] = uv[a] + c * n[a];
  Rm[4 * 5 + 4] = H + un * c;
  /* left eigenvectors (rows) */
  double h2 = 0.5 / c2;
  Lm[0 * 5 + 0] = h2 * (0.5 * b * q2 + un * c);
  for (int a = 0; a < 3; ++a) Lm[0 * 5 + 1 + a] = h2 * (-b * uv[a] - c * n[a]);
  Lm[0 * 5 + 4] = h2 * b;
  Lm[1 * 5 + 0] = 1.0 - b * q2 / (2.0 * c2);
  for (int a = 0; a < 3; ++a) Lm[1 * 5 + 1 + a] = b * uv[a] / c2;
  Lm[1 * 5 + 4] = -b / c2;
  Lm[2 * 5 + 0] = -uv[t1];
  Lm[2 * 5 + 1 + t1] = 1.0;
  Lm[3 * 5 + 0] = -uv[t2];
  Lm[3 * 5 + 1 + t2] = 1.0;
  Lm[4 * 5 + 0] = h2 * (0.5 * b * q2 - un * c);
  for (int a = 0; a < 3; ++a) Lm[4 * 5 + 1 + a] = h2 * (-b * uv[a] + c * n[a]);
  Lm[4 * 5 + 4] = h2 * b;
  return c;
}

/* The same matrices for a general equation of state p(rho, e): chi =
 * (1/rho) dp/de at constant rho (gamma - 1 for a calorically perfect gas,
 * R/c_v(T) for a thermally perfect one) and the speed of sound c are given.
 * The entropy-wave column carries H - c^2/chi in its energy entry (|u|^2/2
 * when c^2 = (gamma-1)(H - |u|^2/2)), and the left rows follow from it with
 * the term K = |u|^2 - (H - c^2/chi) in place of |u|^2/2. */
double or_eigvec_tp(double chi, double c, int dir, const double *uv, double H, double *Lm, double *Rm) {
  double b = chi, c2 = c * c;
  double q2 = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
  double hs = H - c2 / chi, K = q2 - hs;
  double n[3] = {0.0, 0.0, 0.0};
  n[dir] = 1.0;
  int t1 = (dir + 1) % 3, t2 = (dir + 2) % 3;
  double un = uv[dir];
  for (int q = 0; q < 25; ++q) { Lm[q] = 0.0; Rm[q] = 0.0; }
  Rm[0 * 5 + 0] = 1.0;
  for (int a = 0; a < 3; ++a) Rm[(1 + a) * 5 + 0] = uv[a] - c * n[a];
  Rm[4 * 5 + 0] = H - un * c;
  Rm[0 * 5 + 1] = 1.0;
  for (int a = 0; a < 3; ++a) Rm[(1 + a) * 5 + 1] = uv[a];
  Rm[4 * 5 + 1] = hs;
  Rm[(1 + t1) * 5 + 2] = 1.0;
  Rm[4 * 5 + 2] = uv[t1];
  Rm[(1 + t2) * 5 + 3] = 1.0;
  Rm[4 * 5 + 3] = uv[t2];
  Rm[0 * 5 + 4] = 1.0;
  for (int a = 0; a < 3; ++a) Rm[(1 + a) * 5 + 4] = uv[a] + c * n[a];
  Rm[4 * 5 + 4] = H + un * c;
  double h2 = 0.5 / c2;
  Lm[0 * 5 + 0] = h2 * (b * K + un * c);
  for (int a = 0; a < 3; ++a) Lm[0 * 5 + 1 + a] = h2 * (-b * uv[a] - c * n[a]);
  Lm[0 * 5 + 4] = h2 * b;
  Lm[1 * 5 + 0] = 1.0 - b * K / c2;
  for (int a = 0; a < 3; ++a) Lm[1 * 5 + 1 + a] = b * uv[a] / c2;
  Lm[1 * 5 + 4] = -b / c2;
  Lm[2 * 5 + 0] = -uv[t1];
  Lm[2 * 5 + 1 + t1] = 1.0;
  Lm[3 * 5 + 0] = -uv[t2];
  Lm[3 * 5 + 1 + t2] = 1.0;
  Lm[4 * 5 + 0] = h2 * (b * K - un * c);
  for (int a = 0; a < 3; ++a) Lm[4 * 5 + 1 + a] = h2 * (-b * uv[a] + c * n[a]);
  Lm[4 * 5 + 4] = h2 * b;
  return c;
}

/* Roe average of the states a and b (rho, u, v, w, T each): velocity and
 * total enthalpy weighted by sqrt(rho); for a thermally perfect gas also the
 * temperature T~ with h(T~) = H~ - |u~|^2/2 (Newton from the sqrt(rho)-
 * weighted mean of T), chi = R/c_v(T~) and c~ = sqrt(gamma(T~) R T~).  A
 * calorically perfect gas has chi = gamma - 1 and c~^2 = chi (H~ - |u~|^2/2).
 * out: u, v, w, H, chi, c. */
static void roe_state(const ws_t *s, const double *sa, const double *sb, double *out) {
  double ra = sqrt(sa[0]), rb = sqrt(sb[0]);
  double H[2];
  const double *st[2] = {sa, sb};
  for (int m = 0; m < 2; ++m) {
    const double *z = st[m];
    double q2 = z[1] * z[1] + z[2] * z[2] + z[3] * z[3];
    H[m] = (s->tp ? e_of(s, z[4]) + s->R * z[4] : s->cp * z[4]) + 0.5 * q2;
  }
  for (int a = 0; a < 3; ++a) out[a] = (ra * sa[1 + a] + rb * sb[1 + a]) / (ra + rb);
  out[3] = (ra * H[0] + rb * H[1]) / (ra + rb);
  double q2 = out[0] * out[0] + out[1] * out[1] + out[2] * out[2];
  if (!s->tp) {
    out[4] = s->c->gamma - 1.0;
    out[5] = sqrt(out[4] * (out[3] - 0.5 * q2));
    return;
  }
  double T0 = (ra * sa[4] + rb * sb[4]) / (ra + rb);
  double Tt = temperature_of(s, out[3] - 0.5 * q2, 1, T0);
  out[4] = s->R / (cp_of(s, Tt) - s->R);
  out[5] = sqrt(gamma_of(s, Tt) * s->R * Tt);
}

/* value of field f at position "pos" along direction dir of the pencil
 * through (i,j,k) */
static inline size_t at(const ws_t *s, int dir, int pos, int i, int j, int k) {
  if (dir == 0) return PI(s, pos, j, k);
  if (dir == 1) return PI(s, i, pos, k);
  return PI(s, i, j, pos);
}

/* WENO flux of order 2r-1 at interface pos+1/2 (characteristic variables,
 * local Lax-Friedrichs splitting with one dissipation per characteristic
 * field: the largest |eigenvalue| over the stencil points; Roe-averaged
 * eigenvectors). */
static void weno_flux(const ws_t *s, int dir, int pos, int i, int j, int k, double *F) {
  const double gam = s->c->gamma;
  int r = (s->c->weno_order + 1) / 2;
  int np = 2 * r; /* stencil points pos-r+1 .. pos+r */
  size_t a = at(s, dir, pos, i, j, k), bq = at(s, dir, pos + 1, i, j, k);
  /* Roe average of the states at pos and pos+1 */
  double sa[5] = {s->rho[a], s->u[a], s->v[a], s->w[a], s->T[a]};
  double sb[5] = {s->rho[bq], s->u[bq], s->v[bq], s->w[bq], s->T[bq]};
  double roe[6];
  roe_state(s, sa, sb, roe);
  double Lm[25], Rm[25];
  if (!s->tp)
    or_eigvec(gam, dir, roe, roe[3], Lm, Rm);
  else
    or_eigvec_tp(roe[4], roe[5], dir, roe, roe[3], Lm, Rm);
  double V[8][5], G[8][5], lam[8][5];
  for (int m = 0; m < np; ++m) {
    size_t q = at(s, dir, pos - r + 1 + m, i, j, k);
    double rho = s->rho[q], vel[3] = {s->u[q], s->v[q], s->w[q]};
    double p = s->p[q], Hq = s->H[q], un = vel[dir];
    double W[5] = {rho, rho * vel[0], rho * vel[1], rho * vel[2], rho * Hq - p};
    double Fp[5] = {rho * un, rho * un * vel[0], rho * un * vel[1], rho * un * vel[2], rho * un * Hq};
    Fp[1 + dir] += p;
    for (int e = 0; e < 5; ++e) {
      double sv = 0.0, sg = 0.0;
      for (int f = 0; f < 5; ++f) { sv += Lm[e * 5 + f] * W[f]; sg += Lm[e * 5 + f] * Fp[f]; }
      V[m][e] = sv; G[m][e] = sg;
    }
    lam[m][0] = un - s->cs[q];
    lam[m][1] = un; lam[m][2] = un; lam[m][3] = un;
    lam[m][4] = un + s->cs[q];
  }
  double gh[5];
  for (int e = 0; e < 5; ++e) {
    double alpha = 0.0;
    for (int m = 0; m < np; ++m) alpha = fmax(alpha, fabs(lam[m][e]));
    double fp[7], fm[7];
    /* plus flux: left-biased, points pos-r+1 .. pos+r-1 */
    for (int m = 0; m < 2 * r - 1; ++m) fp[m] = 0.5 * (G[m][e] + alpha * V[m][e]);
    /* minus flux: right-biased, mirrored so pos+r .. pos-r+2 */
    for (int m = 0; m < 2 * r - 1; ++m) {
      int mm = np - 1 - m;
      fm[m] = 0.5 * (G[mm][e] - alpha * V[mm][e]);
    }
    gh[e] = or_weno_rec(s->c->weno_order, fp) + or_weno_rec(s->c->weno_order, fm);
  }
  for (int f = 0; f < 5; ++f) {
    double sum = 0.0;
    for (int e = 0; e < 5; ++e) sum += Rm[f * 5 + e] * gh[e];
    F[f] = sum;
  }
}

/* Split-form central flux at interface pos+1/2 (Pirozzoli 2010):
 * F = 2 sum_l a_l sum_{m<l} (rho)(u_n)(phi) over the pairs (pos-m, pos-m+l),
 * (g) the arithmetic mean of the pair, phi = (1, u, v, w, H); the pressure
 * enters the normal momentum as sum_l a_l sum_{m<l} (p_a + p_b). */
static void central_flux(const ws_t *s, int dir, int pos, int i, int j, int k, double *F) {
  const double *un = dir == 0 ? s->u : (dir == 1 ? s->v : s->w);
  const double *A1 = s->ac;
  for (int f = 0; f < 5; ++f) F[f] = 0.0;
  double fp = 0.0;
  for (int l = 1; l <= s->lc; ++l) {
    double acc[5] = {0, 0, 0, 0, 0}, pp = 0.0;
    for (int m = 0; m < l; ++m) {
      size_t a = at(s, dir, pos - m, i, j, k), b = at(s, dir, pos - m + l, i, j, k);
      double rr = 0.5 * (s->rho[a] + s->rho[b]);
      double uu = 0.5 * (un[a] + un[b]);
      double phi[5] = {1.0, 0.5 * (s->u[a] + s->u[b]), 0.5 * (s->v[a] + s->v[b]),
                       0.5 * (s->w[a] + s->w[b]), 0.5 * (s->H[a] + s->H[b])};
      for (int f = 0; f < 5; ++f) acc[f] += rr * uu * phi[f];
      pp += s->p[a] + s->p[b];
    }
    for (int f = 0; f < 5; ++f) F[f] += 2.0 * A1[l] * acc[f];
    fp += A1[l] * pp;
  }
  F[1 + dir] += fp;
}

/* ---------------------------------------------------------------- KEEP-n ---
 * Kinetic-energy and entropy preserving central flux (paper Sec. 2: the
 * optional KEEP-n scheme, which keeps kinetic energy and, for smooth
 * inviscid flow, entropy locally).  Reading: the same flux-differencing
 * form as the split-form flux, F = 2 sum_l a_l sum_{m<l} f*(w_{pos-m},
 * w_{pos-m+l}), with the two-point flux of a calorically perfect gas
 *   f*_rho  = <rho> {u_n}
 *   f*_rhou = f*_rho {u} + {p} n
 *   f*_rhoE = f*_rho (c_v / <1/T> + (u_a . u_b)/2) + (p_a u_n,b + p_b u_n,a)/2
 * ({.} arithmetic, <.> logarithmic mean), which satisfies Tadmor's
 * entropy condition for the entropy -rho s/(gamma-1), s = ln(p rho^-gamma)
 * (Ranocha 2018), so the central scheme conserves that entropy; its
 * momentum flux (mass flux times the mean velocity plus the mean pressure)
 * preserves kinetic energy, and uniform velocity and pressure stay
 * uniform.  KEEP-n takes the logarithmic mean from the first n terms of
 * its series in z = (a-b)/(a+b): <a,b> = {a} / sum_{k<n} z^2k/(2k+1), an
 * entropy error of order z^2n per pair; n = -1 takes the exact mean. */
static double log_mean(double a, double b, int n) {
  double z = (a - b) / (a + b), u = z * z;
  if (n < 0) {
    if (u > 1e-4) return (a - b) / log(a / b);
    n = 6; /* the series' remainder is below u^6/13: below rounding */
  }
  double F = 0.0, zk = 1.0;
  for (int k = 0; k < n; ++k) {
    F += zk / (2.0 * k + 1.0);
    zk *= u;
  }
  return 0.5 * (a + b) / F;
}

/* the two-point flux of points a and b along direction dir */
static void keep_pair(const ws_t *s, int dir, size_t a, size_t b, double *f) {
  const double *un = dir == 0 ? s->u : (dir == 1 ? s->v : s->w);
  double rl = log_mean(s->rho[a], s->rho[b], s->c->keep);
  double bl = log_mean(1.0 / s->T[a], 1.0 / s->T[b], s->c->keep); /* <1/T> */
  double unm = 0.5 * (un[a] + un[b]);
  double fr = rl * unm;
  f[0] = fr;
  f[1] = fr * 0.5 * (s->u[a] + s->u[b]);
  f[2] = fr * 0.5 * (s->v[a] + s->v[b]);
  f[3] = fr * 0.5 * (s->w[a] + s->w[b]);
  f[1 + dir] += 0.5 * (s->p[a] + s->p[b]);
  double uab = s->u[a] * s->u[b] + s->v[a] * s->v[b] + s->w[a] * s->w[b];
  f[4] = fr * (s->cv / bl + 0.5 * uab) + 0.5 * (s->p[a] * un[b] + s->p[b] * un[a]);
}

static void keep_flux(const ws_t *s, int dir, int pos, int i, int j, int k, double *F) {
  for (int f = 0; f < 5; ++f) F[f] = 0.0;
  for (int l = 1; l <= s->lc; ++l)
    for (int m = 0; m < l; ++m) {
      double f2[5];
      keep_pair(s, dir, at(s, dir, pos - m, i, j, k), at(s, dir, pos - m + l, i, j, k), f2);
      for (int f = 0; f < 5; ++f) F[f] += 2.0 * s->ac[l] * f2[f];
    }
}

/* flags: where the per-interface WENO flags are written, or (given != 0)
 * read from: a caller-supplied decision replaces the sensor test. */
static void convective(ws_t *s, int dir, double *rhs, unsigned char *flags, int given) {
  int nx = s->nx, ny = s->ny, nz = s->nz, n = dir == 0 ? nx : (dir == 1 ? ny : nz);
  int r = (s->c->weno_order + 1) / 2;
  int na = dir == 0 ? ny : nx, nb = dir == 2 ? ny : nz; /* transverse extents */
#pragma omp parallel for schedule(static) collapse(2)
  for (int tb = 0; tb < nb; ++tb)
    for (int ta = 0; ta < na; ++ta) {
      int i = 0, j = 0, k = 0;
      if (dir == 0) { j = ta; k = tb; }
      else if (dir == 1) { i = ta; k = tb; }
      else { i = ta; j = tb; }
      double *Fh = (double *)malloc(sizeof(double) * 5 * (size_t)(n + 1));
      for (int pos = -1; pos < n; ++pos) {
        int fl = 0;
        size_t slot = 0;
        if (flags) {
          /* per-direction interface flags, n+1 per pencil, interface pos+1/2 at slot pos+1 */
          if (dir == 0) slot = ((size_t)k * ny + j) * (nx + 1) + (pos + 1);
          else if (dir == 1) slot = ((size_t)k * (ny + 1) + (pos + 1)) * nx + i;
          else slot = ((size_t)(pos + 1) * ny + j) * nx + i;
        }
        if (given) {
          fl = s->c->weno_order > 0 && flags[slot];
        } else {
          if (s->c->weno_order > 0) {
            double mx = 0.0;
            for (int m = pos - r + 1; m <= pos + r; ++m) mx = fmax(mx, s->sens[at(s, dir, m, i, j, k)]);
            fl = mx > s->c->threshold;
          }
          if (flags) flags[slot] = (unsigned char)fl;
        }
        if (fl) {
          OR_SECTION(SEC_WENO);
          weno_flux(s, dir, pos, i, j, k, Fh + 5 * (pos + 1));
        } else {
          OR_SECTION(SEC_CENTRAL);
          if (s->c->keep) keep_flux(s, dir, pos, i, j, k, Fh + 5 * (pos + 1));
          else central_flux(s, dir, pos, i, j, k, Fh + 5 * (pos + 1));
        }
      }
      OR_SECTION(SEC_CENTRAL);
      for (int pos = 0; pos < n; ++pos) {
        int ii = dir == 0 ? pos : i, jj = dir == 1 ? pos : j, kk = dir == 2 ? pos : k;
        double sc = dir == 0 ? 1.0 / s->dx : (dir == 1 ? s->eta_y[jj] : 1.0 / s->dz);
        size_t q = WI(s, ii, jj, kk);
        for (int f = 0; f < 5; ++f)
          rhs[f * s->n + q] -= sc * (Fh[5 * (pos + 1) + f] - Fh[5 * pos + f]);
      }
      free(Fh);
    }
}

/* ---------------------------------------------------------------- viscous ---
 * Viscous and heat-flux terms in Laplacian form (paper Sec. 2):
 *   momentum_i: mu (lap u_i + (1/3) d_i theta) + d_j mu (d_j u_i + d_i u_j)
 *               - (2/3) theta d_i mu
 *   energy:     u_i * momentum_i + tau_ij d_j u_i + k lap T + grad k . grad T
 * with mu = (T/T_ref)^omega / Re, grad mu = (omega mu / T) grad T,
 * k = mu c_p(T) / Pr, tau_ij = mu (d_j u_i + d_i u_j - (2/3) theta delta_ij),
 * theta the stored divergence (its gradient by the same stencil). */
static void viscous(ws_t *s, double *rhs) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  const or_cfg *c = s->c;
  size_t n = s->n;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double *vel[3] = {s->u, s->v, s->w};
        double g[3][3], lap[3], gT[3], gth[3];
        OR_SECTION(SEC_VISC_GRAD);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) g[a][b] = d1(s, vel[a], i, j, k, b); /* d u_a / d x_b */
        OR_SECTION(SEC_VISC);
        for (int a = 0; a < 3; ++a) lap[a] = d2(s, vel[a], i, j, k, 0) + d2(s, vel[a], i, j, k, 1) + d2(s, vel[a], i, j, k, 2);
        for (int b = 0; b < 3; ++b) { gT[b] = d1(s, s->T, i, j, k, b); gth[b] = d1(s, s->div, i, j, k, b); }
        double lapT = d2(s, s->T, i, j, k, 0) + d2(s, s->T, i, j, k, 1) + d2(s, s->T, i, j, k, 2);
        size_t pa = PI(s, i, j, k);
        double T = s->T[pa];
        double mu = pow(T / c->t_ref, c->visc_exp) / c->re;
        double mut = c->visc_exp * mu / T;
        double gmu[3], gk[3], kc;
        if (!s->tp) {
          kc = mu * s->cp / c->prandtl;
          for (int b = 0; b < 3; ++b) { gmu[b] = mut * gT[b]; gk[b] = s->cp / c->prandtl * gmu[b]; }
        } else { /* k = mu c_p(T) / Pr, grad k = (c_p grad mu + mu c_p'(T) grad T) / Pr */
          double cpT = cp_of(s, T), dcpT = dcp_of(s, T);
          kc = mu * cpT / c->prandtl;
          for (int b = 0; b < 3; ++b) {
            gmu[b] = mut * gT[b];
            gk[b] = (cpT * gmu[b] + mu * dcpT * gT[b]) / c->prandtl;
          }
        }
        double th = s->div[pa];
        double uvec[3] = {s->u[pa], s->v[pa], s->w[pa]};
        double mom[3], en = 0.0;
        for (int a = 0; a < 3; ++a) {
          double m = mu * (lap[a] + gth[a] / 3.0);
          for (int b = 0; b < 3; ++b) m += gmu[b] * (g[a][b] + g[b][a]);
          m -= 2.0 / 3.0 * th * gmu[a];
          mom[a] = m;
        }
        for (int a = 0; a < 3; ++a) {
          en += uvec[a] * mom[a];
          for (int b = 0; b < 3; ++b) {
            double tau = mu * (g[a][b] + g[b][a] - (a == b ? 2.0 / 3.0 * th : 0.0));
            en += tau * g[a][b];
          }
        }
        en += kc * lapT;
        for (int b = 0; b < 3; ++b) en += gk[b] * gT[b];
        size_t q = WI(s, i, j, k);
        for (int a = 0; a < 3; ++a) rhs[(1 + a) * n + q] += mom[a];
        rhs[4 * n + q] += en;
      }
}

/* ----------------------------------------------------------------- forcing ---
 * Constant-mass-flow forcing (force_rhs_1 of Table 2): a uniform x body
 * force f = -(sum R_rhou dV)/(sum dV), dV proportional to dy/deta, added to
 * R_rhou and, times u, to R_rhoE; the bulk rho u then stays constant. */
static double forcing(ws_t *s, double *rhs) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  size_t n = s->n;
  OR_SECTION(SEC_FORCE);
  double num = 0.0, den = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j) {
      double dv = 1.0 / s->eta_y[j];
      for (int i = 0; i < nx; ++i) num += rhs[n + WI(s, i, j, k)] * dv;
      den += dv * nx;
    }
  double f = -num / den;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t q = WI(s, i, j, k);
        rhs[n + q] += f;
        rhs[4 * n + q] += f * s->u[PI(s, i, j, k)];
      }
  return f;
}

/* --------------------------------------------------------------------- RHS ---
 * R(w): primitives, sensor, convective fluxes in x, y, z, viscous terms,
 * forcing.  flags{x,y,z} (may be NULL) receive the per-interface WENO flags,
 * (n_dir + 1) per pencil. */
static int rhs_ws(ws_t *s, const double *w, double *rhs, unsigned char *fx, unsigned char *fy,
                  unsigned char *fz, int terms, double *force_out, int given) {
  memset(rhs, 0, sizeof(double) * NV * s->n);
  prims(s, w);
  sensor(s);
  if (terms & OR_CONV) {
    convective(s, 0, rhs, fx, given);
    convective(s, 1, rhs, fy, given);
    convective(s, 2, rhs, fz, given);
  }
  if ((terms & OR_VISC) && s->viscous) viscous(s, rhs);
  double f = 0.0;
  if ((terms & OR_FORCE) && s->c->force) f = forcing(s, rhs);
  if (force_out) *force_out = f;
  return 0;
}

int or_rhs(const or_cfg *c, const double *w, double *rhs, unsigned char *fx, unsigned char *fy,
           unsigned char *fz, int terms, double *force_out) {
  ws_t s;
  if (ws_init(&s, c)) { ws_free(&s); return -1; }
  rhs_ws(&s, w, rhs, fx, fy, fz, terms, force_out, 0);
  ws_free(&s);
  return 0;
}

/* R(w) with the interface WENO flags supplied by the caller (layout as
 * or_rhs writes them) instead of decided by the sensor: isolates the
 * arithmetic of another implementation from its flag decisions. */
int or_rhs_given_flags(const or_cfg *c, const double *w, double *rhs, unsigned char *fx, unsigned char *fy,
                       unsigned char *fz, int terms) {
  if (!fx || !fy || !fz) return -1;
  ws_t s;
  if (ws_init(&s, c)) { ws_free(&s); return -1; }
  rhs_ws(&s, w, rhs, fx, fy, fz, terms, NULL, 1);
  ws_free(&s);
  return 0;
}

/* Sensor and divergence at interior points, for checks. */
int or_sensor(const or_cfg *c, const double *w, double *sens, double *div) {
  ws_t s;
  if (ws_init(&s, c)) { ws_free(&s); return -1; }
  prims(&s, w);
  sensor(&s);
  for (int k = 0; k < c->nz; ++k)
    for (int j = 0; j < c->ny; ++j)
      for (int i = 0; i < c->nx; ++i) {
        sens[WI(&s, i, j, k)] = s.sens[PI(&s, i, j, k)];
        div[WI(&s, i, j, k)] = s.div[PI(&s, i, j, k)];
      }
  ws_free(&s);
  return 0;
}

/* -------------------------------------------------------------------- dt ---
 * compute_dt of Table 2: dt = cfl / max over the interior of
 *   (|u|+c)/dx + (|v|+c) eta_y + (|w|+c)/dz
 *   + gamma mu / (Pr rho) (1/dx^2 + eta_y^2 + 1/dz^2)   (viscous runs),
 * gamma = gamma(T) and c = sqrt(gamma(T) R T) for a thermally perfect gas. */
static double dt_ws(ws_t *s, const double *w, double cfl) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  const or_cfg *c = s->c;
  prims(s, w);
  OR_SECTION(SEC_DT);
  double mx = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t a = PI(s, i, j, k);
        double cs = s->cs[a], ey = s->eta_y[j];
        double sr = (fabs(s->u[a]) + cs) / s->dx + (fabs(s->v[a]) + cs) * ey + (fabs(s->w[a]) + cs) / s->dz;
        if (s->viscous) {
          double mu = pow(s->T[a] / c->t_ref, c->visc_exp) / c->re;
          sr += gamma_of(s, s->T[a]) * mu / (c->prandtl * s->rho[a]) *
                (1.0 / (s->dx * s->dx) + ey * ey + 1.0 / (s->dz * s->dz));
        }
        mx = fmax(mx, sr);
      }
  return cfl / mx;
}

double or_dt(const or_cfg *c, const double *w, double cfl) {
  ws_t s;
  if (ws_init(&s, c)) { ws_free(&s); return -1.0; }
  double dt = dt_ws(&s, w, cfl);
  ws_free(&s);
  return dt;
}

/* ------------------------------------------------------------------- RK3 ---
 * n low-storage RK3 steps of w (in place).  dt: when cfl > 0 it is
 * recomputed at the start of every step whose counter is a multiple of
 * dt_every and frozen within the step; otherwise dt_fixed.  *step_io and
 * *dt_io carry the step counter and the current dt across calls. */
int or_step(const or_cfg *c, double *w, int nsteps, double cfl, double dt_fixed, int dt_every,
            long long *step_io, double *dt_io) {
  ws_t s;
  if (ws_init(&s, c)) { ws_free(&s); return -1; }
  size_t tot = NV * s.n;
  double *R = (double *)malloc(sizeof(double) * tot);
  double *Rp = (double *)calloc(tot, sizeof(double));
  if (!R || !Rp) { free(R); free(Rp); ws_free(&s); return -1; }
  long long step = step_io ? *step_io : 0;
  double dt = dt_io ? *dt_io : dt_fixed;
  if (dt_every < 1) dt_every = 1;
  for (int it = 0; it < nsteps; ++it, ++step) {
    if (cfl > 0.0) {
      if (step % dt_every == 0 || dt <= 0.0) dt = dt_ws(&s, w, cfl);
    } else {
      dt = dt_fixed;
    }
    for (int st = 0; st < 3; ++st) {
      rhs_ws(&s, w, R, NULL, NULL, NULL, OR_CONV | OR_VISC | OR_FORCE, NULL, 0);
      OR_SECTION(SEC_UPDATE);
      for (size_t q = 0; q < tot; ++q) w[q] += dt * (RK_GAMMA[st] * R[q] + RK_RHO[st] * Rp[q]);
      double *t = Rp; Rp = R; R = t;
    }
  }
  if (step_io) *step_io = step;
  if (dt_io) *dt_io = dt;
  free(R); free(Rp);
  ws_free(&s);
  return 0;
}

/* Thermodynamic functions of the configuration's gas at T: c_p, dc_p/dT,
 * e.  Returns -1 if the configuration is invalid. */
int or_thermo(const or_cfg *c, double T, double *cp, double *dcp, double *e) {
  ws_t s;
  memset(&s, 0, sizeof(s));
  gas_init(&s, c);
  *cp = cp_of(&s, T);
  *dcp = dcp_of(&s, T);
  *e = e_of(&s, T);
  return 0;
}

/* T from the internal energy e (enthalpy = 0, the primitive recovery's
 * inversion) or from the enthalpy h (enthalpy = 1, from T0). */
double or_temperature(const or_cfg *c, double target, int enthalpy, double T0) {
  ws_t s;
  memset(&s, 0, sizeof(s));
  gas_init(&s, c);
  return enthalpy ? temperature_of(&s, target, 1, T0) : T_of_e(&s, target);
}

/* Roe state of the WENO flux between the states a and b (rho, u, v, w, T):
 * out = (u, v, w, H, chi, c). */
int or_roe_state(const or_cfg *c, const double *a, const double *b, double *out) {
  ws_t s;
  memset(&s, 0, sizeof(s));
  gas_init(&s, c);
  roe_state(&s, a, b, out);
  return 0;
}

/* RK3 on the scalar ODE y' = lambda y with the same coefficient table. */
double or_rk3_scalar(double lambda, double y0, double dt, int nsteps) {
  double y = y0, rp = 0.0;
  for (int it = 0; it < nsteps; ++it) {
    rp = 0.0;
    for (int st = 0; st < 3; ++st) {
      double r = lambda * y;
      y += dt * (RK_GAMMA[st] * r + RK_RHO[st] * rp);
      rp = r;
    }
  }
  return y;
}
