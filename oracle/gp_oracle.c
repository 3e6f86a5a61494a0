/*
 * gp_oracle.c -- plain FP64 CPU oracle for the 3D split-step Crank-Nicolson (SSCN)
 * Gross-Pitaevskii step.  TEST INFRASTRUCTURE ONLY: the test suite, the smoke
 * check and the benchmark's CPU-baseline leg are its only users.  Nothing here is
 * blocked, fused or reordered beyond the definitions below; it is meant to be read
 * against the method statement line by line.
 *
 * Sources (the paper prints the method's name, not its formulas):
 *   - Program summary, "Solution method" and the imag3d/real3d summaries: the GP
 *     equation is solved by the split-step Crank-Nicolson method, discretising in
 *     space and time and propagating over small steps in imaginary or real time.
 *   - "Nature of problem": fully anisotropic harmonic trap in 3D.
 *   - "Summary of revisions": the programs compute the dimensionless nonlinearity
 *     from the number of atoms, scattering length and oscillator length; outputs
 *     are energy, chemical potential, rms sizes and integrated densities (Eq. 1).
 *
 * Readings of what the paper leaves open (each is the textbook form):
 *   GP equation, dimensionless, oscillator units of the x trap frequency:
 *       i d(psi)/dt = [ -(1/2) Lap + V + g |psi|^2 ] psi,
 *       V = (gamma^2 x^2 + nu^2 y^2 + lambda^2 z^2) / 2,   g = 4 pi N a_s / l_osc.
 *   Imaginary time replaces t by -i tau; every imaginary step is followed by a
 *   renormalisation to unit norm.
 *   One step with tau = dt (imaginary) or tau = i dt (real):
 *     (1) pointwise potential + nonlinear substep
 *             psi <- psi * exp(-tau (V + g |psi|^2)),  |psi|^2 taken before the update;
 *     (2) for each axis a = x, y, z in that order, every grid line along a gets one
 *         Crank-Nicolson solve of the free kinetic step
 *             (1 + 2 al) u_j - al (u_{j-1} + u_{j+1}) = (1 - 2 al) v_j + al (v_{j-1} + v_{j+1}),
 *             al = tau / (4 h_a^2),  zero values on the ghost points j = -1 and j = n;
 *         solved by the Thomas recurrence with precomputed elimination coefficients;
 *     (3) imaginary time only: psi <- psi / sqrt(sum |psi|^2 dV).
 *   Grid: x_i = (i - (n-1)/2) h, every stored point an unknown, psi = 0 on the ghosts.
 *   2D (the imag2d / real2d programs; nz = 1): the same equation in the xy plane,
 *   V = (gamma^2 x^2 + nu^2 y^2) / 2, CN solves along x and y only, dV = hx hy; g is
 *   then the 2D nonlinearity (the paper does not print its reduction from the 3D
 *   inputs).
 */
#include "gp_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846264338327950288;
static int orc_threads = 1;

int orc_set_threads(int n) {
#ifdef _OPENMP
  orc_threads = n < 1 ? 1 : n;
  return orc_threads;
#else
  (void)n;
  orc_threads = 1;
  return 1;
#endif
}

/* ---------------------------------------------------------------- helpers -- */

/* Neumaier compensated sum. */
typedef struct { double s, c; } orc_sum;

static void sum_add(orc_sum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

static double sum_val(const orc_sum* a) { return a->s + a->c; }

static long npoints(const orc_problem* p) { return (long)p->nx * p->ny * p->nz; }

/* nz = 1 is a 2D problem in the xy plane: no z solve, cell area hx hy, z = 0. */
static int is2d(const orc_problem* p) { return p->nz == 1; }
static double cell(const orc_problem* p) { return p->hx * p->hy * (is2d(p) ? 1.0 : p->hz); }

static long index3(const orc_problem* p, int i, int j, int k) {
  return ((long)k * p->ny + j) * p->nx + i;
}

double orc_g_physical(double natoms, double a_s, double l_osc) {
  return 4.0 * ORC_PI * natoms * a_s / l_osc;
}

double orc_coord(int i, int n, double h) { return (i - 0.5 * (n - 1)) * h; }

static double potential(const orc_problem* p, int i, int j, int k) {
  double x = orc_coord(i, p->nx, p->hx);
  double y = orc_coord(j, p->ny, p->hy);
  double z = orc_coord(k, p->nz, p->hz);
  return 0.5 * (p->gamma * p->gamma * x * x + p->nu * p->nu * y * y +
                p->lambda * p->lambda * z * z);
}

static double complex value(const double* psi, int is_complex, long idx) {
  if (is_complex) return psi[2 * idx] + I * psi[2 * idx + 1];
  return psi[idx];
}

static double abs2(double complex v) { return creal(v) * creal(v) + cimag(v) * cimag(v); }

/* ------------------------------------------------------- Thomas, one line -- */

/* Elimination coefficients of the constant-coefficient CN matrix
 * diag b = 1 + 2a, off-diagonals -a:
 *   m_0 = 1/b,                  cp_0 = -a m_0,
 *   m_j = 1/(b + a cp_{j-1}),   cp_j = -a m_j.                                  */
static void coeffs_complex(int n, double complex a, double complex* cp, double complex* m) {
  double complex b = 1.0 + 2.0 * a;
  m[0] = 1.0 / b;
  cp[0] = -a * m[0];
  for (int j = 1; j < n; ++j) {
    m[j] = 1.0 / (b + a * cp[j - 1]);
    cp[j] = -a * m[j];
  }
}

static void coeffs_real(int n, double a, double* cp, double* m) {
  double b = 1.0 + 2.0 * a;
  m[0] = 1.0 / b;
  cp[0] = -a * m[0];
  for (int j = 1; j < n; ++j) {
    m[j] = 1.0 / (b + a * cp[j - 1]);
    cp[j] = -a * m[j];
  }
}

void orc_thomas_coeffs(int n, double are, double aim, double* cp, double* m) {
  coeffs_complex(n, are + I * aim, (double complex*)cp, (double complex*)m);
}

/* CN update of one real line v[0], v[s], ..., v[(n-1)s]; d is scratch of n. */
static void cn_line_real(int n, double a, const double* cp, const double* m, double* v,
                         long s, double* d) {
  for (int j = 0; j < n; ++j) {
    double left = j > 0 ? v[(j - 1) * s] : 0.0;
    double right = j < n - 1 ? v[(j + 1) * s] : 0.0;
    d[j] = (1.0 - 2.0 * a) * v[j * s] + a * (left + right);
  }
  d[0] = d[0] * m[0];                                       /* forward elimination */
  for (int j = 1; j < n; ++j) d[j] = (d[j] + a * d[j - 1]) * m[j];
  v[(n - 1) * s] = d[n - 1];                                /* back substitution */
  for (int j = n - 2; j >= 0; --j) v[j * s] = d[j] - cp[j] * v[(j + 1) * s];
}

/* Same for one complex line. */
static void cn_line_complex(int n, double complex a, const double complex* cp,
                            const double complex* m, double complex* v, long s,
                            double complex* d) {
  for (int j = 0; j < n; ++j) {
    double complex left = j > 0 ? v[(j - 1) * s] : 0.0;
    double complex right = j < n - 1 ? v[(j + 1) * s] : 0.0;
    d[j] = (1.0 - 2.0 * a) * v[j * s] + a * (left + right);
  }
  d[0] = d[0] * m[0];
  for (int j = 1; j < n; ++j) d[j] = (d[j] + a * d[j - 1]) * m[j];
  v[(n - 1) * s] = d[n - 1];
  for (int j = n - 2; j >= 0; --j) v[j * s] = d[j] - cp[j] * v[(j + 1) * s];
}

void orc_cn_line(int n, double are, double aim, double* v) {
  double complex a = are + I * aim;
  double complex* cp = malloc(sizeof(double complex) * n);
  double complex* m = malloc(sizeof(double complex) * n);
  double complex* d = malloc(sizeof(double complex) * n);
  coeffs_complex(n, a, cp, m);
  cn_line_complex(n, a, cp, m, (double complex*)v, 1, d);
  free(cp);
  free(m);
  free(d);
}

/* ---------------------------------------------------------- axis sweeps -- */

/* One CN solve along every line of axis 0 (x), 1 (y) or 2 (z), real field. */
static void sweep_real(const orc_problem* p, double* psi, int axis, double a) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  int n = axis == 0 ? nx : axis == 1 ? ny : nz;
  double* cp = malloc(sizeof(double) * n);
  double* m = malloc(sizeof(double) * n);
  coeffs_real(n, a, cp, m);
  if (axis == 0) {
#pragma omp parallel for collapse(2) schedule(static) num_threads(orc_threads)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j) {
        double d[n];
        cn_line_real(n, a, cp, m, psi + index3(p, 0, j, k), 1, d);
      }
  } else if (axis == 1) {
#pragma omp parallel for collapse(2) schedule(static) num_threads(orc_threads)
    for (int k = 0; k < nz; ++k)
      for (int i = 0; i < nx; ++i) {
        double d[n];
        cn_line_real(n, a, cp, m, psi + index3(p, i, 0, k), nx, d);
      }
  } else {
#pragma omp parallel for collapse(2) schedule(static) num_threads(orc_threads)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double d[n];
        cn_line_real(n, a, cp, m, psi + index3(p, i, j, 0), (long)nx * ny, d);
      }
  }
  free(cp);
  free(m);
}

static void sweep_complex(const orc_problem* p, double complex* psi, int axis,
                          double complex a) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  int n = axis == 0 ? nx : axis == 1 ? ny : nz;
  double complex* cp = malloc(sizeof(double complex) * n);
  double complex* m = malloc(sizeof(double complex) * n);
  coeffs_complex(n, a, cp, m);
  if (axis == 0) {
#pragma omp parallel for collapse(2) schedule(static) num_threads(orc_threads)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j) {
        double complex d[n];
        cn_line_complex(n, a, cp, m, psi + index3(p, 0, j, k), 1, d);
      }
  } else if (axis == 1) {
#pragma omp parallel for collapse(2) schedule(static) num_threads(orc_threads)
    for (int k = 0; k < nz; ++k)
      for (int i = 0; i < nx; ++i) {
        double complex d[n];
        cn_line_complex(n, a, cp, m, psi + index3(p, i, 0, k), nx, d);
      }
  } else {
#pragma omp parallel for collapse(2) schedule(static) num_threads(orc_threads)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double complex d[n];
        cn_line_complex(n, a, cp, m, psi + index3(p, i, j, 0), (long)nx * ny, d);
      }
  }
  free(cp);
  free(m);
}

/* ----------------------------------------------------------------- state -- */

static double norm_of(const orc_problem* p, const double* psi, int is_complex) {
  orc_sum s = {0.0, 0.0};
  long n = npoints(p);
  for (long idx = 0; idx < n; ++idx) sum_add(&s, abs2(value(psi, is_complex, idx)));
  return sum_val(&s) * cell(p);
}

void orc_init_gaussian(const orc_problem* p, double wx, double wy, double wz, double* psi) {
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        double x = orc_coord(i, p->nx, p->hx);
        double y = orc_coord(j, p->ny, p->hy);
        double z = orc_coord(k, p->nz, p->hz);
        psi[index3(p, i, j, k)] = exp(-0.5 * (wx * x * x + wy * y * y + wz * z * z));
      }
  double sc = 1.0 / sqrt(norm_of(p, psi, 0));
  long n = npoints(p);
  for (long idx = 0; idx < n; ++idx) psi[idx] *= sc;
}

/* ------------------------------------------------------------ time steps -- */

int orc_step_imag(const orc_problem* p, double* psi, long nsteps) {
  long n = npoints(p);
  for (long step = 0; step < nsteps; ++step) {
    /* (1) psi <- psi exp(-dt (V + g psi^2)) */
    for (int k = 0; k < p->nz; ++k)
      for (int j = 0; j < p->ny; ++j)
        for (int i = 0; i < p->nx; ++i) {
          long idx = index3(p, i, j, k);
          double v = psi[idx];
          psi[idx] = v * exp(-p->dt * (potential(p, i, j, k) + p->g * v * v));
        }
    /* (2) CN kinetic solves along x, y, z with al = dt / (4 h^2) */
    sweep_real(p, psi, 0, p->dt / (4.0 * p->hx * p->hx));
    sweep_real(p, psi, 1, p->dt / (4.0 * p->hy * p->hy));
    if (!is2d(p)) sweep_real(p, psi, 2, p->dt / (4.0 * p->hz * p->hz));
    /* (3) renormalise to unit norm */
    double nrm = norm_of(p, psi, 0);
    if (!(nrm > 0.0) || !isfinite(nrm)) return -4;
    double sc = 1.0 / sqrt(nrm);
    for (long idx = 0; idx < n; ++idx) psi[idx] *= sc;
  }
  return 0;
}

int orc_step_real(const orc_problem* p, double* psi_interleaved, long nsteps) {
  double complex* psi = (double complex*)psi_interleaved;
  for (long step = 0; step < nsteps; ++step) {
    /* (1) psi <- psi exp(-i dt (V + g |psi|^2)) */
    for (int k = 0; k < p->nz; ++k)
      for (int j = 0; j < p->ny; ++j)
        for (int i = 0; i < p->nx; ++i) {
          long idx = index3(p, i, j, k);
          double complex v = psi[idx];
          double theta = p->dt * (potential(p, i, j, k) + p->g * abs2(v));
          psi[idx] = v * cexp(-I * theta);
        }
    /* (2) CN kinetic solves along x, y, z with al = i dt / (4 h^2) */
    sweep_complex(p, psi, 0, I * (p->dt / (4.0 * p->hx * p->hx)));
    sweep_complex(p, psi, 1, I * (p->dt / (4.0 * p->hy * p->hy)));
    if (!is2d(p)) sweep_complex(p, psi, 2, I * (p->dt / (4.0 * p->hz * p->hz)));
  }
  for (long idx = 0; idx < npoints(p); ++idx)
    if (!isfinite(creal(psi[idx])) || !isfinite(cimag(psi[idx]))) return -4;
  return 0;
}

/* ------------------------------------------------- Strang-split steps -- */
/* The symmetric (Strang) splitting, a variant beside the Lie step above: one step is
 *   (1) pointwise substep with tau / 2, (2) the CN solves along x, y, z with tau,
 *   (3) pointwise substep with tau / 2, each pointwise substep taking |psi|^2 before
 *   its own update; imaginary time then renormalises.  Second order in dt, where
 *   the Lie step is first order.                                                  */

static void half_pointwise_real(const orc_problem* p, double* psi) {
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        long idx = index3(p, i, j, k);
        double v = psi[idx];
        psi[idx] = v * exp(-0.5 * p->dt * (potential(p, i, j, k) + p->g * v * v));
      }
}

static void half_pointwise_complex(const orc_problem* p, double complex* psi) {
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        long idx = index3(p, i, j, k);
        double complex v = psi[idx];
        double theta = 0.5 * p->dt * (potential(p, i, j, k) + p->g * abs2(v));
        psi[idx] = v * cexp(-I * theta);
      }
}

int orc_step_imag_strang(const orc_problem* p, double* psi, long nsteps) {
  long n = npoints(p);
  for (long step = 0; step < nsteps; ++step) {
    half_pointwise_real(p, psi);
    sweep_real(p, psi, 0, p->dt / (4.0 * p->hx * p->hx));
    sweep_real(p, psi, 1, p->dt / (4.0 * p->hy * p->hy));
    if (!is2d(p)) sweep_real(p, psi, 2, p->dt / (4.0 * p->hz * p->hz));
    half_pointwise_real(p, psi);
    double nrm = norm_of(p, psi, 0);
    if (!(nrm > 0.0) || !isfinite(nrm)) return -4;
    double sc = 1.0 / sqrt(nrm);
    for (long idx = 0; idx < n; ++idx) psi[idx] *= sc;
  }
  return 0;
}

int orc_step_real_strang(const orc_problem* p, double* psi_interleaved, long nsteps) {
  double complex* psi = (double complex*)psi_interleaved;
  for (long step = 0; step < nsteps; ++step) {
    half_pointwise_complex(p, psi);
    sweep_complex(p, psi, 0, I * (p->dt / (4.0 * p->hx * p->hx)));
    sweep_complex(p, psi, 1, I * (p->dt / (4.0 * p->hy * p->hy)));
    if (!is2d(p)) sweep_complex(p, psi, 2, I * (p->dt / (4.0 * p->hz * p->hz)));
    half_pointwise_complex(p, psi);
  }
  for (long idx = 0; idx < npoints(p); ++idx)
    if (!isfinite(creal(psi[idx])) || !isfinite(cimag(psi[idx]))) return -4;
  return 0;
}

/* ----------------------------------------------------------- observables -- */

/* Sum over the edges of every line along one axis, ghost edges included, of
 * |psi_{j+1} - psi_j|^2 with psi_{-1} = psi_n = 0.                             */
static double edge_sum(const orc_problem* p, const double* psi, int is_complex, int axis) {
  orc_sum s = {0.0, 0.0};
  int nx = p->nx, ny = p->ny, nz = p->nz;
  int n = axis == 0 ? nx : axis == 1 ? ny : nz;
  int la = axis == 0 ? ny : nx;  /* the two axes other than `axis` */
  int lb = axis == 2 ? ny : nz;
  for (int b = 0; b < lb; ++b)
    for (int a = 0; a < la; ++a)
      for (int j = -1; j < n; ++j) {
        double complex lo = 0.0, hi = 0.0;
        int i0, j0, k0;
        if (axis == 0) { i0 = j; j0 = a; k0 = b; }
        else if (axis == 1) { i0 = a; j0 = j; k0 = b; }
        else { i0 = a; j0 = b; k0 = j; }
        if (j >= 0) lo = value(psi, is_complex, index3(p, i0, j0, k0));
        if (j + 1 < n) {
          int i1 = i0 + (axis == 0), j1 = j0 + (axis == 1), k1 = k0 + (axis == 2);
          hi = value(psi, is_complex, index3(p, i1, j1, k1));
        }
        sum_add(&s, abs2(hi - lo));
      }
  return sum_val(&s);
}

void orc_observables(const orc_problem* p, const double* psi, int is_complex, double* out) {
  orc_sum nrm = {0, 0}, ep = {0, 0}, e4 = {0, 0}, sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        double d = abs2(value(psi, is_complex, index3(p, i, j, k)));
        double x = orc_coord(i, p->nx, p->hx);
        double y = orc_coord(j, p->ny, p->hy);
        double z = orc_coord(k, p->nz, p->hz);
        sum_add(&nrm, d);
        sum_add(&ep, potential(p, i, j, k) * d);
        sum_add(&e4, d * d);
        sum_add(&sx, x * x * d);
        sum_add(&sy, y * y * d);
        sum_add(&sz, z * z * d);
      }
  double dV = cell(p);
  double norm = sum_val(&nrm) * dV;
  double ekin = 0.5 * dV *
                (edge_sum(p, psi, is_complex, 0) / (p->hx * p->hx) +
                 edge_sum(p, psi, is_complex, 1) / (p->hy * p->hy) +
                 (is2d(p) ? 0.0 : edge_sum(p, psi, is_complex, 2) / (p->hz * p->hz)));
  double epot = sum_val(&ep) * dV;
  double eint = 0.5 * p->g * sum_val(&e4) * dV;
  double x2 = sum_val(&sx) * dV / norm;
  double y2 = sum_val(&sy) * dV / norm;
  double z2 = sum_val(&sz) * dV / norm;
  out[0] = norm;
  out[1] = ekin + epot + 2.0 * eint; /* chemical potential */
  out[2] = ekin + epot + eint;       /* energy */
  out[3] = ekin;
  out[4] = epot;
  out[5] = eint;
  out[6] = sqrt(x2);
  out[7] = sqrt(y2);
  out[8] = sqrt(z2);
  out[9] = sqrt(x2 + y2 + z2);
}

/* ------------------------------------------------------------- densities -- */

void orc_density1d(const orc_problem* p, const double* psi, int is_complex, int axis,
                   double* out) {
  int n = axis == 0 ? p->nx : axis == 1 ? p->ny : p->nz;
  const double hz = is2d(p) ? 1.0 : p->hz;
  double w = axis == 0 ? p->hy * hz : axis == 1 ? p->hx * hz : p->hx * p->hy;
  orc_sum* s = calloc(n, sizeof(orc_sum));
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        int o = axis == 0 ? i : axis == 1 ? j : k;
        sum_add(&s[o], abs2(value(psi, is_complex, index3(p, i, j, k))));
      }
  for (int o = 0; o < n; ++o) out[o] = sum_val(&s[o]) * w;
  free(s);
}

void orc_density2d(const orc_problem* p, const double* psi, int is_complex, int plane,
                   double* out) {
  long n = plane == 0 ? (long)p->nx * p->ny : plane == 1 ? (long)p->nx * p->nz
                                                         : (long)p->ny * p->nz;
  double w = plane == 0 ? (is2d(p) ? 1.0 : p->hz) : plane == 1 ? p->hy : p->hx;
  orc_sum* s = calloc(n, sizeof(orc_sum));
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        long o = plane == 0 ? (long)j * p->nx + i
                 : plane == 1 ? (long)k * p->nx + i
                              : (long)k * p->ny + j;
        sum_add(&s[o], abs2(value(psi, is_complex, index3(p, i, j, k))));
      }
  for (long o = 0; o < n; ++o) out[o] = sum_val(&s[o]) * w;
  free(s);
}
