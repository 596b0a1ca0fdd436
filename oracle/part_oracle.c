/*
 * part_oracle.c -- plain FP64 CPU oracle for the particle advance.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  Shares no code
 * with the CUDA library.  Build: gcc -O2 -ffp-contract=off -fopenmp -shared.
 *
 * Every routine states the definition it writes out.  Loops over particles in
 * the per-particle routines are independent (OpenMP may split them); sums that
 * combine particles (the deposit) run strictly in particle index order.
 *
 * Parity unpinned: the code-unit synchrotron coefficient c_r = c0 (|B|^2/2 +
 * U_rad) (the paper prints c_r only in cgs units, Eq. rad_losses).
 */
#include "part_oracle.h"
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

/* ---- shape functions (textbook; the paper only says LPs "sample" fluid
 * quantities, Sec. 2).  xi = (cell centre - particle) in cell units.        */
double or_shape(int shape, double xi) {
  double a = fabs(xi);
  if (shape == OR_CIC) {              /* hat function, support |xi| < 1     */
    return a < 1.0 ? 1.0 - a : 0.0;
  }
  /* TSC: quadratic B-spline, support |xi| < 3/2 */
  if (a <= 0.5) return 0.75 - a * a;
  if (a < 1.5) { double b = 1.5 - a; return 0.5 * b * b; }
  return 0.0;
}

/* Cell index j = floor((x - xmin) / dx) with 1/dx formed once; the upper edge
 * tie (rounding to j == n) goes to n-1.  delta = (s - j) - 1/2.  On an open
 * axis s is first clamped to [0, n]: beyond the boundary a particle samples
 * (and deposits at) the boundary itself, which with the zero-gradient ghost
 * layer below continues the edge values outwards.                          */
void or_cell_coord(const or_grid* g, const double* x, int* j, double* delta) {
  for (int a = 0; a < 3; ++a) {
    if (a >= g->dim) { j[a] = 0; delta[a] = 0.0; continue; }
    double inv = 1.0 / g->dx[a];
    double s = (x[a] - g->xmin[a]) * inv;
    if (g->open[a]) {
      if (s < 0.0) s = 0.0;
      if (s > (double)g->n[a]) s = (double)g->n[a];
    }
    double f = floor(s);
    int jj = (int)f;
    if (jj >= g->n[a]) jj = g->n[a] - 1;
    if (jj < 0) jj = 0;
    j[a] = jj;
    delta[a] = (s - (double)jj) - 0.5;
  }
}

/* Periodic wrap by one domain length L = n dx into [xmin, xmin + L); an open
 * axis is not wrapped. */
double or_wrap(const or_grid* g, int axis, double x) {
  if (g->open[axis]) return x;
  double L = (double)g->n[axis] * g->dx[axis];
  double xmax = g->xmin[axis] + L;
  if (x < g->xmin[axis]) x = x + L;
  else if (x >= xmax) x = x - L;
  return x;
}

static int64_t cell_linear(const or_grid* g, int jx, int jy, int jz) {
  return ((int64_t)jz * g->n[1] + jy) * g->n[0] + jx;
}

static int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* Neighbour index along an axis: periodic, or clamped to the edge cell on an
 * open axis (a zero-gradient ghost layer; deposits there fold onto the edge
 * cell, the exact adjoint of that gather). */
static int nbr(const or_grid* g, int a, int j) {
  if (!g->open[a]) return pmod(j, g->n[a]);
  return j < 0 ? 0 : (j >= g->n[a] ? g->n[a] - 1 : j);
}

int or_outside(const or_grid* g, const double* x) {
  for (int a = 0; a < g->dim; ++a) {
    if (!g->open[a]) continue;
    double L = (double)g->n[a] * g->dx[a];
    if (x[a] < g->xmin[a] || x[a] >= g->xmin[a] + L) return 1;
  }
  return 0;
}

/* F(x_p) = sum_k W(k_x - d_x) W(k_y - d_y) W(k_z - d_z) f[j + k], periodic,
 * k in {-1,0,1}^dim, cell-centred fields [comp][z][y][x].                   */
void or_gather(const or_grid* g, int shape, const double* fields, int ncomp,
               const double* x, double* out) {
  int j[3]; double d[3];
  or_cell_coord(g, x, j, d);
  int64_t G = (int64_t)g->n[0] * g->n[1] * g->n[2];
  for (int c = 0; c < ncomp; ++c) out[c] = 0.0;
  int kz0 = g->dim == 3 ? -1 : 0, kz1 = g->dim == 3 ? 1 : 0;
  for (int kz = kz0; kz <= kz1; ++kz) {
    double wz = g->dim == 3 ? or_shape(shape, kz - d[2]) : 1.0;
    for (int ky = -1; ky <= 1; ++ky) {
      double wy = or_shape(shape, ky - d[1]);
      for (int kx = -1; kx <= 1; ++kx) {
        double wx = or_shape(shape, kx - d[0]);
        double w = (wz * wy) * wx;
        int64_t cell = cell_linear(g, nbr(g, 0, j[0] + kx), nbr(g, 1, j[1] + ky),
                                   nbr(g, 2, j[2] + kz));
        for (int c = 0; c < ncomp; ++c) out[c] += w * fields[(int64_t)c * G + cell];
      }
    }
  }
}

/* Relativistic Boris (Boris 1970; Birdsall & Langdon Sec. 15-4), c = 1:
 *   h = (q/m) dt/2;  u- = u + h E;  g- = sqrt(1 + |u-|^2)
 *   t = h B / g-;  s = 2 t / (1 + |t|^2)
 *   u' = u- + u- x t;  u+ = u- + u' x s;  u_new = u+ + h E                   */
void or_boris_kick(double* u, const double* E, const double* B, double qm, double dt) {
  double h = qm * dt * 0.5;
  double um[3], t[3], s[3], up[3], upl[3];
  for (int a = 0; a < 3; ++a) um[a] = u[a] + h * E[a];
  double gm = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]));
  for (int a = 0; a < 3; ++a) t[a] = (h / gm) * B[a];
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + t2);
  upl[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  upl[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  upl[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  up[0] = um[0] + (upl[1] * s[2] - upl[2] * s[1]);
  up[1] = um[1] + (upl[2] * s[0] - upl[0] * s[2]);
  up[2] = um[2] + (upl[0] * s[1] - upl[1] * s[0]);
  for (int a = 0; a < 3; ++a) u[a] = up[a] + h * E[a];
}

/* One step: fields sampled at x^n (E = comps 0-2, B = comps 3-5), Boris kick,
 * drift x^{n+1} = x^n + dt u^{n+1}/gamma^{n+1} on the dim spatial axes, wrap.
 * The force deposited later is F_p = w_p (u^{n+1} - u^n)/dt (m = 1).        */
void or_boris_step(const or_grid* g, int shape, const double* fields6, int64_t n,
                   double* x, double* u, const double* w, double qm, double dt,
                   double* F_out, double* x_old_out) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    double xp[3], up[3], f[6], u0[3];
    for (int a = 0; a < 3; ++a) { xp[a] = x[a * n + p]; up[a] = u[a * n + p]; u0[a] = up[a]; }
    if (x_old_out) for (int a = 0; a < 3; ++a) x_old_out[a * n + p] = xp[a];
    or_gather(g, shape, fields6, 6, xp, f);
    or_boris_kick(up, f, f + 3, qm, dt);
    double gam = sqrt(1.0 + (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]));
    for (int a = 0; a < g->dim; ++a) xp[a] = or_wrap(g, a, xp[a] + dt * (up[a] / gam));
    for (int a = 0; a < 3; ++a) { x[a * n + p] = xp[a]; u[a * n + p] = up[a]; }
    if (F_out) {
      double wp = w ? w[p] : 1.0;
      for (int a = 0; a < 3; ++a) F_out[a * n + p] = wp * ((up[a] - u0[a]) / dt);
    }
  }
}

/* F_g = sum_p W(x_g - x_p) F_p with the gather's shape and stencil; particle
 * index order, then the stencil order of or_gather.                         */
void or_deposit(const or_grid* g, int shape, int64_t n, const double* x,
                const double* F, double* out) {
  int64_t G = (int64_t)g->n[0] * g->n[1] * g->n[2];
  memset(out, 0, sizeof(double) * 3 * G);
  int kz0 = g->dim == 3 ? -1 : 0, kz1 = g->dim == 3 ? 1 : 0;
  for (int64_t p = 0; p < n; ++p) {
    double xp[3] = {x[p], x[n + p], x[2 * n + p]};
    int j[3]; double d[3];
    or_cell_coord(g, xp, j, d);
    for (int kz = kz0; kz <= kz1; ++kz) {
      double wz = g->dim == 3 ? or_shape(shape, kz - d[2]) : 1.0;
      for (int ky = -1; ky <= 1; ++ky) {
        double wy = or_shape(shape, ky - d[1]);
        for (int kx = -1; kx <= 1; ++kx) {
          double wx = or_shape(shape, kx - d[0]);
          double w = (wz * wy) * wx;
          int64_t cell = cell_linear(g, nbr(g, 0, j[0] + kx), nbr(g, 1, j[1] + ky),
                                     nbr(g, 2, j[2] + kz));
          for (int c = 0; c < 3; ++c) out[(int64_t)c * G + cell] += w * F[(int64_t)c * n + p];
        }
      }
    }
  }
}

void or_deposit_cell(const or_grid* g, int shape, int64_t n, const double* x,
                     const double* F, int64_t cell, double* out3) {
  out3[0] = out3[1] = out3[2] = 0.0;
  int kz0 = g->dim == 3 ? -1 : 0, kz1 = g->dim == 3 ? 1 : 0;
  for (int64_t p = 0; p < n; ++p) {
    double xp[3] = {x[p], x[n + p], x[2 * n + p]};
    int j[3]; double d[3];
    or_cell_coord(g, xp, j, d);
    for (int kz = kz0; kz <= kz1; ++kz) {
      for (int ky = -1; ky <= 1; ++ky) {
        for (int kx = -1; kx <= 1; ++kx) {
          int64_t c0 = cell_linear(g, nbr(g, 0, j[0] + kx), nbr(g, 1, j[1] + ky),
                                   nbr(g, 2, j[2] + kz));
          if (c0 != cell) continue;
          double wz = g->dim == 3 ? or_shape(shape, kz - d[2]) : 1.0;
          double w = (wz * or_shape(shape, ky - d[1])) * or_shape(shape, kx - d[0]);
          for (int c = 0; c < 3; ++c) out3[c] += w * F[(int64_t)c * n + p];
        }
      }
    }
  }
}

/* Cell key: the grid is cut into bricks of b[0] x b[1] x b[2] cells (the last
 * brick on an axis may be partial); key = brick index * brick volume + cell
 * index inside the brick, both x-fastest.  A bijection from cells to keys.  */
uint32_t or_cell_key(const or_grid* g, const int* b, const int* j) {
  int nb0 = (g->n[0] + b[0] - 1) / b[0], nb1 = (g->n[1] + b[1] - 1) / b[1];
  int64_t V = (int64_t)b[0] * b[1] * b[2];
  int64_t brick = ((int64_t)(j[2] / b[2]) * nb1 + j[1] / b[1]) * nb0 + j[0] / b[0];
  int64_t local = ((int64_t)(j[2] % b[2]) * b[1] + j[1] % b[1]) * b[0] + j[0] % b[0];
  return (uint32_t)(brick * V + local);
}

int64_t or_key_count(const or_grid* g, const int* b) {
  int64_t nb = 1;
  for (int a = 0; a < 3; ++a) nb *= (g->n[a] + b[a] - 1) / b[a];
  return nb * b[0] * b[1] * b[2];
}

void or_keys(const or_grid* g, const int* b, int64_t n, const double* x, uint32_t* keys) {
  for (int64_t p = 0; p < n; ++p) {
    double xp[3] = {x[p], x[n + p], x[2 * n + p]};
    int j[3]; double d[3];
    or_cell_coord(g, xp, j, d);
    keys[p] = or_cell_key(g, b, j);
  }
}

typedef struct { uint32_t key; uint32_t idx; } kv_t;
static int kv_cmp(const void* a, const void* b) {
  const kv_t* x = (const kv_t*)a; const kv_t* y = (const kv_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/* Stable sort by key: ordering (key, original index) pairs lexicographically
 * keeps equal keys in their current order.                                  */
void or_stable_sort(int64_t n, const uint32_t* keys, uint32_t* perm) {
  kv_t* t = (kv_t*)malloc(sizeof(kv_t) * (n > 0 ? n : 1));
  for (int64_t p = 0; p < n; ++p) { t[p].key = keys[p]; t[p].idx = (uint32_t)p; }
  qsort(t, (size_t)n, sizeof(kv_t), kv_cmp);
  for (int64_t p = 0; p < n; ++p) perm[p] = t[p].idx;
  free(t);
}

void or_cell_start(int64_t nkeys, int64_t n, const uint32_t* sk, uint32_t* cs) {
  int64_t p = 0;
  for (int64_t c = 0; c <= nkeys; ++c) {
    while (p < n && (int64_t)sk[p] < c) ++p;
    cs[c] = (uint32_t)p;
  }
}

/* LP advection, Eq. push, with a second-order Runge-Kutta (Heun) step:
 *   v1 = v(x^n); x* = x^n + dt v1; v2 = v(x*); x^{n+1} = x^n + dt (v1+v2)/2
 * then samples at x^{n+1}: n_new = rho, gamma_g = 1/sqrt(1-|v|^2) (proper
 * time d tau = dt/gamma_g, Sec. 2), b2m = (|B(x^n)|^2 + |B(x^{n+1})|^2)/2.  */
void or_lp_rk2_step(const or_grid* g, int shape, const double* vel, const double* rho,
                    const double* bfield, int64_t n, double* x, double dt,
                    double* n_new, double* b2m, double* gam) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    double x0[3], xs[3], x1[3], v1[3], v2[3], b0[3], b1[3], v3[3], r;
    for (int a = 0; a < 3; ++a) x0[a] = xs[a] = x1[a] = x[a * n + p];
    or_gather(g, shape, vel, 3, x0, v1);
    or_gather(g, shape, bfield, 3, x0, b0);
    for (int a = 0; a < g->dim; ++a) xs[a] = or_wrap(g, a, x0[a] + dt * v1[a]);
    or_gather(g, shape, vel, 3, xs, v2);
    for (int a = 0; a < g->dim; ++a)
      x1[a] = or_wrap(g, a, x0[a] + dt * (0.5 * (v1[a] + v2[a])));
    or_gather(g, shape, rho, 1, x1, &r);
    or_gather(g, shape, bfield, 3, x1, b1);
    or_gather(g, shape, vel, 3, x1, v3);
    for (int a = 0; a < 3; ++a) x[a * n + p] = x1[a];
    double bb0 = b0[0] * b0[0] + b0[1] * b0[1] + b0[2] * b0[2];
    double bb1 = b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2];
    double vv = v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2];
    n_new[p] = r;
    b2m[p] = 0.5 * (bb0 + bb1);
    gam[p] = 1.0 / sqrt(1.0 - vv);
  }
}

/* Third-order LP advection: the three-stage strong-stability-preserving
 * Runge-Kutta scheme (Shu & Osher 1988) applied to Eq. push, written with
 * the stage velocities so that the periodic wrap only enters the positions
 * where v is sampled:
 *   k1 = v(x),  k2 = v(x + dt k1),  k3 = v(x + dt (k1 + k2)/4),
 *   x' = x + dt (k1 + k2 + 4 k3)/6.
 * (Its Shu-Osher form x1 = x + dt v(x), x2 = 3/4 x + 1/4 (x1 + dt v(x1)),
 * x' = 1/3 x + 2/3 (x2 + dt v(x2)) expands to exactly these stages.)
 * Samples at x^{n+1} as in the second-order step.                          */
void or_lp_rk3_step(const or_grid* g, int shape, const double* vel, const double* rho,
                    const double* bfield, int64_t n, double* x, double dt,
                    double* n_new, double* b2m, double* gam) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    double x0[3], xa[3], xb[3], x1[3], k1[3], k2[3], k3[3], b0[3], b1[3], v3[3], r;
    for (int a = 0; a < 3; ++a) x0[a] = xa[a] = xb[a] = x1[a] = x[a * n + p];
    or_gather(g, shape, vel, 3, x0, k1);
    or_gather(g, shape, bfield, 3, x0, b0);
    for (int a = 0; a < g->dim; ++a) xa[a] = or_wrap(g, a, x0[a] + dt * k1[a]);
    or_gather(g, shape, vel, 3, xa, k2);
    for (int a = 0; a < g->dim; ++a)
      xb[a] = or_wrap(g, a, x0[a] + dt * (0.25 * (k1[a] + k2[a])));
    or_gather(g, shape, vel, 3, xb, k3);
    for (int a = 0; a < g->dim; ++a)
      x1[a] = or_wrap(g, a, x0[a] + dt * ((k1[a] + k2[a] + 4.0 * k3[a]) / 6.0));
    or_gather(g, shape, rho, 1, x1, &r);
    or_gather(g, shape, bfield, 3, x1, b1);
    or_gather(g, shape, vel, 3, x1, v3);
    for (int a = 0; a < 3; ++a) x[a * n + p] = x1[a];
    double bb0 = b0[0] * b0[0] + b0[1] * b0[1] + b0[2] * b0[2];
    double bb1 = b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2];
    double vv = v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2];
    n_new[p] = r;
    b2m[p] = 0.5 * (bb0 + bb1);
    gam[p] = 1.0 / sqrt(1.0 - vv);
  }
}

/* Spectral update away from shocks, Eq. cr_chi, by exact characteristics.
 * Along a characteristic d eps/d tau = -a3 eps - c_r eps^2, a3 = div(u)/3
 * (Eqs. cr_N, rad_losses).  With y = 1/eps this is linear, dy/dtau = a3 y +
 * c_r, so over d tau with a3, c_r frozen:  y1 = A y0 + C,
 *   A = exp(a3 dtau),  C = c_r dtau expm1(a3 dtau)/(a3 dtau).
 * Continuity (div(n u) = 0, Sec. 2) gives a3 dtau = ln(n_old/n_new)/3.
 * chi dEps is conserved along characteristics (Eq. cr_chi is a conservation
 * law in eps), so with s = A + C eps0: eps1 = eps0/s, chi1 = chi0 s^2/A.
 * c_r = c0 (|B|^2/2 + U_rad) in code units, dtau = dt/gamma_g.             */
void or_spec_update(int nb, int64_t n, double* chi, double* eng, double* n_old,
                    const double* n_new, const double* b2m, const double* gam,
                    double dt, double c0, double u_rad) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    double dtau = dt / gam[p];
    double L = log(n_old[p] / n_new[p]) / 3.0;
    double A = exp(L);
    double cr = c0 * (0.5 * b2m[p] + u_rad);
    double C = cr * dtau * (L == 0.0 ? 1.0 : expm1(L) / L);
    for (int i = 0; i < nb; ++i) {
      double e = eng[(int64_t)i * n + p];
      double s = A + C * e;
      eng[(int64_t)i * n + p] = e / s;
      chi[(int64_t)i * n + p] = (chi[(int64_t)i * n + p] * (s * s)) / A;
    }
    n_old[p] = n_new[p];
  }
}

/* Eq. initSpec on N_b log-spaced nodes from emin to emax (both included). */
void or_init_spectrum(int nb, double emin, double emax, double p, double N0,
                      double* eng, double* chi) {
  double la = log(emin), lb = log(emax);
  double norm = N0 * (1.0 - p) / (pow(emax, 1.0 - p) - pow(emin, 1.0 - p));
  for (int i = 0; i < nb; ++i) {
    double e = nb > 1 ? exp(la + (lb - la) * ((double)i / (double)(nb - 1))) : emin;
    eng[i] = e;
    chi[i] = norm * pow(e, -p);
  }
}

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
 * -> 64-bit multiplies with a word permutation and a Weyl-sequence key.    */
void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw r in (0,1) from a 32-bit word: (r + 1/2) 2^-32 (exact in double). */
static double u01(uint32_t r) { return ((double)r + 0.5) * 2.3283064365386963e-10; }

/* Particle p: key = seed; counter (p, 0) gives the position (uniform over
 * the domain), counter (p, 1) gives three Box-Muller normals for u (each
 * component N(0, u_th^2)); w = 1; id = p.                                   */
void or_init_particles(const or_grid* g, int64_t n, uint64_t seed, double u_th,
                       double* x, double* u, double* w, uint64_t* id) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    uint32_t c0[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), 0u, 0u};
    uint32_t c1[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), 1u, 0u};
    uint32_t r0[4], r1[4];
    or_philox4x32_10(c0, key, r0);
    or_philox4x32_10(c1, key, r1);
    for (int a = 0; a < 3; ++a) {
      double L = (double)g->n[a] * g->dx[a];
      x[a * n + p] = or_wrap(g, a, g->xmin[a] + L * u01(r0[a]));
    }
    double rad0 = sqrt(-2.0 * log(u01(r1[0])));
    double rad1 = sqrt(-2.0 * log(u01(r1[2])));
    double ph0 = (2.0 * M_PI) * u01(r1[1]);
    double ph1 = (2.0 * M_PI) * u01(r1[3]);
    u[p] = u_th * (rad0 * cos(ph0));
    u[n + p] = u_th * (rad0 * sin(ph0));
    u[2 * n + p] = u_th * (rad1 * cos(ph1));
    if (w) w[p] = 1.0;
    if (id) id[p] = (uint64_t)p;
  }
}

/* Compaction after deletions, following the five steps of Sec. 3.2:
 *  1. flag and count the N_del particles to delete (holes);
 *  2. save the hole indices, in increasing order;
 *  3. if there are holes, collect the fillers: particles stored at an index
 *     at or beyond N_p - N_del that are not deleted, in increasing order;
 *  4. copy the k-th filler into the k-th hole below N_p - N_del;
 *  5. shrink to N_p - N_del.
 * The result is given as the source index of every kept slot.               */
int64_t or_compact_map(int64_t n, const uint8_t* del, int64_t* src) {
  int64_t ndel = 0;
  for (int64_t i = 0; i < n; ++i) ndel += del[i] ? 1 : 0;              /* step 1 */
  const int64_t nkeep = n - ndel;
  int64_t* holes = (int64_t*)malloc(sizeof(int64_t) * (ndel > 0 ? ndel : 1));
  int64_t nh = 0;
  for (int64_t i = 0; i < n; ++i)                                       /* step 2 */
    if (del[i]) holes[nh++] = i;
  for (int64_t j = 0; j < nkeep; ++j) src[j] = j;
  if (ndel > 0) {
    int64_t k = 0;
    for (int64_t i = nkeep; i < n; ++i) {                               /* step 3 */
      if (del[i]) continue;
      /* step 4: the k-th filler goes to the k-th hole (all holes that lie
       * below nkeep come first in the sorted hole list) */
      src[holes[k]] = i;
      ++k;
    }
  }
  free(holes);
  return nkeep;                                                         /* step 5 */
}

/* ---- diffusive shock acceleration (Sec. 2, Eqs. convolution_spectra, slope)
 *
 * Compression ratio of a hydrodynamic shock from the Rankine-Hugoniot jump
 * conditions (Sec. 4.1.2): r = (gamma+1) M^2 / (2 + (gamma-1) M^2).        */
double or_rh_compression(double gamma, double mach) {
  double m2 = mach * mach;
  return (gamma + 1.0) * m2 / (2.0 + (gamma - 1.0) * m2);
}

/* Power-law index of the accelerated spectrum, Eq. slope, non-relativistic
 * shock (the relativistic correction q_R is zero): q = 3r/(r-1).            */
double or_dsa_index(double r) { return 3.0 * r / (r - 1.0); }

/* Eq. slope for a relativistic shock.  The paper adds a correction q_R that
 * depends on the upstream and downstream flow speeds and takes its form from
 * the literature; this oracle takes the index of Keshet & Waxman (2005) for
 * isotropic small-angle scattering, with beta_u > beta_d the normal flow
 * speeds on either side in the shock's rest frame, in units of c:
 *   q = (3 beta_u - 2 beta_u beta_d^2 + beta_d^3) / (beta_u - beta_d),
 * i.e. q_R = q - 3r/(r-1).  At small speeds mass conservation gives
 * beta_u / beta_d = r and q -> 3r/(r-1); an ultra-relativistic shock
 * (beta_u -> 1, beta_d -> 1/3) gives q = 38/9, the energy index 20/9.      */
double or_kw_index(double beta_u, double beta_d) {
  return (3.0 * beta_u - 2.0 * beta_u * beta_d * beta_d + beta_d * beta_d * beta_d) /
         (beta_u - beta_d);
}

/* Normal flow speeds on both sides of a shock in its rest frame.  Inputs:
 * the lab-frame velocity component v along the shock normal, the squared
 * speed s2 = |v|^2 (all components; c = 1), and the proper density rho, for
 * the upstream (u) and downstream (d) states.  The lab-frame mass density is
 * D = rho / sqrt(1 - s2); continuity, d_t D + d_n (D v) = 0, across a front
 * moving at v_sh requires v_sh (D_d - D_u) = D_d v_d - D_u v_u.  A boost
 * along the normal by v_sh turns a normal velocity v into
 * (v - v_sh) / (1 - v v_sh) (relativistic velocity addition); the speeds are
 * the magnitudes of those.  Returns 0 (no frame) if a speed is not below 1,
 * D_d = D_u, |v_sh| >= 1, or the flow does not slow down across the front
 * (beta_d >= beta_u); NaN inputs fail these tests too.                     */
int or_shock_frame_speeds(double v_u, double s2_u, double rho_u, double v_d, double s2_d,
                          double rho_d, double* beta_u, double* beta_d) {
  if (!(s2_u < 1.0 && s2_d < 1.0)) return 0;
  double D_u = rho_u / sqrt(1.0 - s2_u);
  double D_d = rho_d / sqrt(1.0 - s2_d);
  if (!(D_d != D_u)) return 0;
  double v_sh = (D_d * v_d - D_u * v_u) / (D_d - D_u);
  if (!(fabs(v_sh) < 1.0)) return 0;
  double bu = fabs((v_u - v_sh) / (1.0 - v_u * v_sh));
  double bd = fabs((v_d - v_sh) / (1.0 - v_d * v_sh));
  if (!(bd < bu)) return 0;
  *beta_u = bu;
  *beta_d = bd;
  return 1;
}

/* Index q of Eq. slope for every shock cell of or_shock_cells (r_cell > 0;
 * q_cell = 0 elsewhere).  relativistic = 0: q = 3r/(r-1).  relativistic = 1:
 * along the axis that set r (the first axis with the largest ratio, as in
 * or_shock_cells) the lower-density neighbour is upstream and the other one
 * downstream; q = or_kw_index of their shock-frame speeds
 * (or_shock_frame_speeds), or 3r/(r-1) where no shock frame exists.        */
void or_shock_slopes(const or_grid* g, const double* vel, const double* rho,
                     const double* r_cell, int relativistic, double* q_cell) {
  int64_t G = (int64_t)g->n[0] * g->n[1] * g->n[2];
  for (int jz = 0; jz < g->n[2]; ++jz)
    for (int jy = 0; jy < g->n[1]; ++jy)
      for (int jx = 0; jx < g->n[0]; ++jx) {
        int64_t c = cell_linear(g, jx, jy, jz);
        double r = r_cell[c];
        if (!(r > 0.0)) {
          q_cell[c] = 0.0;
          continue;
        }
        double q = or_dsa_index(r);
        if (relativistic) {
          int j[3] = {jx, jy, jz};
          double best = 0.0;
          int64_t up = -1, down = -1;
          int axis = -1;
          for (int a = 0; a < g->dim; ++a) {
            int jp[3] = {jx, jy, jz}, jm[3] = {jx, jy, jz};
            jp[a] = nbr(g, a, j[a] + 1);
            jm[a] = nbr(g, a, j[a] - 1);
            int64_t cp = cell_linear(g, jp[0], jp[1], jp[2]);
            int64_t cm = cell_linear(g, jm[0], jm[1], jm[2]);
            if (vel[a * G + cp] - vel[a * G + cm] < 0.0) {
              int64_t dn = rho[cp] > rho[cm] ? cp : cm;   /* denser side: downstream */
              int64_t un = dn == cp ? cm : cp;
              double rr = rho[dn] / rho[un];
              if (rr > best) {
                best = rr;
                axis = a;
                down = dn;
                up = un;
              }
            }
          }
          if (axis >= 0) {
            double s2u = 0.0, s2d = 0.0;
            for (int a = 0; a < 3; ++a) {
              s2u += vel[a * G + up] * vel[a * G + up];
              s2d += vel[a * G + down] * vel[a * G + down];
            }
            double bu, bd;
            if (or_shock_frame_speeds(vel[axis * G + up], s2u, rho[up], vel[axis * G + down],
                                      s2d, rho[down], &bu, &bd))
              q = or_kw_index(bu, bd);
          }
        }
        q_cell[c] = q;
      }
}

/* Shock cells.  The paper leaves the detection criterion to the fluid code;
 * this oracle uses: cell c is a shock cell if, along some axis a < dim, the
 * flow converges across c (v_a(c + e_a) - v_a(c - e_a) < 0) and the density
 * ratio of those two neighbours, max/min, is at least r_min.  Its
 * compression ratio is the largest such ratio over the axes; 0 elsewhere.
 * Periodic neighbours; vel [3][G], rho [G] cell-centred.                    */
void or_shock_cells(const or_grid* g, const double* vel, const double* rho, double r_min,
                    double* r_cell) {
  int64_t G = (int64_t)g->n[0] * g->n[1] * g->n[2];
  for (int jz = 0; jz < g->n[2]; ++jz)
    for (int jy = 0; jy < g->n[1]; ++jy)
      for (int jx = 0; jx < g->n[0]; ++jx) {
        int j[3] = {jx, jy, jz};
        double best = 0.0;
        for (int a = 0; a < g->dim; ++a) {
          int jp[3] = {jx, jy, jz}, jm[3] = {jx, jy, jz};
          jp[a] = nbr(g, a, j[a] + 1);
          jm[a] = nbr(g, a, j[a] - 1);
          int64_t cp = cell_linear(g, jp[0], jp[1], jp[2]);
          int64_t cm = cell_linear(g, jm[0], jm[1], jm[2]);
          double dv = vel[a * G + cp] - vel[a * G + cm];
          if (dv < 0.0) {
            double hi = rho[cp] > rho[cm] ? rho[cp] : rho[cm];
            double lo = rho[cp] > rho[cm] ? rho[cm] : rho[cp];
            double ratio = hi / lo;
            if (ratio > best) best = ratio;
          }
        }
        r_cell[cell_linear(g, jx, jy, jz)] = best >= r_min ? best : 0.0;
      }
}

/* Eq. convolution_spectra on one spectrum of nb bins (energies increasing):
 *   chi_out(eps_i) = cn * integral_{eps_0}^{eps_i} chi_in(e) (eps_i/e)^(2-q) de/e.
 * Between adjacent bins chi_in is the power law through the two bin values
 * (the bins are log-spaced; a power-law spectrum is represented exactly), so
 * each segment integral is closed-form: with R = e1/e0 and local index
 * s = ln(c1/c0)/ln R, a = s + q - 2,
 *   integral_{e0}^{e1} c0 (e/e0)^s (eps_i/e)^(2-q) de/e
 *     = c0 (eps_i/e0)^(2-q) (R^a - 1)/a,   (R^a - 1)/a = expm1(a ln R)/a.
 * A segment with a zero endpoint contributes 0 (the limit of the power law
 * through a vanishing value).  chi_out at the lowest bin is 0.              */
void or_shock_convolve(int nb, const double* eng, const double* chi_in, double q, double cn,
                       double* chi_out) {
  for (int i = 0; i < nb; ++i) {
    double sum = 0.0;
    for (int j = 1; j <= i; ++j) {
      double e0 = eng[j - 1], e1 = eng[j], c0 = chi_in[j - 1], c1 = chi_in[j];
      if (!(c0 > 0.0 && c1 > 0.0 && e1 > e0)) continue;
      double lnR = log(e1 / e0);
      double s = log(c1 / c0) / lnR;
      double a = s + q - 2.0;
      double I = a == 0.0 ? lnR : expm1(a * lnR) / a;
      sum += c0 * pow(eng[i] / e0, 2.0 - q) * I;
    }
    chi_out[i] = cn * sum;
  }
}

/* Shock update of the LP spectra after a step's smooth update.  An LP whose
 * cell at x (the cell containing it) is a shock cell, and that was not in a
 * shock cell at the end of its previous step (state[p] == 0), takes
 * Eq. convolution_spectra with the cell's q (q_cell, or or_dsa_index(r) when
 * q_cell is NULL) and cn = q / r: the non-relativistic test-particle solution
 * conserves particle number per unit fluid density, chi = N/n (Eq. chi),
 * across a jump n_d = r n_u.  state[p] becomes 1 in a shock cell and 0
 * elsewhere.  chi, eng bin-major [nb][n].                                   */
void or_lp_shock(const or_grid* g, const double* r_cell, const double* q_cell, int nb,
                 int64_t n, const double* x, double* chi, const double* eng, uint8_t* state) {
#pragma omp parallel
  {
    double* e = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    double* ci = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    double* co = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
#pragma omp for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
      double xp[3] = {x[p], x[n + p], x[2 * n + p]};
      int j[3]; double d[3];
      or_cell_coord(g, xp, j, d);
      int64_t c = cell_linear(g, j[0], j[1], j[2]);
      double r = r_cell[c];
      if (r > 0.0) {
        if (!state[p]) {
          double q = q_cell ? q_cell[c] : or_dsa_index(r);
          for (int i = 0; i < nb; ++i) {
            e[i] = eng[(int64_t)i * n + p];
            ci[i] = chi[(int64_t)i * n + p];
          }
          or_shock_convolve(nb, e, ci, q, q / r, co);
          for (int i = 0; i < nb; ++i) chi[(int64_t)i * n + p] = co[i];
        }
        state[p] = 1;
      } else {
        state[p] = 0;
      }
    }
    free(e); free(ci); free(co);
  }
}

/* Threads the OpenMP loops above may use (timing runs; results do not depend
 * on it: every parallel loop writes disjoint particles). */
void or_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int or_max_threads(void) { return omp_get_max_threads(); }
