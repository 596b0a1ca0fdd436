/*
 * part_oracle.h -- plain FP64 CPU oracle for the particle advance.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path.  Everything is double precision, processed in particle
 * index order, compiled without floating-point contraction (-ffp-contract=off).
 *
 * Sources (the paper: "The PLUTO Code on GPUs: Offloading Lagrangian Particle
 * Methods"):
 *   Eq. push            LP advection dx/dt = v(x)                 (Sec. 2)
 *   proper time         d tau = dt / gamma_g                       (Sec. 2)
 *   Eq. rad_losses      d eps/d tau = -c_r eps^2                   (Sec. 2)
 *   Eq. cr_chi          d chi/d tau + d_eps[(-eps/3 div u - c_r eps^2) chi] = 0
 *   Eq. initSpec        chi_i = N0 (1-p)/(emax^(1-p)-emin^(1-p)) eps_i^-p  (Sec. 4.1.2)
 *   Eq. convolution_spectra  chi_out = C int chi_in (eps/eps')^(2-q) d eps'/eps'  (Sec. 2)
 *   Eq. slope           q(r) = 3r/(r-1) + q_R(r, beta_u, beta_d)
 *   Rankine-Hugoniot    r = (gamma+1) M^2/(2 + (gamma-1) M^2)      (Sec. 4.1.2)
 *   Appendix A          particle record: pos, speed, chi[128], eng[128], id
 * Where the paper is silent the oracle uses textbook definitions:
 *   TSC / CIC shape functions (Hockney & Eastwood), relativistic Boris push
 *   (Boris 1970; Birdsall & Langdon), Philox4x32-10 (Salmon et al., SC'11),
 *   and for q_R of Eq. slope the index of Keshet & Waxman (2005, PRL 94,
 *   111102), one of the works the paper cites for it.
 *
 * Parity unpinned: the absolute synchrotron coefficient scaling (c0, U_B in
 * code units) -- the paper gives c_r only in cgs form.
 */
#ifndef PART_ORACLE_H
#define PART_ORACLE_H
#include <stdint.h>

typedef struct {
  int dim;          /* 2 or 3 spatial dimensions                         */
  int n[3];         /* cells per axis; n[2] == 1 when dim == 2            */
  double xmin[3];   /* lower domain corner                               */
  double dx[3];     /* cell width per axis                               */
  int open[3];      /* 1: open (outflow) axis, 0: periodic               */
} or_grid;

enum { OR_CIC = 1, OR_TSC = 2 };

/* shape function W(xi), xi in cell units */
double or_shape(int shape, double xi);
/* cell coordinate j and offset delta = s - j - 1/2 of position x, per axis */
void or_cell_coord(const or_grid* g, const double* x, int* j, double* delta);
/* wrap one coordinate periodically into [xmin, xmin + n dx); identity on an
 * open axis */
double or_wrap(const or_grid* g, int axis, double x);
/* 1 if x lies outside the domain along an open axis (the particle has left) */
int or_outside(const or_grid* g, const double* x);
/* interpolate ncomp cell-centred fields [comp][z][y][x] at x */
void or_gather(const or_grid* g, int shape, const double* fields, int ncomp,
               const double* x, double* out);
/* relativistic Boris kick (c = 1, u = gamma v), fields at the particle */
void or_boris_kick(double* u, const double* E, const double* B, double qm, double dt);
/* one Boris step for n particles: gather at x^n, kick, drift, wrap.
 * x, u: [3][n]; w: [n] (may be NULL => 1); F_out [3][n] (may be NULL) gets
 * w (u^{n+1}-u^n)/dt; x_old_out [3][n] (may be NULL) gets x^n.            */
void or_boris_step(const or_grid* g, int shape, const double* fields6, int64_t n,
                   double* x, double* u, const double* w, double qm, double dt,
                   double* F_out, double* x_old_out);
/* scatter F [3][n] at positions x [3][n] onto out [3][G] (overwritten) */
void or_deposit(const or_grid* g, int shape, int64_t n, const double* x,
                const double* F, double* out);
/* deposit onto one cell only (sampling check); out3 gets the 3 components */
void or_deposit_cell(const or_grid* g, int shape, int64_t n, const double* x,
                     const double* F, int64_t cell, double* out3);
/* brick-ordered cell key of cell coordinates j with brick dims b */
uint32_t or_cell_key(const or_grid* g, const int* b, const int* j);
int64_t or_key_count(const or_grid* g, const int* b);
/* keys of n positions [3][n] */
void or_keys(const or_grid* g, const int* b, int64_t n, const double* x, uint32_t* keys);
/* stable sort: perm gets the particle indices ordered by key */
void or_stable_sort(int64_t n, const uint32_t* keys, uint32_t* perm);
/* cs[c] = #particles with key < c for c in [0, nkeys] (sorted keys input) */
void or_cell_start(int64_t nkeys, int64_t n, const uint32_t* sorted_keys, uint32_t* cs);
/* Heun RK2 LP advection on velocity fields vel [3][G]; samples at x^{n+1} */
void or_lp_rk2_step(const or_grid* g, int shape, const double* vel, const double* rho,
                    const double* bfield, int64_t n, double* x, double dt,
                    double* n_new, double* b2m, double* gam);
/* third-order SSP Runge-Kutta LP advection (same arguments as RK2) */
void or_lp_rk3_step(const or_grid* g, int shape, const double* vel, const double* rho,
                    const double* bfield, int64_t n, double* x, double dt,
                    double* n_new, double* b2m, double* gam);
/* exact-characteristic spectral update; chi, eng are bin-major [nb][n] */
void or_spec_update(int nb, int64_t n, double* chi, double* eng, double* n_old,
                    const double* n_new, const double* b2m, const double* gam,
                    double dt, double c0, double u_rad);
/* initial power-law spectrum on log-spaced nodes, Eq. initSpec */
void or_init_spectrum(int nb, double emin, double emax, double p, double N0,
                      double* eng, double* chi);
/* Philox4x32-10 block function */
void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out);
/* particle initialisation from Philox draws: uniform x, Maxwellian u */
void or_init_particles(const or_grid* g, int64_t n, uint64_t seed, double u_th,
                       double* x, double* u, double* w, uint64_t* id);
/* Hole/filler compaction of Sec. 3.2 (the paper's five steps): given the
 * deletion flags of n particles, returns n_keep and src[j] (j < n_keep) = the
 * old index of the particle that ends up in slot j.                        */
int64_t or_compact_map(int64_t n, const uint8_t* del, int64_t* src);
/* Rankine-Hugoniot compression ratio r(gamma, M) */
double or_rh_compression(double gamma, double mach);
/* Eq. slope without the relativistic correction: q = 3r/(r-1) */
double or_dsa_index(double r);
/* per-cell compression ratio of detected shocks (0: no shock), [G] */
void or_shock_cells(const or_grid* g, const double* vel, const double* rho, double r_min,
                    double* r_cell);
/* Eq. convolution_spectra on one spectrum (piecewise power law in chi_in) */
void or_shock_convolve(int nb, const double* eng, const double* chi_in, double q, double cn,
                       double* chi_out);
/* Eq. slope for a relativistic shock: the index from the upstream and
 * downstream normal flow speeds in the shock frame (units of c) */
double or_kw_index(double beta_u, double beta_d);
/* shock-frame normal speeds from lab-frame normal velocities v, squared
 * speeds s2 (all components, for the Lorentz factors) and proper densities;
 * 1 on success, 0 where no shock frame exists */
int or_shock_frame_speeds(double v_u, double s2_u, double rho_u, double v_d, double s2_d,
                          double rho_d, double* beta_u, double* beta_d);
/* per-cell q of Eq. slope for the shock cells r_cell > 0 (0 elsewhere);
 * relativistic = 0: 3r/(r-1); 1: with q_R from the cell's neighbours */
void or_shock_slopes(const or_grid* g, const double* vel, const double* rho,
                     const double* r_cell, int relativistic, double* q_cell);
/* shock update of n LP spectra at positions x; state[n] = inside a shock cell;
 * q_cell = the per-cell index (NULL: 3r/(r-1)) */
void or_lp_shock(const or_grid* g, const double* r_cell, const double* q_cell, int nb,
                 int64_t n, const double* x, double* chi, const double* eng, uint8_t* state);
/* OpenMP thread count of the loops above (timing only) */
void or_set_threads(int n);
int or_max_threads(void);
#endif
