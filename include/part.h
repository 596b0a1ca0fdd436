/*
 * part.h -- C ABI of the B300 particle-advance library (libpart.so).
 *
 * The library advances particles on a periodic Cartesian grid, one CUDA
 * stream per context:
 *   - Lagrangian particles (LPs): advection with the fluid velocity (Eq. push,
 *     Sec. 2) by a two- or three-stage Runge-Kutta step (Sec. 3.3, Table
 *     codeTiming: Particles_RK#1 / Particles_RK#2; Sec. 4.1.1), the
 *     per-particle energy-spectrum update of Eq. cr_chi (Sec. 2;
 *     Particles_Spectra in Table codeTiming) and, at shocks, the diffusive
 *     shock acceleration of Eq. convolution_spectra with Eq. slope;
 *   - charged test/cosmic-ray particles: relativistic Boris push with fields
 *     gathered by TSC or CIC weights, and the deposit of the particle force
 *     density back onto the grid (the MHD-PIC coupling named in Sec. 1).
 * Particles are stored as structures of arrays (Sec. 3.2, "Ensure coalesced
 * access to memory"), with the record of Appendix A (pos, speed, chi[nb],
 * eng[nb], id); deleted particles are removed by the hole/filler compaction
 * of Sec. 3.2 (part_compact).
 *
 * Conventions (all entry points):
 *   - Every call returns a part_status and never aborts.  Argument errors are
 *     found on the host before any launch and return PART_EINVAL with a
 *     message in part_last_error().
 *   - Work is enqueued asynchronously on the context's stream.  Errors found
 *     by kernels (non-finite state, a particle outside its sorted cell, a
 *     bounded wait that ran out) are latched in a device status word and
 *     reported by the next part_sync().
 *   - The library allocates no device memory.  All device memory is passed in
 *     by the caller: a workspace of part_workspace_size() bytes (256-byte
 *     aligned) and the particle/field/output arrays.  The caller keeps every
 *     buffer alive until the work that uses it has completed (part_sync or a
 *     stream synchronisation).
 *   - Pointers to particle, field and output data are device pointers of the
 *     context's device (or managed memory, or pinned host memory mapped into
 *     the unified address space, which the kernels then reach over the host
 *     link).  Pageable host memory is refused with PART_EINVAL.
 *   - Units: c = 1, particle mass m = 1, u = gamma v.
 *   - Grid: cell-centred fields, layout [comp][z][y][x] (x fastest), cell
 *     (jx,jy,jz) centred at xmin + (j + 1/2) dx.  For dim == 2 the grid has
 *     n[2] == 1 and only x, y move (2D3V).
 *   - Boundaries, per axis: periodic (wrap), or open (outflow, as the x axis
 *     of the paper's shock test, Sec. 4.1.2).  On an open axis the fields are
 *     continued by a zero-gradient ghost layer; a particle samples at its
 *     position clamped into the domain; deposits beyond the face fold onto
 *     the edge cell (the adjoint of that gather); positions are not wrapped,
 *     and a particle that ends a push outside the domain is flagged in the
 *     outflow mask (part_set_outflow) for removal by part_compact before the
 *     next sort or push.  The serving API needs periodic grids.
 */
#ifndef PART_H
#define PART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct part_ctx part_ctx; /* opaque; one per stream and particle set */

typedef enum {
  PART_OK = 0,
  PART_EINVAL = 1,        /* bad argument (host-side check)                 */
  PART_ENOMEM = 2,        /* workspace too small                            */
  PART_ECUDA = 3,         /* a CUDA runtime call failed                     */
  PART_ETIMEOUT = 4,      /* a bounded device wait ran out                  */
  PART_ENONFINITE = 5,    /* NaN/Inf met in particle state or samples       */
  PART_EUNSUPPORTED = 6,  /* valid request the library does not implement  */
  PART_EDOMAIN = 7        /* a particle was not in the cell it was sorted by */
} part_status;

typedef enum { PART_FP64 = 0, PART_MIXED = 1 } part_prec;
typedef enum { PART_CIC = 1, PART_TSC = 2 } part_shape;
typedef enum { PART_BORIS = 0, PART_LP_RK2 = 1 } part_mode;

typedef struct {
  int dim;          /* 2 or 3                                              */
  int n[3];         /* cells per axis, each >= 1; n[2] must be 1 if dim==2 */
  double xmin[3];   /* lower corner                                        */
  double dx[3];     /* cell widths (> 0)                                   */
  int periodic[3];  /* 1: periodic; 0: open (outflow) axis, see below      */
} part_grid;

/* Brick (cell tile) dimensions the library sorts and stages by: 8x8x8 in 3D,
 * 16x16x1 in 2D.  A cell's sort key is
 *   key = brick_index * (b0*b1*b2) + local_index,
 * brick_index = (bz*nby + by)*nbx + bx with nb_a = ceil(n_a/b_a), local_index
 * = (lz*b1 + ly)*b0 + lx, (b, l) = (j / b_a, j % b_a) per axis.  The last
 * brick on an axis may be partial; keys then skip the missing cells.
 * nkeys gets the key-space size nbx*nby*nbz*b0*b1*b2.                      */
part_status part_brick_dims(const part_grid* grid, int brick[3], int64_t* nkeys);

/* Workspace bytes for a context: padded field copy (and, for FP64 fields,
 * its x quadratics: the TSC gathers read each stencil row as q0 + d (q1 +
 * d q2), 32 bytes per component and padded cell), sort buffers, cell_start,
 * deposit partials, LP samples, status word.  capacity = maximum particles,
 * nbins = spectral bins (LP mode; ignored otherwise).                     */
part_status part_workspace_size(const part_grid* grid, part_prec prec, part_mode mode,
                                int64_t capacity, int nbins, size_t* bytes);

/* Create a context.  workspace: device memory of at least
 * part_workspace_size() bytes, 256-byte aligned, owned by the caller and
 * kept alive until part_destroy.  cuda_stream: a cudaStream_t (NULL = the
 * legacy default stream).  Supported: PART_BORIS with PART_FP64 or
 * PART_MIXED; PART_LP_RK2 with PART_FP64.  Returns PART_ENOMEM if ws_bytes
 * is too small.                                                            */
part_status part_init(part_ctx** out, const part_grid* grid, part_prec prec,
                      part_shape shape, part_mode mode, int64_t capacity, int nbins,
                      void* workspace, size_t ws_bytes, void* cuda_stream);
part_status part_destroy(part_ctx* ctx);

/* Copy a field snapshot into the context's padded, ghost-filled copy.
 * fields: device, [ncomp][z][y][x] contiguous, element type f64 (PART_FP64
 * context) or f32 (PART_MIXED context); field_prec must match.
 * PART_BORIS: ncomp = 6 (E then B).  PART_LP_RK2: ncomp = 7 (fluid velocity
 * v[3], density rho, B[3]) -- the fluid quantities LPs sample (Sec. 2).
 * The copy (with the x quadratics of FP64 fields) is stream-ordered; the
 * source may be freed once it completes.
 * fields must be aligned to its element size, and be device memory of the
 * context's device, managed memory, or pinned host memory (read once by the
 * padding kernel over the host link); anything else, such as pageable host
 * memory, is refused with PART_EINVAL before any launch.  The same rule
 * holds for every array argument of the library.                          */
part_status part_set_fields(part_ctx* ctx, const void* fields, int ncomp, part_prec field_prec);

/* Bind caller-owned particle arrays (device, component-major, row stride n):
 *   PART_FP64 / BORIS : x_or_cell = double[3][n] positions, off = NULL,
 *                       u = double[3][n], w = double[n] or NULL (w = 1)
 *   PART_MIXED / BORIS: x_or_cell = int32[n] linear cell (jz*ny+jy)*nx+jx,
 *                       off = float[3][n] offsets from the cell centre in
 *                       cell units, in [-1/2, 1/2]; u = float[6][n], the
 *                       momentum as a compensated pair: rows 0-2 its f32
 *                       value, rows 3-5 the f32 residual (u = hi + lo; start
 *                       the residual at 0, or at u - hi when u is known more
 *                       precisely); w = float[n] or NULL
 *   PART_LP_RK2       : x_or_cell = double[3][n], chi, eng = double[nb][n]
 *                       (bin-major), n_old = double[n] (density sampled at
 *                       the previous step); u, w = NULL
 * id (uint64[n]) is optional in every mode; when given it is permuted with
 * the particles so the caller can undo a sort.  0 <= n <= capacity.  Every
 * array must be aligned to its element size (PART_EINVAL otherwise).     */
part_status part_bind_particles(part_ctx* ctx, int64_t n, void* x_or_cell, void* off,
                                void* u, void* w, uint64_t* id, double* chi, double* eng,
                                double* n_old);

/* Sort the bound particles by cell key (stable: equal keys keep their current
 * order), permuting every bound array, and rebuild cell_start.  Required
 * before a push with deposit enabled.
 * Boris modes: the sort only computes the permutation.  The next one-step
 * push reads the particles through it and writes them, sorted, into a second
 * copy in the workspace, which then holds the current state (the copies
 * alternate from step to step).  part_flush, part_sync, part_bind_particles,
 * part_compact and a multi-step push first bring the current state into the
 * bound arrays, in sorted order.  Between part_sort and the next of those
 * calls the caller must neither read nor write the bound arrays.
 * When the previous sort's order has been kept and every push since moved
 * each particle by less than one cell (sum of nsteps * |dt| below the
 * smallest dx; |v| < c = 1), a per-brick incremental sort replaces the radix
 * passes; the permutation is the same.                                     */
part_status part_sort(part_ctx* ctx);

/* Bring the current particle state into the bound arrays, in sorted order,
 * asynchronously on the context's stream (see part_sort).                  */
part_status part_flush(part_ctx* ctx);

/* Remove the particles flagged in deleted (device uint8[n], nonzero = delete)
 * by the hole/filler compaction of Sec. 3.2 ("Ensure coalesced access to
 * memory"): the k-th deleted slot below n_new = n - N_del receives the k-th
 * surviving particle stored at or beyond n_new (both in index order), then the
 * set shrinks to n_new.  Every bound array is updated and re-laid out with row
 * stride n_new (component a of particle p at a*n_new + p); the context's n
 * becomes n_new.  Synchronises the stream once to read N_del.  Invalidates
 * the sort.                                                                 */
part_status part_compact(part_ctx* ctx, const uint8_t* deleted, int64_t* n_new);

/* Append k >= 0 particles at run time (the injection of Sec. 3.2, "Minimize
 * memory allocation/deallocation": the set grows inside memory allocated
 * once, up to the context's capacity).  Every bound array is re-laid out
 * from row stride n to row stride n + k (component a of particle p at
 * a*(n+k) + p) and the new particles fill slots n .. n+k-1; the context's n
 * becomes n + k.  Each bound array must therefore hold rows x (n + k)
 * elements (bind arrays allocated at capacity).  Sources are device arrays
 * in the bound layout with row stride k: x_or_cell, and u (Boris), off
 * (PART_MIXED), chi, eng, n_old (LP); w and id are read only when the bound
 * set has w and id planes, and are then required.  Shock flags, when
 * enabled, are cleared for the new particles.  PART_EINVAL if n + k exceeds
 * the capacity or a required source is NULL.  Invalidates the sort.        */
part_status part_inject(part_ctx* ctx, int64_t k, const void* x_or_cell, const void* off,
                        const void* u, const void* w, const uint64_t* id, const double* chi,
                        const double* eng, const double* n_old);

/* Outflow mask (grids with an open axis): every push writes, per bound
 * particle, 1 if it ended outside the domain along an open axis, else 0
 * (device uint8[n], caller-owned, in the order of the bound arrays after the
 * push).  A fused multi-step push stops advancing a particle once it is out.
 * Pass the mask to part_compact to remove those particles.  NULL: not
 * written.  part_bind_particles resets it to NULL.                         */
part_status part_set_outflow(part_ctx* ctx, uint8_t* mask);

/* Device pointer to cell_start[nkeys + 1] (valid after part_sort): the
 * particles of key k are [cell_start[k], cell_start[k+1]).                */
part_status part_cell_start(part_ctx* ctx, const uint32_t** cell_start, int64_t* nkeys);

/* Turn on (1) or off (0) the fused force deposit of part_gather_push.     */
part_status part_enable_deposit(part_ctx* ctx, int on);

/* PART_BORIS: nsteps steps of gather (fields at x^n with the context's
 * shape) + relativistic Boris kick + drift + periodic wrap.  With deposit on,
 * nsteps must be 1, the particles must have been sorted since the last push,
 * and the kick's force density F_p = w_p (u^{n+1} - u^n)/dt is reduced onto
 * the grid with the weights at x^n (see part_deposit).
 * PART_LP_RK2: nsteps Heun steps x* = x + dt v(x), x' = x + dt (v(x)+v(x*))/2
 * of Eq. push, then samples at the new position for spec_update: density,
 * the mean of |B|^2 at the old and new position, and gamma_g.  q_over_m is
 * ignored in LP mode.  The fluid v and B sampled at the new positions are
 * kept (workspace) and stand for the samples at the old positions of the
 * next push, one stencil pass fewer per LP; part_set_fields, part_sort,
 * part_compact, part_bind_particles and part_init_particles drop them.  A
 * caller that moves the LPs itself binds them again.                       */
part_status part_gather_push(part_ctx* ctx, double q_over_m, double dt, int nsteps);

/* Time marching of the LP push (PART_LP_RK2 contexts; default 2).
 * order 2: Heun, as part_gather_push states.  order 3: the three-stage
 * strong-stability-preserving Runge-Kutta scheme of Shu & Osher (the paper
 * runs its advection test with 2nd- and 3rd-order RK, Sec. 4.1.1), in
 * stage-velocity form: k1 = v(x), k2 = v(x + dt k1),
 * k3 = v(x + dt (k1 + k2)/4), x' = x + dt (k1 + k2 + 4 k3)/6; each sampled
 * position is wrapped, the samples at x' are as for order 2.
 * Other orders or modes: PART_EINVAL.                                      */
part_status part_set_lp_order(part_ctx* ctx, int order);

/* Arithmetic of the LP push (PART_LP_RK2 contexts; default 0).
 * paired = 0: FP64.  paired = 1: paired f32 -- every value of the step
 * (offsets, weights, stencil sums, position updates, samples) is carried as
 * the unevaluated sum of two floats, about 48 significant bits, built from
 * error-free transformations (TwoSum, FMA product errors) and evaluated on
 * the f32 pipes, two field components per packed f32x2 instruction; the
 * stencil sums are Dot2 accumulations (Ogita, Rump & Oishi 2005).  B300
 * runs FP64 at about 1/64 of its f32 rate, and the FP64 push is bound by
 * it.  Positions, spectra and everything the caller sees stay FP64; the
 * step agrees with the FP64 one to ~1e-15 in position and ~1e-13 relative
 * in the samples (offsets within ~1e-13 cell).  The spectral update
 * (spec_update) stays FP64 in both.  Changing it drops the cached v, B
 * (the next push gathers them again).  Other values or modes: PART_EINVAL. */
part_status part_set_lp_arith(part_ctx* ctx, int paired);

/* How spec_update keeps the LP spectra (PART_LP_RK2 contexts; default 0).
 * The step of Eq. cr_chi (spec_update) is, for every bin of an LP, the same
 * affine map in y = 1/eps and psi = chi eps^2: y <- A y + C, psi <- psi / A
 * (A, C from the LP's samples).  lazy = 0: every bin is updated every step.
 * lazy = 1: the bins stay as they were, and each LP keeps the composition of
 * its steps' maps, y = alpha y0 + beta, psi = S psi0 (alpha <- A alpha,
 * beta <- A beta + C, S <- S / A per step): O(1) work per LP and step
 * instead of O(N_b).  The bins are brought up to date where the spectra are
 * handed back anyway -- part_sync, part_flush, part_sort, part_compact,
 * part_inject, the exchange calls, a rebind -- as eps = eps0 / t,
 * chi = S chi0 t^2 with t = alpha + beta eps0; an LP that a shock update
 * takes has its bins brought up to date and its map reset first.  The
 * results agree with lazy = 0 to rounding (the composed map rounds
 * differently from the steps one by one).  Changing it brings the bound
 * spectra up to date first.  Other values or modes: PART_EINVAL.          */
part_status part_set_spec_lazy(part_ctx* ctx, int lazy);

/* Write the force density deposited by the last part_gather_push into
 * grid_out (device, double[3][G], overwritten):
 *   F_g = sum_p W(x_g - x_p^n) F_p.
 * Deterministic: no floating-point atomics; the same inputs give the same
 * bits on every run.  grid_out must be 8-byte aligned (PART_EINVAL); it may
 * be pinned host memory, written directly over the host link.             */
part_status part_deposit(part_ctx* ctx, double* grid_out);

/* Spectral update of every LP (Eq. cr_chi with Eq. rad_losses), using the
 * samples of the last PART_LP_RK2 push.  Per LP: dtau = dt/gamma_g (Sec. 2),
 * A = (n_old/n_new)^{1/3}, c_r = c0 (|B|^2/2 + u_rad),
 * C = c_r dtau expm1(ln A)/ln A; per bin, s = A + C eps:
 *   eps <- eps/s,  chi <- chi s^2/A;  then n_old <- n_new.
 * With shocks enabled, every LP that the last push moved into a shock cell
 * (from outside one) then takes the shock update of part_enable_shocks.
 * part_sort or part_compact between the push and this call invalidate the
 * samples (PART_EINVAL).
 * The step is applied in the variables it is linear in, y = 1/eps and
 * psi = chi eps^2 (y <- A y + C, psi <- psi/A: the same update exactly), and
 * the bound chi and eng arrays hold psi and y from the first update until the
 * next part_flush, part_sync, part_bind_particles, part_compact or
 * part_inject, which turn them back into chi and eps.  In between the caller
 * must neither read nor write them.  Energies must be positive.            */
part_status spec_update(part_ctx* ctx, double dt, double c0, double u_rad);

/* Diffusive shock acceleration of the LP spectra (PART_LP_RK2 only).
 * Shock cells are found in the current fields (recomputed by every
 * part_set_fields): along an axis a < dim, a cell whose neighbours' flow
 * converges (v_a(j+1) - v_a(j-1) < 0) and whose neighbour density ratio
 * max/min is >= r_min is a shock cell with compression ratio r = the largest
 * such ratio.  (The paper leaves the criterion to the fluid code.)
 * state: device uint8[n], caller-owned and caller-initialised (0 = not in a
 * shock cell), one flag per bound LP; it is permuted by part_sort and moved
 * by part_compact with the LPs.  part_bind_particles disables shocks; call
 * this again after binding.  NULL disables shocks.  r_min must be > 1.
 * After a push, an LP whose cell at x^{n+1} is a shock cell and whose flag is
 * 0 is listed; its flag then follows its cell (1 in a shock cell, 0
 * elsewhere).  spec_update applies Eq. convolution_spectra to each listed LP
 * after the smooth update:
 *   chi(eps_i) <- cn * integral_{eps_0}^{eps_i} chi(e) (eps_i/e)^(2-q) de/e,
 * q = the index of Eq. slope of the LP's shock cell (part_set_shock_slope),
 * cn = q/r (for a non-relativistic shock, particle number per unit fluid
 * density is conserved across the jump n_d = r n_u), the q and r being those
 * of the cell at the push, chi between adjacent bins taken as the power law through
 * the two bin values, eps_0 = the LP's lowest bin energy (chi there becomes
 * 0).  Bin energies are unchanged.  Requires bound particles and fields.   */
part_status part_enable_shocks(part_ctx* ctx, double r_min, uint8_t* state);

/* Device pointer to the shock cells r[G] (cell order as the fields; 0 = no
 * shock), valid while shocks are enabled and the fields are unchanged.     */
part_status part_shock_cells(part_ctx* ctx, const double** r_cell, int64_t* ncells);

/* Index q of Eq. slope, q(r) = 3r/(r-1) + q_R (PART_LP_RK2 only).
 * relativistic = 0 (the default): q_R = 0, the non-relativistic shock.
 * relativistic = 1: q_R from the flow speeds on both sides of the shock
 * (velocities in units of c, as in the LP push's gamma_g).  The paper takes
 * q_R from the literature; this library uses the index of Keshet & Waxman
 * (2005, PRL 94, 111102), one of the works it cites:
 *   q = (3 b_u - 2 b_u b_d^2 + b_d^3) / (b_u - b_d),
 * b_u > b_d the normal flow speeds upstream and downstream in the shock's
 * rest frame.  For a shock cell whose ratio r was set along axis a, the
 * neighbour along a with the lower density is upstream and the other one
 * downstream; the shock moves at v_sh = (D_d v_d - D_u v_u)/(D_d - D_u), the
 * speed that conserves the lab-frame mass D = rho/sqrt(1 - |v|^2) across it
 * (v: the a components; |v|: all three), and there the normal speeds are
 * |v - v_sh|/(1 - v v_sh).  Where that frame does not exist (a speed >= 1,
 * D_d = D_u, |v_sh| >= 1, or b_d >= b_u) the cell keeps 3r/(r-1).
 * Recomputes the shock cells when shocks are enabled; otherwise the setting
 * is taken up by part_enable_shocks.  It survives part_bind_particles.
 * Errors: PART_EINVAL for another mode or relativistic not 0/1.           */
part_status part_set_shock_slope(part_ctx* ctx, int relativistic);

/* Device pointer to the per-cell index q[G] of Eq. slope (0 = no shock),
 * valid like part_shock_cells.                                             */
part_status part_shock_slopes(part_ctx* ctx, const double** q_cell, int64_t* ncells);

/* Initialise the bound particles on the device from Philox4x32-10 draws
 * (key = seed; counter (p, 0) -> uniform position over the domain, counter
 * (p, 1) -> Maxwellian u with per-component std u_th by Box-Muller), w = 1,
 * id = p.  LP mode: u_th ignored; every LP gets the power law of Eq. initSpec
 * on nb log-spaced energies in [eps_min, eps_max] with index p_index and
 * integral N0, and n_old = density sampled at its position.              */
part_status part_init_particles(part_ctx* ctx, uint64_t seed, double u_th, double eps_min,
                                double eps_max, double p_index, double N0);

/* part_flush, then wait for the context's stream; return (and clear) the
 * first latched device error, else PART_OK.                                */
part_status part_sync(part_ctx* ctx);

/* Message for the last non-OK status of this context (never NULL).        */
const char* part_last_error(const part_ctx* ctx);

/* Kernel launches this context has enqueued since creation.               */
int64_t part_launch_count(const part_ctx* ctx);

/* Self-test of the bounded device waits (failure detection without a
 * fault).  Enqueues one kernel whose thread waits on a shared-memory
 * mbarrier with the wait every TMA-fed kernel uses, limited to limit_ns
 * (0 < limit_ns <= 1e10).  arrive = 1: the thread arrives first and the wait
 * succeeds.  arrive = 0: nothing arrives, the wait gives up after limit_ns,
 * and the next part_sync returns PART_ETIMEOUT (and clears it); the context
 * stays usable.  The kernels' own limit is 1 s.  PART_EINVAL on bad
 * arguments.                                                               */
part_status part_selftest_wait(part_ctx* ctx, int64_t limit_ns, int arrive);

/* ---- Serving: continuous batching of test-particle requests --------------
 * Test particles (no deposit) of many independent requests advance against
 * field snapshots that stay resident on the device, each snapshot being a
 * PART_MIXED / PART_BORIS context whose fields are set.  The caller (the
 * scheduler) cuts the active requests into work items each round; one
 * persistent kernel, replayed from a CUDA graph, advances every item.  Every
 * particle is advanced with the same arithmetic as part_gather_push with
 * nsteps > 1, so a request's result does not depend on what else is batched
 * with it or on how its steps are sliced.  Not in the paper: it serves the
 * particle push of Sec. 2 to many clients at once.                          */
typedef struct {
  int32_t* cell;       /* request state, device: int32 cell[stride]          */
  float* off;          /*   f32 off[3][stride] (cell units, [-1/2, 1/2))     */
  float* u;            /*   f32 u[6][stride]: hi rows 0-2, residual 3-5      */
  int64_t stride;      /* particles of the request (row stride of off, u)    */
  int64_t first;       /* first particle of this item                        */
  int32_t count;       /* particles in this item, >= 0                       */
  int32_t nsteps;      /* steps this item advances, >= 0                     */
  int32_t snapshot;    /* index into the server's snapshot list              */
  int32_t reserved;    /* 0                                                  */
  double q_over_m;     /* charge-to-mass ratio of the request                */
  double dt;           /* time step of the request, != 0                     */
} part_work_item;      /* 72 bytes                                           */

typedef struct part_server part_server;

/* Device workspace and pinned host staging bytes of a server for nsnap
 * snapshots and at most max_items items per round.                         */
part_status part_server_sizes(int nsnap, int max_items, size_t* device_bytes,
                              size_t* host_bytes);

/* Create a server over nsnap snapshot contexts (all PART_MIXED, PART_BORIS,
 * fields set, one shape and dim).  workspace: device, 256-byte aligned;
 * host_stage: pinned host memory (cudaHostAlloc / pinned tensor) of
 * host_bytes, in which the caller writes the work list (part_server_items).
 * threads: CTA size (128..512, multiple of 32); ctas_per_sm: persistent CTAs
 * per SM.  cuda_stream must be a created stream (not a default stream: the
 * round is captured into a CUDA graph); the snapshot contexts should use the
 * same stream.  The snapshot contexts must outlive the server.             */
part_status part_server_init(part_server** out, part_ctx* const* snapshots, int nsnap,
                             int max_items, void* workspace, size_t ws_bytes,
                             void* host_stage, size_t host_bytes, void* cuda_stream,
                             int threads, int ctas_per_sm);

/* Host pointer to the work-item array inside the pinned staging buffer.    */
part_work_item* part_server_items(part_server* s);

/* Validate the first nitems items on the host (PART_EINVAL on a bad item,
 * nothing launched), then enqueue one round: the copy of the work list to
 * the device and the persistent kernel, as one CUDA graph (captured on the
 * first call).  The staging buffer must not be rewritten until the round has
 * completed (part_server_sync).                                            */
part_status part_server_run(part_server* s, int nitems);

/* Wait for the last round; return (and clear) a latched device error.      */
part_status part_server_sync(part_server* s);
part_status part_server_destroy(part_server* s);

/* ---- Several ranks (Sec. 3.3, "Multi-core communication") ----------------
 * A run split over ranks gives each rank a context whose grid is its box of
 * cells plus, along every split axis, one halo cell on each side holding the
 * neighbour's fields (those axes are open in the context's grid, so nothing
 * wraps there).  Particles live in the interior; after a push, the ones in a
 * halo cell belong to a neighbour.  Per split axis, in turn (the paper's
 * three directions), the caller:
 *   1. part_exchange_pack: flags and counts the leaving particles and packs
 *      them into one buffer per neighbour (the paper's steps 1, 3, 4);
 *   2. exchanges the counts, then the buffers, with both neighbours
 *      (non-blocking sends and receives, steps 2, 5, 7);
 *   3. part_compact with the flags, then part_exchange_unpack of what came
 *      from the left and from the right (steps 6, 8).
 * Positions are moved into the receiver's frame while packing: FP64 and LP
 * positions are global coordinates and only change across the periodic seam
 * of the whole domain (x_axis += dx, the same rounding as the wrap of a
 * one-rank run); the mixed form's cell index is local and is re-based
 * (j_axis += dj) and re-linearised with the receiver's n_axis.             */
typedef struct {
  double dx;       /* added to the position along the axis (FP64, LP)       */
  int32_t dj;      /* added to the cell index along the axis (mixed)        */
  int32_t n_axis;  /* receiver's cells along the axis (mixed; >= 1)         */
} part_xshift;

/* Bytes of a packed exchange buffer holding k particles of this context
 * (every bound plane at row stride k, 8-byte planes first).                */
part_status part_exchange_bytes(const part_ctx* ctx, int64_t k, size_t* bytes);

/* Classify the bound particles along axis (0 <= axis < dim) against the
 * interior cell range [lo, hi) of the context's grid (FP64 and LP: s = (x -
 * xmin)/dx with the library's roundings, left if s < lo, right if s >= hi;
 * mixed: the cell index), write leaving[n] (device uint8, 1 = leaves), and
 * set counts[0] (left) and counts[1] (right).  If send_left / send_right hold
 * part_exchange_bytes(count) bytes (device, 8-byte aligned; NULL allowed for
 * a count of 0), pack the leaving particles into them in index order, moved
 * into the receiver's frame by to_left / to_right; otherwise return
 * PART_ENOMEM with the counts set and nothing packed, so the caller can
 * resize and call again.  Brings the current state home first (part_flush)
 * and synchronises the stream once, to read the counts.  PART_EINVAL on bad
 * arguments.                                                                */
part_status part_exchange_pack(part_ctx* ctx, int axis, int lo, int hi,
                               const part_xshift* to_left, const part_xshift* to_right,
                               void* send_left, size_t left_bytes, void* send_right,
                               size_t right_bytes, uint8_t* leaving, int64_t counts[2]);

/* Append k particles from a buffer packed by part_exchange_pack on a rank
 * with the same bound planes (recv: device, 8-byte aligned, at least
 * part_exchange_bytes(k) bytes); as part_inject, and LP shock flags are
 * carried along.  PART_EINVAL if n + k exceeds the capacity.               */
part_status part_exchange_unpack(part_ctx* ctx, int64_t k, const void* recv, size_t recv_bytes);

/* Deposit halos.  part_box_pack copies the box [lo, lo + ext) of a device
 * array double[ncomp][dims[2]][dims[1]][dims[0]] into dst, packed
 * [ncomp][ext[2]][ext[1]][ext[0]]; part_box_add adds such a packed src into
 * the box of dst (one rounded add per element).  Asynchronous on
 * cuda_stream (NULL = legacy default stream).  PART_EINVAL if the box leaves
 * the array, a pointer is NULL, unaligned or unreachable.                   */
part_status part_box_pack(const double* src, int ncomp, const int dims[3], const int lo[3],
                          const int ext[3], double* dst, void* cuda_stream);
part_status part_box_add(double* dst, int ncomp, const int dims[3], const int lo[3],
                         const int ext[3], const double* src, void* cuda_stream);

/* Replicated grids (particles partitioned over ranks, fields replicated):
 * out[i] = (((parts[0][i] + parts[1][i]) + parts[2][i]) + ...), parts laid
 * out [nparts][count], summed in that order, so every rank that holds the
 * same parts gets the same bits.  out may alias parts' first row.
 * Asynchronous on cuda_stream.  PART_EINVAL on bad arguments.              */
part_status part_sum_ordered(double* out, const double* parts, int64_t count, int nparts,
                             void* cuda_stream);

/* ---- Measurement -----------------------------------------------------------
 * FP64 fused multiply-add rate of the current device, measured: the
 * denominator of the arithmetic roofline of this library's FP64 kernels (on
 * B300 every FP64 kernel that does real arithmetic per byte is bound by the
 * FP64 pipe, not by HBM).  Not in the paper.  Runs ctas_per_sm CTAs of 256
 * threads on every SM, each thread 16 independent chains of iters dependent
 * fma steps, once untimed and then reps times, each timed with CUDA events
 * on cuda_stream (NULL = legacy default stream); synchronises that stream.
 * *tflops = 2 flop x threads x 16 x iters / best time (TFLOP/s); *best_ms
 * (may be NULL) = that time.  sink: device memory of one double, caller-owned
 * (never written in practice; it keeps the chains from being optimised away).
 * Errors: PART_EINVAL for NULL sink/tflops, an unaligned or unreachable
 * sink, ctas_per_sm outside 1..8, iters outside 1..2^20, reps outside 1..100;
 * PART_ECUDA if a launch or event call fails.  Nothing is allocated.        */
part_status part_probe_fp64_fma(void* cuda_stream, double* sink, int ctas_per_sm, int iters,
                                int reps, double* tflops, double* best_ms);

/* ---- Sort without any device allocation ----------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need a sort, so cannot provide the
 * workspace that part_init requires.  Examples: a plug-in inside a host code
 * that owns every device byte through its own memory pool, or a
 * latency-critical loop where a cudaMalloc (which may synchronise the device)
 * is not acceptable.
 *
 * Same result as part_sort on a PART_FP64 / PART_BORIS context: the particles
 * are stably sorted by the brick cell key (see part_brick_dims) and x[3][n],
 * u[3][n], w[n] (may be NULL) and id[n] (may be NULL) are permuted in place;
 * cell_start receives nkeys + 1 entries.  All pointers are device pointers
 * owned by the caller; the work is enqueued on cuda_stream (NULL = legacy
 * default stream).
 *
 * Scratch: a static array of PART_NOALLOC_SORT_SCRATCH_BYTES compiled into
 * libpart.so.  Each device holds it until the process exits: from the
 * library's load when CUDA loads modules eagerly, else (CUDA_MODULE_LOADING
 * = LAZY, the default) from the first use of the library's kernels on that
 * device.  The first call on each device (with that device current) looks up
 * the array's device address and caches it per device ordinal; the cache
 * assumes the device's primary context (the one the CUDA runtime uses) for
 * the life of the process, so do not call this entry point again after a
 * cudaDeviceReset or from another driver-API context.  Make that first call
 * before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU race: serialise them.  Nothing is allocated or freed.
 * Errors (message in part_last_error(NULL)):
 *   PART_EINVAL       n < 0 or n > PART_NOALLOC_SORT_MAX_N; x or u NULL with
 *                     n > 0; cell_start NULL; an array not aligned to its
 *                     element size; an array the kernels cannot reach
 *                     (pageable host memory, another device's memory);
 *                     an invalid grid;
 *   PART_EUNSUPPORTED the current device's ordinal is 128 or more;
 *   PART_ECUDA        a CUDA runtime call (device query, symbol lookup,
 *                     launch) failed.
 * Non-finite positions are sorted as if in cell 0 of that axis and are not
 * reported by this entry point.                                             */
#define PART_NOALLOC_SORT_MAX_N 1048576
#define PART_NOALLOC_SORT_SCRATCH_BYTES 25428736
part_status part_sort_fp64_noalloc(const part_grid* grid, int64_t n, double* x, double* u,
                                   double* w, uint64_t* id, uint32_t* cell_start,
                                   void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PART_H */
