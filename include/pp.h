/*
 * pp.h -- C ABI of the GB300 (sm_103a) Photon-Plasma particle step.
 *
 * Method: Haugboelle, Frederiksen & Nordlund, "Photon-Plasma: a modern
 * high-order particle-in-cell code" (arXiv:1211.4575).  The library advances a
 * 3D periodic relativistic Maxwell-Vlasov system (Sec. II, eq:vlasov ..
 * eq:ampere) with macro-particles of B-spline shape (eq:pseudop,
 * eq:weightfunction), leap-frog time staggering (Sec. III, step order 1-5),
 * a Vay or Boris push, a charge-conserving high-order current (Sec. III
 * "Charge conserving current density", eq:cc1 .. eq:penta) and the implicit
 * de-centred field update (eq:bnplus1, eq:enplus1, eq:EllipticB).
 *
 * Units and normalisation: c = eps0 = mu0 = 1 (the fields c and eps0 of the
 * grid descriptor must be 1).  Positions are physical, x in [0, nx*dx).
 * Proper velocity u = gamma*v, staggered half a step back in time.
 *
 * Mesh layout seen through the ABI (pp_load_fields, pp_get_fields,
 * pp_get_rho): FP64 arrays of nx*ny*nz values, x fastest
 * (a[i + nx*(j + ny*k)]), Yee-staggered as in Sec. III (Fig. "Spatial
 * staggering"): E_x, J_x at ((i+1/2)dx, j dy, k dz); B_x at
 * (i dx, (j+1/2)dy, (k+1/2)dz); cyclic for y and z; rho at (i dx, j dy, k dz).
 *
 * Conventions common to every entry point:
 *  - Return value: PP_OK (0) or one of the PP_E* codes below.  No exception or
 *    abort crosses the ABI.  pp_last_error(ctx) describes the last failure.
 *  - Ownership: the caller owns every host buffer it passes; the library
 *    copies in and out and keeps no pointer to them after the call returns.
 *    Device buffers passed with on_device = 1 are read during the call only.
 *    The library owns all device state of a context (fields, particles,
 *    scratch), allocated in pp_init_grid / pp_init_species and freed by
 *    pp_destroy.
 *  - Streams: all device work of a context is issued on the stream given in
 *    pp_grid_desc.stream (a cudaStream_t; NULL = the legacy default stream).
 *    pp_step, pp_deposit, pp_field_update and pp_sort only enqueue work;
 *    calls that return data to the host synchronise that stream.
 *  - Threading: calls on one context are not thread-safe; distinct contexts
 *    may be used from distinct threads.
 */
#ifndef PP_GB300_PP_H
#define PP_GB300_PP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PP_OK 0
#define PP_EINVAL 1     /* invalid argument or descriptor                        */
#define PP_ENOMEM 2     /* device or host allocation failed, or capacity exceeded */
#define PP_EBUSY 3      /* no free slot (batched form)                           */
#define PP_ECUDA 4      /* a CUDA runtime call failed                            */
#define PP_ETIMEOUT 5   /* a bounded device-side wait ran out                    */
#define PP_ENOCONV 6    /* field relaxation could not reach its tolerance       */
#define PP_ECFL 7       /* a particle moved a cell or more in one step           */
#define PP_ENAN 8       /* a non-finite particle value was met                   */
#define PP_WSTAB 9      /* warning: alpha < 0.525 with 6th order + PCS (Sec. III) */
#define PP_EBOUNDS 10   /* checked build (-DPP_CHECKED) only: a kernel index left its
                           array; that access was skipped                          */

/* ---- enumerations ---- */
#define PP_VAY 0
#define PP_BORIS 1
#define PP_FP64 0       /* FP64 positions (cell units), momenta, fields, current   */
#define PP_MIXED32 1    /* int32 cell + FP32 offset, FP32 momenta/fields/current;
                           FP64 global reductions                                 */
#define PP_DEPOSIT_AUTO 0
#define PP_DEPOSIT_GLOBAL 1  /* one thread per particle, L2 atomics                */
#define PP_DEPOSIT_TILED 2   /* cell tiles staged in shared memory (PP_MIXED32), cell
                                sort every sort_interval steps                     */
#define PP_DEPOSIT_CELLS 3   /* PP_MIXED32: particles sorted by cell at the start of
                                every particle pass (Sec. III, the sort between the
                                deposit and the field update of every step); the
                                E/B window of each 8^3 tile arrives by TMA tensor
                                copies (bounded wait, PP_ETIMEOUT); the current of
                                the particles of one cell that cross no support
                                boundary, and of those that cross it on the same
                                single axis in the same direction, is summed in
                                registers, then in an int32 fixed-point tile
                                window.  Needs the
                                charge-conserving current and mesh sizes that are
                                multiples of 8; PP_DEPOSIT_AUTO takes it wherever it
                                applies                                             */

#define PP_FIELD_IMPLICIT 0  /* de-centred implicit update, eq:EllipticB (default)    */
#define PP_FIELD_EXPLICIT 1  /* explicit FDTD leap-frog (cold-beam comparison)         */
#define PP_CURRENT_CONSERVING 0  /* charge-conserving high-order current (default)    */
#define PP_CURRENT_DIRECT 1      /* direct current eq:jj2 (the original method)        */
#define PP_BOUNDARY_PERIODIC 0   /* x periodic like y and z (default)                  */
#define PP_BOUNDARY_WALLS 1      /* reflecting walls at x = 0 and x = nx*dx            */

#define PP_MAX_SPECIES 8

typedef struct pp_ctx pp_ctx;

/* Grid and solver parameters (Sec. III).  Validation (PP_EINVAL): n >= 1 per
 * axis and <= 1023, at most 2^28 cells once each size is rounded up to a
 * multiple of 8; d > 0; dt > 0 with c*dt/d < 1 on every axis (a particle
 * crosses at most one cell face per step); c = eps0 = 1; field_order in
 * {2,4,6}; 0.5 <= alpha < 1 (eq:bnplus1); shape_order in {1,2,3} (CIC, TSC,
 * PCS of Sec. II); pusher PP_VAY or PP_BORIS; precision PP_FP64 or
 * PP_MIXED32.  alpha < 0.525 with field_order 6 and PCS returns PP_WSTAB but
 * still creates the context (the paper reports instability below 0.525).
 *
 * boundary_x = PP_BOUNDARY_WALLS puts reflecting walls at x = 0 and
 * x = L = nx*dx (Sec. V "Boundary conditions"); boundary_y and boundary_z do
 * the same on y and z, on any set of axes (the others stay periodic).  The
 * walls sit on integer (charge-density) nodes.  A particle that crosses a wall
 * deposits its current as if streaming freely, its virtual mirror image
 * deposits the mirrored current (rho and the components along the wall added
 * across it, the normal component subtracted), and only then is it reflected:
 * x_a -> 2 x_b - x_a, u_a -> -u_a.  The fields keep the paper's parities
 * across each wall: components staggered along its normal a (E_a; B_b, b != a)
 * odd, the others even.  The library holds the mesh as the mirror-extended
 * periodic box, 2*n_a cells on each walled axis a, whose added half is the
 * mirror image of the physical one, and every mesh array of the ABI
 * (pp_load_fields, pp_get_fields, pp_get_rho) has that shape (e.g.
 * 2*nx*ny*nz values, x fastest, with walls on x).  pp_load_fields projects
 * its arrays onto the mirror-symmetric state (each value and its image
 * replaced by their parity-signed mean).  Particle positions stay physical:
 * x_a in [0, L_a] on a walled axis.  Needs 2*n_a <= 1023 (and a multiple of 8
 * for the tiled deposit). */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double dt;
    double c, eps0;
    int field_order;
    double alpha;
    int shape_order;
    int pusher;
    int precision;
    int sort_interval;    /* cell sort every this many steps; 0 = only at load   */
    int relax_max_iter;   /* cap on relaxation sweeps of eq:EllipticB            */
    double relax_tol;     /* target relative residual of eq:EllipticB            */
    int deposit_mode;     /* PP_DEPOSIT_*                                         */
    void *stream;         /* cudaStream_t                                          */
    int boundary_x;       /* PP_BOUNDARY_PERIODIC or PP_BOUNDARY_WALLS             */
    int boundary_y;       /* the same for y and z (walls on any set of axes)      */
    int boundary_z;
} pp_grid_desc;

/* One particle species: charge q, mass m, and w = number density represented
 * by one macro-particle (eq:pseudop, eq:rho2); capacity = maximum number of
 * macro-particles the species may hold. */
typedef struct {
    double q, m, w;
    int64_t capacity;
} pp_species_desc;

/* FP64 global diagnostics (Sec. III eq:gauss, eq:divb, eq:rho2; Sec. VIII
 * field-energy series).  dV = dx*dy*dz.  Between walls the field energies and
 * the charge are those of the physical box (the sums over the mirror-extended
 * mesh over 2^k, k walled axes); maxima are taken over the extended mesh,
 * which holds the same values 2^k times. */
typedef struct {
    int64_t step;              /* steps taken since pp_init_grid                 */
    double time;               /* step * dt                                       */
    double energy_E;           /* sum 1/2 |E|^2 dV                                */
    double energy_B;           /* sum 1/2 |B|^2 dV                                */
    double energy_Ex;          /* sum 1/2 E_x^2 dV                                */
    double kinetic[PP_MAX_SPECIES]; /* sum over particles w m (gamma - 1) dV     */
    double kinetic_total;
    double charge;             /* sum rho dV                                       */
    double rho_max;            /* max |rho|                                        */
    double gauss_max;          /* max |div^- E - rho/eps0|                         */
    double gauss_drift_max;    /* max |G - G_0|, G_0 taken at the first load      */
    double divB_max;           /* max |div^+ B|                                    */
    double relax_residual;     /* max|(1 - a^2 dt^2 L)B - rhs| / max|rhs|, last solve
                                  (with the B a divergence filter, an outflow layer
                                  or a window shift left after it; PP_ENOCONV is
                                  then not raised from it)                          */
    int relax_iters;           /* relaxation sweeps of the last solve             */
    int status;                /* PP_* code of the device status word             */
    int64_t n_particles;       /* all species                                      */
    int64_t n_slow;            /* particles sent to the fallback path, last step   */
} pp_diag;

/* Per-phase device time of a context, measured with CUDA events recorded on
 * the context's own stream around every phase while profiling is enabled. */
typedef struct {
    double particle_ms;        /* fused gather/push/move/deposit kernels          */
    int64_t particle_launches;
    double current_ms;         /* ghost fold + high-order current solve           */
    double field_ms;           /* implicit field update + ghost fill              */
    double sort_ms;            /* cell sorts                                       */
    int64_t steps;             /* steps (or deposit/field halves) recorded         */
    int64_t kernel_launches;   /* every kernel this context enqueued while enabled */
} pp_profile;

/* Create a context: validates the descriptor, allocates the padded Yee mesh
 * (fields zeroed, E = B = J = 0) and binds the stream.  *out receives the
 * context, or NULL on failure (the error text is then available through
 * pp_last_error(NULL)). */
int pp_init_grid(pp_ctx **out, const pp_grid_desc *desc);

/* Add a species (at most PP_MAX_SPECIES); allocates its particle storage for
 * desc->capacity macro-particles.  *species_id receives its index 0, 1, ... */
int pp_init_species(pp_ctx *ctx, const pp_species_desc *desc, int *species_id);

/* Radiative cooling of species sid (Sec. "Radiative cooling", eq:prad,
 * eq:udot): after each Lorentz push the proper velocity loses
 *   pdot_rad dt = -coef gamma0 / p0^2 [pdot0^2 + |pdot0 x p0|^2] p0 dt,
 * with p0 = (p+ + p-)/2, pdot0 = (p+ - p-)/dt of that push, gamma0 =
 * sqrt(1 + p0^2), explicit and not iterated (the paper's choice).  coef is
 * mu0 q^2 / (6 pi m c) of eq:udot in the library's units: it depends on the
 * physical length unit of the run, so the caller supplies it.  0 (the
 * default) turns cooling off.  The explicit form assumes that one step
 * changes the energy by a small fraction.  Errors: PP_EINVAL for a bad sid
 * or a coefficient that is negative or not finite.  Takes effect at the next
 * pp_step / pp_deposit. */
int pp_set_radiative_cooling(pp_ctx *ctx, int sid, double coef);

/* Time integrator of pp_step (Sec. III, the symmetric fourth-order
 * symplectic integrator of Yoshida / Forest & Ruth / Candy & Rozmus).
 * order 2 (default): the leap-frog step; proper velocities are staggered
 * half a step behind the positions.  order 4: each step is four kick-drift
 * substeps, kick b_i dt then drift a_i dt with b = (0, w1, w0, w1) and
 * a = (w1/2, (w0+w1)/2, (w0+w1)/2, w1/2), w1 = 1/(2 - 2^(1/3)),
 * w0 = -2^(1/3) w1, so that every kick is centred on the position time.  The
 * fields advance with the drifts (field update with dt -> a_i dt and the
 * current of that drift).  In order 4 the proper velocities are synchronous
 * with the positions at step boundaries (load u at t, read back u at the new
 * t).  A step costs four particle passes and four field solves.  Errors:
 * PP_EINVAL for another order.  Takes effect at the next pp_step; pp_deposit
 * and pp_field_update always take one leap-frog step. */
int pp_set_integrator(pp_ctx *ctx, int order);

/* Step graphs (no counterpart in the paper: a launch-overhead measure for
 * small runs).  With enable = 1, pp_step captures each step as a CUDA graph
 * the first time the context is in that state, and replays the capture
 * afterwards.  A state is whether the step sorts, which of the two current
 * buffers holds J, and which of its two buffers holds each species; at most
 * 8 captures are kept, the oldest replaced first.  Results equal those of
 * the eager path.  Every call that changes what a step launches (species,
 * particle loads, cooling, integrator, tuning) drops the captures.  Graphs
 * are not used while profiling is enabled.  Needs a context stream other
 * than the legacy default (PP_EINVAL otherwise).  If a capture fails the
 * context returns to eager steps for good.  enable = 0 frees the captures.
 * A runtime setting: checkpoints do not keep it. */
int pp_set_graphs(pp_ctx *ctx, int enable);

/* Steps captured as graphs and steps replayed from a capture since
 * pp_init_grid (either pointer may be NULL). */
int pp_get_graph_stats(pp_ctx *ctx, int64_t *captures, int64_t *replays);

/* Field solver of pp_step / pp_field_update.  PP_FIELD_IMPLICIT (default)
 * is the de-centred implicit update of eq:bnplus1 / eq:enplus1 relaxed
 * through eq:EllipticB.  PP_FIELD_EXPLICIT is the explicit FDTD solver the
 * paper compares against in its cold-beam test (Sec. VIII, fig:coldbeam):
 * Yee's leap-frog with the same staggered differences of field_order, B in
 * two half steps so that E and B stay at the same time level,
 *   B^{n+1/2} = B^n - dt/2 curl^+ E^n,
 *   E^{n+1} = E^n + dt (curl^- B^{n+1/2} - J),
 *   B^{n+1} = B^{n+1/2} - dt/2 curl^+ E^{n+1}.
 * It has no damping (alpha plays no part) and is stable only for
 * dt sqrt(sum_a Kmax_a^2) < 2, Kmax_a the largest symbol of the staggered
 * difference along axis a.  Errors: PP_EINVAL for another solver, or for
 * PP_FIELD_EXPLICIT when dt breaks that limit (the message gives the
 * largest stable dt).  Takes effect at the next field update. */
int pp_set_field_solver(pp_ctx *ctx, int solver);

/* Current deposit.  PP_CURRENT_CONSERVING (default) is the charge-conserving
 * high-order current of Sec. III (eq:cc1 .. eq:penta).  PP_CURRENT_DIRECT is
 * eq:jj2, the paper's original method: J = sum q w v W(x - x_c) with each
 * component on its staggered nodes, W at the middle of the move and v the
 * new velocity, with no high-order current solve.  It does not satisfy the
 * discrete continuity equation; the paper pairs it with a divergence filter
 * of E (pp_set_divergence_filter).  Errors: PP_EINVAL for another mode. */
int pp_set_current_deposit(pp_ctx *ctx, int mode);

/* Divergence filter (Sec. III after eq:penta: the filtering of E that the
 * direct current needs, and the occasional filtering of E and B in long FP32
 * runs).  After every interval-th step, `passes` simultaneous smoothing steps
 *   E += tau grad^+ (div^- E - rho),   B += tau grad^- (div^+ B),
 * tau = 1 / max(sum_a K_a^2) (the largest eigenvalue of -div grad), rho
 * deposited from the particles' positions at that time.  A pass removes the
 * Nyquist-scale error and damps every other non-constant mode; it changes E
 * and B by gradients only.  The paper describes a Gauss-Seidel sweep; the
 * simultaneous form damps the same error in parallel.  passes = 0 (the
 * default) turns it off.  Errors: PP_EINVAL for passes < 0 or interval < 1. */
int pp_set_divergence_filter(pp_ctx *ctx, int passes, int interval);

/* ---- open end, injector and sliding window (PP_BOUNDARY_WALLS only) -------
 * Sec. V "Boundary conditions" (outflow) and "Sliding window and injection
 * of particles".  The upper wall at x = L stays a reflecting wall; the lower
 * end x = 0 becomes open.  pp_step applies them after each full step, in this
 * order: damping of the layer, injection, window shift (the particles that
 * leave through the open end do so in the step's own particle pass).  Steps of
 * a context that uses any of them run eagerly (no step graphs) and
 * synchronise at every sort.  A particle that leaves keeps its slot until the
 * next sort; pp_get_count, pp_get_particles, pp_diagnostics and pp_save sort
 * first when one may have left.  Errors of all three: PP_EINVAL without walls
 * or for a value outside the stated range. */

/* Outflow layer at x = 0: every step the field components chosen by
 * `components` (bit a = E_a, bit 3 + a = B_a; the paper damps those
 * perpendicular to the boundary normal, E_y E_z B_y B_z = 0x36) are multiplied
 * by 1 - damping ((cells - d) / cells)^2 at distance d < cells from x = 0,
 * taken at each component's staggered position; a particle that ends a step
 * closer than `escape` cells to x = 0 and moving outward (u_x < 0) leaves the
 * box; until then it deposits like any other.  The paper gives no profile and
 * uses about 20 cells.  cells in [0, nx] (0 = closed again: the reflecting
 * wall), damping in [0, 1], escape in [0, nx] (cells), components < 64. */
int pp_set_open_boundary(pp_ctx *ctx, int cells, double damping, double escape, int components);

/* Inflow of species sid through the open end x = 0: at the k-th step after
 * this call, floor(k r) - floor((k-1) r) particles, r = ppc ny nz v_x dt / dx
 * with v the drift velocity (the flux of a density of ppc per cell), uniform
 * in [0, v_x dt) x [0, Ly) x [0, Lz), with proper velocity u + u_th (three
 * standard normals).  Draws: Philox4x32-10 (Salmon et al., SC'11) keyed by
 * the seed; positions come from one stream for all species, so two species
 * injected with the same ppc, drift and seed enter at the same points (a
 * neutral inflow keeps Gauss's law).  The sliding window also fills its new
 * bottom layer from the injectors: round(ppc ny nz) particles uniform in
 * [0, dx) per species.  ppc = 0 turns it off.  PP_ENOMEM from pp_step when an
 * injection would exceed the species' capacity. */
int pp_set_injector(pp_ctx *ctx, int sid, double ppc, const double u[3], double u_th, uint64_t seed);

/* Sliding window moving at speed v (0 <= v < c) against x: whenever the
 * window has travelled a further cell, v (t - t_set) / dx passing an integer
 * (so its mean speed is v), the content of the box moves one cell up in x:
 * fields shift (zero in the new bottom layer), particles move up by dx, those
 * that pass the top wall leave, the injectors fill the bottom layer, and the
 * species are re-sorted.  The current J is left as the last deposit made it.
 * v = 0 turns it off. */
int pp_set_sliding_window(pp_ctx *ctx, double v);

/* Append n macro-particles to species sid (eq:pseudop): positions x,y,z
 * (physical, any real value: wrapped periodically into the box) and proper
 * velocities ux,uy,uz = gamma*v at t - dt/2.  Six FP64 arrays of n values,
 * host memory (on_device = 0) or device memory (on_device = 1); page-locked
 * host arrays are read in place by the device, pageable ones are staged.
 * On an axis between walls (PP_BOUNDARY_WALLS) x_a must lie in [0, n_a*d_a].
 * Errors: PP_ENOMEM if the count would exceed the capacity, PP_ENAN if a
 * value is not finite, PP_EINVAL for a position outside the walls (nothing is
 * appended then).  Loading re-sorts the
 * species by cell and resets the Gauss reference G_0 of pp_diagnostics (taken
 * from the loaded state before the next step or diagnostics). */
int pp_load_particles(pp_ctx *ctx, int sid, int64_t n, const double *x, const double *y, const double *z,
                      const double *ux, const double *uy, const double *uz, int on_device);

/* Replace E and B with caller values (initial condition), three FP64 arrays
 * each in the mesh layout above; on_device as in pp_load_particles.  Resets
 * the Gauss reference G_0. */
int pp_load_fields(pp_ctx *ctx, const double *const E[3], const double *const B[3], int on_device);

/* Advance nsteps full leap-frog steps (Sec. III step order 1-5): per step,
 * [cell sort when due] -> per species gather (eq:pfields) + push (Vay/Boris)
 * + move + charge-conserving deposit (eq:cc1, eq:jj3) -> ghost fold ->
 * high-order current solve (eq:jj6 .. eq:penta) -> implicit field update
 * (eq:EllipticB, eq:enplus1) -> ghost fill.  Asynchronous: the device status
 * word is examined by the next synchronising call (pp_sync, pp_diagnostics,
 * pp_get_*). */
int pp_step(pp_ctx *ctx, int nsteps);

/* The particle half of one step only (Sec. III steps 1-3): gather, push,
 * move and deposit for species sid (or every species when sid = -1), then
 * the ghost fold and the high-order current solve, leaving J^{n+1} on the
 * mesh.  Fields are not advanced and the step counter is not incremented. */
int pp_deposit(pp_ctx *ctx, int sid);

/* The field half of one step only (Sec. III steps 4-5): eq:EllipticB with the
 * current J on the mesh, then eq:enplus1, then the periodic ghost fill. */
int pp_field_update(pp_ctx *ctx);

/* Stable-order-free counting sort of every species by cell (Sec. III, the
 * sort by cell position between the deposit and the field update). */
int pp_sort(pp_ctx *ctx);

/* Change the cell-sort interval (>= 0) and the deposit mode (PP_DEPOSIT_*) of
 * a live context; both take effect from the next step and change only how
 * fast a step runs, not what it computes (the tuning knobs of the
 * autotuner; with PP_DEPOSIT_CELLS every particle pass sorts, whatever the
 * interval).  PP_EINVAL for values the context cannot use (the tiled
 * deposits need PP_MIXED32 and grid sizes that are multiples of 8). */
int pp_set_tuning(pp_ctx *ctx, int sort_interval, int deposit_mode);

/* Synchronise the context's stream and return the device status word as a
 * PP_* code (PP_ECFL, PP_ENAN, PP_ENOCONV, ...; PP_OK when clean).  Clears it. */
int pp_sync(pp_ctx *ctx);

/* Check of the bounded device-side wait.  The per-step sorted kernel
 * (PP_DEPOSIT_CELLS) stages each tile's E/B window into shared memory with TMA
 * tensor copies that complete on an mbarrier; every thread's wait on it gives
 * up after one second, records PP_ETIMEOUT in the device status word and
 * stops its CTA (later tiles see the status and stop too), so that no wait can
 * hold the GPU.  This call runs that same wait in one CTA on the context's
 * stream with a limit of limit_ns nanoseconds (1 .. 10^10): with deliver != 0
 * the barrier's phase completes and the call returns PP_OK; with deliver == 0
 * the phase waits for 16 bytes that no copy delivers, the wait runs out and
 * the call returns PP_ETIMEOUT (after about 2 limit_ns: the timed-out CTA
 * waits once more, bounded, for copies in flight).  The context stays
 * usable.  PP_EINVAL for a limit outside the range. */
int pp_check_bounded_wait(pp_ctx *ctx, int deliver, long long limit_ns);

/* Global FP64 diagnostics into *out (synchronises). */
int pp_diagnostics(pp_ctx *ctx, pp_diag *out);

/* FP64 host copies of the fields in the mesh layout; any of E, B, J (each an
 * array of three host pointers to nx*ny*nz doubles) may be NULL. */
int pp_get_fields(pp_ctx *ctx, double *const E[3], double *const B[3], double *const J[3]);

/* FP64 host copy of the charge density of eq:rho2 at the integer nodes
 * (nx*ny*nz doubles). */
int pp_get_rho(pp_ctx *ctx, double *rho);

/* Copy of the context's grid descriptor into *desc (stream included) and
 * the number of species into *nspecies (either pointer may be NULL). */
int pp_get_grid(pp_ctx *ctx, pp_grid_desc *desc, int *nspecies);

/* Number of macro-particles of species sid. */
int pp_get_count(pp_ctx *ctx, int sid, int64_t *n);

/* FP64 host copies of species sid (positions physical in [0, L), proper
 * velocities), each array of pp_get_count values, in the library's current
 * (cell-sorted) order.  Particles that left through an open end or a sliding
 * window are dropped first (a sort), so call pp_get_count before sizing the
 * arrays. */
int pp_get_particles(pp_ctx *ctx, int sid, double *x, double *y, double *z, double *ux, double *uy,
                     double *uz);

/* Start (enable = 1, totals reset) or stop (enable = 0) recording per-phase
 * CUDA events.  Recording adds two event records per phase and no
 * synchronisation. */
int pp_profile_enable(pp_ctx *ctx, int enable);

/* Totals since the last pp_profile_enable(ctx, 1) (synchronises). */
int pp_profile_read(pp_ctx *ctx, pp_profile *out);

/* Checkpoint: write the descriptor, integrator order, field solver, current
 * deposit and divergence filter, species parameters (with the cooling
 * coefficient), step counter, FP64 fields and FP64 particle arrays to a file
 * (Sec. IX, each attribute as one 64-bit block so that a restart does not
 * depend on the precision form). */
int pp_save(pp_ctx *ctx, const char *path);

/* Restore a checkpoint written by pp_save into a new context on `stream`. */
int pp_restore(pp_ctx **out, const char *path, void *stream);

/* ---- z-slab decomposition of one run over ranks (one GPU each) ------------
 * Sec. IX: the paper splits a run into domains, moves particles that leave a
 * domain to its neighbour and exchanges the boundary layers of the fields.
 * Here every rank holds the whole mesh and the particles of one z-slab; a
 * step is pp_deposit on every rank, the sum of the ranks' currents
 * (pp_get_current, an allreduce by the caller's communicator, pp_set_current),
 * pp_field_update on every rank (identical inputs give identical fields), and
 * the migration of the particles that left each slab (pp_extract_particles,
 * the caller's exchange, pp_load_particles on the owner).  The driver is
 * paper_1211_4575_gb300/parallel.py. */

/* Declare ctx the rank that owns the particles with physical z in
 * [z_lo, z_hi) of a periodic box (0 <= z_lo < z_hi <= nz*dz).  A rank's charge
 * density is a share of the run's, so from here on loads do not retake the
 * Gauss reference of pp_diagnostics.  Errors: PP_EINVAL for walls on z or
 * bounds outside the box. */
int pp_set_slab(pp_ctx *ctx, double z_lo, double z_hi);

/* Copy the current J on the mesh (after pp_deposit: this rank's high-order
 * current) into three FP64 arrays in the mesh layout, device pointers when
 * on_device = 1 (enqueued on the context's stream; the caller orders its own
 * work after it), else host arrays (synchronises). */
int pp_get_current(pp_ctx *ctx, double *const J[3], int on_device);

/* Replace J on the mesh by three FP64 arrays in the mesh layout (e.g. the sum
 * of every rank's current), ready for pp_field_update; on_device as in
 * pp_get_current.  Drops the step graphs. */
int pp_set_current(pp_ctx *ctx, const double *const J[3], int on_device);

/* Remove from species sid every particle whose z lies outside the slab of
 * pp_set_slab and return their FP64 state (physical x, y, z; proper
 * velocities) in six arrays of capacity cap (device pointers when
 * on_device = 1, else host); *n_out receives the count.  Synchronises.
 * Errors: PP_EINVAL without a slab, PP_ENOMEM when more than cap particles
 * left (nothing is removed then; *n_out = 0). */
int pp_extract_particles(pp_ctx *ctx, int sid, int64_t cap, double *x, double *y, double *z, double *ux,
                         double *uy, double *uz, int on_device, int64_t *n_out);

/* Allocation-free FP64 field energies: out[0] = sum 1/2 |E|^2 dV,
 * out[1] = sum 1/2 |B|^2 dV, out[2] = sum 1/2 E_x^2 dV over an nx*ny*nz mesh,
 * the same sums pp_diagnostics reports.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * need the energies (loops that forbid allocation after start-up, because an
 * allocation may block or fail at any time; hosts that own all device memory
 * and hand over pre-allocated buffers only).
 * E, B: arrays of three DEVICE pointers to nx*ny*nz FP64 values each (the
 * mesh layout above; the caller owns them).  out: DEVICE pointer to three
 * FP64 values, written on `stream` (cudaStream_t, NULL = legacy default).
 * The call allocates nothing: its scratch (1024 x 3 FP64 partial sums, 24 KiB)
 * is a fixed array inside the library, one per device, held until the process
 * exits.  The first call on a device looks that array up (with the device
 * current) and keeps its address; make it before any stream capture.  After
 * cudaDeviceReset that address is stale: do not call this entry point on a
 * device the process has reset.  Calls whose kernels overlap
 * on the GPU share the array and race.  Errors: PP_EINVAL for NULL pointers or
 * a mesh of more than 1023^3 cells, PP_ECUDA for a failed lookup or launch;
 * pp_field_energy_noalloc_error() then returns the message (per host thread). */
int pp_field_energy_noalloc(const double *const E[3], const double *const B[3], int nx, int ny, int nz, double dV,
                            double *out, void *stream);
const char *pp_field_energy_noalloc_error(void);

/* ---- batched / served form ---------------------------------------------
 * Independent periodic runs (one context each, loaded by the caller) admitted
 * into the slots of a batch by device-memory budget and advanced together:
 * each slot's steps go to its context's own stream, so runs of different
 * sizes overlap on the GPU.  The paper runs one simulation per job; the
 * method inside a slot is exactly pp_step.  The batch does not own the
 * contexts: a slot refers to one until the slot is reported done or failed. */
typedef struct pp_batch pp_batch;

#define PP_BATCH_FREE 0     /* slot unused                                     */
#define PP_BATCH_RUNNING 1  /* steps left to enqueue, or enqueued and running  */
#define PP_BATCH_DONE 2     /* all steps finished on the device (reported once) */
#define PP_BATCH_FAILED 3   /* a step returned an error (reported once)         */

/* Device bytes a context holds (mesh, scratch and particle storage). */
int64_t pp_device_bytes(pp_ctx *ctx);

/* The device bytes of a context that pp_init_grid(desc) and nspecies
 * pp_init_species calls with the given capacities would create, before any
 * of it exists (pp_device_bytes of that context returns the same figure): a
 * server checks a run against its memory budget before building it.  0 for an
 * invalid argument. */
int64_t pp_estimate_device_bytes(const pp_grid_desc *desc, int nspecies, const int64_t *capacities);

/* New batch admitting contexts while their device bytes sum to at most
 * budget_bytes, in at most max_slots (1..4096) slots.  PP_EINVAL, PP_ENOMEM. */
int pp_batch_create(pp_batch **out, int64_t budget_bytes, int max_slots);

/* Admit ctx for `steps` steps into a free slot (*slot receives it).
 * PP_EBUSY when no slot is free or the budget would be exceeded (nothing
 * changes then); PP_EINVAL for a context that already holds a slot.  Give
 * every admitted context its own stream for overlap: such a context steps
 * through captured graphs (pp_set_graphs) while it holds the slot, and gets
 * its previous setting back when the slot is released. */
int pp_batch_admit(pp_batch *b, pp_ctx *ctx, int64_t steps, int *slot);

/* Enqueue up to max_steps steps of every running slot, one step per slot in
 * turn, then record each slot's completion event.  Does not synchronise. */
int pp_batch_advance(pp_batch *b, int max_steps);

/* Fused rounds (enable = 1): each round of pp_batch_advance then takes one
 * step of every running slot with the particle kernels of all of them in one
 * persistent launch per group of runs that share shape order, pusher and
 * boundary kind: persistent CTAs, one per SM, take the (run, tile) work items
 * of the group from a device counter, largest runs first; each slot's sort
 * before it and its current solve and field update after it run on the slot's
 * own stream.  Applies while every running slot steps through the per-step
 * sorted kernel as a leap-frog step with no open end, injector, window or
 * profiling; otherwise rounds take the per-slot path.  Results equal those of
 * the per-slot path.  Creates the batch's own stream. */
int pp_batch_set_fused(pp_batch *b, int enable);

/* Non-blocking state of a slot (PP_BATCH_*), and the steps enqueued so far.
 * A slot reported DONE or FAILED is released (its bytes return to the
 * budget); its return value is then the failing step's code.  A FAILED slot
 * is released only after the context's stream has drained (this call then
 * blocks on it). */
int pp_batch_poll(pp_batch *b, int slot, int64_t *steps_done, int *state);

/* Bytes admitted and slots in use. */
int pp_batch_used(pp_batch *b, int64_t *bytes, int *active);

const char *pp_batch_last_error(const pp_batch *b);

/* Free the batch (not the contexts). */
int pp_batch_destroy(pp_batch *b);

/* Free all device and host state of the context (NULL is accepted). */
int pp_destroy(pp_ctx *ctx);

/* Text of the last error of ctx (or of the last failed pp_init_grid /
 * pp_restore when ctx is NULL).  Static storage owned by the library. */
const char *pp_last_error(const pp_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PP_GB300_PP_H */
