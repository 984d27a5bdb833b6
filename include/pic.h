/*
 * pic.h -- C ABI of libpic, a single-GPU (GB300, sm_103a) implementation of the
 * hot path of the charge-conserving particle-in-cell step of I. V. Sokolov,
 * "Alternating-Order Interpolation in a Charge-Conserving Scheme for
 * Particle-In-Cell Simulations" (arXiv:1101.0809).
 *
 * State follows the paper's statement of the problem (Sec. 2 and Appendix):
 * on a periodic Yee grid the library holds E^n and B^{n-1/2}; per particle it
 * holds x^n and w^{n-1/2}, w = gamma*v the momentum-to-mass ratio (Eq. 1).
 * Coordinates are normalized, x~ = x/dx (Eq. coorddimless); units are Gaussian.
 *
 * Staggering (Sec. 2).  Field arrays are x-fastest, element [i,j,k] at linear
 * index (k*ny + j)*nx + i, and hold
 *     Ex at (i, j+1/2, k+1/2)   Ey at (i+1/2, j, k+1/2)   Ez at (i+1/2, j+1/2, k)
 *     Bx at (i+1/2, j, k)       By at (i, j+1/2, k)       Bz at (i, j, k+1/2)
 * J is placed like E.  A 2D3V grid (dims = 2) has an ignorable z and nz = 1.
 *
 * Precision.  PIC_FP64 runs every particle and field operation in double.
 * PIC_FP32 stores int32 cell + float offsets, float momenta and fields, and
 * accumulates currents in float; its diagnostics are still computed in double.
 * Field arrays passed to pic_set_fields / pic_get_fields use the grid's
 * precision (double for PIC_FP64, float for PIC_FP32).  Particle momenta and
 * offsets returned by pic_get_particles use it too.
 *
 * Conventions shared by every call:
 *   - every call returns int: PIC_OK (0) or one PIC_ERR_* code; the message of
 *     the last failure on the calling thread is returned by pic_last_error();
 *   - no call aborts, traps or throws across the ABI;
 *   - the library owns all device memory of a grid; inputs are copied;
 *   - on_device = 1 means the pointers are device pointers, ordered on the
 *     grid's CUDA stream; on_device = 0 means host pointers (the call then
 *     synchronizes the stream before returning);
 *   - work is enqueued on the grid's stream; pic_step, pic_gather_push,
 *     pic_deposit_current, pic_yee_update and pic_sort return without waiting.
 *     Device-side failures (a non-finite momentum) are latched in an error word
 *     that pic_sync and pic_diagnostics read and report as PIC_ERR_NONFINITE.
 */
#ifndef PIC_H
#define PIC_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PIC_OK = 0,
    PIC_ERR_INVALID_ARG = 1,  /* a null pointer, a size out of range, a bad enum */
    PIC_ERR_CFL = 2,          /* c*dt/d_a >= 1 on some axis, or the Yee limit violated */
    PIC_ERR_OOM = 3,          /* a device allocation failed */
    PIC_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
    PIC_ERR_NONFINITE = 5,    /* a particle momentum became NaN or infinite */
    PIC_ERR_OUT_OF_TILE = 6,  /* reserved: particles are never dropped, out-of-tile ones take the global path */
    PIC_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
    PIC_ERR_STATE = 8         /* call out of order (e.g. deposit before gather_push) */
};

enum { PIC_FP64 = 0, PIC_FP32 = 1 };
enum { PIC_B_HALF = 1, PIC_E_FULL = 2 };

typedef struct pic_grid pic_grid;   /* opaque */

/* Geometry and run parameters.  dt and c are in the same units as dx; the
 * Courant numbers are c_a = c*dt/d_a (Sec. 2). */
typedef struct {
    int dims;               /* 2 (z ignorable) or 3 */
    int nx, ny, nz;         /* cells per axis; nz must be 1 when dims == 2 */
    double dx, dy, dz;      /* cell sizes (dz ignored when dims == 2) */
    double dt, c;           /* time step; speed of light */
    int precision;          /* PIC_FP64 or PIC_FP32 */
    int order2;             /* twice the alternating order l_a (Sec. 4.5): 3 (or 0) for l_a = 1 1/2,
                               5 for l_a = 2 1/2; 4 selects the uniform-order l = 2 comparison
                               scheme of Eq. wrong1 (Sec. 5: fields interpolated with the
                               cell-centred weights averaged over the faces, l_a = 1 1/2 charge
                               and current).  Orders 4 and 5 run the fused, split and
                               diagnostics paths; the persistent batch step and the adjoint
                               are l_a = 1 1/2 only */
    int tile[3];            /* tile extents in cells for the sort and the shared-memory
                               stages (0 = default: 8x8x8 in 3D, 16x16 in 2D) */
    int halo;               /* drift guard in cells around a tile (0..2; -1 = default 1) */
    int sort_interval;      /* sort the particles by tile every K steps (>= 1; 0 = default 10) */
    int particles_per_block;/* particles per thread block work item (0 = default 8192) */
    double rho_bg;          /* uniform immobile background charge density (enters rho only) */
    void *cuda_stream;      /* cudaStream_t to enqueue on; NULL = the legacy default stream */
    int sort_order;         /* PIC_SORT_AUTO (0, default), PIC_SORT_STABLE, PIC_SORT_BANKED or
                               PIC_SORT_CELL_LANES; see the enum below */
} pic_grid_desc;

/* Order of the tile sort.  Every order sorts by tile key first (the tile of
 * the particle's cell, tiles numbered (tk*nty + tj)*ntx + ti per run and
 * species); they differ inside a tile.
 * PIC_SORT_STABLE keeps the input order inside a tile.
 * PIC_SORT_BANKED orders a tile's particles by (r, b): b = base mod 32 with
 * base = (i-ox+h+2) + P0*((j-oy+h+2) + P1*(k-oz+h+2))
 * (h = the halo, plus one for l_a = 2 1/2, whose current tile is one cell wider)
 * (no k term in 2D) the shared-memory bank of the particle's cell in the
 * current tile of its tile (tile origin (ox, oy, oz), halo h, tile pitches
 * P0, P1 as reported by pic_tile_layout), and r the number of earlier
 * particles (input order) of the same tile with the same b; so that 32
 * consecutive particles fall on 32 different banks.  For l_a = 2 1/2 the
 * interpolation is anchored at the base index, the cell plus (offset >= 1/2)
 * per axis, so i, j, k in base are those of the base index.
 * PIC_SORT_CELL_LANES (tiles of at most 128 cells) gives each cell of a tile,
 * c = (i-ox) + Tx*((j-oy) + Ty*(k-oz)), a lane L(c): the cells ranked by
 * descending particle count, ties by c.  The particle of rank r among its
 * cell's particles (input order) takes slot P(r) + L(c) of the tile, with
 * P(r) = sum over the tile's cells of min(count, r).  A thread per lane then
 * walks the particles of one cell while the threads of a warp read
 * consecutive slots; the FP32 fused step of 3D grids with 8x4x4 tiles, halo 1
 * and l_a = 1 1/2 runs that way when this order is requested (the particles
 * that have left their cell since the sort take a general path, so the order
 * pays off for slow species and short sort intervals).
 * PIC_SORT_AUTO (0, the default) is PIC_SORT_BANKED. */
enum { PIC_SORT_AUTO = 0, PIC_SORT_STABLE = 1, PIC_SORT_BANKED = 2, PIC_SORT_CELL_LANES = 3 };

/* One species.  The macro-particle charge is q_p = weight*q, its mass m_p = weight*m;
 * the push uses q/m (Eq. 1), the deposit q_p/V (Eq. xi). */
typedef struct {
    double q, m, weight;
} pic_species_desc;

/* FP64 diagnostics at time level n, i.e. between two pic_step calls where the
 * state is E^n, B^{n-1/2}, x^n, w^{n-1/2}:
 *   kinetic        sum m_p c (sqrt(w^2 + c^2) - c)
 *   field_E        V/(8 pi) sum E^2
 *   field_B        V/(8 pi) sum B^2 with B^n = B^{n-1/2} - (1/2) c curl E^n
 *   half_step_corr sum (q_p dt/2) u^{n-1/2} . E(x^n)       (energy integral, Sec. 4.1)
 *   total          kinetic + field_E + field_B + half_step_corr
 *   momentum       sum m_p w
 *   total_charge   V * sum_cells rho (particles and background)
 *   gauss_resid_*  max and root-mean-square over cells of |r^n - r^ref|, where
 *                  r = div E - 4 pi rho (Eq. chargelaw) and r^ref is the residual
 *                  at the first pic_diagnostics call after the last load or set.
 */
typedef struct {
    double kinetic, field_E, field_B, half_step_corr, total;
    double momentum[3];
    double total_charge;
    double gauss_resid_max, gauss_resid_rms;
    long long n_particles;
    int error_word;
} pic_diag;

/* Create a grid with zero fields and no particles.  The grid uses the stream in
 * desc->cuda_stream for all its work.  Returns PIC_ERR_CFL when a Courant number
 * c*dt/d_a is >= 1 (the deposit window assumes a particle crosses at most one
 * face per axis per step) or when c*dt*sqrt(sum 1/d_a^2) >= 1 (Yee stability). */
int pic_create_grid(const pic_grid_desc *desc, pic_grid **out);

/* Free a grid and all its device memory.  Null is accepted. */
int pic_destroy(pic_grid *g);

/* Copy E^n and B^{n-1/2} in.  Each pointer holds nx*ny*nz values of the grid's
 * precision.  Clears the residual reference of pic_diagnostics. */
int pic_set_fields(pic_grid *g, const void *const E[3], const void *const B[3], int on_device);

/* Copy E, B and the last deposited J (J^{n+1/2} after pic_step or
 * pic_deposit_current) out.  Any of the three arrays of pointers may be null. */
int pic_get_fields(pic_grid *g, void *E[3], void *B[3], void *J[3], int on_device);

/* Load (replace) one species.  x[a] are n normalized absolute positions per
 * axis (any real value; wrapped periodically into [0, N_a)), w[a] the momenta
 * w^{n-1/2}; both double.  x[2] is ignored in 2D.  species is 0..31 and may
 * skip indices.  All particles of the grid are re-sorted by tile on return.
 * Particle k of this call gets id k (see pic_get_particles). */
int pic_load_particles(pic_grid *g, int species, const pic_species_desc *sp, long long n,
                       const double *const x[3], const double *const w[3], int on_device);

/* Layout chosen at creation: out[0..2] tile extents, out[3] halo, out[4..5] the
 * x and y pitch of the shared-memory field and current tiles. */
int pic_tile_layout(pic_grid *g, int out[6]);

/* Number of particles of a species (0 if not loaded). */
long long pic_num_particles(pic_grid *g, int species);

/* Copy one species out in the library's current storage order: cell (linear
 * cell index (k*ny + j)*nx + i), offset[a] in [0, 1) so that x_a = i_a + offset_a,
 * w[a], and id (the particle's index in its pic_load_particles call).  Any
 * pointer may be null; offset[2] is not written in 2D. */
int pic_get_particles(pic_grid *g, int species, int *cell, void *offset[3], void *w[3], int *id,
                      int on_device);

/* Appendix step 2a-2c for every particle: alternating-order form factor at x^n
 * (Sec. 4.5), gather of E (Eq. alphax) and B (Eq. betax), relativistic push
 * (Eq. 1, Appendix), new position (Eq. coordscheme).  Needs B^n: call
 * pic_yee_update(g, PIC_B_HALF) first.  Keeps x^n for pic_deposit_current. */
int pic_gather_push(pic_grid *g);

/* Appendix step 2d: J^{n+1/2} = sum_p (q_p/V) xi(x^n, x^{n+1}) by the six-box-path
 * virtual-path current (Eq. current) from the positions kept by the last
 * pic_gather_push and the current ones.  J is zeroed first.  Returns
 * PIC_ERR_STATE if no pic_gather_push preceded it since the last load or sort. */
int pic_deposit_current(pic_grid *g);

/* Yee updates (Appendix).  PIC_B_HALF: B -= (1/2) c curl_h E (Eq. updateB).
 * PIC_E_FULL: E += -4 pi dt J + c curl_h B (Eq. escheme). */
int pic_yee_update(pic_grid *g, int which);

/* ---- Plane-wave antenna ------------------------------------------------------
 * The paper motivates laser-plasma runs but gives no injection; this antenna is
 * a one-way source on a plane of constant x (a total-field / scattered-field
 * boundary), uniform in y and z, so it adds no charge and leaves the discrete
 * continuity equation untouched.  The incident wave travels in +x:
 *   E_inc(x, t) = amplitude * g(tau) * sin(omega * tau),  tau = t - (x - plane) dx / c,
 *   g = sin^2(pi tau / (2 ramp)) for 0 < tau < ramp, 1 after, 0 before;
 * polarization PIC_POL_Y: E_y = E_inc, B_z = E_inc; PIC_POL_Z: E_z = E_inc, B_y = -E_inc.
 * The total field starts at the B node x = plane.  Each B half step of step n
 * adds (c_x/2) E_inc(plane - 1/2, t^n) to B_z (PIC_POL_Y) or subtracts it from
 * B_y (PIC_POL_Z) on the cells i = plane; the E step adds
 * c_x E_inc(plane, t^n + dt/2) to E_y or E_z on the cells i = plane - 1.  t^n =
 * n dt counts the E steps since the antenna was set, plus `start` (the
 * antenna's clock, kept on the device, saved in state snapshots).  The box stays periodic: the wave
 * must not reach the plane again from the other side.  a == NULL removes the
 * antenna.  Errors: PIC_ERR_INVALID_ARG for a bad run, polarization or plane
 * (1 <= plane < nx required). */
enum { PIC_POL_Y = 1, PIC_POL_Z = 2 };
typedef struct {
    int polarization;   /* PIC_POL_Y or PIC_POL_Z */
    int plane;          /* x index of the first total-field B node */
    double amplitude;   /* E_0 */
    double omega;       /* angular frequency */
    double ramp;        /* rise time of the sin^2 envelope (0: none) */
    long long start;    /* initial value of the antenna's clock (E steps already taken) */
} pic_antenna_desc;
int pic_set_antenna(pic_grid *g, int run, const pic_antenna_desc *a);

/* Sort policy of pic_step.  By default particles are re-sorted by tile every
 * sort_interval steps.  With adaptive != 0, pic_step times every step's
 * particle kernel and counts the particles that ran more than `halo` cells
 * past their tile since the last sort (they take the slower global-memory
 * path).  While there are such particles it sums the kernel's time above that
 * of the first step after the last sort, and sorts before the next step once
 * the sum, plus the last step's excess again (the next step costs at least as
 * much), exceeds the measured time of a sort.  A sort so triggered after k
 * steps sets the interval to k - 1 (drift that builds up coherently, as in a
 * laser-driven plasma, arrives all at once); after a growing number of cycles
 * without drift the interval is tried one step longer.  sort_interval stays
 * the longest interval.  The measurement costs one stream synchronization per step, so the
 * adaptive policy applies to pic_step only (pic_step_persistent and
 * pic_step_graph keep the fixed interval), and the sort schedule follows the
 * timings.  Errors: PIC_ERR_INVALID_ARG for a null grid. */
int pic_set_sort_policy(pic_grid *g, int adaptive);

/* nsteps full steps of the Appendix: B half step, [tile sort every
 * sort_interval steps], gather + push + deposit fused in one pass over the
 * tile-sorted particles, B half step, E full step. */
int pic_step(pic_grid *g, int nsteps);

/* Sort all particles by tile (order inside a tile: see PIC_SORT_AUTO). */
int pic_sort(pic_grid *g);

/* FP64 diagnostics (see pic_diag).  Synchronizes the grid's stream. */
int pic_diagnostics(pic_grid *g, pic_diag *out);

/* Synchronize the grid's stream and report a latched device error, if any. */
int pic_sync(pic_grid *g);

/* Message of the last failure on the calling thread ("" if none). */
const char *pic_last_error(void);

/* Allocation-failure injection, for testing the failure paths (the paper has
 * no counterpart).  After the call, the library's next `after` device
 * allocations succeed and the one after them fails as an out-of-memory
 * condition would; the call that made it returns PIC_ERR_OOM.  One failure per
 * arming; after < 0 disarms.  Process-wide.  A load that fails this way leaves
 * the grid usable: a failure while the new particle pool is allocated keeps
 * the previous particles, a later one leaves the grid with its fields and no
 * particles. */
int pic_inject_alloc_failure(long long after);

/* Number of kernels this grid has launched since creation (for accounting). */
long long pic_kernel_launches(pic_grid *g);

/* ---- Batched form -------------------------------------------------------------
 * pic_create_batch makes nruns independent periodic runs in one grid object.
 * They share dims, precision, tile, halo, sort interval, particles per block
 * and stream (all taken from descs[0]); each run keeps its own cell counts, cell
 * sizes, dt, c and rho_bg, checked as in pic_create_grid.  Fields are stored run
 * after run; one particle pool holds every (run, species), sorted together, and
 * every kernel launch covers all runs.  The *_run calls address one run
 * (0 .. nruns-1); the calls without _run address run 0.  pic_step,
 * pic_step_persistent and pic_step_graph advance every run. */
int pic_create_batch(const pic_grid_desc *descs, int nruns, pic_grid **out);
int pic_num_runs(pic_grid *g);
int pic_set_fields_run(pic_grid *g, int run, const void *const E[3], const void *const B[3], int on_device);
int pic_get_fields_run(pic_grid *g, int run, void *E[3], void *B[3], void *J[3], int on_device);
int pic_load_particles_run(pic_grid *g, int run, int species, const pic_species_desc *sp, long long n,
                           const double *const x[3], const double *const w[3], int on_device);
/* Bulk form of pic_load_particles_run for one species index over `count` runs
 * with a single pool re-layout and sort: runs[r], sp[r], n[r], and the arrays
 * x[3*r + a], w[3*r + a] (a = 0, 1, 2) for entry r. */
int pic_load_particles_runs(pic_grid *g, int count, const int *runs, int species, const pic_species_desc *sp,
                            const long long *n, const double *const *x, const double *const *w, int on_device);
long long pic_num_particles_run(pic_grid *g, int run, int species);
int pic_get_particles_run(pic_grid *g, int run, int species, int *cell, void *offset[3], void *w[3], int *id,
                          int on_device);
int pic_diagnostics_run(pic_grid *g, int run, pic_diag *out);

/* The same steps as pic_step, one kernel launch per step: a cooperative
 * persistent kernel runs the B half step (with the J clear), the fused particle
 * work of every run, the second B half step and the E step, separated by
 * grid-wide barriers (its grid is the number of blocks that can be resident at
 * once).  The tile sort adds its own launches every sort_interval steps.
 * Built for l_a = 1 1/2: PIC_ERR_INVALID_ARG on a grid with order2 = 5 (as
 * for pic_step_graph). */
int pic_step_persistent(pic_grid *g, int nsteps);

/* pic_step_persistent replayed from a CUDA graph of 2*sort_interval steps
 * (two sorts, so that the double-buffered particle pool returns to the buffer
 * it started in).  The graph is captured on first use, on the grid's stream,
 * which must not be the legacy default stream; loading particles or calling
 * pic_sort / pic_step / pic_step_persistent discards it.  Steps that do not
 * fill a whole graph run uncaptured. */
int pic_step_graph(pic_grid *g, int nsteps);

/* Launch-group timing with CUDA events recorded on the grid's stream.
 * pic_profile(g, 1) clears the totals and starts recording an event pair around
 * every launch group below; pic_profile(g, 0) stops.  pic_profile_read
 * synchronizes the stream and returns, per group, the summed device time in
 * milliseconds and the number of groups timed since the last pic_profile(g, 1). */
enum {
    PIC_PROF_YEE_B = 0,       /* B half steps (with the J clear) */
    PIC_PROF_PARTICLES = 1,   /* the particle kernel(s): fused step, gather_push or deposit */
    PIC_PROF_YEE_E = 2,       /* E full step */
    PIC_PROF_SORT = 3,        /* the tile sort and work-list build */
    PIC_PROF_N = 4
};
int pic_profile(pic_grid *g, int enable);
int pic_profile_read(pic_grid *g, double ms[PIC_PROF_N], long long count[PIC_PROF_N]);

/* ---- Vector-potential formulation (Sec. 4.2) -----------------------------------------
 * pic_set_vector_potential starts tracking the vector potential A^{n-1/2} on the
 * E points (three arrays of the grid's precision, runs concatenated like the
 * fields; host or device memory, copied).  From then on every E step (pic_step,
 * pic_yee_update(PIC_E_FULL)) first advances it by Eq. dadt,
 * A^{n+1/2} = A^{n-1/2} - c dt E^n.  With set_B != 0 the call also sets
 * B^{n-1/2} = curl_h A^{n-1/2} (Eq. viaA, grid form:
 * Bx[i,j,k] = (Az[i,j,k] - Az[i,j-1,k])/dy - (Ay[i,j,k] - Ay[i,j,k-1])/dz,
 * cyclically), so that B stays the curl of A.  A = NULL stops tracking.  The
 * vector potential is not part of a state snapshot, and pic_step_persistent and
 * pic_step_graph refuse a grid that tracks it (PIC_ERR_INVALID_ARG).
 * pic_generalized_momentum_run returns P = sum_p m_p w_p^{n-1/2} +
 * (q_p/c) A^{n-1/2}(x_p^n - (dt/2) u_p^{n-1/2}) over the run's particles, A
 * interpolated with the E weights alpha of the grid's interpolation (Eq. A),
 * summed in FP64; it is conserved along an axis the fields do not depend on
 * (Sec. 4.2, up to the time discretization).  Errors: PIC_ERR_INVALID_ARG for
 * null arguments or a bad run; PIC_ERR_STATE when no vector potential is
 * tracked. */
int pic_set_vector_potential(pic_grid *g, const void *const A[3], int on_device, int set_B);
int pic_get_vector_potential(pic_grid *g, void *A[3], int on_device);
int pic_generalized_momentum(pic_grid *g, double P[3]);
int pic_generalized_momentum_run(pic_grid *g, int run, double P[3]);

/* ---- State snapshots ------------------------------------------------------------
 * A snapshot is one contiguous blob: a 64-byte header ("PICS", version 4,
 * dims, precision, group count, sort phase, particle, cell, tile and run
 * counts, whether cell-lane tables follow, and a checksum of the header)
 * followed by the particle arrays (cell, id, offsets, momenta, in storage
 * order), the fields E^n, B^{n-1/2}, the tile starts of the particle order
 * (from the last tile sort), the antenna clock of every run (pic_set_antenna)
 * and, for a grid in the cell-lane order, every tile's lane cells (128 bytes)
 * and lane counts (128 int32), each array starting at the next multiple of
 * 16 bytes.  A device snapshot is copied by one kernel.  pic_state_bytes gives its
 * size.  pic_state_save writes it to dst (device memory if on_device, else host
 * memory); pic_state_restore reads one taken from a grid with the same layout
 * (same runs, species, particle counts and tiles), rebuilds the work items from
 * the saved tile starts, continues the saved sort schedule (steps since the
 * last sort) and clears the residual references, so that a restored grid steps
 * on exactly as the saved one would have.  Used for checkpoints, for restart
 * from a file written by the caller, and by the adjoint's recompute. */
long long pic_state_bytes(pic_grid *g);
int pic_state_save(pic_grid *g, void *dst, int on_device);
int pic_state_restore(pic_grid *g, const void *src, int on_device);

/* pic_state_restore without the final wait: the header is read and checked
 * at once (a device snapshot's header after a synchronization of the grid's
 * stream), and the copies are only enqueued on the grid's stream, so that a
 * host-to-device restore of one grid can run under the kernels of another
 * grid on another stream.  The caller keeps src allocated and unchanged until
 * the grid's stream has passed the copies (pic_sync, or a call that returns
 * results, such as pic_diagnostics).  Errors: those of pic_state_restore; a
 * CUDA error of a copy may be reported by a later call. */
int pic_state_restore_async(pic_grid *g, const void *src, int on_device);

/* The recompute pass of a checkpointed adjoint: nsteps steps as
 * pic_step(g, 1) each, with a device snapshot of the state before step s
 * written to states[s] (nsteps device buffers of pic_state_bytes(g) bytes,
 * owned by the caller).  Everything is enqueued on the grid's stream; unlike
 * pic_state_save the call does not wait for the copies (pic_sync does).
 * Errors: PIC_ERR_INVALID_ARG for a null grid, a null list or buffer, or a
 * negative count; the errors of pic_step. */
int pic_step_saving(pic_grid *g, int nsteps, void *const *states);

/* ---- Discrete adjoint of the step -----------------------------------------------
 * pic_adjoint_step takes the grid's current state as level n (E^n, B^{n-1/2},
 * x^n, w^{n-1/2}) and maps the adjoints of level n+1 to those of level n, in
 * place: lamE, lamB are field arrays (nx*ny*nz values of the grid's precision
 * per component, runs concatenated like the fields); lamx, lamw are particle
 * arrays of the grid's precision, one value per particle, indexed by the
 * species' position in the pool plus the particle id, i.e. for one species in
 * its load order (lamx[2] is unused in 2D).  All are device pointers.  The
 * step is the reverse of pic_step: transposes of the E step and of both B half
 * steps, and for every particle the gather of lamJ over its current window, the
 * hand-derived reverse of the deposit (Eq. current), move (Eq. coordscheme),
 * push (Eq. 1) and gather (Eqs. alphax, betax), with the transposed gather
 * scattered into lamE and lamB by atomics.  The particle part runs over the
 * last tile sort's work items with each item's E, B and lamJ staged in shared
 * memory (particles that drifted past their tile's halo read the global
 * arrays), or untiled (one thread per particle, all reads global; the same
 * arithmetic); see pic_set_adjoint_tiled.
 * The adjoint is derived for l_a = 1 1/2: PIC_ERR_INVALID_ARG on a grid with
 * order2 = 5 (also for pic_adjoint_steps).
 * pic_adjoint_yee_half_B adds (-(1/2) C_B)^T lamB to lamE (the transpose of one
 * B half step), e.g. to seed a loss that uses B^n = B^{n-1/2} - (1/2) c curl E^n. */
int pic_adjoint_step(pic_grid *g, void *lamE[3], void *lamB[3], void *lamx[3], void *lamw[3]);
/* Adjoint steps back through nstates device snapshots of consecutive levels
 * (states[s] holds level n0 + s, e.g. from pic_step_saving): for
 * s = nstates-1 ... 0, restore states[s] as pic_state_restore does, then
 * pic_adjoint_step with the same adjoint arrays.  The headers of all snapshots
 * are read and checked first, with one host synchronization; nothing else
 * waits.  On return the grid holds the state of states[0].  Errors: those of
 * pic_state_restore (checked for every snapshot before any is restored) and
 * of pic_adjoint_step; PIC_ERR_INVALID_ARG for a null list or buffer or a
 * negative count. */
int pic_adjoint_steps(pic_grid *g, void *const *states, int nstates, void *lamE[3], void *lamB[3], void *lamx[3],
                      void *lamw[3]);

/* tiled != 0: the tiled particle adjoint (the default in FP32); 0: the
 * untiled one (the default in FP64, where the FP64 pipe bounds the kernel and
 * the per-block staging of the tiles costs more than it saves, and the form
 * used whenever the tiled one's shared tiles would not fit the device).
 * Errors: PIC_ERR_INVALID_ARG for a null grid. */
int pic_set_adjoint_tiled(pic_grid *g, int tiled);
int pic_adjoint_yee_half_B(pic_grid *g, void *const lamB[3], void *lamE[3]);

/* ---- The FP32 form's renormalization -----------------------------------------
 * After the move of Eq. coordscheme (Appendix, step 2c) the FP32 form stores a
 * position as an int32 cell and a float offset in [0, 1).  Moving offset o by a
 * displacement d (|d| < 1 cell, the Courant limit) gives the cell shift
 * k = floor(o + d) and the new offset, the float nearest to the exact o + d - k
 * (round to nearest even), as a double-precision renormalization rounded once
 * would give; an offset that rounds to 1 becomes offset 0 of the next cell
 * (k + 1).  pic_renormalize_f32 applies the device function the FP32 particle
 * kernels use to n pairs: offset[p], delta[p] (device memory, float) give
 * shift[p] (int) and offset_out[p] (float), device memory owned by the caller.
 * Enqueued on cuda_stream (NULL = legacy default stream); returns without
 * waiting.  Errors: PIC_ERR_INVALID_ARG for null arrays or n < 0; PIC_ERR_CUDA
 * for a failed launch.  Inputs with |delta| >= 1 or offsets outside [0, 1)
 * are outside the contract (the result is then unspecified, never a fault). */
int pic_renormalize_f32(const float *offset, const float *delta, long long n, int *shift, float *offset_out,
                        void *cuda_stream);

/* ---- FP64 FMA rate ---------------------------------------------------------------
 * The paper has no counterpart: a measurement aid for the roofline of the FP64
 * path, which is bound by the FP64 pipe.  Enqueues on cuda_stream one launch of
 * blocks_per_sm blocks of 256 threads per SM, each thread running 8 independent
 * chains of iters FP64 fused multiply-adds, and returns in *fma_count the FMAs
 * it executes; the caller times the launch (e.g. with events on the stream).
 * sink: one device double the kernel may write (never read back).  Errors:
 * PIC_ERR_INVALID_ARG for non-positive counts or null pointers, PIC_ERR_CUDA
 * for a failed launch. */
int pic_measure_fp64_fma(long long iters, int blocks_per_sm, double *sink, long long *fma_count, void *cuda_stream);

/* ---- Tile sort without device allocation -----------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory: code running inside a memory budget that another
 * runtime owns (a framework's caching allocator, a coupler that reserved the
 * whole GPU up front) or on a path where a cudaMalloc would synchronize the
 * device.  It computes the same stable permutation by tile as pic_sort (ties
 * keep their input order) but keeps every temporary in one fixed device array
 * of the library (16.25 MiB, held on every GPU that loads libpic until the
 * process exits) and never calls cudaMalloc, cudaFree or an allocating library
 * routine.
 *   cell        n linear cell indices (k*ny + j)*nx + i, device memory
 *   n           0 .. PIC_NOALLOC_MAX_PARTICLES; larger n returns PIC_ERR_INVALID_ARG
 *   dims        2 or 3; ncell[3], tile[3] as in pic_grid_desc (z ignored in 2D)
 *   perm        n outputs, device memory: perm[o] = input index of sorted slot o
 *   tile_start  ntiles+1 outputs (device memory, may be null): first sorted slot
 *               of every tile, tile_start[ntiles] = n; tiles numbered
 *               (tk*nty + tj)*ntx + ti
 *   cuda_stream stream to run on (NULL = legacy default stream)
 * A cell index outside the grid returns PIC_ERR_INVALID_ARG.  The call
 * synchronizes the stream once (after checking the cells) and returns with the
 * sort enqueued.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture.  All calls share the one array: two calls whose work overlaps
 * on the GPU (different streams, or different host threads) race and must be
 * serialized by the caller. */
#define PIC_NOALLOC_MAX_PARTICLES 1048576
int pic_tile_sort_perm_noalloc(const int *cell, long long n, int dims, const int ncell[3], const int tile[3],
                               int *perm, long long *tile_start, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
