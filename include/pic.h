/*
 * pic.h -- C ABI of libpic, a single-GPU (GB300, sm_103a) particle-in-cell
 * step for the three box methods of "Particle-in-Cell Methods for Simulations
 * of Sheared, Expanding, or Escaping Astrophysical Plasma" (arXiv 2602.15939):
 * the kinetic shearing box with orbital advection (KSB-OA, Sec. 2), the
 * kinetic expanding box (KEB, Sec. 3) and the leaky box (Sec. 4).
 *
 * Units and layout shared by every call:
 *  - code units dx = dt = 1; `c` is the Courant number c dt/dx (cells/step);
 *    Gaussian units as in the paper (4 pi in Ampere's law);
 *  - momentum u is the spatial part of the four-velocity, u = gamma v, in
 *    cells/step, gamma = sqrt(1 + (u/c)^2);
 *  - positions are absolute cell coordinates, x in [0,nx), y in [0,ny),
 *    z in [0,nz); node (i,j,k) sits at (i,j,k);
 *  - fields use Yee staggering: Ex (i+1/2,j,k), Ey (i,j+1/2,k), Ez (i,j,k+1/2),
 *    Bx (i,j+1/2,k+1/2), By (i+1/2,j,k+1/2), Bz (i+1/2,j+1/2,k); J like E.
 *    Host field arrays are float64 [3][nz][ny][nx], index ((c*nz+k)*ny+j)*nx+i;
 *  - 2D runs set the ignorable axis to one cell (plane XY: nz = 1; plane XZ:
 *    ny = 1); all three vector components are kept (2D3V); the ignorable
 *    coordinate of a particle is not tracked and reads back as 0.5;
 *  - shearing box: the radial coordinate in v_s = -s Omega0 x e_y is measured
 *    from the box centre (x - nx/2); E passed in and out is the comoving E'
 *    and u the comoving u' (Sec. 2.1);
 *  - expanding box: positions are the comoving x' and fields and momenta the
 *    lab-frame values on the x' grid (Sec. 3.2); l_i(t) = exp(rate_i t).
 *
 * Ownership: the library owns all device memory (allocated at pic_init and
 * at particle load).  Host arrays passed in are copied before the call
 * returns and never retained; host arrays passed out are filled by the call.
 * Errors: every call returns a pic_status; nothing is thrown across the ABI.
 * After a non-OK status, pic_last_error(h) describes it.  Device-side
 * failures (a bounded wait that expired, a non-finite momentum) are recorded
 * in a device error word and reported by the next pic_step or
 * pic_diagnostics as PIC_ERR_TIMEOUT or PIC_ERR_NUMERIC.
 * Streams: all work of a handle is ordered on its stream (pic_set_stream);
 * pic_step returns without waiting for the GPU.  Calls on one handle must
 * not run concurrently from several host threads.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 1
#define PIC_MAX_SPECIES 4
#define PIC_NOALLOC_MAX_COMPONENTS 8

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,     /* invalid argument or configuration */
    PIC_ERR_OOM = 2,     /* device or host allocation failed */
    PIC_ERR_CUDA = 3,    /* a CUDA runtime call failed (no device, launch error) */
    PIC_ERR_TIMEOUT = 4, /* a bounded device-side wait expired */
    PIC_ERR_STATE = 5,   /* call not valid in the handle's current state */
    PIC_ERR_NUMERIC = 6  /* non-finite particle momentum detected */
} pic_status;

typedef enum {
    PIC_BOX_PERIODIC = 0, /* standard periodic PIC */
    PIC_BOX_SHEAR = 1,    /* KSB-OA shearing box, Sec. 2 */
    PIC_BOX_EXPAND = 2,   /* KEB expanding box, Sec. 3 */
    PIC_BOX_LEAKY = 3,    /* leaky box, Sec. 4 */
    PIC_BOX_SHEAR_EXPAND = 4 /* shearing box that also expands: the combination Sec. 5 names as
                             future work, in this library's formulation.  The KSB-OA system of
                             Sec. 2.1 in the expanding coordinates xi = L^{-1} x of Sec. 3.1
                             (s_shear, Omega0, fp_iters as for PIC_BOX_SHEAR; expand_rate as for
                             PIC_BOX_EXPAND).  Positions are xi, momenta the comoving u', fields
                             E' and B on the xi grid.  The push solves the discrete momentum
                             equations of Secs. 2.2 and 3.2 together; the position update adds
                             the shear motion v_{s,y}/l_2; the x faces are shear-periodic with
                             Dxi_s(t) = s Omega0 nx int_0^t l_1/l_2 dt'; the fields are advanced
                             by the implicit midpoint sweeps of Sec. 2.2 on X^ = ell L^{-1} X,
                             each shear term multiplied by ell L^{-1}. */
} pic_box;

enum { PIC_PLANE_XY = 0, PIC_PLANE_XZ = 1 };
enum { PIC_FP32 = 0, PIC_FP64 = 1 };
enum { PIC_KEB_CLOSED_FORM = 0, PIC_KEB_EXACT = 1 };
enum { PIC_ESC_NONE = 0, PIC_ESC_DISPLACEMENT = 1, PIC_ESC_PROBABILISTIC = 2 };

typedef struct pic_config {
    int32_t box;          /* pic_box */
    int32_t ndim;         /* 2 or 3 */
    int32_t plane;        /* 2D only: PIC_PLANE_XY (z ignorable) or PIC_PLANE_XZ (y ignorable) */
    int32_t nx, ny, nz;   /* cells per axis; the 2D ignorable axis must be 1 */
    int32_t shape_order;  /* 1 (linear) or 2 (quadratic) particle shapes */
    int32_t precision;    /* PIC_FP32 (int32 cell + float offset, float u) or PIC_FP64 */
    int32_t fp_iters;     /* shearing box: fixed-point sweeps of the implicit Maxwell
                             solve (Sec. 2.2); counts of 3, 4, 7, 8, ... are stable */
    int32_t keb_push;     /* expanding box: PIC_KEB_CLOSED_FORM (the operator of Sec. 3.2)
                             or PIC_KEB_EXACT (direct 3x3 solve of its defining equation) */
    int32_t escape_mode;  /* PIC_ESC_*: the leaky box's escape and reinjection (Sec. 4.1).
                             PIC_ESC_PROBABILISTIC also runs in the shearing, expanding
                             and combined boxes (the reinjected momentum replaces the
                             momentum that box evolves; positions are kept);
                             PIC_ESC_DISPLACEMENT there is PIC_ERR_ARG */
    int32_t escape_dims;  /* leaky displacement test over (x,y) [2] or (x,y,z) [3] */
    int32_t tile[3];      /* particle tile in cells per axis; 0 = automatic.  3D: 4x4x4 or
                             8x8x8.  2D: 8x8, 16x16 or, FP32 only, 32x32 on the active
                             plane (the ignorable axis' entry is not read); other shapes
                             are PIC_ERR_ARG.  Automatic: in 3D 4x4x4 when 8x8x8 tiles
                             would be fewer than two per SM, else 8x8x8; in 2D 8x8 when
                             16x16 tiles would be fewer than two per SM, 32x32 (FP32) when
                             those are still eight per SM, else 16x16.  See
                             pic_autotune_tile. */
    int32_t device;       /* CUDA device ordinal the handle lives on */
    uint32_t seed;        /* key word of the Philox streams (escape, reinjection, loading) */
    uint32_t kernel_variant; /* particle-kernel launch shape: 0 = automatic (the tuned choice
                             for the precision and geometry); k >= 1 forces variant k (see
                             pic_kernel_variant_info); a variant that does not fit is PIC_ERR_ARG */
    double c;             /* Courant number; 0 < c, and c * sqrt(ndim) < 1 */
    double s_shear;       /* shearing box: s in v_s = -s Omega0 x e_y (3/2 Keplerian) */
    double Omega0;        /* shearing box: rotation frequency per step */
    double expand_rate[3];/* expanding box: l_i(t) = exp(expand_rate[i] * t) */
    double l_esc;         /* leaky box, displacement mode: escape distance in cells */
    double p_esc;         /* leaky box, probabilistic mode: escape probability per step */
    double theta_inj;     /* leaky box: temperature k T / m c^2 of the reinjection law */
    double capacity_slack;/* spare particle slots per tile as a fraction; 0 = 0.3 */
} pic_config;

typedef struct pic_diag {
    int64_t step;             /* n: state is at t = n */
    double t;
    double shear_shift;       /* Dy_s(t) mod ny (shearing box), cells */
    double l[3];              /* l_i(t) (expanding box) */
    double field_energy_E[3]; /* sum over cells of E_c^2 / (8 pi), cell volume 1 */
    double field_energy_B[3];
    double kinetic_energy[PIC_MAX_SPECIES]; /* sum of m c^2 (gamma - 1) */
    int64_t count[PIC_MAX_SPECIES];
    int64_t escaped_total;    /* leaky box: reinjections since load */
    int64_t superluminal_total; /* shearing box: |u'/gamma' + v_s| >= c occurrences */
    int64_t loose;            /* particles currently outside the tile layout (slow path) */
    int32_t error_word;       /* device error bits (0 = none) */
    int32_t reserved;
} pic_diag;

typedef struct pic_profile {
    double ms_particle;       /* accumulated device time of the fused particle kernels */
    double ms_field;          /* field solve, guard fill, current fold */
    double ms_other;          /* loose-particle path, bookkeeping */
    int64_t launches;         /* kernels launched by the library since the last reset */
    int64_t particle_launches;
    int64_t particle_steps;   /* sum over steps of the particle count */
} pic_profile;

typedef struct pic_handle pic_handle;

/* Library version string and ABI version. */
const char *pic_version(void);
int pic_abi_version(void);

/* Validate *cfg, select the current CUDA device, allocate the grid state and
 * return a new handle in *out (NULL on failure).  Fields start at zero.
 * The configuration carries each box's parameters as the paper states them:
 * shearing box (Sec. 2.1): s and Omega0 of the shear flow v_s = -s Omega0 x e_y,
 * the shearing-periodic x boundary with Dy_s = s Omega0 (x_o - x_i) t, and the
 * number of fixed-point sweeps of the implicit Maxwell solve (Sec. 2.2);
 * expanding box (Sec. 3.1): the diagonal L = diag(l_i(t)) through
 * l_i(t) = exp(rate_i t); leaky box (Sec. 4.1): the escape distance l_esc, the
 * displacement components tested (x,y or x,y,z) and the temperature of the
 * reinjection law.  Errors: PIC_ERR_ARG (text in pic_last_error(NULL)) for a
 * configuration outside these ranges; PIC_ERR_OOM; PIC_ERR_CUDA. */
pic_status pic_init(const pic_config *cfg, pic_handle **out);

/* Release everything the handle owns; h may be NULL. */
pic_status pic_destroy(pic_handle *h);

/* Text of the last error on h (or of the last failed pic_init when h is NULL). */
const char *pic_last_error(pic_handle *h);

/* Order all of h's work on `stream` (a cudaStream_t; NULL = the handle's own stream). */
pic_status pic_set_stream(pic_handle *h, void *stream);

/* Wait for all of h's queued work. */
pic_status pic_synchronize(pic_handle *h);

/* Load (replacing) species `species` (< PIC_MAX_SPECIES) with n particles of
 * macro-charge q and macro-mass m from arrays x[n][3] (cells) and u[n][3]
 * (cells/step), in host (pageable or pinned) or device memory.  The state
 * loaded is each box's evolving particle state: positions x and comoving
 * momenta u' = u - gamma' v_s for the shearing box (Sec. 2.1); comoving
 * positions x' and lab-frame momenta u for the expanding box (Sec. 3.1); for
 * the leaky box the displacement Delta r starts at zero (Sec. 4.1).  Momenta
 * are u^{n-1/2} of the leapfrog, positions x^n.  The caller keeps ownership
 * of the arrays; errors: PIC_ERR_ARG (bad species, n < 0, NULL x or u),
 * PIC_ERR_OOM, PIC_ERR_CUDA.  id (nullable)
 * gives particle ids (default 0..n-1); ids key the leaky box's random streams.
 * Positions are wrapped into the box.  The arrays are read twice (a tile
 * count of the positions, then the scatter), in chunks of at most 2^23
 * particles through device staging buffers.  Synchronizes the handle's
 * stream.  The particle-step order within a tile is not preserved. */
pic_status pic_load_particles(pic_handle *h, int species, double q, double m, int64_t n,
                              const double *x, const double *u, const uint32_t *id);

/* Device-side loader: ppc particles per cell, positions uniform in each cell,
 * momenta isotropic Maxwell-Juettner at temperature theta (k T / m c^2), plus
 * drift[3] (cells/step) and independent Gaussian noise of deviation
 * noise_sigma (cells/step) per component.  ids are assigned 0.. in cell order
 * offset by id_base.  Random numbers come from Philox4x32-10 keyed on
 * (id, seed). */
/* The load is queued on the handle's stream (the call does not wait for it). */
pic_status pic_load_maxwellian(pic_handle *h, int species, double q, double m, int ppc,
                               double theta, const double drift[3], double noise_sigma,
                               uint32_t seed, uint32_t id_base);

/* Set E and B from host arrays [3][nz][ny][nx] (copied; the caller keeps
 * them).  The shearing box evolves the comoving E' = E + (v_s / c) x B and B
 * (Sec. 2.1), so E here is E'.  The expanding box passes the lab-frame E and
 * B sampled on the comoving x' grid (Sec. 3.1; the solver transforms them to
 * E' = ell L^{-1} E, B' = ell L^{-1} B itself, Sec. 3.2).  Guard cells are
 * filled for the handle's time (shearing-periodic with Dy_s(t)).  Errors:
 * PIC_ERR_ARG (NULL array), PIC_ERR_CUDA. */
pic_status pic_set_fields(pic_handle *h, const double *E, const double *B);

/* Set uniform E and B (3 components each). */
pic_status pic_set_uniform_fields(pic_handle *h, const double E[3], const double B[3]);

/* Set the step counter n (time t = n): the time of the state already loaded.
 * Used to restart a run; the shearing shift Dy_s(t) and the expansion factors
 * l_i(t) follow from it.  Guard cells are refilled for the new time. */
pic_status pic_set_step(pic_handle *h, int64_t step);

/* Advance nsteps steps (asynchronous on the handle's stream).  One step is
 * the box's step list: the standard PIC step (gather at x^n, Boris push,
 * position update, charge-conserving current, leapfrog Maxwell update) for the
 * periodic box; the five steps of Sec. 2.2 for the shearing box (Boris-like
 * push with the shear, Coriolis and tidal terms; partial move x^n -> x';
 * current J' from x' - x^n advected along y by v_{s,y} dt / 2; full move
 * adding the shear motion; implicit Maxwell solve by fixed-point sweeps); the
 * four steps of Sec. 3.2 for the expanding box (modified Boris push with
 * Lambda; comoving move with L^{-1}(t^{n+1/2}); current ell J'; leapfrog on the
 * transformed fields); and the escape algorithm of Sec. 4.1 after the
 * standard step for the leaky box.  Errors found on the device (a bounded
 * wait that expired, a non-finite momentum, a fixed-point current beyond its
 * range) are reported by the next call that synchronises: PIC_ERR_TIMEOUT,
 * PIC_ERR_NUMERIC, PIC_ERR_STATE (particles lost to a full loose list).
 * PIC_ERR_STATE also for a handle with no particles loaded or in a batch. */
pic_status pic_step(pic_handle *h, int nsteps);

/* Synchronize and fill *out with FP64 sums over the current state: the
 * energies whose time histories the paper's examples follow (Secs. 2.3, 3.3,
 * 4.2): field energy per component, sum E_c^2 / (8 pi) and B_c^2 / (8 pi)
 * over the cells (E' for the shearing box), and per species the kinetic
 * energy sum m c^2 (gamma - 1); plus Dy_s(t) (Sec. 2.1), l_i(t) (Sec. 3.1), the
 * leaky box's reinjection count (Sec. 4.1) and the shearing box's count of
 * superluminal effective velocities |u'/gamma' + v_s| >= c (Sec. 2.1).  The
 * sums are taken in FP64 whatever the particle precision.  Errors: the
 * device error word as for pic_step; PIC_ERR_ARG for out == NULL. */
pic_status pic_diagnostics(pic_handle *h, pic_diag *out);

/* Clear the handle's device error word.  A device-side error (see pic_step)
 * stays recorded, and every later pic_step or pic_diagnostics reports it,
 * until this call; clear it once the state that caused it has been replaced
 * (pic_load_particles, pic_set_fields, pic_set_step).  Synchronizes the
 * handle's stream.  Errors: PIC_ERR_ARG (NULL handle), PIC_ERR_CUDA. */
pic_status pic_clear_error(pic_handle *h);

/* Number of particles of a species. */
pic_status pic_get_count(pic_handle *h, int species, int64_t *n);

/* Copy a species to arrays sized by pic_get_count: x[n][3], u[n][3], id[n]
 * and dr[n][3] (leaky displacement); each pointer may be NULL.  The arrays may
 * be pageable or pinned host memory or device memory (pinned host memory
 * transfers fastest).  The particles pass through device staging buffers of at
 * most 2^23 particles, so no device memory in proportion to n is needed.
 * Synchronizes the handle's stream.  The order is the device's tile order;
 * match particles by id. */
pic_status pic_get_particles(pic_handle *h, int species, double *x, double *u, uint32_t *id,
                             double *dr);

/* Copy the particles of a species whose id is remainder (mod modulus) --
 * the same subset at every step, for following particles through a large
 * run -- to host arrays with room for max_out entries (x[max_out][3], u, id,
 * dr; each may be NULL), in any order.  *n_out is the number in the subset
 * (entries beyond max_out are not copied). */
pic_status pic_get_particles_sampled(pic_handle *h, int species, uint32_t modulus, uint32_t remainder,
                                     int64_t max_out, double *x, double *u, uint32_t *id, double *dr,
                                     int64_t *n_out);

/* Copy E (E'), B and the current J of the last step (after folding, and for
 * the shearing box after the y advection) to host arrays [3][nz][ny][nx];
 * each pointer may be NULL.  J is the source term of the box's Maxwell
 * update: J' advected to the lab-frame grid for the shearing box (Sec. 2.2),
 * ell J' for the expanding box (Sec. 3.1), J otherwise; ghost currents are
 * folded back with the shearing-periodic identification of Sec. 2.1.
 * Synchronizes the handle's stream.  Errors: PIC_ERR_CUDA. */
pic_status pic_get_fields(pic_handle *h, double *E, double *B, double *J);

/* Per-kernel device timing (CUDA events on the handle's stream). */
pic_status pic_set_profiling(pic_handle *h, int enable);
pic_status pic_get_profile(pic_handle *h, pic_profile *out);
pic_status pic_reset_profile(pic_handle *h);

/* Tile capacity.  Each tile holds a fixed number of particle slots (set at
 * load from the fullest tile and cfg.capacity_slack); particles crowding into
 * a tile beyond it take a loose list, and beyond the loose list's room are
 * lost (PIC_ERR_STATE).  Every step keeps each species' fullest-tile
 * occupancy on the device; pic_step checks it every 8 steps it runs (an
 * asynchronous snapshot of the maxima since the last one, acted on one check
 * later) and, when a species' fullest tile passes 90% of its slots or its
 * loose list a quarter of its room, lays every species out again with more
 * slots (the fullest tile x max(1 + slack, 1.25) + 32) and a larger loose
 * list.  Particle states and results do not change.  pic_rebalance runs the
 * check now and synchronizes the handle's stream (force != 0: re-layout
 * regardless; *grown, nullable, says whether it did); PIC_ERR_OOM if the new
 * layout does not fit (the old one is kept), PIC_ERR_STATE on a batched box.
 * pic_get_capacity reports a species' slots per tile, loose-list room and
 * the re-layouts so far (each output nullable; PIC_ERR_ARG for a bad
 * species).  Not a part of the paper's method: the bookkeeping of the
 * tile-sorted particle layout. */
pic_status pic_rebalance(pic_handle *h, int32_t force, int32_t *grown);
/* Capacity checks every `every` steps (default 8; 0: none; every < 0 is
 * PIC_ERR_ARG).  block != 0 (default): a check waits for the snapshot taken
 * one check earlier, which also keeps the host at most about two checks ahead
 * of the GPU; block = 0: a check whose snapshot has not landed is skipped
 * (for callers that bound their own lead, like the server). */
pic_status pic_set_capacity_check(pic_handle *h, int32_t every, int32_t block);
pic_status pic_get_capacity(pic_handle *h, int species, int64_t *slots_per_tile, int64_t *loose_capacity,
                            int64_t *relayouts);

/* Regrouping by cell.  Every `every` steps (0: never) pic_step first rewrites
 * each tile's particles into the other particle buffer ordered by cell (a
 * counting sort per tile: one read and one write of the particle arrays).
 * Warps of the particle kernel then hold particles of one or two cells, which
 * makes their field reads and current adds conflict less in shared memory;
 * the order decays as particles change cells.  Default: 3 for 3D FP32 boxes,
 * 0 otherwise (FP64 boxes should keep 0: the order of their current's
 * floating-point adds, and so its last bits, would vary from run to run).
 * FP32 results are bit-identical for every interval.  A tile whose slots
 * exceed the sort's shared memory (65536 or more) is copied in order instead.
 * pic_set_regroup_interval synchronizes the handle's stream and drops its
 * captured step graphs; every < 0 is PIC_ERR_ARG.  Not a part of the paper's
 * method. */
pic_status pic_set_regroup_interval(pic_handle *h, int32_t every);
pic_status pic_get_regroup_interval(pic_handle *h, int32_t *every);

/* Load the library's particle kernels for one precision on `device` now
 * rather than at their first use (CUDA loads code lazily: the first box of
 * each geometry otherwise pays some tens of milliseconds).  It also loads
 * the allocation-free field-energy reduction (both precisions) and its
 * scratch array on `device` (see pic_field_energy_noalloc).  The server calls
 * it for FP32 when it starts. */
pic_status pic_preload_kernels(int32_t device, int32_t precision);

/* Particle-kernel variants: launch shapes of the fused particle kernel (no
 * counterpart in the paper, which gives no kernel design), numbered
 * 1..pic_kernel_variant_count().  Variant k runs *threads_per_cta threads per
 * CTA, one CTA per tile.  *stable = 1: each tile's stayers are written in
 * their input order (one barrier per chunk; particles stay grouped by cell as
 * the device loader stores them); 0: warps write in any order.  *copies: 1, 2
 * or 4 copies of the tile's shared current box, 32/copies banks apart, each
 * particle's adds dealt onto a copy so that a warp's adds spread over the
 * banks (FP64: lanes alternate between copies).
 * All variants compute the same result; particle states and FP32 currents are
 * bit-identical.  Outputs may be NULL; k out of range is PIC_ERR_ARG. */
int pic_kernel_variant_count(void);
pic_status pic_kernel_variant_info(int32_t k, int32_t *threads_per_cta, int32_t *stable, int32_t *copies);
/* The variant handle h runs (1-based) / switch it to variant k (takes effect at
 * the next pic_step; PIC_ERR_ARG if its shared memory does not fit the
 * configuration).  Switching drops the handle's captured step graphs. */
pic_status pic_get_kernel_variant(pic_handle *h, int32_t *k);
pic_status pic_set_kernel_variant(pic_handle *h, int32_t k);

/* Autotuner: run each variant that fits for trial_steps ordinary steps of
 * this box (two interleaved rounds, the first step after each switch
 * untimed), time its particle kernel with CUDA events, and keep the fastest.
 * The trial steps advance the simulation like pic_step (all variants give
 * the same result), so tuning costs no extra work beyond those steps.
 * Outputs (nullable): *best (1-based), ms_per_variant[pic_kernel_variant_count()]
 * (mean particle-kernel ms per step; -1 where the variant does not fit) and
 * *steps_taken.  Synchronizes the handle's stream; captured step graphs are
 * dropped. */
pic_status pic_autotune(pic_handle *h, int32_t trial_steps, int32_t *best, double *ms_per_variant,
                        int64_t *steps_taken);

/* Particle tiles (no counterpart in the paper).  pic_get_tile: the tile in
 * cells per axis (1 on the ignorable axis).  pic_set_tile (2D: side 8, 16, or
 * 32 in FP32; 3D: 4 or 8): re-lay the particles out in tiles of that side.  Every
 * species is read out into flat device arrays (cell + offset in FP64, which
 * holds FP32 state exactly), its arrays are freed and it is loaded again
 * under the new tiling, so the particles and every later result are
 * unchanged (FP32: bit-identical); the order within tiles is not kept.
 * Needs device memory for the flat copy (about 52 bytes per particle of the
 * largest species); PIC_ERR_OOM leaves the tiling as it was, PIC_ERR_STATE
 * for a batched box.  Synchronizes the handle's stream; drops its captured
 * step graphs.
 * pic_autotune_tile: for each tile shape (2D: 8x8, 16x16 and, FP32, 32x32;
 * 3D: 4x4x4 and 8x8x8) in turn, switch to it, run pic_autotune(trial_steps)
 * for its best launch variant, then one untimed and trial_steps timed
 * ordinary steps (all kernels, CUDA events); keep the tiles and variant with
 * the least time per step.  The trial steps advance the simulation like
 * pic_step.  Outputs (nullable): *best_side and ms_per_side[3] (2D: sides 8,
 * 16, 32; 3D: 4, 8; -1 for a side not tried). */
pic_status pic_get_tile(pic_handle *h, int32_t tile[3]);
pic_status pic_set_tile(pic_handle *h, int32_t side);
pic_status pic_autotune_tile(pic_handle *h, int32_t trial_steps, int32_t *best_side, double *ms_per_side);

/* Regroup-interval autotuner (FP32 boxes; FP64 boxes keep 0): for each of
 * the n candidate intervals (0 = never), run one untimed cycle and then
 * `cycles` whole cycles of ordinary steps (interval x cycles steps; pairs of
 * steps for 0), time every kernel of those steps with CUDA events, and keep
 * the interval with the least device time per step.  The particles' order
 * decays at a rate set by their speeds, so the best interval depends on the
 * box.  The trial steps advance the simulation like pic_step (FP32 results do
 * not depend on the interval).  Outputs (nullable): *best and
 * ms_per_step[n].  Synchronizes the handle's stream; drops its captured step
 * graphs.  PIC_ERR_ARG for an FP64 box, n < 1, cycles < 1 or a negative
 * candidate.  No counterpart in the paper. */
pic_status pic_autotune_regroup(pic_handle *h, const int32_t *candidates, int32_t n, int32_t cycles, int32_t *best,
                                double *ms_per_step);

/* ---- batches: many boxes of one kind stepped together --------------------------
 * (no counterpart in the paper; the ensembles of independent boxes the method
 * is run on).  A batch steps n boxes together: each step launches one
 * persistent particle kernel over the tiles of all boxes (at most
 * pic_batch_max_boxes_per_launch boxes per launch; more make several
 * launches), while each box's own field update, current fold and bookkeeping
 * run as parallel branches; each cycle of steps (a regroup by cell and the
 * steps up to the next, or a pair of steps) is captured in one CUDA graph and
 * replayed.  The boxes must share device, precision, geometry (3D, 2D x-y, 2D
 * x-z), shape order and box type; they may differ in grid, parameters, species
 * and particle counts.  Members run on the plain tiles of their geometry
 * (8x8x8, 16x16): members on other tile shapes are first re-laid out
 * (pic_set_tile).  They must be loaded before pic_batch_create and stay
 * owned by the caller; until pic_batch_destroy they are stepped only through
 * the batch (pic_step on a member is PIC_ERR_STATE), may be read back after
 * pic_batch_synchronize, and must not be destroyed.  The particle kernel of a
 * batch uses the default launch variant of its kind.  Results are those of
 * stepping each box alone (FP32: bit-identical). */
typedef struct pic_batch pic_batch;
pic_status pic_batch_create(pic_handle *const *boxes, int32_t n, pic_batch **out);
pic_status pic_batch_step(pic_batch *b, int32_t nsteps);   /* asynchronous */
pic_status pic_batch_synchronize(pic_batch *b);
pic_status pic_batch_destroy(pic_batch *b);                 /* synchronizes; members are free again */
/* Regroup every member by cell every `every` steps (see
 * pic_set_regroup_interval; the default is that of the members' kind).
 * Batches make no tile-capacity checks: to re-lay out crowded members, call
 * pic_rebalance on them after pic_batch_destroy. */
pic_status pic_batch_set_regroup_interval(pic_batch *b, int32_t every);
int32_t pic_batch_max_boxes_per_launch(int32_t precision);

/* ---- serving: continuous batching of independent runs ------------------------
 * A run is one box advanced for nsteps from a device Maxwellian load and
 * uniform initial fields.  The server admits queued runs in arrival order as
 * soon as their estimated device footprint fits the HBM budget and an active
 * slot is free; every active run has its own stream, so their kernels overlap
 * on the GPU; finished runs free their memory for the next ones.  Results are
 * the same alone and in a mix: each run's state is private and the FP32 path
 * is bitwise reproducible.  (Service layer of the library; the paper has no
 * counterpart -- its runs are single boxes.) */
typedef struct pic_run_spec {
    pic_config cfg;       /* box configuration (cfg.device is overridden by the server's) */
    int32_t nspecies;     /* species loaded with pic_load_maxwellian, 1..PIC_MAX_SPECIES */
    int32_t ppc;          /* particles per cell per species */
    double theta;         /* temperature of the load, k T / m c^2 */
    double q[PIC_MAX_SPECIES], m[PIC_MAX_SPECIES];
    double drift[3];
    double noise_sigma;
    double E0[3], B0[3];  /* uniform initial fields */
    uint32_t load_seed;
    uint32_t keep_state;  /* 1: keep the finished run's box for pic_take_result */
    int64_t nsteps;
} pic_run_spec;

typedef struct pic_server_info {
    int32_t queued, active;
    int64_t completed;
    uint64_t bytes_in_use, peak_bytes;
    int32_t peak_active;
    int32_t cohorts_formed;  /* batches formed from active runs so far (pic_server_set_batching) */
} pic_server_info;

typedef struct pic_server pic_server;

/* Estimated device bytes a run holds while active (host arithmetic only). */
pic_status pic_run_footprint(const pic_run_spec *spec, uint64_t *bytes);

/* How many runs at the front of a queue (device footprints queued_bytes[0..n))
 * to admit now, given the budget, the bytes and slots in use: the longest
 * prefix that fits (a run is always admitted when nothing else is active).
 * Host arithmetic only; the server's admission rule. */
int pic_admission_count(uint64_t budget, uint64_t in_use, int active, int max_active,
                        const uint64_t *queued_bytes, int nqueued);

/* Start a server on `device` with an HBM budget, at most max_active runs at
 * once, advancing each active run steps_per_round steps per round. */
pic_status pic_server_create(int device, uint64_t hbm_budget_bytes, int max_active,
                             int steps_per_round, pic_server **out);

/* Batching of served runs: min_batch = 0 (the default) steps every active
 * run on its own stream; min_batch >= 2 groups runs of one kind (precision,
 * geometry and tile shape, shape order, box type and escape rule) that were
 * admitted in the same round and have at least 4 x steps_per_round steps
 * left, at least min_batch of them, into a cohort stepped as one pic_batch
 * (no graph capture: a cohort may not live long enough to repay one).  A
 * cohort advances by chunks of at most steps_per_round steps and no more than
 * its shortest remaining run; when a member is done the cohort is dissolved
 * after its queued chunks complete, the finished runs retire and the others
 * step alone.  Results are those of each run stepped alone (FP32:
 * bit-identical).  PIC_ERR_ARG for min_batch < 0 or 1.  Takes effect from
 * the worker's next round. */
pic_status pic_server_set_batching(pic_server *s, int min_batch);

/* Queue a run (the spec is copied); *ticket identifies it. */
pic_status pic_submit(pic_server *s, const pic_run_spec *spec, uint64_t *ticket);

/* *done = 1 once the run has finished; then *out holds its final diagnostics
 * and *latency_s the time from submission to result.  Returns the run's
 * status once done. */
pic_status pic_poll(pic_server *s, uint64_t ticket, int *done, pic_diag *out, double *latency_s);

/* Hand over the box of a finished run submitted with keep_state = 1: *out
 * becomes the caller's handle (state at step nsteps, on its own stream; free
 * it with pic_destroy), from which pic_get_particles and pic_get_fields read
 * the run's final particles and fields.  Until it is taken, the box keeps
 * its device memory and counts against the server's budget; the server
 * destroys boxes never taken when it is destroyed.  PIC_ERR_STATE if the run
 * has not finished, failed, was not submitted with keep_state, or was taken
 * already; PIC_ERR_ARG for an unknown ticket. */
pic_status pic_take_result(pic_server *s, uint64_t ticket, pic_handle **out);

/* Block until run `ticket` (0: every submitted run) has finished, or timeout_s
 * seconds pass (PIC_ERR_TIMEOUT). */
pic_status pic_server_wait(pic_server *s, uint64_t ticket, double timeout_s);

pic_status pic_server_stats(pic_server *s, pic_server_info *out);

/* Stop the server: runs not yet admitted are dropped (PIC_ERR_STATE), active
 * runs are finished first. */
pic_status pic_server_destroy(pic_server *s);

/* Field energy without any device allocation.  The paper has no counterpart:
 * this is a service entry point of the library.
 *
 * Some callers cannot call cudaMalloc: a host application whose device memory
 * is owned up front by its own pool allocator (a new allocation would fail or
 * fragment that pool), a latency-critical loop where an allocation call (which
 * may synchronise the device) is not allowed, or a plug-in running inside a
 * framework callback that forbids allocation.  For them this call computes
 * what pic_diagnostics reports as field energy -- out[c] = sum_i F[c][i]^2 /
 * (8 pi) for c < ncomp -- on a caller-owned device array, using a fixed
 * scratch array compiled into the library instead of allocated memory.
 *
 * d_field: device pointer, ncomp component arrays of n values each, component
 *          after component (float for PIC_FP32, double for PIC_FP64).
 * d_out:   device pointer to ncomp doubles, written by the call.
 * stream:  cudaStream_t the work is ordered on (NULL = the legacy default
 *          stream of the current device); the call returns without waiting.
 * Limits:  1 <= ncomp <= PIC_NOALLOC_MAX_COMPONENTS; otherwise PIC_ERR_ARG.
 * Scratch: a 64 KB static device array, held on a device from the moment
 *          the library's module is loaded there until the process exits.  CUDA
 *          loads modules lazily: the first call on a device (or
 *          pic_preload_kernels for that device, which does the same set-up
 *          ahead of time) maps the array and the kernels and looks up the
 *          array's device address with that device current.  Make that first
 *          call, or pic_preload_kernels, before any stream capture.  All calls
 *          on a device share the array, so calls whose work can overlap on the
 *          GPU race and return wrong sums: order them (one stream, or events).
 *          Each call overwrites every partial sum it reads, so nothing needs
 *          clearing between calls.
 * Errors:  PIC_ERR_ARG / PIC_ERR_CUDA with text in pic_last_error(NULL).
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library call. */
pic_status pic_field_energy_noalloc(const void *d_field, int precision, int64_t n, int ncomp,
                                    double *d_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif
