/*
 * apic.h -- C ABI of the GB300 (sm_103a) APIC / explicit MPM hot path.
 *
 * Method: Jiang, Schroeder & Teran, "An angular momentum conserving Affine-Particle-In-
 * Cell method" (arXiv:1603.06188).  One step is the particle-to-grid transfer of mass and
 * affine momentum (Sec. 3.2) with the elastic force (Sec. 3.3), the explicit grid update
 * (Sec. 3.3, lambda = 0) and the grid-to-particle transfer of v_p, B_p with advection of
 * x_p and F_p (Sec. 3.4, in the lambda = 0 form of Sec. 5.7).
 *
 * General rules
 *   - Every call returns an apic_status and never aborts.  apic_last_error() gives a
 *     human-readable reason for the last failure of a simulation.
 *   - The library allocates no device memory: the caller passes one device workspace of
 *     apic_workspace_size() bytes to apic_create() and keeps it alive until
 *     apic_destroy().  Host-side bookkeeping (a small struct) is malloc'ed.
 *   - All kernels are launched on the stream given to apic_create() (a cudaStream_t
 *     passed as void*; NULL = the legacy default stream).  Calls are asynchronous except
 *     those documented as synchronising.
 *   - Device-side checks (a particle whose stencil leaves the grid, a timed-out wait) are
 *     latched in an error word that synchronising calls read; they then return
 *     APIC_ERR_NUMERIC / APIC_ERR_TIMEOUT.
 *   - Positions cross the boundary as FP64 absolute coordinates.  Inside, a particle's
 *     position is an integer cell index plus an offset in [0,1) (FP32 for precision 32),
 *     so weights keep full precision on large grids.
 *   - Particles are reordered internally every step (sorted by cell key); downloads
 *     return them in upload order.
 *   - Row-major matrices: B[a*d+b] = B_ab = sum_i w_ip v~_ia (x_i - x_p)_b (Sec. 3.4),
 *     F[a*d+b] = F_ab.
 *   - Grid nodes sit at x_i = origin + i*dx, 0 <= i_a < res[a].  Dense grid arrays
 *     exchanged with the caller use node index i0 + res0*(i1 + res1*i2).
 */
#ifndef APIC_H
#define APIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct apic_sim apic_sim;

typedef enum {
    APIC_OK = 0,
    APIC_ERR_ARG = 1,          /* invalid argument or call order */
    APIC_ERR_OOM = 2,          /* workspace too small or particle capacity exceeded */
    APIC_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    APIC_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out */
    APIC_ERR_NUMERIC = 5,      /* a particle's stencil left the grid (it was clamped), or a
                                  non-finite value was uploaded */
    APIC_ERR_UNSUPPORTED = 6   /* configuration the library does not implement */
} apic_status;

enum { APIC_TRANSFER_APIC = 0, APIC_TRANSFER_PIC = 1, APIC_TRANSFER_FLIP = 2 };
enum { APIC_BOUNDARY_NONE = 0, APIC_BOUNDARY_STICKY = 1, APIC_BOUNDARY_SLIP = 2 };
enum { APIC_MODEL_NONE = 0, APIC_MODEL_FIXED_COROTATED = 1, APIC_MODEL_NEOHOOKEAN = 2 };
enum { APIC_WHERE_PARTICLES = 0, APIC_WHERE_GRID = 1 };
enum { APIC_GRID_MOMENTUM = 0, APIC_GRID_VELOCITY = 1 };

typedef struct {
    int dim;                 /* 2 or 3 */
    int order;               /* 2 = quadratic, 3 = cubic B-spline (Sec. 3.5); 1 (multilinear)
                                is rejected with APIC_ERR_UNSUPPORTED: the B_p transfer is
                                unstable for it (Sec. 5.9) */
    int precision;           /* 32 or 64: arithmetic type of particle and grid state */
    int transfer;            /* APIC_TRANSFER_APIC, APIC_TRANSFER_PIC (C_p = 0, Sec. 5.6), or
                                APIC_TRANSFER_FLIP: PIC's transfer to the grid and the FLIP
                                velocity update of Sec. 1, blended with PIC's by flip_alpha */
    int res[3];              /* grid nodes per axis (res[2] ignored in 2-D); <= 1024 in 3-D */
    double dx;               /* grid spacing */
    double origin[3];        /* position of node 0 */
    double dt;               /* time step */
    double gravity[3];       /* added to v~ of nodes with mass (not in the paper) */
    int boundary;            /* APIC_BOUNDARY_NONE, _STICKY (v~ = 0 on nodes within `wall`
                                nodes of a face) or _SLIP (only the component of v~ normal to
                                that face is zeroed; the paper's Sec. 6.2 test uses slip) */
    int wall;                /* wall thickness in nodes */
    int model;               /* APIC_MODEL_NONE (transfer only), _FIXED_COROTATED
                                (P = 2 mu (F - R) + lam (J - 1) J F^-T) or _NEOHOOKEAN
                                (P = mu (F - F^-T) + lam log(J) F^-T, the model of the
                                paper's Sec. 6 experiments) */
    double E, nu;            /* Young's modulus, Poisson's ratio */
    double particle_mass;    /* m_p, the same for every particle of a simulation */
    double particle_volume;  /* V_p (reference volume), the same for every particle */
    int tile_particles;      /* particles per P2G / G2P tile (power of two, 256..4096);
                                0 = default */
    int p2g_kernel;          /* P2G kernel: 0 = default (2); 1 = component-
                                split (3-D only: the lanes of a group per base cell each sum two
                                of the four node sums); 2 = cell-parallel (lanes of a group
                                share a cell's particles and reduce their full sums); results
                                agree to rounding */
    double flip_alpha;       /* APIC_TRANSFER_FLIP only: v_p <- a (v_p + sum w (v~_i - v_i)) +
                                (1 - a) sum w v~_i, a in [0, 1] (1 = the paper's FLIP); the
                                velocities v_i before the grid update are kept (+32 B per
                                node); not available in batches */
    int p2g_group;           /* lanes that share one base cell in the cell-parallel P2G: 2 or
                                4; 0 = chosen after the first sort following each upload from
                                the particles per occupied node block (2 below 16 particles
                                per cell, else 4) -- that apic_p2g reads the tile count back
                                and so synchronises once.  Results agree to rounding. */
    int integrator;          /* member of the Sec. 3.3 family: APIC_INTEGRATOR_LAMBDA0 (0, the
                                explicit symplectic Euler step), APIC_INTEGRATOR_LAMBDA1 (1:
                                the force at F^{n+1} = (I + dt sum_i v_i grad w^T) F^n from the
                                grid velocities before the update, particles moved with them,
                                the general transfer of Sec. 3.4) or APIC_INTEGRATOR_MIDPOINT
                                (2: the implicit midpoint rule lambda = 1/2, solved on the grid
                                by Newton iterations with mass-inner-product conjugate gradients,
                                Sec. 4.1-4.2 and Algorithm 1; neither gravity nor walls, which
                                the paper's solve does not have).  lambda = 1 and the midpoint
                                rule are for single APIC / PIC simulations (not FLIP, batches or
                                adaptive steps) */
    int newton_max;          /* midpoint rule: Newton iterations per step at most (0 = 20) */
    int cg_max;              /* midpoint rule: CG iterations per Newton system at most (0 = 200) */
    double solve_tol;        /* midpoint rule: a Newton loop ends when |dt M^-1 f - dv|_M <=
                                solve_tol |v|_M, a CG solve when its residual has dropped by
                                solve_tol (0 = 1e-6 in FP32, 1e-12 in FP64) */
} apic_config;

enum { APIC_INTEGRATOR_LAMBDA0 = 0, APIC_INTEGRATOR_LAMBDA1 = 1, APIC_INTEGRATOR_MIDPOINT = 2 };

/* Bytes of device workspace a simulation with this config and capacity needs.
 * Errors: APIC_ERR_ARG (NULL pointer, bad config), APIC_ERR_UNSUPPORTED. */
apic_status apic_workspace_size(const apic_config* cfg, int64_t max_particles, size_t* bytes);

/* Create a simulation.  `workspace` is a device pointer (256-byte aligned) to at least
 * apic_workspace_size() bytes, owned by the caller, used exclusively by this simulation
 * until apic_destroy().  `stream` is a cudaStream_t (or NULL).  Zeroes the grid on the
 * stream.  Errors: APIC_ERR_ARG, APIC_ERR_UNSUPPORTED, APIC_ERR_OOM (workspace too small). */
apic_status apic_create(const apic_config* cfg, int64_t max_particles, void* workspace,
                        size_t workspace_bytes, void* stream, apic_sim** out);

/* Release the host-side state.  Synchronises the stream.  The workspace is the caller's. */
apic_status apic_destroy(apic_sim* sim);

/* Load n particles (n <= max_particles) from FP64 arrays: x (n*d), v (n*d), B (n*d*d),
 * F (n*d*d).  v, B may be NULL (zero); F may be NULL (identity).  `on_device` = 1 if the
 * pointers are device memory, 0 for host memory.  The data are copied; the library keeps
 * no pointer.  Synchronising when on_device = 0.
 * Every value is checked on the device.  A NaN or Inf anywhere in x, v, B or F gives
 * APIC_ERR_NUMERIC: for host input from this call, which then discards the upload (the
 * simulation holds no particles); for device input from the next synchronising call.  A
 * position outside the grid is clamped into it and also gives APIC_ERR_NUMERIC; the
 * particles are kept.
 * Errors: APIC_ERR_ARG, APIC_ERR_OOM (n > capacity), APIC_ERR_NUMERIC, APIC_ERR_CUDA. */
apic_status apic_upload(apic_sim* sim, int64_t n, const double* x, const double* v,
                        const double* B, const double* F, int on_device);

/* A material per particle: Young's modulus E[i] > 0 and Poisson's ratio nu[i] in (-1, 0.5)
 * for the particle uploaded at index i (n = the count of the last apic_upload), turned into
 * Lame parameters mu = E / (2 (1 + nu)), lam = E nu / ((1 + nu)(1 - 2 nu)) that replace the
 * configuration's in the particle's stress from now on (the first "next" extension of the
 * paper's Sec. 3.3 force: the constitutive model is per particle; the paper's experiments
 * use one material per body).  The current stress is recomputed.  Valid until the next
 * apic_upload, which returns to the configuration's material.  `on_device` as in
 * apic_upload; host values are checked, device values are not.  Not allowed between
 * apic_p2g and apic_g2p, nor while the simulation is in a batch.  Synchronising when
 * on_device = 0.  Errors: APIC_ERR_ARG, APIC_ERR_CUDA. */
apic_status apic_upload_materials(apic_sim* sim, int64_t n, const double* E, const double* nu, int on_device);

/* A mass and a volume per particle: mass[i] = m_p and vol[i] = V_p of the particle uploaded at
 * index i (n = the count of the last apic_upload), each finite and > 0, in place of the
 * configuration's `mass` and `vol`.  Sec. 3.2 gives every particle its own constant mass m_p
 * (in m_i = sum_p m_p w_ip and the affine momentum sum), and Sec. 3.3 its own volume V_p (in
 * the potential sum_p V_p Psi_p and the force sum_p V_p P_p F_p^T grad w_ip); the momentum
 * diagnostics use m_p too.  The values are stored in the state's precision (FP32 in an FP32
 * simulation) and the current stress is recomputed with V_p.  This call and
 * apic_upload_materials set parts of the same per-particle parameters: what one of them
 * does not give keeps its earlier per-particle value, or the configuration's if none was
 * set.  Valid until the next apic_upload, which returns to the configuration's values.
 * `on_device` as in apic_upload; host values are checked, device values are not.  Not
 * allowed between apic_p2g and apic_g2p, nor while the simulation is in a batch (a member
 * keeps its values in the batch).  Synchronising when on_device = 0.
 * Errors: APIC_ERR_ARG, APIC_ERR_CUDA. */
apic_status apic_upload_mass_volume(apic_sim* sim, int64_t n, const double* mass, const double* vol, int on_device);

/* Copy the particle state back in upload order (any pointer may be NULL to skip that
 * field).  Synchronising.  Errors: APIC_ERR_ARG, APIC_ERR_CUDA, and a latched device error. */
apic_status apic_download(apic_sim* sim, double* x, double* v, double* B, double* F, int on_device);

/* Positions in their internal form, upload order: integer cell (n*d int32) and offset in
 * [0,1) widened exactly to FP64 (n*d).  Synchronising, host pointers. */
apic_status apic_download_positions(apic_sim* sim, int32_t* cell, double* offset);

/* Sec. 3.2 (+ Sec. 3.3 force): cell keys, stable radix sort by key, tile list, and the
 * scatter m_i = sum_p w_ip m_p, (m v)_i = sum_p w_ip m_p (v_p + B_p D_p^{-1} (x_i - x_p)),
 * with dt f_i = -dt sum_p V_p P(F_p) F_p^T grad w_ip added into the momentum when a
 * constitutive model is set.  D_p = (dx^2/4) I (quadratic) / (dx^2/3) I (cubic), the
 * constants Sec. 5.6 prints for B-splines.  Asynchronous. */
apic_status apic_p2g(apic_sim* sim);

/* Sec. 3.3, lambda = 0: v~_i = ((m v)_i + dt f_i) / m_i + dt g, sticky walls, v~ = 0 where
 * m_i = 0.  Clears the accumulation grid for the next step.  Asynchronous.
 * lambda = 1 (APIC_INTEGRATOR_LAMBDA1; apic_p2g then transfers mass and momentum only):
 * v_i = (m v)_i / m_i, the force f_i = -sum_p V_p P(F_p^{n+1}) (F_p^n)^T grad w_ip at
 * F_p^{n+1} = (I + dt sum_i v_i grad w_ip^T) F_p^n, then v~_i = v_i + dt f_i / m_i + dt g and
 * the walls; v_i is kept for apic_g2p. */
apic_status apic_grid_update(apic_sim* sim);

/* Sec. 3.4 with Sec. 5.7 (lambda = 0): v_p = sum_i w_ip v~_i, B_p = sum_i w_ip v~_i
 * (x_i - x_p)^T (zero for PIC), F_p <- (I + dt sum_i v~_i grad w_ip^T) F_p,
 * x_p <- x_p + dt v_p.  Writes the particles in sorted order and their next cell keys.
 * lambda = 1: the general form of Sec. 3.4 with x~_i = x_i + dt v_i: v_p = sum_i w v~_i,
 * x_p <- sum_i w x~_i, F_p <- (I + dt sum_i v_i grad w^T) F_p, and the symmetrised B_p of
 * Sec. 3.4 (which adds to the lambda = 0 sum dt/2 times the antisymmetric
 * sum_i w (v~_i v_i^T - v_i v~_i^T) - (v_p vbar_p^T - vbar_p v_p^T), vbar_p = sum_i w v_i).
 * Asynchronous. */
apic_status apic_g2p(apic_sim* sim);

/* n whole steps (apic_p2g, apic_grid_update, apic_g2p).  Asynchronous. */
apic_status apic_step(apic_sim* sim, int n);

/* nsteps explicit steps whose time step follows the Sec. 4.3 bound: before each step
 * dt = min(dt_max, nu * dx / max_p(|v_p| + 6 sqrt(d)/dx |B_p|_F)) (nu = the CFL number; the
 * paper uses nu = 1 with its implicit integrator -- an explicit elastic run also needs
 * dt_max under its wave-speed limit).  The first maximum is reduced from the current state
 * in FP64; each later one is reduced by G2P from the state it writes (FP32 in the FP32
 * build), and the time step is set on the device, so the steps run without host
 * synchronisation.  The configured dt is not changed.  `elapsed` (may be NULL) receives
 * the simulated time of the steps; then the call synchronises.  Not allowed between
 * apic_p2g and apic_g2p, nor in a batch.  Errors: as apic_step, APIC_ERR_ARG for nu or
 * dt_max <= 0. */
apic_status apic_step_adaptive(apic_sim* sim, int nsteps, double nu, double dt_max, double* elapsed);

/* Total linear momentum p and angular momentum l about the world origin, accumulated in
 * FP64 (Sec. 3.1; Sec. 5.3 for the particle form l = sum x_p x m_p v_p + m_p B_p^T : eps).
 * where = APIC_WHERE_PARTICLES, or APIC_WHERE_GRID: after apic_p2g, sum (m v)_i (which
 * includes dt f_i) and sum x_i x (m v)_i; after apic_grid_update, sum m_i v~_i and
 * sum x_i x m_i v~_i.  In 2-D, l[0] is the z component.  Synchronising, host pointers. */
apic_status apic_momentum(apic_sim* sim, int where, double p[3], double l[3]);

/* The particle momentum of apic_momentum (APIC_WHERE_PARTICLES) of the state as it stands
 * after the work queued so far, read without synchronising: the reduction runs on a stream
 * of its own (with its own scratch) once that work is done, overlapping whatever is queued
 * next, and writes out[0..2] = p, out[3..5] = l (in 2-D out[3] is the z component and
 * out[2] = out[4] = out[5] = 0).  `out` (6 doubles, host or device memory, caller-owned)
 * must stay valid until apic_momentum_wait returns; with pinned host or device memory the
 * call returns at once, with pageable host memory only when the read is done.  A later
 * call that overwrites the state copy that was read (apic_g2p two steps on, an upload, new
 * materials or masses) waits for the read on the device first, so the value is that of the
 * state at the time of the call.  Not for members of a batch (APIC_ERR_ARG). */
apic_status apic_momentum_async(apic_sim* sim, double* out);

/* Waits until every apic_momentum_async read of this simulation has written its output. */
apic_status apic_momentum_wait(apic_sim* sim);

/* Sec. 4.3 time-step bound: *max_speed = max_p (|v_p| + (6 sqrt(d) / dx) |B_p|_F), the
 * (kappa / k) dx factor being the same for quadratic and cubic B-splines; a step with
 * dt <= nu dx / *max_speed moves no particle more than nu dx at the grid velocity.
 * Synchronising, host pointer. */
apic_status apic_cfl(apic_sim* sim, double* max_speed);

/* Dense copy of the grid (host pointers, res-box node order): which =
 * APIC_GRID_MOMENTUM after apic_p2g: m (nodes) and (m v)_i + dt f_i (nodes*d);
 * APIC_GRID_VELOCITY after apic_grid_update: m and v~.  Synchronising. */
apic_status apic_grid_download(apic_sim* sim, int which, double* m, double* mv);

/* The last sort (host pointers, n entries each): sorted keys, and perm[k] = internal
 * index, at sort time, of the k-th sorted particle (right after apic_upload the internal
 * order is the upload order).  Synchronising. */
apic_status apic_keys_download(apic_sim* sim, uint32_t* keys, uint32_t* perm);

/* Active node blocks (4^d nodes each) of the grid after apic_p2g: out[b] = 1 if block b
 * (linear index, axis 0 fastest, ceil(res/4) blocks per axis) takes part in the grid
 * update, else 0.  n_blocks must equal the block count.  Synchronising, host pointer. */
apic_status apic_grid_occupancy(apic_sim* sim, uint8_t* out, int64_t n_blocks);

/* Counters: [0] particles, [1] blocks of the grid, [2] tiles of the last sort,
 * [3] FP64 fallbacks of the 3x3 polar decomposition since creation, [4] kernels launched
 * by this simulation since creation.  Synchronising. */
apic_status apic_stats(apic_sim* sim, int64_t out[5]);

/* Phases of a step, for apic_profile_read. */
enum { APIC_PHASE_KEYS = 0, APIC_PHASE_SORT, APIC_PHASE_TILES, APIC_PHASE_P2G, APIC_PHASE_GRID,
       APIC_PHASE_G2P, APIC_NPHASE };

/* Start (enable = 1, clearing earlier records) or stop (0) per-phase timing: CUDA events
 * recorded on the simulation's stream around each phase's kernels.  No device work
 * changes.  Host-only bookkeeping; asynchronous. */
apic_status apic_profile(apic_sim* sim, int enable);

/* Accumulated device time (ms) and launch count per phase since apic_profile(sim, 1).
 * Synchronising, host pointers of APIC_NPHASE entries. */
apic_status apic_profile_read(apic_sim* sim, double ms[APIC_NPHASE], int64_t launches[APIC_NPHASE]);

/* ------------------------------------------------------------------------------------
 * Batched stepping (no counterpart in the paper): many independent simulations of the
 * same dimension, B-spline order and precision -- each with its own grid, size, material
 * and time step -- advanced together, one persistent kernel launch per phase over a work
 * list that spans all members.  A member keeps its own workspace; the batch adds a
 * workspace for the shared work lists.  While a simulation is a member, apic_p2g /
 * apic_grid_update / apic_g2p / apic_step / apic_upload on it return APIC_ERR_ARG;
 * apic_download, apic_download_positions and apic_momentum synchronise with the batch
 * first.
 * ------------------------------------------------------------------------------------ */
typedef struct apic_batch apic_batch;

typedef struct {
    int dim, order, precision;   /* shared by every member */
    int max_sims;                /* member capacity, 1..12000 */
    int64_t max_particles;       /* total particles over the members */
    int64_t max_blocks;          /* total node blocks (4^d nodes) over the members' grids */
    int tile_particles;          /* 1024, 2048 or 4096 particles per tile; 0 = 4096 */
    int group;                   /* P2G: lanes sharing one cell in the cell-parallel kernel, 1, 2,
                                    4 or 8, or APIC_BATCH_SPLIT for the component-split kernel
                                    (3-D); 0 = APIC_BATCH_SPLIT in 3-D, 8 in 2-D */
    int use_graph;               /* 1 = replay each step as a captured CUDA graph (needs a
                                    non-NULL stream) */
} apic_batch_config;

/* apic_batch_config.group value selecting the component-split P2G kernel (3-D) */
#define APIC_BATCH_SPLIT 16

apic_status apic_batch_workspace_size(const apic_batch_config* cfg, size_t* bytes);

/* `workspace`: caller-owned device memory (256-byte aligned), kept until apic_batch_destroy.
 * Errors: APIC_ERR_ARG, APIC_ERR_UNSUPPORTED, APIC_ERR_OOM (workspace too small). */
apic_status apic_batch_create(const apic_batch_config* cfg, void* workspace, size_t workspace_bytes,
                              void* stream, apic_batch** out);

/* Removes every member (as apic_batch_remove) and frees the host-side state. */
apic_status apic_batch_destroy(apic_batch* batch);

/* Add a simulation with n > 0 particles already uploaded.  Synchronises the simulation's
 * stream.  Errors: APIC_ERR_ARG (incompatible, empty, or already a member),
 * APIC_ERR_UNSUPPORTED (a FLIP simulation), APIC_ERR_OOM (member, particle or block
 * capacity), APIC_ERR_CUDA. */
apic_status apic_batch_add(apic_batch* batch, apic_sim* sim);

/* Take a simulation out; its state is current as of the last batched step.
 * Synchronising. */
apic_status apic_batch_remove(apic_batch* batch, apic_sim* sim);

/* n batched steps of every member (each member does exactly what apic_step(sim, 1)
 * would).  Asynchronous on the batch's stream. */
apic_status apic_batch_step(apic_batch* batch, int n);

/* Serving (continuous batching; no counterpart in the paper).  Admit a simulation that will
 * run `steps` batched steps and occupies `footprint_bytes` of device memory while resident
 * (typically its apic_workspace_size): if the footprints of the members admitted this way
 * plus this one exceed `budget_bytes`, nothing changes and APIC_ERR_OOM is returned (the
 * caller keeps it queued and retries after a completion); otherwise it joins the batch as
 * apic_batch_add would.  Synchronises the simulation's stream.
 * Errors: APIC_ERR_ARG (steps <= 0, negative sizes, as apic_batch_add), APIC_ERR_OOM (over
 * the budget, or a batch capacity), APIC_ERR_UNSUPPORTED, APIC_ERR_CUDA. */
apic_status apic_batch_admit(apic_batch* batch, apic_sim* sim, int steps, int64_t footprint_bytes,
                             int64_t budget_bytes);

/* Step every member min(max_steps, the fewest steps any admitted member has left) batched
 * steps -- so no admitted member passes its completion -- then take the admitted members
 * whose steps are done out of the batch (as apic_batch_remove: their state is current and
 * their memory counts no more against the budget) and write them to finished[0 ..
 * *n_finished - 1] in membership order.  Members added with apic_batch_add have no step
 * count and stay.  `finished` needs room for every admitted member.  *steps_done (may be
 * NULL) receives the steps taken.  Synchronises when a member finishes.
 * Errors: APIC_ERR_ARG, and those of apic_batch_step / apic_batch_remove. */
apic_status apic_batch_run(apic_batch* batch, int max_steps, apic_sim** finished, int max_finished,
                           int* n_finished, int* steps_done);

/* Device bytes of the members admitted with apic_batch_admit and still resident. */
apic_status apic_batch_resident_bytes(apic_batch* batch, int64_t* bytes);

/* Tile size and P2G lane group (as apic_batch_config.group) for the following steps (0 keeps
 * the current value). */
apic_status apic_batch_set_tuning(apic_batch* batch, int tile_particles, int group);

/* Autotuner: times `steps` batched steps for every candidate (tile 1024 / 2048 / 4096 x
 * group 1 / 2 / 4 / 8 / APIC_BATCH_SPLIT in 3-D), keeps the fastest and reports it.  The trial steps are real steps of the
 * members.  Results are cached per (dim, order, precision, particle-count bucket) for the
 * life of the process; force = 1 re-measures.  Synchronising. */
apic_status apic_batch_autotune(apic_batch* batch, int steps, int force, int* tile_particles, int* group);

/* [0] members, [1] particles, [2] batched steps done, [3] kernels launched,
 * [4] work tiles of the last step.  Synchronising. */
apic_status apic_batch_stats(apic_batch* batch, int64_t out[5]);

const char* apic_batch_last_error(apic_batch* batch);

/* Stable radix sort of 32-bit keys that allocates nothing.  The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory -- a host framework
 * that owns all device memory and gives plug-ins no allocator, or a real-time loop that
 * must not call cudaMalloc after start-up (it can synchronise the device and take
 * unbounded time).  Such a caller passes only its inputs and outputs; the sort's own
 * scratch (ping-pong keys and indices, digit histograms, scan partials) lives in a
 * fixed-size static device array inside the library, which every GPU that loads the
 * library holds until the process exits (about 9 MB).  It is a plain LSD radix sort, one
 * pass per 8-bit digit (a histogram, a device-wide exclusive scan, a stable scatter); it
 * does not use the one-sweep and incremental kernels of apic_p2g's sort, but gives the
 * same result: the stable sort of the keys.
 *   keys        device pointer, n keys (read only)
 *   key_bits    number of low key bits to sort on, 1..32 (higher bits must be zero)
 *   sorted_keys device pointer, n entries: the keys in ascending order
 *   perm        device pointer, n entries: perm[k] = input index of the k-th sorted key;
 *               equal keys keep their input order (stable)
 *   stream      cudaStream_t (or NULL); the call is asynchronous on it.
 * The three buffers must not overlap (a pass reads its input while other CTAs write its
 * output); overlapping buffers return APIC_ERR_ARG.
 * n <= APIC_SORT_NOALLOC_MAX_KEYS; larger n returns APIC_ERR_OOM before any launch.
 * The first call on each device looks up the static array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that first call
 * before any stream capture.  Every call reuses the same array, so calls whose work
 * overlaps on the GPU (other streams, other threads) race on it: serialise them.
 * Every scratch word a call reads is written earlier in the same call, so nothing left
 * by a previous call is used.  A CUDA error already pending on the calling thread when
 * the call starts is left pending, nothing is launched, and APIC_ERR_CUDA is returned.
 * Errors: APIC_ERR_ARG (NULL pointer, n < 0, key_bits out of range, overlapping buffers),
 * APIC_ERR_OOM, APIC_ERR_CUDA. */
#define APIC_SORT_NOALLOC_MAX_KEYS (1 << 20)
apic_status apic_sort_keys_noalloc(const uint32_t* keys, int64_t n, int key_bits, uint32_t* sorted_keys,
                                   uint32_t* perm, void* stream);

/* Fault-injection hook for tests of the timeout path (the paper has no counterpart): the
 * number of polls G2P's first wait for a tile's staged grid blocks makes before it gives up
 * (default 4194304, several seconds).  With 0 the wait gives up at once: the CTA latches
 * APIC_ERR_TIMEOUT, waits (bounded) for its copies in flight to land, and leaves without
 * writing its particles, so the next synchronising call returns APIC_ERR_TIMEOUT and the
 * particle state of that step is not valid; the device stays usable.  Host-only
 * bookkeeping.  Errors: APIC_ERR_ARG (NULL, or the simulation is in a batch). */
apic_status apic_set_wait_limit(apic_sim* sim, unsigned polls);

/* The last grid solve of the implicit midpoint rule: out[0] Newton iterations (systems
 * solved), out[1] conjugate-gradient iterations over them, out[2] the final Newton residual
 * |dt M^-1 f - dv|_M / |v|_M.  Zeros for the explicit members.  Host-only, no
 * synchronisation (apic_grid_update already read the scalars back).  Errors: APIC_ERR_ARG. */
apic_status apic_solve_stats(apic_sim* sim, double out[3]);

/* Reason for the last failing call on this simulation ("" if none). */
const char* apic_last_error(apic_sim* sim);

#ifdef __cplusplus
}
#endif

#endif /* APIC_H */
