/*
 * amr.h -- C ABI of the B300 block-AMR hot path.
 *
 * The library keeps a quadtree/octree forest of N^d-cell blocks on the host
 * and the block data on one GPU, and executes the per-time-step work of the
 * method of "foap4: adaptive mesh refinement with OpenACC, MPI, and p4est":
 * the ghost-cell pattern (same-level copies, fine-to-coarse restriction,
 * coarse-to-fine limited prolongation, physical boundaries; Sec. 2.6) and the
 * explicit finite-volume Runge-Kutta update of the Euler equations with flux
 * fixing at refinement boundaries (Sec. 2.7, Sec. 3.1-3.5).
 *
 * Conventions shared by every call:
 *  - Every call returns an amr_status and never aborts the process.  The
 *    message of the last failure of a forest is available from
 *    amr_last_error().  Errors found on the device (non-physical states,
 *    expired device waits) are latched in a device status word and reported
 *    by amr_sync_status().
 *  - The forest owns every host and device buffer it allocates (through the
 *    dev_alloc/dev_free hook of amr_config when given, cudaMalloc otherwise).
 *    Pointers passed in are borrowed for the duration of the call only.
 *    Streams are owned by the caller; an amr_stream is a cudaStream_t (NULL =
 *    the legacy default stream).
 *  - Block data layout is Eq. 3 of the paper, uu(i, j, k, ivar, iblock) with
 *    i fastest and ghost layers included: element (i, j, k, v, b) of state
 *    slot s sits at index
 *        (((s * max_blocks + b) * n_var + v) * S + (k + ng)) * S + j + ng) * S + i + ng
 *    with S = block_n + 2 n_ghost and i, j, k in [-ng, block_n + ng)
 *    (k absent in 2D).  Elements are float (precision 32) or double (64).
 *  - Blocks are numbered in leaf order: trees row-major (x fastest), Morton
 *    order inside a tree with x the lowest bit (Sec. 2.2: the n-th quadrant
 *    is the n-th block).
 *  - A forest is not thread safe; distinct forests are independent.
 */
#ifndef AMR_B300_H
#define AMR_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMR_OK = 0,
    AMR_EINVAL = 1,      /* invalid argument or configuration */
    AMR_ENOMEM = 2,      /* host or device allocation failed */
    AMR_ECAPACITY = 3,   /* a regrid would exceed max_blocks; mesh and data unchanged */
    AMR_ECUDA = 4,       /* a CUDA runtime call failed */
    AMR_ETIMEOUT = 5,    /* a bounded device wait expired */
    AMR_EBOUNDS = 6,     /* a checked index fell outside its buffer */
    AMR_ENONPHYS = 7,    /* density or pressure <= 0 met by a stage */
    AMR_ESTATE = 8       /* call out of order (e.g. no ghost pattern yet) */
} amr_status;

/* Physical boundary kinds per face direction (Sec. 2.4). */
typedef enum {
    AMR_BC_PERIODIC = 0,   /* through the connectivity; the dimension must be periodic */
    AMR_BC_DIRICHLET = 1,  /* uniform value bc_val[face][var] */
    AMR_BC_NEUMANN = 2,    /* uniform outward normal derivative bc_val[face][var] */
    AMR_BC_DATA = 3        /* Dirichlet values per boundary-face cell, amr_set_bc_data() */
} amr_bc;

/* Ghost-strip kinds by direction of data flow (Sec. 2.6). */
typedef enum {
    AMR_GHOST_SRL = 0,     /* same refinement level: copy */
    AMR_GHOST_F2C = 1,     /* fine -> coarse: restriction into the coarse block's ghosts */
    AMR_GHOST_BC = 2,      /* physical boundary */
    AMR_GHOST_C2F = 3,     /* coarse -> fine: limited prolongation, second round */
    AMR_GHOST_DIAG = 4,    /* edge / corner region held by a same-level leaf: copy
                              (only with amr_config.diagonal_ghosts); face =
                              (dx+1) + 3 (dy+1) + 9 (dz+1) for the direction */
    AMR_GHOST_DIAG_F2C = 5,/* edge / corner region covered by finer leaves:
                              restriction, round 1, one entry per fine leaf;
                              offset = its half along a 3D edge (else 0) */
    AMR_GHOST_DIAG_C2F = 6,/* edge / corner region inside a coarser leaf: limited
                              prolongation, round 2; offset bit d = parity of the
                              same-size box's coordinate along dimension d */
    AMR_GHOST_DIAG_BC = 7  /* edge / corner region outside a non-periodic domain
                              (no counterpart in the paper, which fills face
                              ghosts only): the boundary formula of face
                              `offset` -- the face across the region's lowest
                              dimension that leaves the domain -- applied to
                              the cell mirrored across it; src = -1, aux = that
                              face's boundary-face index; after round 2, edges
                              before corners */
} amr_ghost_kind;

typedef struct amr_forest amr_forest;
typedef void *amr_stream;  /* cudaStream_t */

typedef void *(*amr_dev_alloc_fn)(size_t bytes, void *ctx);
typedef void (*amr_dev_free_fn)(void *ptr, void *ctx);

/* Problem statement.  Sec. 2.2 (brick of trees, max refinement), Sec. 2.3
 * (N^d blocks, N even and N >= n_ghost; this library also needs
 * N >= 2 n_ghost so that a coarse ghost layer maps inside one fine block),
 * Sec. 2.3 static capacity max_blocks x n_states blocks (Sec. 3.1),
 * Sec. 2.4 boundary kinds in the face order -x, +x, -y, +y, -z, +z. */
typedef struct {
    int ndim;              /* 2 or 3 */
    int block_n;           /* N: 8, 16 or 32 */
    int n_ghost;           /* ghost layers, 1..4 (the Euler stage needs >= 2) */
    int n_var;             /* Euler: ndim + 2 (rho, rho v, E); advection: 1 */
    int ntrees[3];         /* brick of trees (unused entries 1) */
    int periodic[3];
    double lo[3], len[3];  /* domain corner and extent */
    int max_level;         /* finest level, <= 12 */
    int max_blocks;        /* capacity in blocks per state slot */
    int n_states;          /* state slots (Heun needs 2) */
    int precision;         /* 32 or 64 */
    double gamma, cfl;
    int bc[6];             /* amr_bc per face direction */
    double bc_val[6][8];   /* per face direction and variable */
    amr_dev_alloc_fn dev_alloc;   /* optional allocation hook (NULL: cudaMalloc) */
    amr_dev_free_fn dev_free;
    void *alloc_ctx;
    int host_only;         /* 1: mesh and ghost pattern only -- no device memory
                              is touched; calls on block data return AMR_ESTATE
                              and amr_flag_and_regrid needs explicit flags */
    int limiter;           /* amr_limiter: MUSCL slope limiter (Sec. 3.2) */
    int flux;              /* amr_flux: numerical flux (Sec. 3.2) */
    double gravity[3];     /* g of the source term S = (0, rho g, rho g.u) added to
                              every stage (Sec. 4.2); zero: no source */
    int diagonal_ghosts;   /* 1: the pattern also fills the edge and corner ghost
                              regions (AMR_GHOST_DIAG copies and
                              AMR_GHOST_DIAG_F2C restrictions in round 1,
                              AMR_GHOST_DIAG_C2F prolongations in round 2,
                              AMR_GHOST_DIAG_BC boundary formulas outside a
                              non-periodic domain after them); the paper and the
                              stage kernels use face ghosts only (Sec. 2.1) */
    int physics;           /* amr_physics: equations of the stage (Sec. 3.4, 3.5) */
    double velocity[3];    /* uniform velocity of the scalar advection equation
                              (Eq. 13); ignored for Euler */
} amr_config;

/* Equations the stage solves.  Euler gas dynamics (Sec. 3.5, Eq. 14-16):
 * n_var = ndim + 2.  Scalar advection (Sec. 3.4, Eq. 13) with the uniform
 * velocity amr_config.velocity: n_var = 1, primitive = conservative, wave
 * speeds min(v_d, 0) and max(v_d, 0) (so Rusanov and HLL both upwind; the
 * HLL flux is 0 where v_d = 0), CFL limit sum_d |v_d| / dx_d, no gravity;
 * the refinement criterion looks at the scalar; the learned flag predictor
 * (whose features are Euler quantities) is refused with AMR_EINVAL. */
typedef enum { AMR_PHYS_EULER = 0, AMR_PHYS_ADVECTION = 1 } amr_physics;

/* Face reconstructions of Sec. 3.2.  MUSCL slope limiters (two ghost
 * layers); the slope of a cell from its one-sided differences a, b: minmod =
 * Eq. 1 with theta = 1; MC (monotonized central) = Eq. 1 with theta = 2; van
 * Leer = 2ab / (a + b) when ab > 0, else 0; face values w -/+ slope / 2.
 * Koren: the right face w + a phi(b/a) / 2, the left face w - b phi(a/b) / 2,
 * phi(r) = max(0, min(2r, (1 + 2r) / 3, 2)).  WENO3: candidates -a/2 + 3b/2
 * and (b + c)/2, weights (1/3, 2/3) / (1e-6 + beta)^2.  Upwind: first order
 * (face values = cell values; this library still needs n_ghost >= 2).
 * WENO5 (Jiang & Shu, weights (1/10, 6/10, 3/10) / (1e-6 + beta)^2) from
 * five cells on each side: needs n_ghost >= 3 and ignores halo gathering.
 * The FP32 pair kernels take minmod, MC and van Leer (with either flux); the
 * others run in the per-cell kernel. */
typedef enum {
    AMR_LIM_MINMOD = 0, AMR_LIM_MC = 1, AMR_LIM_VANLEER = 2, AMR_LIM_WENO5 = 3,
    AMR_LIM_KOREN = 4, AMR_LIM_WENO3 = 5, AMR_LIM_UPWIND = 6
} amr_limiter;

/* Numerical fluxes of Sec. 3.2, both with Einfeldt's signal speeds
 * u_roe -/+ d (Sec. 3.5): Rusanov (local Lax-Friedrichs, a = |u_roe| + d)
 * and HLL (Harten, Lax and van Leer). */
typedef enum { AMR_FLUX_RUSANOV = 0, AMR_FLUX_HLL = 1 } amr_flux;

/* One canonical ghost-pattern entry: one per (receiving block, face), and one
 * per fine source block for F2C.  face = direction from dst towards src;
 * offset = position of the fine block inside the coarse face (bit 0 along the
 * lower tangential dimension); aux = boundary-face index for BC entries
 * (row of the bc_data array), else 0; src = -1 for BC.  Entries are sorted by
 * (kind, face, dst, offset) -- the paper sorts its index arrays by neighbour
 * type, face direction, receiving block and hanging offset (Sec. 2.6). */
typedef struct {
    int32_t kind, face, dst, src, offset, aux;
} amr_ghost_entry;

/* One forward-Euler sub-step of Eq. 5 (Sec. 3.1):
 *   u(s_out) = w_dt * dt * F(u(s_deriv)) + sum_i w_prev[i] u(s_prev[i])
 * dt is the device-resident time step of the forest.  update_dt = 1 marks
 * the last stage of a step: the stage also reduces the CFL limit of its own
 * output (after flux fixing) into the next dt.  gather_halo = 1: halo cells
 * across same-level (SRL) faces are read straight from the neighbour's
 * interior instead of from s_deriv's ghost cells, which then only need the
 * non-SRL part of the pattern (amr_step with AMR_STEP_GATHER does that). */
typedef struct {
    int s_out, s_deriv;
    int n_prev;
    int s_prev[4];
    double w_prev[4];
    double w_dt;
    int update_dt;
    int gather_halo;
} amr_stage;

/* Flags of amr_step(). */
#define AMR_STEP_GRAPH 1   /* capture one step as a CUDA graph and replay it */
#define AMR_STEP_GATHER 2  /* stages gather same-level halos from neighbours;
                              the ghost fill runs only the entries that still
                              need ghost cells (state ghosts are then stale) */
#define AMR_STEP_SSP3 4    /* three-stage strong-stability-preserving RK
                              (Shu-Osher form) instead of Heun; n_states >= 3 */
#define AMR_STEP_RK4 8     /* classical four-stage RK instead of Heun;
                              n_states >= 4 */
#define AMR_STEP_SSP43 16  /* optimal four-stage, third-order SSP RK instead
                              of Heun; n_states >= 3 */

/* Refinement-criterion constants of Eq. 12 (Sec. 3.3).  The criterion is
 * evaluated on density and pressure; a cell's value is the larger one (for
 * scalar advection: on the scalar). */
typedef struct {
    double c_refine, c_derefine, eps, eps_abs;
} amr_flag_params;

/* Creates the brick of Sec. 2.2 refined uniformly to init_level, allocates
 * n_states x max_blocks blocks of device state (Sec. 2.3 static allocation;
 * zero-filled) and builds the ghost pattern.  *out receives the forest.
 * Errors: AMR_EINVAL (bad config), AMR_ECAPACITY (init mesh larger than
 * max_blocks), AMR_ENOMEM, AMR_ECUDA. */
amr_status amr_create_forest(const amr_config *cfg, int init_level, amr_forest **out);

/* Creates one forest holding n independent mesh instances (many meshes of
 * uneven size advanced together): instance i is the brick of cfgs[i] refined
 * uniformly to init_levels[i].  The blocks of all instances are numbered
 * consecutively in instance order, so every call below works on all of them
 * at once -- one kernel launch per phase sweeps every block of every
 * instance.  Each instance keeps its own domain, brick, periodicity,
 * max_level, boundaries, CFL number and time step; ndim, block_n, n_ghost,
 * precision, n_states, gamma, limiter, flux, gravity, diagonal_ghosts,
 * host_only and the allocation hook must be the same for all.  Capacity is the sum of the instances' max_blocks; each
 * instance is also held to its own max_blocks on regrid.  amr_create_forest
 * is the n = 1 case.  Errors as amr_create_forest. */
amr_status amr_create_batch(const amr_config *cfgs, const int *init_levels, int n, amr_forest **out);

/* Number of mesh instances of the forest. */
amr_status amr_n_instances(const amr_forest *f, int *n);

/* Block range of instance inst: blocks first .. first + n - 1 (either
 * pointer may be NULL).  Ranges change after a regrid. */
amr_status amr_instance_blocks(const amr_forest *f, int inst, int64_t *first, int64_t *n);

/* Frees everything the forest owns.  NULL is accepted. */
amr_status amr_destroy_forest(amr_forest *f);

/* Number of leaf blocks (of all instances). */
amr_status amr_n_blocks(const amr_forest *f, int64_t *n);

/* Level and integer block coordinates (at the block's own level, counted over
 * the whole brick; coords[3b+2] = 0 in 2D) of the first min(cap, n) blocks
 * in block order (Sec. 2.2).  Either array may be NULL.  *n = block count. */
amr_status amr_get_blocks(const amr_forest *f, int32_t *level, int64_t *coords, int64_t cap, int64_t *n);

/* Classifies every block face as SRL / F2C / C2F / BC from the forest's face
 * connectivity and uploads the index lists to the device (Sec. 2.6: built on
 * the CPU, executed on the GPU).  A no-op when the mesh revision has not
 * changed since the last build (Sec. 2.2 mesh revision number). */
amr_status amr_build_ghost_pattern(amr_forest *f);

/* Copies the canonical pattern (see amr_ghost_entry) into out[0..cap).
 * *n = total number of entries (call with cap = 0 to size the buffer). */
amr_status amr_get_ghost_pattern(const amr_forest *f, amr_ghost_entry *out, int64_t cap, int64_t *n);

/* Copies n_blocks blocks of state slot s (layout above, ghosts included) from
 * src, which is a host pointer (on_device = 0) or a device pointer of the
 * current device (on_device = 1).  Ordered on `stream`; host copies are
 * complete when the call returns. */
amr_status amr_set_state(amr_forest *f, int s, const void *src, int on_device, amr_stream stream);

/* Copies n_blocks blocks of state slot s into dst (host or device pointer);
 * host copies are complete when the call returns. */
amr_status amr_get_state(const amr_forest *f, int s, void *dst, int on_device, amr_stream stream);

/* Device pointer of state slot s (max_blocks blocks); valid until the forest
 * is destroyed. */
amr_status amr_state_ptr(const amr_forest *f, int s, void **ptr);

/* Dirichlet values for the AMR_BC_DATA faces (Sec. 2.4, Eq. 4 bc_data):
 * host array [n_bf][n_var][N^(d-1)] in double, n_bf = number of BC entries of
 * the current pattern in canonical order (row = entry's aux), face-cell index
 * with the lower tangential dimension fastest.  Must be set again after a
 * regrid (the paper refreshes it through a callback; out of scope here). */
amr_status amr_set_bc_data(amr_forest *f, const double *values, int64_t n_values);

/* Fills the face ghost cells of state slot s: round 1 (SRL copies, physical
 * boundaries, F2C restriction), then round 2 (C2F limited prolongation, which
 * reads round-1 ghosts of the coarse blocks) -- Sec. 2.6.  Edge and corner
 * ghost cells are not filled (Sec. 2.1). */
amr_status amr_fill_ghosts(amr_forest *f, int s, amr_stream stream);

/* Sets the device time step to cfl / max over leaf cells of
 * sum_d (|v_d| + c) / dx_d of state slot s (Sec. 3.2, step 2c). */
amr_status amr_compute_dt(amr_forest *f, int s, amr_stream stream);

/* Overwrites every instance's device time step / reads instance 0's
 * (synchronises `stream`). */
amr_status amr_set_dt(amr_forest *f, double dt, amr_stream stream);
amr_status amr_get_dt(amr_forest *f, double *dt, amr_stream stream);

/* Time step of every instance into dts[0 .. n_instances) (synchronises). */
amr_status amr_get_dts(amr_forest *f, double *dts, amr_stream stream);

/* One stage of Eq. 5 on every block: primitive reconstruction with the minmod
 * limiter, Rusanov fluxes with Einfeldt wave speeds, divergence, Runge-Kutta
 * combination (Sec. 3.2), then flux fixing at refinement boundaries (Sec. 2.7)
 * with the stage's time step w_dt * dt.  s_deriv's ghosts must be filled.
 * s_out may equal one of s_prev. */
amr_status amr_advance_stage(amr_forest *f, const amr_stage *st, amr_stream stream);

/* n_steps steps of Heun's method (Eq. 6-7) on slot 0 (slot 1 as the stage
 * state): fill ghosts, stage 1, fill ghosts, stage 2 with the dt update.
 * With AMR_STEP_SSP3 or AMR_STEP_RK4 the step is the three-stage SSP or the
 * classical four-stage Runge-Kutta method (Sec. 3.1 lists both), each stage
 * a sub-step of Eq. 5 (L = flux divergence with flux fixing):
 *   SSP3: u1 = u0 + dt L(u0); u2 = 3/4 u0 + 1/4 (u1 + dt L(u1));
 *         u0 <- 1/3 u0 + 2/3 (u2 + dt L(u2))                    (slots 1, 2)
 *   SSP43: u1 = u0 + dt/2 L(u0); u2 = u1 + dt/2 L(u1);
 *         u1 <- 2/3 u0 + 1/3 u2 + dt/6 L(u2); u0 <- u1 + dt/2 L(u1) (slots 1, 2)
 *   RK4:  u1 = u0 + dt/2 L(u0); u2 = u0 + dt/2 L(u1); u3 = u0 + dt L(u2);
 *         u0 <- -1/3 u0 + 1/3 u1 + 2/3 u2 + 1/3 u3 + dt/6 L(u3)  (slots 1-3),
 * the last form being u0 + dt/6 (k1 + 2 k2 + 2 k3 + k4) written with the
 * stage states; the last stage updates dt.
 * flags: AMR_STEP_GRAPH captures one step in a CUDA graph on first use and
 * replays it (re-captured after a regrid or a change of flags);
 * AMR_STEP_GATHER lets the stage kernel read same-level halos directly (the
 * ghost cells of the state are not all refreshed; amr_fill_ghosts() refills
 * them).  The dt must be set (amr_compute_dt).  Errors: AMR_EINVAL (more
 * than one scheme flag, or too few state slots for the scheme). */
amr_status amr_step(amr_forest *f, int n_steps, int flags, amr_stream stream);

/* Integral of every conserved variable over the leaves of slot s, summed in
 * double on the device in a fixed order (Eq. 18), for instance 0 (n_var
 * values).  Synchronises `stream`. */
amr_status amr_conserved(amr_forest *f, int s, double *sums, amr_stream stream);

/* The same for every instance: sums[inst * n_var + v]. */
amr_status amr_conserved_all(amr_forest *f, int s, double *sums, amr_stream stream);

/* Refinement flags of slot s from the criterion of Eq. 12 (ghosts must be
 * filled): +1 refine, -1 derefine, 0 keep, per block.  Copied to flags_out
 * (host, n_blocks entries); synchronises `stream`. */
amr_status amr_flag(amr_forest *f, int s, const amr_flag_params *prm, int8_t *flags_out, amr_stream stream);

/* Adapts the mesh (Sec. 2.2): flags from `flags` (host, one per block) or,
 * when flags is NULL, from amr_flag() on slot 0 after a ghost fill; refine,
 * coarsen (a family only when all of its children are flagged -1), 2:1
 * balance across faces, edges and corners; then, if the mesh changed, moves
 * slot 0's data to the new blocks on the GPU (copy / prolong / restrict),
 * rebuilds the ghost pattern and sets every instance's dt to the CFL limit of
 * slot 0 on the new mesh (Sec. 3.2).  Slot 0's ghosts are filled first.
 * Other slots are scratch afterwards.  AMR_ECAPACITY leaves mesh and data
 * unchanged.
 * *changed (may be NULL) = 1 when the mesh changed. */
amr_status amr_flag_and_regrid(amr_forest *f, const amr_flag_params *prm, const int8_t *flags,
                               int *changed, amr_stream stream);

/* Autotuner: times the stage kernel on this forest's mesh for each
 * candidate launch shape -- (block, tile) items per CTA 1, 2 or 4, or a
 * persistent grid of SMs x resident CTAs sweeping all items -- and, for FP32
 * 3D with two ghost layers and the Rusanov flux, the kernel and staging tile
 * (packed cell-pair kernel with 16 x 16 or, for blocks above 8^3, 8 x 8 column
 * tiles, versus one cell per thread); keeps the fastest for later stages and
 * steps.  The timed stages write slot 1 only: slot 0's interior is not
 * advanced (its ghost cells are refilled).  *choice (may be NULL) =
 * 1000 x (pair tile 8) + 100 x (per-cell kernel) + items per CTA, 0 for
 * persistent; *best_ms = mean time of one stage launch of the choice. */
amr_status amr_autotune(amr_forest *f, int *choice, double *best_ms, amr_stream stream);

/* Sets the stage launch shape directly, with amr_autotune's choice code
 * (items per CTA 1..64 or 0 for a persistent grid; +100 per-cell kernel;
 * +1000 pair kernel with 8 x 8 tiles, FP32 3D blocks above 8^3 only).
 * Errors: AMR_EINVAL (a code this forest cannot run). */
amr_status amr_set_launch_shape(amr_forest *f, int choice);

/* ---- learned refinement flags ------------------------------------------
 * A small network predicts the flags of the criterion of Eq. 12 (Sec. 3.3)
 * from pooled block data; the criterion stays as fallback for blocks the
 * network is unsure about and as the judge of its flags.  Network: F inputs
 * -> 64 -> 64 (GELU) -> 3 logits (derefine / keep / refine) -> softmax; the
 * passes use BF16 copies of the FP32 master weights with FP32 accumulation.
 * Parameters are packed FP32 [W1 (F x 64), b1, W2 (64 x 64), b2, W3 (64 x
 * 3), b3]; labels are classes 0, 1, 2 = flags -1, 0, +1. */
typedef struct amr_mlp amr_mlp;

/* Features of every block of slot s into device memory x[f * n_blocks + b]
 * (feature-major): for each of 4^d pools of (N/4)^d cells the mean density
 * and pressure over the block means, minus one, and the mean speed over the
 * block-mean sound speed, then level / max_level; F = 3 * 4^d + 1 (193 in
 * 3D).  x may be NULL to only query *n_features.  Needs block_n % 4 == 0
 * and Euler physics (AMR_EINVAL otherwise). */
amr_status amr_features(amr_forest *f, int s, float *x, int *n_features, amr_stream stream);

/* Model on the current device with n_features inputs, weights drawn
 * uniformly in +-1/sqrt(fan_in) from `seed`, zero biases. */
amr_status amr_mlp_create(int n_features, uint64_t seed, amr_mlp **out);
amr_status amr_mlp_destroy(amr_mlp *m);
amr_status amr_mlp_n_params(const amr_mlp *m, int64_t *n);

/* FP32 master parameters to / from the host (n = amr_mlp_n_params);
 * setting them also refreshes the BF16 copy and resets the optimiser. */
amr_status amr_mlp_get_params(const amr_mlp *m, float *host, int64_t n);
amr_status amr_mlp_set_params(amr_mlp *m, const float *host, int64_t n);

/* Arithmetic of the passes: bits = 16 (the default) runs the products on
 * BF16 tensor cores (mma.sync m16n8k16, FP32 accumulation), with features,
 * hidden activations and hidden-layer deltas rounded to BF16 (nearest even)
 * where they enter a product; bits = 32 runs them on FP32 CUDA cores with
 * FP32 activations (the weights are BF16 in both).  Errors: AMR_EINVAL. */
amr_status amr_mlp_set_precision(amr_mlp *m, int bits);

/* Softmax probabilities prob[s * 3 + c] of n samples x[f * n + s] (device). */
amr_status amr_mlp_forward(amr_mlp *m, const float *x, int64_t n, float *prob, amr_stream stream);

/* Gradient of the mean cross-entropy over all n samples (labels y, device)
 * into grad[0 .. P) (device), and the loss into grad[P]. */
amr_status amr_mlp_gradient(amr_mlp *m, const float *x, const int8_t *y, int64_t n, float *grad, amr_stream stream);

/* One AdamW step (Loshchilov & Hutter 2019: beta 0.9 / 0.999, eps 1e-8,
 * bias-corrected moments, decay lr * weight_decay * w decoupled from the
 * gradient) of the FP32 master weights with the caller's gradient grad[0 ..
 * P) (device, FP32), then their BF16 copy; the step counter of the bias
 * correction advances by one (amr_mlp_set_params resets it and the moments).
 * Enqueued on `stream`.  Errors: AMR_EINVAL, AMR_ECUDA. */
amr_status amr_mlp_adamw_step(amr_mlp *m, const float *grad, double lr, double weight_decay, amr_stream stream);

/* AdamW (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay) on shuffled
 * mini-batches for `epochs` passes; *final_loss = mean loss of the last
 * epoch's batches. */
amr_status amr_mlp_train(amr_mlp *m, const float *x, const int8_t *y, int64_t n, int epochs, int batch, double lr,
                         double weight_decay, uint64_t seed, double *final_loss, amr_stream stream);

/* Refinement flags of slot s from the model: the most probable class when
 * its probability is at least tau, else the criterion of Eq. 12 with `prm`
 * (ghost cells of slot s are filled for those blocks).  flags_out: host,
 * one per block; *n_fallback = blocks that used the criterion. */
amr_status amr_mlp_flags(amr_forest *f, amr_mlp *m, int s, const amr_flag_params *prm, double tau, int8_t *flags_out,
                         int64_t *n_fallback, amr_stream stream);

/* Reads and clears the device status word (synchronises `stream`): AMR_OK or
 * the first device-side error (AMR_ENONPHYS, AMR_ETIMEOUT, AMR_EBOUNDS). */
amr_status amr_sync_status(amr_forest *f, amr_stream stream);

/* Message of the last failed call on f ("" if none).  Never NULL. */
const char *amr_last_error(const amr_forest *f);

/* Kernel launches issued by the library since the forest was created. */
amr_status amr_launch_count(const amr_forest *f, int64_t *n);

/* ---- per-phase timing ----------------------------------------------------
 * A debug mode that splits the time of the calls above into the phases of
 * one time step, as the timers of Sec. 2.8 and the breakdowns of Sec. 5.2 and
 * 5.4 do (ghost-cell updates against the flux computation and solution
 * update; mesh adaptation and pattern updates in the AMR run).  Device phases are timed by a pair of CUDA events
 * recorded on the call's stream around their launches, host phases by the
 * wall clock.  While tracing is on, amr_step runs every step as separate
 * launches even when AMR_STEP_GRAPH is given (a replayed graph cannot be
 * split into phases), and amr_autotune pauses it.  Off by default; tracing
 * never changes results. */
typedef enum {
    AMR_PHASE_GHOST_R1 = 0,   /* ghost fill round 1: same level, restriction, boundaries (Sec. 2.6) */
    AMR_PHASE_GHOST_R2,       /* ghost fill round 2: limited prolongation (Sec. 2.6) */
    AMR_PHASE_STAGE,          /* flux computation and solution update (Eq. 5), all passes */
    AMR_PHASE_FLUXFIX,        /* flux fixing at refinement faces (Sec. 2.7) */
    AMR_PHASE_DT,             /* CFL time step: maximum speed and the per-mesh commit */
    AMR_PHASE_CONSERVED,      /* conserved sums */
    AMR_PHASE_FLAGS,          /* refinement flags (Eq. 12) and model features */
    AMR_PHASE_TRANSFER,       /* regrid data transfer on the device */
    AMR_PHASE_MESH_HOST,      /* host: adapting and balancing the forest, the old -> new map */
    AMR_PHASE_PATTERN_HOST,   /* host: building and uploading the ghost-cell pattern */
    AMR_N_PHASES
} amr_phase;

/* Switches tracing on (on != 0) or off.  The totals are kept across
 * switches; amr_trace_read clears them.  Errors: AMR_EINVAL (f NULL). */
amr_status amr_trace(amr_forest *f, int on);

/* Waits for every phase recorded so far (so it synchronises with the
 * streams they were recorded on), then writes per phase the total
 * milliseconds to ms[0 .. AMR_N_PHASES) and the number of timed records to
 * count[0 .. AMR_N_PHASES) (host arrays; either may be NULL).  reset != 0
 * clears the totals afterwards.  Errors: AMR_EINVAL; AMR_ECUDA when a
 * phase traced since the last read with reset could not be timed (its
 * events could not be created or recorded, or not read back, including at
 * the automatic drain of a long traced run); such phases are left out of the
 * totals, which are still written, and the condition is cleared by reset. */
amr_status amr_trace_read(amr_forest *f, double *ms, int64_t *count, int reset);

/* ---- checkpoint, restart and output --------------------------------------
 * The configuration of instance `inst` as given at creation (the batch
 * capacity is in f's max_blocks only through amr_n_blocks; here max_blocks
 * is the instance's own).  Errors: AMR_EINVAL. */
amr_status amr_get_config(const amr_forest *f, int inst, amr_config *out);

/* Writes a checkpoint of f to the file `path`: per instance its
 * configuration (allocation hooks excepted), its leaves and its dt, then
 * state slot 0 of every block including ghost cells (host-only forests: the
 * meshes only).  Binary, native byte order, versioned ("AMRCKPT1").
 * Synchronises `stream`.  Errors: AMR_EINVAL (null argument), AMR_ESTATE
 * (the file cannot be written), AMR_ECUDA. */
amr_status amr_save(const amr_forest *f, const char *path, amr_stream stream);

/* Creates a forest from a checkpoint written by amr_save: the saved meshes,
 * configurations, dt and slot 0.  `opts` (may be NULL) supplies n_states,
 * host_only and the allocation hooks (other fields are ignored); NULL keeps
 * the saved n_states on the device with cudaMalloc.  Slots other than 0
 * start zeroed.  Errors: AMR_EINVAL, AMR_ESTATE (unreadable, truncated or
 * foreign file, or a host-only checkpoint loaded onto the device),
 * AMR_ECAPACITY, AMR_ENOMEM, AMR_ECUDA. */
amr_status amr_load(const char *path, const amr_config *opts, amr_forest **out, amr_stream stream);

/* Writes slot s in the XDMF format the paper uses for output (Sec. 2.8):
 * `base`.bin holds, block after block and variable after variable, the
 * N^d interior cells of each block (i fastest) in the forest's precision;
 * `base`.xmf describes every block as a uniform grid (origin and spacing of
 * its level) whose cell-centred attributes (rho, mx, my[, mz], E) point into
 * the binary file by byte offset, one spatial collection per instance.  The
 * data file name is written without directories, so keep both files
 * together.  Synchronises `stream`.  Errors: AMR_EINVAL, AMR_ESTATE (file),
 * AMR_ECUDA. */
amr_status amr_write_xdmf(const amr_forest *f, int s, const char *base, amr_stream stream);

/* Largest block count amr_conserved_static() accepts. */
#define AMR_STATIC_MAX_BLOCKS 65536

/* Conserved integrals of a block array without any device allocation.
 * The paper has no counterpart: this is for callers that cannot call
 * cudaMalloc when they need the sums -- their device memory is reserved up
 * front by another allocator (a framework's caching pool, a fixed arena), or
 * they must not trigger the device-wide synchronisation that cudaMalloc and
 * cudaFree may cause.  It computes what amr_conserved() computes, but takes
 * plain device pointers and needs no forest:
 *   state       : n_blocks blocks in the layout above (one state slot),
 *                 float (precision 32) or double (64);
 *   cell_volume : device array, volume of one cell of each block (double);
 *   sums        : device array of ndim + 2 doubles, written on `stream`
 *                 (the Euler layout; advection states use amr_conserved).
 * The per-block partial sums go to a scratch array of
 * AMR_STATIC_MAX_BLOCKS x 5 doubles (2.6 MB) that is part of the library's
 * device image: every GPU that loads the library holds it until the process
 * exits.  Calls share that array, so calls that overlap on the GPU (on
 * different streams, or from different threads) race and give wrong sums;
 * each call overwrites the entries it reads, so nothing carries over between
 * calls that are ordered.  Every call looks up the array's device address
 * on the current device (nothing is cached, so the call stays valid after
 * cudaDeviceReset or a new primary context); the first call on a device
 * also loads the library's device code there, so make that first call
 * before any stream capture.  Errors: AMR_EINVAL (null pointer, bad shape or
 * precision), AMR_ECAPACITY (n_blocks > AMR_STATIC_MAX_BLOCKS), AMR_ECUDA. */
amr_status amr_conserved_static(const void *state, int precision, int ndim, int block_n, int n_ghost,
                                int64_t n_blocks, const double *cell_volume, double *sums, amr_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* AMR_B300_H */
