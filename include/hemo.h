/*
 * hemo.h - C ABI of the GB300 library for the coupled lattice-Boltzmann /
 * immersed-boundary time step of cellular blood flow (HemoCell method,
 * Zavodszky et al., "Cellular blood flow modelling with HemoCell").
 *
 * One simulation = a D3Q19 BGK plasma lattice (Sec. 2.2) plus triangulated
 * cell membranes coupled to it by the immersed-boundary method (Sec. 2.3),
 * with periodic, resting-wall and moving-wall boundaries (Sec. 2.5) and
 * Euler vertex integration every fluid step (Sec. 2.6).  Optional: membrane
 * forces every N fluid steps and the Adams-Bashforth integrator (Sec. 2.6),
 * nonlinear bending and local area terms (Sec. 2.3), an internal viscosity
 * ratio (Sec. 1, Sec. 3) and a Lees-Edwards boundary (Sec. 2.5).  Every step
 * runs in this library's CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Lattice units: dx = 1, dt = 1.  Lattice arrays are indexed
 *    n = x + nx * (y + ny * z) (x fastest); vector fields are [n][3].
 *  - Return value: HEMO_OK (0) or a negative hemo_status; the message of the
 *    last failure on the calling thread is returned by hemo_last_error().
 *  - Pointers documented "host" are read or written during the call only;
 *    pointers documented "any" may be host (pageable or pinned) or device
 *    memory of the simulation's GPU.  The library owns every buffer it
 *    allocates and frees them in hemo_destroy().
 *  - All work is enqueued on the simulation's CUDA stream; a call that
 *    returns data to the caller synchronises that stream first.
 *  - Nothing traps or aborts on the device: device-side problems set a
 *    status word that the host reads (see hemo_step).
 */
#ifndef HEMO_H
#define HEMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hemo_sim hemo_sim;

enum hemo_status {
    HEMO_OK = 0,
    HEMO_ERR_ARG = -1,      /* invalid argument (null, size, range)           */
    HEMO_ERR_OOM = -2,      /* device allocation failed                        */
    HEMO_ERR_CUDA = -3,     /* a CUDA call or kernel launch failed             */
    HEMO_ERR_NUMERIC = -4,  /* non-finite or |u| > 0.3 velocity seen on device */
    HEMO_ERR_DOMAIN = -5,   /* a vertex left the domain across a wall axis     */
    HEMO_ERR_STATE = -6     /* call not valid in the simulation's state        */
};

/* Storage of the populations.  F64: FP64 everything (parity path).  F32:
 * populations stored as FP32 deviations f_i - w_i, FP32 arithmetic.
 * F16DEV / BF16DEV: populations stored as FP16 / BF16 deviations f_i - w_i,
 * less a per-row reference equilibrium (hemo_set_velocity), FP32
 * arithmetic.  In every mode per-cell area and volume sums and cell
 * centroids are FP64; vertex positions are the FP64 centroid plus an offset
 * in the arithmetic precision. */
enum hemo_precision { HEMO_F64 = 0, HEMO_F32 = 1, HEMO_F16DEV = 2, HEMO_BF16DEV = 3 };

/* Device memory provider.  alloc returns a device pointer of at least
 * `bytes` bytes (256-byte aligned) or NULL; release frees it.  When both are
 * NULL the library uses cudaMalloc / cudaFree. */
typedef void *(*hemo_alloc_fn)(size_t bytes, void *ctx);
typedef void (*hemo_free_fn)(void *ptr, void *ctx);

typedef struct {
    int nx, ny, nz;              /* lattice size, each >= 1                        */
    double tau;                  /* BGK relaxation time (Sec. 2.2), > 0.5;
                                    viscosity nu = (tau - 1/2) / 3                 */
    int precision;               /* enum hemo_precision                            */
    int periodic[3];             /* 1 = periodic along x / y / z (Sec. 2.5);
                                    0 = nodes beyond the edge act as resting walls */
    const uint8_t *wall_mask;    /* host, nx*ny*nz or NULL: 0 fluid, 1 resting
                                    wall, 2 / 3 walls moving at wall_velocity[0/1]
                                    (halfway bounce-back, Sec. 2.5 no-slip)       */
    double wall_velocity[2][3];  /* velocities of mask ids 2 and 3                 */
    double body_force[3];        /* constant force density g on every fluid node   */
    void *cuda_stream;           /* cudaStream_t for all work; NULL = default     */
    hemo_alloc_fn alloc;         /* optional device memory provider                */
    hemo_free_fn release;
    void *alloc_ctx;
    unsigned options;            /* bit mask of HEMO_OPT_*; 0 = defaults           */
} hemo_lattice_desc;

/* Staged collision: tiles of wall-free rows go through shared memory by
 * bulk copies (on odd steps the rows shifted by the velocities, the
 * one-node x-shift applied in shared memory) instead of every node through
 * the per-node kernel; the rows next to walls stay per node.  It applies to
 * 16-bit storage with x periodic and rows of at most 1024 nodes whose bytes
 * are a multiple of 16, and is used by default where rows hold at least 512
 * nodes (where it is the faster of the two).  HEMO_OPT_STAGED_COLLISION:
 * also for shorter rows; HEMO_OPT_UNSTAGED_COLLISION: never (it wins over
 * the former).  The results are the same bits in every case. */
enum { HEMO_OPT_STAGED_COLLISION = 1u, HEMO_OPT_UNSTAGED_COLLISION = 64u };

/* 16-bit storage with nx even computes the post-streaming velocity two
 * nodes per thread (32-bit population pairs) and, where the collision is
 * not staged, collides one node per thread.  HEMO_OPT_NODE_COLLISION: one
 * node per thread in both kernels; HEMO_OPT_PAIR_COLLISION: two nodes per
 * thread in both (the unstaged collision only).  The results are the same
 * bits in every case; the options exist to compare the kernels. */
enum { HEMO_OPT_NODE_COLLISION = 2u, HEMO_OPT_PAIR_COLLISION = 8u };

/* HEMO_OPT_TEST_STALLED_WAIT: a test of the failure path of the kernels
 * that wait on copies: the staged collision (HEMO_OPT_STAGED_COLLISION,
 * 16-bit storage) and the FP32 interpolation's tensor copy.  Each
 * first waits, at most 2 ms, on a barrier that no copy completes (before
 * issuing any); the wait runs out, the kernel returns without its work, and
 * the step reports HEMO_ERR_CUDA ("a copy pipeline wait timed out") through
 * the device status, as a real stalled copy would.  Not for production
 * runs. */
enum { HEMO_OPT_TEST_STALLED_WAIT = 4u };

/* HEMO_OPT_WIDE_INDEX: the lattice kernels form population indices i N + n
 * in 64 bits on every lattice.  By default they use 32-bit indices whenever
 * 19 N < 2^32 (N = nx ny nz), and 64-bit ones above, from about 226 M
 * nodes on.  The results are the same bits; the option exists so that the
 * 64-bit variants can be tested on small lattices. */
enum { HEMO_OPT_WIDE_INDEX = 16u };

/* HEMO_OPT_NODE_STAGING: the FP32 interpolation stages each bin's lattice
 * neighbourhood node by node (4-byte asynchronous copies) instead of by one
 * tensor copy (used by default where nx is a multiple of 4 and the
 * neighbourhood does not wrap around a periodic edge).  The results are the
 * same bits. */
enum { HEMO_OPT_NODE_STAGING = 32u };

/* One membrane mesh type (Sec. 2.3: triangulated membrane whose vertices are
 * Lagrangian points).  Energies (F_total = F_link + F_bend + F_area +
 * F_volume, Sec. 2.3; forms chosen where the paper refers elsewhere):
 *   link   per edge  K L0 [eps^2/2 - 1/2 ln(1 - eps^2/max_strain^2)],
 *                    K = k_link kbt / persistence, eps = (L - L0) / L0
 *   bend   per edge  1/2 k_bend kbt (theta - theta0)^2, theta the signed
 *                    angle between the outward normals of the edge's triangles
 *   area   per cell  1/2 k_area ((A - A0) / A0)^2
 *   volume per cell  1/2 k_volume ((V - V0) / V0)^2
 * with L0, theta0, A0, V0 taken from rest_xyz.  Two optional terms for large
 * deformations (Sec. 2.3: the response is highly non-linear; the paper
 * prints no formula, these are this library's forms), off when 0:
 *   nonlinear bending (theta_m > 0) replaces the bending term by
 *                    k_bend kbt theta_m^2 (-1/2) ln(1 - (theta - theta0)^2 /
 *                    theta_m^2): harmonic for small deviations, stiffening
 *                    without bound as |theta - theta0| approaches theta_m
 *   local area       per triangle 1/2 k_local (A_t - A_t0)^2 / A_t0
 * The differentiation form (hemo_record) supports the four-term model only. */
typedef struct {
    int nv, nt;                  /* vertices and triangles; closed, oriented      */
    const int32_t *tri;          /* host, nt*3, counter-clockwise seen from outside */
    const double *rest_xyz;      /* host, nv*3, rest shape                        */
    double k_link, k_bend;       /* in units of kbt                               */
    double k_area, k_volume;     /* lattice energy units                          */
    double kbt;                  /* k_B T in lattice energy units                 */
    double persistence;          /* spectrin persistence length p (lattice units) */
    double max_strain;           /* link strain at which the energy diverges      */
    double k_local;              /* local area modulus, lattice energy per lattice
                                    area; 0 = off                                 */
    double theta_m;              /* maximum bending deviation (rad); 0 = harmonic */
} hemo_mesh_desc;

/* Create a simulation: allocates the lattice, sets every fluid node to rest
 * (f_i = w_i), builds the wall links.  *out receives the handle, or NULL on
 * failure.  HEMO_ERR_ARG for sizes below 1 or nx*ny*nz >= 2^30, tau <= 1/2
 * or NaN, an unknown precision, periodic flags other than 0/1, wall mask
 * values above 3, or only one of alloc / release; HEMO_ERR_OOM when a
 * device allocation fails. */
int hemo_create_lattice(const hemo_lattice_desc *desc, hemo_sim **out);

/* Set the populations of every fluid node to the equilibrium (Sec. 2.2)
 * with rho = 1 and the given velocity.  u: any, nx*ny*nz*3 doubles, or NULL
 * for rest.  Only valid before the first step.  With 16-bit storage the
 * mean x-velocity of each row (x-line) of u over its fluid nodes becomes
 * that row's reference: every population of direction i with c_i,x != 0 is
 * stored minus the equilibrium deviation w_i (3 c_i,x U + 3 U^2) of the
 * row's reference velocity (U, 0, 0), so that the 2-byte values carry the
 * departure from that profile (none without u, and none with the
 * Lees-Edwards boundary). */
int hemo_set_velocity(hemo_sim *sim, const double *u);

/* Add `ncells` cells of a new mesh type: vertex v of cell c is placed at
 * rot[c] * rest_xyz[v] + centers[c] (rot row-major 3x3).  centers, rot: host.
 * *first_cell_id (may be NULL) receives the id of the first added cell;
 * cells and vertices are numbered in the order added.  Only valid before
 * the first step.  Fails with HEMO_ERR_ARG if the mesh is not a closed
 * consistently oriented 2-manifold. */
int hemo_add_cells(hemo_sim *sim, const hemo_mesh_desc *mesh, int ncells, const double *centers,
                   const double *rot, int *first_cell_id);

/* Advance `nsteps` coupled time steps, each in the order of Sec. 2.3:
 * membrane forces at X^n, spreading onto the lattice, BGK collision with the
 * force term and streaming, lattice velocity, interpolation to the vertices
 * and the vertex move (Sec. 2.6; Euler X^{n+1} = X^n + U^n unless
 * hemo_set_time_scales chose otherwise).  Asynchronous on the
 * simulation's stream.  Returns HEMO_OK or the sticky device status
 * (HEMO_ERR_NUMERIC / HEMO_ERR_DOMAIN) of earlier steps that has already
 * reached the host; hemo_sync() waits for it. */
int hemo_step(hemo_sim *sim, int nsteps);

/* Vertex integrators of Sec. 2.6. */
enum hemo_integrator {
    HEMO_EULER = 0,  /* X^{n+1} = X^n + U^n                                  */
    HEMO_AB2 = 1     /* X^{n+1} = X^n + 3/2 U^n - 1/2 U^{n-1}, dt = 1; the
                        first step after hemo_set_time_scales is an Euler
                        step (no U^{n-1} yet)                                */
};

/* Time-scale separation of the cell and fluid updates (Sec. 2.6: the cell
 * equations are integrated by Euler or Adams-Bashforth, and the constitutive
 * model may be evaluated less often than the fluid is updated, with a
 * constant separation).  From the current step on, the membrane forces are
 * evaluated on every `force_every`-th step (the next step is one of them)
 * and held unchanged on the steps in between; spreading, the lattice update,
 * interpolation and the vertex move still run every step.  `integrator` is a
 * hemo_integrator.  The default is force_every = 1 with HEMO_EULER.  May be
 * called before or between steps.  Errors: HEMO_ERR_ARG for force_every < 1
 * or an unknown integrator; HEMO_ERR_STATE while recording for hemo_backward
 * (the differentiation form supports the default only, and hemo_record
 * refuses other settings). */
int hemo_set_time_scales(hemo_sim *sim, int force_every, int integrator);

/* Adaptive time-scale separation (Sec. 2.6: the separation of the cell and
 * fluid updates may be constant or adaptive; the paper's adaptive criterion
 * is in a cited work, so this one is the library's own).  With delta >= 0
 * the membrane forces are evaluated on the next step and from then on at
 * every step at whose start the largest vertex displacement since the last
 * evaluation, |X_v - X_v(last evaluation)|, exceeds delta (lattice units),
 * or at which force_every steps (hemo_set_time_scales) have passed since the
 * last evaluation; they are held in between.  The decision is taken on the
 * device each step (no host synchronisation); the displacement includes the
 * cells' translation, so the criterion is conservative.  delta = 0 evaluates
 * on every step in which anything moved (the default schedule); delta < 0
 * returns to the constant schedule.  hemo_set_time_scales and
 * hemo_set_vertices restart it (the next step evaluates).  Errors:
 * HEMO_ERR_ARG for NaN; HEMO_ERR_STATE while recording for hemo_backward
 * and with the Lees-Edwards boundary; HEMO_ERR_OOM. */
int hemo_set_force_tolerance(hemo_sim *sim, double delta);

/* Membrane-force evaluations (Sec. 2.6: the steps on which the cell forces
 * are computed rather than held) since the simulation was created, over
 * every schedule it has run with, into *count.  With the adaptive
 * separation the count is kept on the device and read here (the call waits
 * for the stream).  Errors: HEMO_ERR_ARG for null pointers; HEMO_ERR_CUDA. */
int hemo_get_force_evaluations(hemo_sim *sim, long long *count);

/* Internal viscosity (Sec. 1: the cytosol is five times as viscous as the
 * plasma; Sec. 3: the red-cell model carries an internal viscosity ratio).
 * From the next step on, fluid nodes inside a cell membrane (at the vertex
 * positions X^n of the step) relax with tau_in = 1/2 + ratio (tau - 1/2),
 * i.e. viscosity ratio * nu; 1 (the default) turns it off.  A node is inside
 * when the upward (+z) ray from it crosses the membrane with a net signed
 * count of one (tie rules: hemo_get_inside).  Errors: HEMO_ERR_ARG for a
 * ratio that is not finite and > 0; HEMO_ERR_STATE while recording for
 * hemo_backward (hemo_record refuses a ratio other than 1), and with the
 * Lees-Edwards boundary (the indicator's rays would cross the displaced
 * plane). */
int hemo_set_viscosity_ratio(hemo_sim *sim, double ratio);

/* Lees-Edwards boundary along z (Sec. 2.5: the domain is periodic in every
 * direction while opposing velocities are imposed on two parallel
 * boundaries, a uniform shear without walls; cells crossing the boundary
 * continue on the other side).  The periodic image above the box is
 * displaced by D_n = U n (mod nx) in x at step n and moves with U x^; the
 * image below by -D_n and -U.  A population streaming across the plane z = 0
 * / nz takes the linear interpolation in x, at the displaced position, of
 * the post-collision populations of the two bracketing nodes of the
 * opposite plane, each shifted by f_eq(rho*, u* +/- U) - f_eq(rho*, u*) (rho*,
 * u* that node's post-collision moments).  Interpolation and spreading treat
 * every z-layer of a vertex's 4x4x4 stencil that falls in an image with the
 * vertex's position displaced by -/+D_n in x (and, interpolating, the image
 * velocity +/-U x^).  At the start of a step a cell whose centroid lies
 * above the box moves by (-D_n, 0, -nz), below it by (+D_n, 0, +nz).  The
 * lattice uses two population arrays from then on.  Call once, before the
 * first step, on a lattice periodic on every axis without walls, with the
 * default time scales.  Errors: HEMO_ERR_ARG (|U| >= 0.3, walls or a
 * non-periodic axis), HEMO_ERR_STATE (after the first step, twice, time
 * scales other than every step with Euler, an internal viscosity ratio
 * other than 1, recording), HEMO_ERR_OOM.
 * hemo_record refuses a simulation with the boundary. */
int hemo_set_lees_edwards(hemo_sim *sim, double U);

/* The inside/outside indicator of the current vertex positions: inside
 * (any, N bytes, [z][y][x]) receives 1 for nodes inside a cell membrane, 0
 * elsewhere.  A column passing exactly through a projected triangle edge
 * belongs to the triangle for which that edge, counter-clockwise seen from
 * +z, points in -y (in +x when horizontal); a crossing exactly at a node's
 * height counts as below the node.  Synchronises. */
int hemo_get_inside(hemo_sim *sim, uint8_t *inside);

/* Wait for the stream and return the device status of all steps so far. */
int hemo_sync(hemo_sim *sim);

enum hemo_field {
    HEMO_RHO = 1,        /* density of the current populations, [n]         */
    HEMO_U = 2,          /* velocity (post-streaming, with F/2), [n][3]     */
    HEMO_VERTS = 4,      /* absolute vertex positions, [v][3] double        */
    HEMO_FORCES = 8,     /* membrane forces of the last step, [v][3] double */
    HEMO_CELLSTATS = 16  /* per cell: centroid xyz, area, volume, Taylor
                            deformation index, [c][6] double                */
};

/* Copy fields out (bitmask of hemo_field).  rho and u are double for
 * HEMO_F64 and float otherwise; rho is 0 and u the wall velocity at wall
 * nodes.  All pointers: any, caller-owned; NULL skips a field.
 * Synchronises the stream and returns the device status. */
int hemo_get_fields(hemo_sim *sim, unsigned what, void *rho, void *u, double *verts,
                    double *forces, double *cellstats);

/* Sizes of the simulation (any pointer may be NULL). */
int hemo_get_sizes(const hemo_sim *sim, long long *n_nodes, long long *n_vertices, int *n_cells,
                   int *n_bins);

/* ---- inspection of integer work and raw state (tests, tools) ----------- */

/* How the collision is split (see the staged collision): plan[0] tiles of
 * wall-free rows staged through shared memory, plan[1] other rows with fluid
 * (per-node kernel), plan[2] rows per tile at most, plan[3] ring stages.
 * All zero when every node goes through the per-node kernel.  plan: host, 4
 * ints, caller-owned. */
int hemo_get_lattice_plan(const hemo_sim *sim, int *plan);

/* The library's D3Q19 velocity order: c (host, 19*3 int), w (host, 19). */
int hemo_velocity_set(int32_t *c, double *w);

/* Populations f_i (not deviations) in the library's velocity order, in
 * natural layout regardless of the in-place streaming parity: any,
 * nx*ny*nz*19 doubles indexed [n][i].  Synchronises. */
int hemo_get_populations(hemo_sim *sim, double *f);

/* Per-node wall links: bits 2i..2i+1 of links[n] give, for direction i of
 * the library's order, 0 if node + c_i is fluid, else the wall id (1 resting,
 * 2 / 3 moving; nodes beyond a non-periodic edge count as 1); 0 at wall
 * nodes.  links: any, nx*ny*nz uint64.  Synchronises. */
int hemo_get_links(hemo_sim *sim, uint64_t *links);

/* Edge table of mesh type `type`: ne*4 int32 (v0, v1, a, b) with triangles
 * (v0, v1, a) and (v1, v0, b); edges numbered in order of first appearance
 * in the triangle list (triangles in order, edges t0t1, t1t2, t2t0).
 * edges: host, capacity 3*nt/2*4; *ne receives the count. */
int hemo_get_edges(hemo_sim *sim, int type, int32_t *edges, int *ne);

/* Replace the absolute vertex positions (any, nv*3 double).  Only valid
 * before the first step. */
int hemo_set_vertices(hemo_sim *sim, const double *verts);

/* Bin the current vertex positions by lattice block of `block` = 8 nodes
 * per axis: key[v] = bx + nbx * (by + nby * bz) of floor(X) (wrapped on
 * periodic axes), perm = vertex ids sorted stably by key, start[k] = first
 * position of block k (nbins + 1 entries).  Same kernels as the step.
 * key, perm: any, nv int32; start: any, nbins+1 int32.  Synchronises. */
int hemo_get_bins(hemo_sim *sim, int32_t *key, int32_t *perm, int32_t *start);

/* ---- checkpoint and resume -------------------------------------------- */

/* Sec. 2.6: a run is paused, its state kept, and continued.  The state is
 * what changes from step to step: the populations (in the in-place layout
 * of the step count's parity; with 16-bit storage also the rows' reference
 * they are stored against), the velocity field, the FP64 cell centroids and
 * the vertex offsets, the membrane forces (held between force evaluations),
 * the previous vertex velocity (Adams-Bashforth), the step count and the
 * time-scale setting, and the Lees-Edwards step counter.  Lattice, walls,
 * parameters and cells are not part of it: load it into a simulation created
 * and filled with cells the same way (same sizes, precision and boundary),
 * which then continues bit for bit as the saved one would have.
 * hemo_state_bytes: *bytes (host) receives the size.  hemo_save_state /
 * hemo_load_state: buf any (host or device of the simulation's GPU),
 * caller-owned, at least that size; both synchronise.  Errors: HEMO_ERR_ARG
 * (null, too small, a state of another simulation), HEMO_ERR_STATE while
 * recording for hemo_backward. */
int hemo_state_bytes(hemo_sim *sim, size_t *bytes);
int hemo_save_state(hemo_sim *sim, void *buf, size_t bytes);
int hemo_load_state(hemo_sim *sim, const void *buf, size_t bytes);

/* ---- differentiation form --------------------------------------------- */

/* Start recording for hemo_backward: checkpoint the full state (populations,
 * centroids, vertex offsets) now and every `checkpoint_every` steps after
 * (even, >= 2), and take the current cell centroids as the reference of the
 * loss's drift term.  The current step count must be even.  Checkpoints are
 * device memory owned by the library: (steps / checkpoint_every + 1) copies
 * of the state.  Needs the default time scales (forces every step, Euler)
 * and the four-term membrane model (k_local = theta_m = 0 for every mesh
 * type): HEMO_ERR_STATE otherwise. */
int hemo_record(hemo_sim *sim, int checkpoint_every);

/* Deformation loss of the current vertices (its own definition; the paper
 * gives none): the mean over cells of the Taylor deformation index
 * (sqrt(l1) - sqrt(l3)) / (sqrt(l1) + sqrt(l3)) of the gyration tensor
 * G = mean_v (X_v - c)(X_v - c)^T (eigenvalues l1 >= l2 >= l3) plus
 * |c - c_ref|^2 (c_ref: centroids at hemo_record, else at the first call).
 * loss: host, 1 double; dL_dverts: any, nv*3 doubles, or NULL.
 * Synchronises. */
int hemo_deformation_loss(hemo_sim *sim, double *loss, double *dL_dverts);

/* Reverse-mode gradient of a loss of the final vertex positions, given
 * dL_dverts = dL/dX at the current step (any, nv*3 doubles), with respect to
 * the parameters of the steps recorded since hemo_record: grad (host,
 * ngrad >= 4 * mesh types + 4 doubles) receives, per mesh type t in the
 * order added, dL/dk_link, dL/dk_bend, dL/dk_area, dL/dk_volume at
 * 4t..4t+3, then dL/ds for a common scale s of both wall velocities, then
 * dL/dg (3).  Each step is differentiated exactly as computed: the
 * adjoint of the interpolation and Euler move, of the post-streaming
 * velocity, of streaming with bounce-back, of the BGK collision with the
 * force term, of the spreading, and of the membrane forces (a Hessian-vector
 * product).  Segments between checkpoints are recomputed forward, keeping
 * each step's populations and positions, then swept backwards; gradients
 * accumulate in FP64.  The state after the call is the state before it.
 * Synchronises. */
int hemo_backward(hemo_sim *sim, const double *dL_dverts, double *grad, int ngrad);

/* ---- measurement ------------------------------------------------------ */

/* Phases of one step, in order. */
enum hemo_phase {
    HEMO_PHASE_MEMBRANE = 0,  /* re-base, area/volume, membrane forces        */
    HEMO_PHASE_BINS = 1,      /* vertex binning and gather in bin order       */
    HEMO_PHASE_SPREAD = 2,    /* force spreading onto the lattice             */
    HEMO_PHASE_COLLIDE = 3,   /* fused BGK collision + streaming              */
    HEMO_PHASE_MOMENTS = 4,   /* post-streaming velocity                      */
    HEMO_PHASE_INTERP = 5,    /* interpolation and Euler move                 */
    HEMO_NUM_PHASES = 6
};

/* on = 1: record a CUDA event before and after every phase of every step
 * (event-record nodes inside the step's CUDA graph, on the stream the
 * kernels run on); on = 0: plain step.  Takes effect at the next step. */
int hemo_set_phase_timing(hemo_sim *sim, int on);

/* Device durations in milliseconds of the phases of the most recent step
 * (ms: host, HEMO_NUM_PHASES floats; phases a step does not run report 0),
 * and the number of kernel launches one step makes (may be NULL).
 * Synchronises.  HEMO_ERR_STATE if timing is off or no step ran yet. */
int hemo_get_phase_times(hemo_sim *sim, float *ms, int *kernels_per_step);

/* ---- binning without device allocation -------------------------------- */

/* The paper has no counterpart: this entry point exists for callers that
 * cannot let a library allocate device memory (code inside another
 * framework's memory budget, latency-critical loops where cudaMalloc's
 * implicit device synchronisation is not acceptable, tools that hold vertex
 * positions in their own buffers and no simulation handle).
 *
 * Bins `nv` absolute FP64 vertex positions with the key rule and the
 * counting-sort kernels of hemo_get_bins (8^3 lattice blocks of floor(X),
 * wrapped on periodic axes, clamped to the edge block on the others; perm =
 * stable sort by key; start = first position of each block, nbins + 1
 * entries) and allocates nothing.  Given the positions hemo_get_fields
 * returns (HEMO_VERTS), the result equals hemo_get_bins bit for bit for a
 * lattice without the Lees-Edwards boundary (that boundary adds a bin).  The
 * step's own binning floors X formed from the centroid and an offset in the
 * arithmetic precision (and, between two force evaluations, from a two-float
 * centroid), which can fall on the other side of a lattice plane than the
 * FP64 absolute position does.  verts: device, nv*3 double; periodic: host, 3 ints; key, perm:
 * device, nv int32; start: device, nbins + 1 int32, nbins = ceil(nx/8) *
 * ceil(ny/8) * ceil(nz/8); cuda_stream: cudaStream_t or NULL.  Asynchronous:
 * outputs are ready when the stream reaches the end of the call's work.
 *
 * Scratch (block counts, cursors, unsorted permutation) is a 5 MiB array in
 * the library's device image, held by every GPU that loads the library until
 * the process exits.  Limits: nv <= 1,048,576 and nbins <= 131,072; larger
 * sizes return HEMO_ERR_ARG with a message.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls
 * share the one array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and give wrong results; serialise them. */
int hemo_bin_vertices_noalloc(const double *verts, int nv, int nx, int ny, int nz, const int32_t *periodic,
                              int32_t *key, int32_t *perm, int32_t *start, void *cuda_stream);

/* Release every resource of the simulation (NULL is allowed). */
void hemo_destroy(hemo_sim *sim);

/* Message of the last failure on the calling thread ("" if none). */
const char *hemo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HEMO_H */
