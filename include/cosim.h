/*
 * cosim.h -- C ABI of the B300 transient EM-thermal-mechanical package solver.
 *
 * One context owns the device state of one voxelised package on one GPU:
 * material IDs, per-axis cell sizes, the E/H fields (with CPML auxiliaries),
 * the Joule-energy accumulator, temperature, and the thermoelastic solution.
 * Every call enqueues its work on the context's CUDA stream; only
 * cosim_read_fields, cosim_stress_solve and the reductions that return a
 * number to the host synchronise that stream.
 *
 * Units are SI. Grids: cells (i,j,k) with 0 <= i < nx ...; nodes 0 <= i <= nx.
 * Node-sized host/device buffers exchanged through this ABI are dense arrays of
 * (nx+1)(ny+1)(nz+1) values, x fastest; cell-sized ones have nx*ny*nz values.
 * An E unknown of axis a is named by the lower node of its edge; an H unknown
 * of axis a by the lowest corner node of its face (see the field list below).
 *
 * Errors: every function returns a cosim_status; nothing throws across the
 * ABI. COSIM_ERR_INVALID leaves the context unchanged. COSIM_ERR_CUDA is
 * sticky: the context must be destroyed. cosim_last_error() describes the
 * most recent failure of a context in words.
 */
#ifndef COSIM_H
#define COSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cosim_ctx cosim_ctx;

typedef enum {
  COSIM_OK = 0,
  COSIM_ERR_INVALID = 1,        /* bad argument or descriptor */
  COSIM_ERR_OOM = 2,            /* device allocation failed */
  COSIM_ERR_CUDA = 3,           /* CUDA runtime error (sticky) */
  COSIM_ERR_NOT_CONVERGED = 4,  /* stress solve hit maxit (result still readable) */
  COSIM_ERR_TIMEOUT = 5,        /* bounded device wait expired */
  COSIM_ERR_NONFINITE = 6       /* NaN/Inf detected in a reduction */
} cosim_status;

/* arithmetic of the field sweeps */
enum { COSIM_FP64 = 0, COSIM_FP32 = 1 };

/* EM wall conditions, per face (x-, x+, y-, y+, z-, z+) */
enum { COSIM_BC_PEC = 0, COSIM_BC_PMC = 1, COSIM_BC_CPML = 2 };

/* Voxel material (Sec. II and III-A). sigma0 is the conductivity at T0 and
 * tcr the temperature coefficient of resistance of Eq. 6; k the thermal
 * conductivity, rho_cp the volumetric heat capacity (Eq. 4); E, nu, alpha_L
 * the isotropic elastic constants and linear CTE (Eqs. 7-8). */
typedef struct {
  double eps_r, mu_r, sigma0, tcr, T0, k, rho_cp, E, nu, alpha_L;
} cosim_material;

/* Problem statement (Sec. II, III). All pointers are host pointers; the
 * library copies what it needs during cosim_create (caller keeps ownership).
 *   dx[nx], dy[ny], dz[nz]: cell sizes [m] (non-uniform grid, Sec. II-A);
 *   mat[nz*ny*nx]: voxel material index < nmat, x fastest;
 *   em_bc[6]: COSIM_BC_* per face. CPML faces are terminated by PEC; an axis
 *     needs at least (number of its CPML faces) * cpml_cells + 2 cells;
 *   cpml_cells, cpml_order (polynomial grading m), cpml_eps_r (background
 *     relative permittivity used for sigma_max);
 *   h_conv[6]: convective film coefficient per face [W/(m^2 K)] (0 = adiabatic,
 *     the paper's thermal condition); T_amb [K]; T_init: initial temperature. */
typedef struct {
  int32_t nx, ny, nz;
  const double *dx, *dy, *dz;
  const uint8_t *mat;
  int32_t nmat;
  const cosim_material *mats;
  int32_t em_bc[6];
  int32_t cpml_cells;
  double cpml_order;
  double cpml_eps_r;
  double h_conv[6];
  double T_amb;
  double T_init;
} cosim_grid_desc;

/* Soft current-density source (the J of Eq. 1-2) on n_edges edges of one
 * axis. edge_ijk[3*e .. 3*e+2] = lower node (i, j, k) of edge e. amp[n] is J
 * [A/m^2] applied during the E update of step n (time (n + 1/2) dt_em); zero
 * for n >= nsteps. Host pointers, copied. */
typedef struct {
  int32_t axis;
  int32_t n_edges;
  const int32_t *edge_ijk;
  int64_t nsteps;
  const double *amp;
} cosim_source;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc returns a device pointer aligned to 256 bytes, or NULL. */
typedef struct {
  void *(*alloc)(size_t bytes, void *user);
  void (*free)(void *ptr, void *user);
  void *user;
} cosim_allocator;

typedef struct {
  int32_t precision;        /* COSIM_FP64 or COSIM_FP32 (fields, stencils, CG vectors) */
  double cfl;               /* fraction of the Courant limit (<= 0: 0.99) ... */
  double dt_em;             /* ... unless dt_em > 0 gives the EM step [s] explicitly */
  double thermal_safety;    /* fraction of the thermal stability limit (<= 0: 0.9) */
  void *stream;             /* cudaStream_t to enqueue on; NULL = default stream */
  const cosim_allocator *allocator; /* NULL = cudaMalloc / cudaFree */
} cosim_options;

/* Create a context: validates the descriptor, copies geometry and materials
 * to the device, derives the EM step (Courant limit of the finest cells at
 * the fastest wave speed, times cfl) and the thermal stability limit,
 * allocates and zeroes all fields (T = T_init). Sec. II-A, II-B. */
cosim_status cosim_create(const cosim_grid_desc *desc, const cosim_options *opts, cosim_ctx **out);

/* Replace the context's current sources (n may be 0). Sec. III-B excitation. */
cosim_status cosim_set_sources(cosim_ctx *ctx, int32_t n, const cosim_source *src);

/* Flag for cosim_em_steps: accumulate the Joule energy of each step. */
#define COSIM_ACCUM_JOULE 1u
/* Flag for cosim_em_steps: the synchronized electro-thermal marching of
 * Sec. II-A. Each step takes every edge's conductivity at the current
 * temperature, sigma(T) = sigma0 / (1 + tcr (T - T0)) per voxel (material
 * fields sigma0, tcr, T0) at the edge temperature (mean of its two end nodes),
 * area-weighted over the edge's voxels as for sigma0; forms the step's Joule
 * power P^{n+1} = D_sigma(T^n) ebar^2 per node (readable as COSIM_F_P, W);
 * and advances the temperature one forward-Euler step of Eq. 5 with the EM
 * time step and that power (convective faces included). Two launches per step
 * (the EM step, then the thermal step). Combines with COSIM_ACCUM_JOULE. */
#define COSIM_COUPLED_THERMAL 2u
/* Flag for cosim_em_steps (implies COSIM_COUPLED_THERMAL): the same coupled
 * step in one launch, the EM kernel taking each node's thermal step once the
 * node's power is complete. Equal to the two-launch form to rounding (the
 * last share of the power enters the update separately). The paper has no
 * counterpart; it is a launch-shape choice (the two-launch form measured
 * faster on B300). */
#define COSIM_COUPLED_FUSED 4u

/* Advance the Maxwell system nsteps leapfrog steps (Eqs. 1-3 in E/H form):
 * H^{n+1/2} = H^{n-1/2} - dt/mu curl E^n;
 * E^{n+1} = ca E^n + cb (curl H^{n+1/2} - J^{n+1/2}),
 * ca = (eps - sigma dt/2)/(eps + sigma dt/2), cb = dt/(eps + sigma dt/2),
 * eps and sigma area-weighted over the voxels of each edge, mu a series mean
 * over each face; CPML auxiliaries in the CPML layers; tangential E held at
 * zero on PEC walls. With COSIM_ACCUM_JOULE each step adds, for every edge,
 * sigma_e V_e ((E^n + E^{n+1})/2)^2 dt / 2 to the Joule energy of both end
 * nodes (P_total = D_sigma e^2, Sec. II-A). One kernel launch per step (two
 * with COSIM_COUPLED_THERMAL). flags: COSIM_ACCUM_JOULE, COSIM_COUPLED_THERMAL,
 * COSIM_COUPLED_FUSED. */
cosim_status cosim_em_steps(cosim_ctx *ctx, int64_t nsteps, uint32_t flags);

/* Peak of the coupled marching since the last reset of cosim_coupled_march. */
typedef struct {
  double T_max;   /* highest nodal temperature seen at a check step [K] (T_init if none) */
  int64_t step;   /* the EM step count (as COSIM_Q_STEP) at that check step; -1 if none */
  int64_t peaks;  /* check steps that set a new peak (each replaced the snapshot) */
} cosim_peak_report;

/* Synchronized marching with peak-temperature snapshots. Sec. IV-A takes the
 * static mechanical solves at peak-temperature snapshots of the coupled
 * electro-thermal marching (Sec. II-A); this call runs nsteps steps of
 * cosim_em_steps(ctx, ., flags | COSIM_COUPLED_THERMAL) and, after every
 * check_every-th step counted from the start of the call and after its last
 * step, compares that step's maximum nodal temperature (a maximum over the
 * owned nodes taken in the step kernel: deterministic, independent of
 * arrival order) with the highest one recorded; a higher one replaces it,
 * with the step count, and the whole temperature field is copied into the
 * peak snapshot (COSIM_F_T_PEAK; cosim_stress_solve with temperature =
 * COSIM_STRESS_T_PEAK takes its load from it). All on the device, no host
 * synchronisation until rep (nullable) is filled at the end. reset != 0 (and
 * the first call on a context) forgets the recorded peak first and sets the
 * snapshot to the current temperature. flags: COSIM_ACCUM_JOULE and
 * COSIM_COUPLED_FUSED (optional).
 * Errors: COSIM_ERR_INVALID (nsteps < 0, check_every <= 0, unknown flags),
 * COSIM_ERR_OOM (first call: 40 bytes + one node-sized field), COSIM_ERR_CUDA,
 * COSIM_ERR_TIMEOUT (a bounded in-kernel wait expired). */
cosim_status cosim_coupled_march(cosim_ctx *ctx, int64_t nsteps, uint32_t flags, int64_t check_every, int32_t reset,
                                 cosim_peak_report *rep);

/* Record nsteps EM steps (flags as for cosim_em_steps) into a CUDA graph held
 * by the context, without running them. nsteps must be a positive multiple of
 * 32 (the Joule window) and at most 2^30; with COSIM_ACCUM_JOULE the context
 * must sit on a window boundary (steps accumulated since the last reset a
 * multiple of 32). The context stream must be a non-default stream. Replaces
 * any earlier graph; cosim_set_sources and cosim_destroy discard it. The paper
 * has no counterpart: this is how the library batches launches on one GPU. */
cosim_status cosim_em_graph_capture(cosim_ctx *ctx, int64_t nsteps, uint32_t flags);

/* Launch the captured graph count times on the context stream (asynchronous):
 * identical results, bit for bit, to cosim_em_steps(ctx, nsteps, flags)
 * called count times. COSIM_ERR_INVALID if no graph is held or the context's
 * E/H parity or Joule window position differs from the captured one. */
cosim_status cosim_em_graph_launch(cosim_ctx *ctx, int64_t count);

/* A batch of contexts (independent package designs of one precision on one
 * GPU, each with its own grid, materials and sources) stepped together: one
 * kernel launch per EM step covers the tiles of every design. The paper has
 * no counterpart; this is how the library serves many design variants at
 * once. Each design's results are those of cosim_em_steps on it alone: the
 * same tiles and formulas, bit for bit in FP64; in FP32 equal to rounding
 * (the batch kernel is compiled apart, and the code generator may contract a
 * packed product into the following addition differently there). */
typedef struct cosim_batch cosim_batch;

/* Create a batch of n distinct contexts. They must have the same precision
 * and share one stream (the batch launches on it, so that their own calls
 * and the batch's stay ordered), and their sources must be set before: a
 * later cosim_set_sources on a member makes the batch calls fail with
 * COSIM_ERR_INVALID (destroy and recreate the batch). persistent != 0: each
 * step is one persistent launch of about as many CTAs as fit on the GPU at
 * once, taking the designs' tiles from a device counter, largest designs
 * first; otherwise one CTA per tile of every design. The batch holds device
 * memory of its own (cudaMalloc: about 28 KB per FP32 design for the
 * per-design step arguments and TMA descriptors) but no field state: the
 * contexts keep theirs. Errors: COSIM_ERR_INVALID (NULL, n < 1, a repeated
 * context, mixed precisions or streams), COSIM_ERR_CUDA; cosim_batch_last_error(NULL)
 * then describes the failure. */
cosim_status cosim_batch_create(cosim_ctx *const *ctxs, int32_t n, int32_t persistent, cosim_batch **out);

/* Advance every design of the batch nsteps EM steps, as cosim_em_steps(ctx,
 * nsteps, flags) would (flags: COSIM_ACCUM_JOULE only). The designs must sit
 * at the same E/H parity and, with COSIM_ACCUM_JOULE, the same position in
 * the 32-step Joule window (else COSIM_ERR_INVALID). Asynchronous on the
 * batch's stream; discards the members' own captured graphs. */
cosim_status cosim_batch_em_steps(cosim_batch *b, int64_t nsteps, uint32_t flags);

/* Record nsteps batch steps (a positive multiple of 32, at most 2^30; with
 * COSIM_ACCUM_JOULE on a window boundary) into a CUDA graph held by the
 * batch, and replay it count times: identical to cosim_batch_em_steps(b,
 * nsteps, flags) called count times. The stream must be a non-default stream. */
cosim_status cosim_batch_graph_capture(cosim_batch *b, int64_t nsteps, uint32_t flags);
cosim_status cosim_batch_graph_launch(cosim_batch *b, int64_t count);

/* The batch's last error in words ("" if none); b may be NULL: then the last
 * failed cosim_batch_create of this thread. Valid until the next call. */
const char *cosim_batch_last_error(const cosim_batch *b);

/* Synchronise the batch's stream and free the batch (not its contexts). */
void cosim_batch_destroy(cosim_batch *b);

/* Flags for cosim_autotune. FORCE: time the variants again even if this
 * grid shape was tuned before in this process. FIXED: no timing; take the
 * shapes from *em_tile_y (8, or 4 for FP32) and *th_block_y (0, 4, 8, 16). */
#define COSIM_TUNE_FORCE 1u
#define COSIM_TUNE_FIXED 2u

/* Pick the launch shapes for this context's grid by timing the variants on
 * the context itself: the EM tile height (8 or 4 rows of threads; FP32
 * contexts, steps without COSIM_COUPLED_THERMAL) and the thermal step kernel
 * (0: TMA-staged 32 x 8 tiles, the default; 4, 8, 16: a per-thread-load
 * kernel with blocks of that height). Timing launches only read the current fields
 * and write spare buffers, so the context's state and step count are
 * unchanged; results are identical for every choice. The choice is cached
 * per (nx, ny, nz, precision) for the process; a later context of the same
 * shape takes it without timing. Synchronises the context stream; discards
 * a captured EM graph. Outputs (nullable) receive the chosen heights. The
 * paper has no counterpart: this is how the library fits tiles to B300. */
cosim_status cosim_autotune(cosim_ctx *ctx, uint32_t flags, int32_t *em_tile_y, int32_t *th_block_y);

/* Joule accumulator operations:
 *   COSIM_JOULE_RESET: zero the per-node energy and the accumulated step count;
 *   COSIM_JOULE_FINALIZE_AVG_POWER: thermal source P_i = Q_i / (n_steps dt_em)
 *     [W per node] (burst-averaged power driving Eq. 5); FP32 contexts form
 *     it in FP32 from Q_i rounded to FP32 (P is stored in FP32);
 *   COSIM_JOULE_FINALIZE_ENERGY: T_i += Q_i / C_i (the burst's energy
 *     deposited adiabatically, C_i the node heat capacity).
 * total_joule_energy_out (nullable): sum_i Q_i [J], deterministic FP64 sum
 * (synchronises the stream). */
enum { COSIM_JOULE_RESET = 0, COSIM_JOULE_FINALIZE_AVG_POWER = 1, COSIM_JOULE_FINALIZE_ENERGY = 2 };
cosim_status cosim_joule_accumulate(cosim_ctx *ctx, int32_t op, double *total_joule_energy_out);

/* Forward-Euler heat diffusion steps (Eq. 5) driven by the current thermal
 * source: T_i += dt/C_i (sum_j G_ij (T_j - T_i) + h_f A_i (T_amb - T_i) + P_i),
 * G_ij = k_e A*_e / l_e over the 7-point nodal stencil (M_kk = V0a^T D_k V0,
 * Eq. 4). dt <= 0 uses thermal_safety x the stability limit. */
cosim_status cosim_thermal_steps(cosim_ctx *ctx, int64_t nsteps, double dt);

/* Mechanical supports (Sec. III-B) */
enum {
  COSIM_MECH_CLAMPED_BOTTOM = 0,   /* all z = 0 nodes fixed in x, y, z */
  COSIM_MECH_KINEMATIC_MOUNT = 1,  /* the paper's 3-node, 6-DOF minimum constraint */
  COSIM_MECH_MASK = 2              /* node_mask[(nx+1)(ny+1)(nz+1)]: bit c = component c fixed */
};

typedef struct {
  int32_t bc;                /* COSIM_MECH_* */
  const uint8_t *node_mask;  /* host pointer, for COSIM_MECH_MASK only */
  double T_ref;              /* stress-free temperature [K] */
  double rtol;               /* stop at ||r|| <= rtol ||f|| (<= 0: 1e-9) */
  int64_t maxit;             /* iteration cap (<= 0: 200000; with refine: per inner solve) */
  int32_t check_every;       /* residual checked on the host every n iterations (<= 0: 32) */
  int32_t refine;            /* 1: FP64 iterative refinement around the context-precision CG */
  double inner_rtol;         /* refine: relative tolerance of each inner CG solve (<= 0: 1e-4) */
  int32_t max_refine;        /* refine: outer step cap (<= 0: 30) */
  int32_t temperature;       /* load from COSIM_STRESS_T_CURRENT (0) or COSIM_STRESS_T_PEAK (1): the peak
                                snapshot of cosim_coupled_march (COSIM_ERR_INVALID if none was taken) */
} cosim_stress_opts;
enum { COSIM_STRESS_T_CURRENT = 0, COSIM_STRESS_T_PEAK = 1 };

typedef struct {
  int64_t iters;             /* CG iterations (summed over inner solves when refining) */
  double relres;             /* ||f - K u|| / ||f||: recursively updated by CG, or the true FP64
                                residual of the refined solution when refine = 1 */
  double seconds;            /* wall time of the solve */
  int64_t refine_steps;      /* outer refinement steps taken (0 without refine) */
} cosim_stress_report;

/* Thermoelastic static solve (Eqs. 7-9): HEX8 elements with exact (2x2x2
 * Gauss) integration, K u = f with f the thermal load of dT = T - T_ref,
 * Jacobi-preconditioned CG (FP64 dot products), then von Mises stress at
 * every element centroid and |u| at every node. Synchronises the stream.
 * With refine = 1 the solve is mixed precision: the FP64 residual
 * r = f - K u (FP64 load, FP64 matvec, FP64 u) drives inner CG solves
 * K d = r in the context's precision to inner_rtol, u += d, until
 * ||r|| <= rtol ||f|| (relres then reports that true FP64 residual).
 * Returns COSIM_ERR_NOT_CONVERGED if maxit (or max_refine) is reached (u is
 * still stored). */
cosim_status cosim_stress_solve(cosim_ctx *ctx, const cosim_stress_opts *opts, cosim_stress_report *rep);

/* y = K u for the supports in opts (constrained rows/columns eliminated,
 * y_c = u_c on constrained DOFs). u, y: 3 node-sized arrays in SoA order
 * (ux | uy | uz), in the context's precision (double for COSIM_FP64, float
 * for COSIM_FP32), host or device memory per on_device. */
cosim_status cosim_stress_apply(cosim_ctx *ctx, const cosim_stress_opts *opts, const void *u, void *y,
                                int32_t on_device);

/* Fields exchanged by cosim_read_fields / cosim_write_fields */
enum {
  COSIM_F_EX = 0, COSIM_F_EY = 1, COSIM_F_EZ = 2,   /* E on edges, node-sized */
  COSIM_F_HX = 3, COSIM_F_HY = 4, COSIM_F_HZ = 5,   /* H on faces, node-sized */
  COSIM_F_T = 6,      /* temperature [K], node-sized */
  COSIM_F_Q = 7,      /* accumulated Joule energy [J], node-sized */
  COSIM_F_P = 8,      /* thermal source [W per node], node-sized */
  COSIM_F_UX = 9, COSIM_F_UY = 10, COSIM_F_UZ = 11, /* displacement [m], node-sized */
  COSIM_F_VM = 12,    /* von Mises stress [Pa], cell-sized */
  COSIM_F_UMAG = 13,  /* |u| [m], node-sized */
  COSIM_F_FX = 14, COSIM_F_FY = 15, COSIM_F_FZ = 16, /* thermal load [N], node-sized */
  COSIM_F_DT = 17,    /* temperature rise T - T_init [K], node-sized: the stored state itself, so
                         small rises keep their full precision (COSIM_F_T adds T_init) */
  COSIM_F_T_PEAK = 18, /* the peak snapshot of cosim_coupled_march [K], node-sized, read only */
  COSIM_NUM_FIELDS = 19
};

/* Copy one field into dst (dense layout above), converting to dtype
 * (COSIM_FP64 -> double, COSIM_FP32 -> float). bytes must equal the field's
 * element count times the dtype size. dst is device memory if dst_is_device,
 * else host memory. Synchronises the stream. Caller owns dst. */
cosim_status cosim_read_fields(cosim_ctx *ctx, int32_t field, int32_t dtype, void *dst, size_t bytes,
                               int32_t dst_is_device);

/* Start copying one field into dst (same layout, dtype and size rules as
 * cosim_read_fields) without waiting for it: the field is converted into a
 * context-owned staging buffer on the context's stream, in order after the
 * work enqueued so far, and copied to dst on a second stream of the context,
 * so the copy overlaps the work enqueued next. Later calls may change the
 * field: the value read is the one the enqueued work had produced. dst must
 * stay valid, and must not be read, until cosim_wait_reads returns; pinned
 * host memory lets the copy run asynchronously. A second asynchronous read
 * first waits for the previous one's copy (one staging buffer). The first
 * call allocates that buffer (8 bytes per node) through the context's
 * allocator and creates the copy stream. Errors: COSIM_ERR_INVALID (unknown
 * field, bad dtype, NULL dst or wrong size; nothing is enqueued),
 * COSIM_ERR_OOM, COSIM_ERR_CUDA. Caller owns dst. */
cosim_status cosim_read_fields_async(cosim_ctx *ctx, int32_t field, int32_t dtype, void *dst, size_t bytes,
                                     int32_t dst_is_device);

/* Wait until every copy started by cosim_read_fields_async has landed in
 * its dst; reports a CUDA error of those copies or a bounded-wait timeout of
 * the context's kernels. */
cosim_status cosim_wait_reads(cosim_ctx *ctx);

/* Overwrite one field from src (same layout and size rules). Entries that are
 * not unknowns (edges beyond the last cell, tangential E on PEC walls) are
 * stored as zero. Writable: E, H, T, DT, Q, P, UX..UZ. */
cosim_status cosim_write_fields(cosim_ctx *ctx, int32_t field, int32_t dtype, const void *src, size_t bytes,
                                int32_t src_is_device);

enum {
  COSIM_Q_DT_EM = 0,          /* EM step [s] */
  COSIM_Q_DT_TH_LIMIT = 1,    /* thermal stability limit [s] */
  COSIM_Q_STEP = 2,           /* EM steps taken */
  COSIM_Q_BYTES_RESIDENT = 3, /* device bytes held by the context */
  COSIM_Q_JOULE_STEPS = 4,    /* steps accumulated since the last reset */
  COSIM_Q_N_CELLS = 5,
  COSIM_Q_N_NODES = 6,
  COSIM_Q_PRECISION = 7,
  COSIM_Q_LAUNCHES = 8,       /* CUDA kernels launched by the context so far */
  COSIM_Q_EM_TILE_Y = 9,      /* EM tile height in use (8, or 4 after autotuning an FP32 context) */
  COSIM_Q_TH_BLOCK_Y = 10     /* thermal step kernel in use: 0 TMA-staged tiles, 4/8/16 classic block height */
};
cosim_status cosim_query(const cosim_ctx *ctx, int32_t what, double *out);

/* Context options for cosim_set_option. */
enum {
  COSIM_OPT_WAIT_CYCLES = 0  /* bound, in SM clock cycles, of every in-kernel wait for staged data
                                (default 2^31, about a second at 2 GHz; >= 1000) */
};
/* Set a context option (value in the option's unit). A wait that runs out
 * abandons its kernel's work and makes the next synchronising call return
 * COSIM_ERR_TIMEOUT; the context stays usable. Discards a captured EM graph.
 * COSIM_ERR_INVALID for an unknown option or a value out of range. The paper
 * has no counterpart. */
cosim_status cosim_set_option(cosim_ctx *ctx, int32_t what, double value);

/* Health check of the bounded waits: one small kernel waits for a barrier
 * phase that nothing completes, runs out after the context's wait bound and
 * takes the solver kernels' error path. Returns COSIM_ERR_TIMEOUT when that
 * path works (and clears the error, so the context stays usable); any other
 * status is a failure of the check (COSIM_ERR_TIMEOUT left from earlier work
 * is reported, and cleared, before the check runs). Synchronises the stream.
 * The paper has no counterpart. */
cosim_status cosim_wait_selftest(cosim_ctx *ctx);

/* Checkpoints of the marching state: E and H with the CPML auxiliaries of the
 * current step, the Joule energy (FP64 total and the short window), the
 * temperature, the thermal source, the step and window counters and the
 * device source time index, in one opaque blob (a header, then raw arrays).
 * The geometry, materials, sources, options and the mechanical solution are
 * not part of it. Stepping on after cosim_checkpoint_load gives the same bits
 * as the saving context stepping on (with the same sources and options). The
 * paper has no counterpart.
 * size: the blob's bytes at the context's present state. */
cosim_status cosim_checkpoint_size(const cosim_ctx *ctx, size_t *bytes);
/* Write the blob to dst (device memory if dst_is_device, else host; caller
 * owns it; bytes must equal cosim_checkpoint_size). Synchronises the stream. */
cosim_status cosim_checkpoint_save(cosim_ctx *ctx, void *dst, size_t bytes, int32_t dst_is_device);
/* Restore a blob written by a context of the same grid, precision and CPML
 * set-up (COSIM_ERR_INVALID otherwise, context unchanged). Discards a captured
 * EM graph. Synchronises the stream. */
cosim_status cosim_checkpoint_load(cosim_ctx *ctx, const void *src, size_t bytes, int32_t src_is_device);

/* Human-readable description of the context's last error ("" if none).
 * Valid until the next call on the context. ctx may be NULL: then the last
 * error of a failed cosim_create on this thread. */
const char *cosim_last_error(const cosim_ctx *ctx);

/* Free all device memory of the context (after synchronising its stream). */
void cosim_destroy(cosim_ctx *ctx);

/* Deterministic FP64 sum of n doubles in device memory, for callers that
 * cannot allocate device memory themselves: an application whose device
 * memory is fully reserved by its own pool or budget, or a latency-critical
 * loop where cudaMalloc's implicit synchronisation and possible failure are
 * not acceptable. The paper has no counterpart; this is a service of the
 * library (the same two-stage reduction that gives cosim_joule_accumulate its
 * total, with its partial sums in a fixed array of the library's device image
 * instead of context scratch).
 *   x: device pointer to n doubles (caller owns it); n <= 268,435,456 (2^28),
 *      larger n returns COSIM_ERR_INVALID before any GPU work;
 *   out: the sum, written to host memory (the call then synchronises stream)
 *      or to device memory when out_is_device != 0;
 *   stream: cudaStream_t to run on (NULL = default stream).
 * Calls no cudaMalloc, cudaFree or any allocating routine. The scratch array
 * (65,568 doubles, 512.25 KiB) is held by every GPU that loads the library
 * until the process exits. The first call on a device resolves the array's
 * device address (cudaGetSymbolAddress) for that device; make that first call
 * before any stream capture. All calls share the array and it keeps the last
 * call's contents: calls that overlap on the GPU (concurrent streams or
 * threads) race and must be serialised by the caller. Nothing needs clearing:
 * every slot a call reads was written earlier in the same call.
 * Errors: COSIM_ERR_INVALID (NULL pointer, n < 0, n over the limit),
 * COSIM_ERR_CUDA; cosim_last_error(NULL) describes the failure. */
cosim_status cosim_sum_f64_noalloc(const double *x, int64_t n, double *out, int32_t out_is_device, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* COSIM_H */
