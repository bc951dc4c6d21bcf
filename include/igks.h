/*
 * igks.h -- C ABI of libigks, the GB300 (sm_103a) implementation of the per-iteration
 * hot path of the implicit gas-kinetic scheme (IGKS) of Pan, Zhong & Zhuo,
 * "An Implicit Gas-Kinetic Scheme for Turbulent Flow on Unstructured Hybrid Mesh",
 * arXiv:1709.00803.
 *
 * A context holds one or more steady solves ("solves"), each a 2D unstructured hybrid
 * mesh with its own flow conditions, resident in GPU memory. One call of igks_iterate
 * advances every live solve of the context by the same number of iterations; each
 * iteration is the paper's steady step:
 *   ghost cells (Section II.E) -> spectral radius and time steps (Eq. 21, 23, 24)
 *   -> least-squares gradients and limiter (Eq. 6-10) -> gas-kinetic interface flux
 *   (Eq. 1-14, 33-34) with the Spalart-Allmaras face terms (Eq. 28-30) -> residual and
 *   SA source (Eq. 16, 27, 28a) -> CFL adaptation (Eq. 25) -> matrix-free LU-SGS forward
 *   and backward sweeps (Eq. 19-22, 31-32) -> update.
 *
 * Conventions
 *  - Every function returns an int status: IGKS_OK (0), IGKS_CONVERGED (1) where noted,
 *    or a negative IGKS_E* code. igks_last_error() gives a message owned by the context.
 *  - All array arguments are HOST pointers owned by the caller. The library copies what
 *    it needs during the call and never keeps a caller pointer.
 *  - Device memory belongs to the context and is released by igks_destroy.
 *  - A context is not thread-safe; distinct contexts may be used from distinct threads.
 *  - Index arrays are int32, zero-based. Field arrays are float64, structure-of-arrays:
 *    component k of cell i is at [k * n_cells + i].
 */
#ifndef IGKS_H
#define IGKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IGKS_OK 0
#define IGKS_CONVERGED 1
#define IGKS_EINVAL (-1)    /* bad argument */
#define IGKS_EMESH (-2)     /* mesh failed validation (index, orientation, closure) */
#define IGKS_ENOMEM (-3)    /* device allocation failed */
#define IGKS_ECUDA (-4)     /* CUDA runtime error */
#define IGKS_DIVERGED (-5)  /* non-positive density/pressure or non-finite state */
#define IGKS_TIMEOUT (-6)   /* a device wait ran out of its spin limit */
#define IGKS_EBUSY (-7)     /* operation not allowed in the current state */

/* boundary tags of face_bc (Section II.E) */
#define IGKS_BC_INTERIOR 0
#define IGKS_BC_FARFIELD 1  /* free stream: the ghost cell holds the free-stream state */
#define IGKS_BC_SYMMETRY 2
#define IGKS_BC_WALL 3      /* adiabatic non-slip wall */
#define IGKS_BC_OUTFLOW 4   /* outflow: boundary-normal velocity from the Riemann invariants,
                               density, tangential velocity, temperature and nu_tilde from inside */
#define IGKS_BC_MOVING_WALL 5 /* adiabatic non-slip wall moving with the tangential part of the
                               free-stream velocity (a lid) */

/* time marching of a solve */
#define IGKS_SCHEME_IMPLICIT 0  /* LU-SGS sweeps (Eq. 22) with the implicit CFL (Eq. 24-25) */
#define IGKS_SCHEME_EXPLICIT 1  /* explicit gas-kinetic scheme, Eq. 15: W += dt M / Omega */

/* precision of the LU-SGS sweeps; flux, residual and state update are always FP64 */
#define IGKS_PREC_FP64 0
#define IGKS_PREC_MIXED 1   /* sweeps and implicit operator in FP32 */
#define IGKS_PREC_DF64 2    /* sweeps in double-float (a pair of FP32 numbers, about 48 bits)
                               on the FP32 pipes: FP64-grade increments at FP32 speed */

#define IGKS_LIMITER_NONE 0
#define IGKS_LIMITER_BJ 1      /* Barth-Jespersen reading of the min-max limiter, Eq. 9 */
#define IGKS_LIMITER_VENKAT 2  /* Venkatakrishnan's smooth variant */

typedef struct igks_options {
  int32_t precision;      /* IGKS_PREC_* */
  int32_t device;         /* CUDA device ordinal */
  void* stream;           /* cudaStream_t to run on, or NULL for a stream of the context */
  int32_t check_every;    /* iterations between host checks of the stopping rule (>=1) */
  int32_t use_graph;      /* capture one iteration (per group) as a CUDA graph and replay it;
                             with 2 <= check_every <= 64 and no timing, also check_every
                             iterations of every group as one graph, launched once per check */
  int32_t sweep_threads;  /* threads per block of the sweep kernels (0: default) */
  int32_t timing;         /* record CUDA events around every kernel (igks_kernel_times) */
  int32_t sweep_mode;     /* 0 automatic, 1 one block per solve walking its levels,
                             2 one launch per level over all solves (low-depth orderings) */
  int32_t sweep_cluster;  /* schedule 1: a thread-block cluster of 1 (0: 1), 2, 4 or 8 blocks per
                             solve shares each level (distributed shared memory, one cluster
                             barrier per level); same arithmetic, same bits */
  int32_t groups;         /* schedule 1 with several solves: split them into this many groups of
                             consecutive solves (0: 1), each iterated by a graph on a stream of
                             its own, so that one group's sweeps (one block per solve) overlap
                             another group's flux; same arithmetic, same bits */
  int32_t wait_limit;     /* tries of a device wait (the one-block-per-solve sweeps wait on an
                             mbarrier for each level's records) before it gives up: the solve
                             stops with state IGKS_TIMEOUT, its fields untouched, and
                             igks_iterate returns IGKS_TIMEOUT (0: 2^24 tries, about 1.4 s) */
  int32_t starve_test;    /* test hook, 0 in use: 1 makes every forward sweep skip the copy of
                             its second level, so that the wait for it runs out */
  int32_t reserved[1];
} igks_options;

/* Flow conditions of one solve. Non-dimensional: free-stream density, speed and the
 * reference length are 1, so p_inf = 1/(gamma Ma^2), mu_inf = 1/Re; gamma = 1.4 (K = 3). */
typedef struct igks_flow {
  double mach, reynolds, aoa_deg;
  double prandtl;          /* one Pr for the laminar and turbulent heat flux */
  double t_ref, s_suth;    /* free-stream temperature and Sutherland constant [K] */
  int32_t sa_on;           /* Spalart-Allmaras turbulence model on/off */
  int32_t limiter;         /* IGKS_LIMITER_* */
  double nut_ratio_inf;    /* free-stream nu_tilde / nu */
  double cfl_exp;          /* CFL of the flux time step (Eq. 23) */
  double cfl_init, cfl_min, cfl_max;   /* implicit CFL (Eq. 24) and Eq. 25 clamp */
  double res_target;       /* stop at L2(M_rho/Omega) <= res_target * first-iteration value */
  double venkat_k;         /* Venkatakrishnan limiter constant */
  double c_num;            /* numerical collision time coefficient (pressure-jump term) */
  int32_t visc_sr;         /* add the viscous term to the face spectral radius */
  int32_t scheme;          /* IGKS_SCHEME_IMPLICIT (LU-SGS) or IGKS_SCHEME_EXPLICIT (Eq. 15) */
  double eq40_target;      /* if > 0, also stop when the Eq. 40 ratio of an update is <= it */
} igks_flow;

typedef struct igks_status {
  int32_t iters;           /* iterations done by this solve */
  int32_t state;           /* 0 running, IGKS_CONVERGED, or a negative code */
  double res_l2_rho;       /* RMS over cells of M_rho / Omega at the last iteration */
  double res_l2_rel;       /* res_l2_rho / its first-iteration value */
  double res_inf;          /* max |M_rho| at the last iteration (Eq. 25) */
  double eq40_ratio;       /* max_i |dW_i| / |W_i| of the last update (Eq. 40) */
  double cfl;              /* implicit CFL used by the last sweep */
  double dt;               /* flux time step of the last iteration (Eq. 23) */
} igks_status;

typedef struct igks_ctx igks_ctx;

/* Create an empty context on opt->device. Errors: IGKS_EINVAL, IGKS_ECUDA. */
int igks_create(const igks_options* opt, igks_ctx** out);

/* Add one solve: a mesh in face/cell form (Section II.D's mesh data reduced to nodes,
 * cells and faces). Cells are CCW node lists (cell_ptr CSR, any polygon); face f joins
 * nodes face_nodes[2f] -> face_nodes[2f+1], CCW around its left cell face_cells[2f];
 * face_cells[2f+1] is the right cell or -1 on a boundary, where face_bc[f] gives the tag.
 * The cell numbering is the sweep order of the LU-SGS method (Eq. 20, j < i).
 * *solve_id receives the solve's index. Must precede the first igks_iterate.
 * Errors: IGKS_EINVAL (null/negative sizes), IGKS_EMESH (index out of range, face with
 * no left cell, non-boundary face without a right cell), IGKS_EBUSY (after iterate). */
int igks_mesh_upload(igks_ctx* ctx, int32_t n_nodes, const double* xy /*[2*n_nodes]*/,
                     int32_t n_cells, const int32_t* cell_ptr /*[n_cells+1]*/,
                     const int32_t* cell_nodes, int32_t n_faces,
                     const int32_t* face_nodes /*[2*n_faces]*/,
                     const int32_t* face_cells /*[2*n_faces]*/,
                     const int32_t* face_bc /*[n_faces]*/, int32_t* solve_id);

/* Set the flow conditions of a solve (before its first iteration, or to restart it). */
int igks_set_flow(igks_ctx* ctx, int32_t solve, const igks_flow* f);

/* Set every cell of a solve to the free stream and reset its iteration state. Builds the
 * device data on first use (geometry, wall distance, sweep levels are computed there;
 * IGKS_EMESH if a cell has non-positive area or a face normal points into its left cell). */
int igks_init_freestream(igks_ctx* ctx, int32_t solve);

/* Advance every live solve by up to max_iters iterations: implicit (LU-SGS) or explicit
 * (Eq. 15) per the solve's igks_flow.scheme. A solve stops on its own at convergence
 * (res_l2_rel <= res_target, or the Eq. 40 ratio <= eq40_target when that is set) or
 * divergence; the host checks every check_every iterations. status (nullable) receives
 * one entry per solve. Returns IGKS_CONVERGED if every solve has converged, IGKS_OK if
 * some are still running, IGKS_TIMEOUT if a solve's sweep wait ran out of its spin limit
 * (that solve stops with its fields as they were before the iteration; the context stays
 * usable), IGKS_DIVERGED if any diverged, or another error. */
int igks_iterate(igks_ctx* ctx, int32_t max_iters, igks_status* status);

/* Enqueue n_iters iterations of every live solve on the context stream and return at
 * once (no host synchronisation, no stopping check on the host; solves still stop on
 * their own on the device). Stream-ordered with anything else the caller puts on the
 * same stream, e.g. CUDA events for timing. */
int igks_enqueue(igks_ctx* ctx, int32_t n_iters);

/* Per-kernel device times of the most recent iteration, in launch order, measured with
 * CUDA events recorded inside the iteration (only when the context was created with
 * igks_options.timing = 1). ms receives up to cap entries; *n the number of kernels.
 * igks_kernel_name(i) names entry i. Call after the stream has been synchronised. */
int igks_kernel_times(igks_ctx* ctx, int32_t cap, float* ms, int32_t* n);
const char* igks_kernel_name(int32_t i);

/* Conserved state + nu_tilde of a solve: W[5*n_cells] SoA (rho, rho U, rho V, rho E, nu_tilde). */
int igks_get_fields(igks_ctx* ctx, int32_t solve, double* W);

/* Overwrite the state of a solve (checkpoint restore / seeded start). The iteration
 * scalars (iteration count, CFL, previous and first residuals) are kept unless
 * igks_set_scalars is called too. */
int igks_set_fields(igks_ctx* ctx, int32_t solve, const double* W);

/* The state of every solve at once (checkpoint / restore of a whole context, and the
 * host round trip of a batched step): W[5 * N] SoA with N the summed cell counts, each
 * variable's block holding the solves in upload order, a solve's cells contiguous
 * (solve k starts at the sum of the cell counts before it). One asynchronous copy per
 * solve on the context stream and one synchronisation. igks_set_fields_all checks each
 * solve's state on the device (density positive, energy finite) and writes only the solves
 * that pass; if any fails it returns IGKS_EINVAL and those solves keep their state. It
 * uses the backward-sweep increment buffer as staging (scratch between iterations).
 * Errors: IGKS_EINVAL, IGKS_ECUDA. */
int igks_get_fields_all(igks_ctx* ctx, double* W);
int igks_set_fields_all(igks_ctx* ctx, const double* W);

/* Iteration scalars of a solve, for checkpoint/resume: out[0] iteration count,
 * out[1] CFL, out[2] previous max|M_rho|, out[3] first-iteration L2 residual,
 * out[4] state. igks_set_scalars takes the same layout. */
int igks_get_scalars(igks_ctx* ctx, int32_t solve, double* out /*[5]*/);
int igks_set_scalars(igks_ctx* ctx, int32_t solve, const double* in /*[5]*/);

/* Intermediate arrays of the last iteration of a solve, for verification. `which`:
 *  IGKS_ARR_GRAD    [4][2][n_cells] unlimited least-squares gradients (Eq. 7)
 *  IGKS_ARR_PHI     [4][n_cells]    limiter factors (Eq. 9)
 *  IGKS_ARR_LAMBDA_F[n_faces]       face spectral radius
 *  IGKS_ARR_LAMBDA_C[n_cells]       per-cell sum of (Lambda_c)_ij
 *  IGKS_ARR_FLUX    [6][n_faces]    time-integrated face flux x S (global frame) and the
 *                                   SA face contributions to the left and right cells
 *  IGKS_ARR_RES     [5][n_cells]    residual M (Eq. 16) and Omega Sr + R (Eq. 27)
 *  IGKS_ARR_DWSTAR  [5][n_cells]    forward sweep result
 *  IGKS_ARR_DW      [5][n_cells]    backward sweep result
 *  IGKS_ARR_GHOST   [5][n_faces]    ghost states (zero on interior faces)
 *  IGKS_ARR_GEOM_CELL[4][n_cells]   area, centroid x, centroid y, wall distance
 *  IGKS_ARR_GEOM_FACE[5][n_faces]   length, normal x, normal y, midpoint x, midpoint y
 * Face arrays follow the uploaded face numbering. */
#define IGKS_ARR_GRAD 1
#define IGKS_ARR_PHI 2
#define IGKS_ARR_LAMBDA_F 3
#define IGKS_ARR_LAMBDA_C 4
#define IGKS_ARR_FLUX 5
#define IGKS_ARR_RES 6
#define IGKS_ARR_DWSTAR 7
#define IGKS_ARR_DW 8
#define IGKS_ARR_GHOST 9
#define IGKS_ARR_GEOM_CELL 10
#define IGKS_ARR_GEOM_FACE 11
int igks_get_array(igks_ctx* ctx, int32_t solve, int32_t which, double* out);

/* Residual history of a solve (Eq. 25's norms, iteration by iteration; kept on the device
 * for the last 1024 iterations): out[3k] the iteration (1-based), out[3k+1] the RMS over
 * cells of M_rho / Omega, out[3k+2] max |M_rho|, oldest first, for the last min(iterations
 * done, 1024, cap) iterations; *n receives the count. */
int igks_get_history(igks_ctx* ctx, int32_t solve, int32_t cap, double* out /*[3*cap]*/, int32_t* n);

/* Sizes of a solve: out[0] n_cells, out[1] n_faces, out[2] forward sweep levels,
 * out[3] backward sweep levels, out[4] boundary faces. */
int igks_mesh_info(igks_ctx* ctx, int32_t solve, int32_t* out /*[5]*/);

/* Pressure and viscous force on the faces tagged bc_tag of a solve, as lift and drag
 * coefficients about the free-stream direction: out[0] Cl, out[1] Cd, out[2] Cd_viscous. */
int igks_get_forces(igks_ctx* ctx, int32_t solve, int32_t bc_tag, double* out /*[3]*/);

/* Launch configuration chosen by igks_autotune. */
typedef struct igks_tuning {
  int32_t sweep_threads;   /* threads per block of the one-block-per-solve sweeps */
  int32_t flux_block;      /* threads per block of the flux kernel */
  int32_t sweep_mode;      /* 1 one block per solve, 2 one launch per level */
  int32_t sweep_cluster;   /* blocks per solve of schedule 1 */
  float ms_per_iter;       /* measured device time of one iteration with it */
  int32_t groups;          /* groups of solves on streams of their own (igks_options.groups) */
} igks_tuning;

/* Time the library's launch configurations (sweep schedule, block size and blocks per
 * solve, flux block size, groups of solves) on the context's live solves, iters_per_trial iterations each after one warm-up
 * iteration, and keep the fastest. Every trial starts from the same saved state and the
 * state is restored afterwards: the configurations do not change the arithmetic, so the
 * solves' iterates are exactly those of an untuned run. Allocates temporary device
 * memory. out (nullable) receives the choice. Errors: IGKS_EINVAL, IGKS_ECUDA. */
int igks_autotune(igks_ctx* ctx, int32_t iters_per_trial, igks_tuning* out);

/* Apply a launch configuration (as igks_autotune returns it; ms_per_iter is ignored) without
 * timing anything: the solves' iterates do not depend on it. Errors: IGKS_EINVAL (a value
 * outside the choices igks_autotune tries), IGKS_ECUDA. */
int igks_set_launch(igks_ctx* ctx, const igks_tuning* t);

/* Number of kernel launches one iteration issues (for launch accounting). */
int igks_launches_per_iteration(igks_ctx* ctx, int32_t* out);

/* Cell numbering for the LU-SGS sweeps (host only, no context). The sweep order of
 * Eq. 20 is the cell numbering, so a renumbering changes the method's iterates (and its
 * convergence rate), not its steady answer; apply the permutation to the mesh before
 * upload (and to any reference run) to use it.
 *   mode 0: identity (the mesh's own numbering)
 *   mode 1: greedy multicolouring of the face-adjacency graph in index order, cells then
 *           sorted by (colour, index): every sweep level is one colour
 * perm[k] = old index of the cell placed at position k; *n_colors receives the number
 * of colours (mode 1) or 1 (mode 0). Errors: IGKS_EINVAL, IGKS_EMESH. */
int igks_order_cells(int32_t n_cells, int32_t n_faces, const int32_t* face_cells /*[2*n_faces]*/,
                     int32_t mode, int32_t* perm /*[n_cells]*/, int32_t* n_colors);

/* Release all device memory and the context. */
int igks_destroy(igks_ctx* ctx);

/* Residual norms of one solve without any allocation by the library (the paper has no
 * counterpart: this is a service for callers that cannot let a library allocate GPU
 * memory -- code running while the stream is being captured into a CUDA graph, hosts
 * whose GPU memory comes only from their own pool or arena, real-time loops that cannot
 * afford an allocation's latency or failure).
 *   m_rho  DEVICE pointer, [n_cells] per-cell density residual (IGKS_ARR_RES component 0)
 *   area   DEVICE pointer, [n_cells] cell areas
 *   out    DEVICE pointer, [2]: out[0] = max |m_rho| over the cells,
 *                               out[1] = RMS over cells of m_rho / area
 *   stream cudaStream_t the two kernels run on (NULL: the legacy default stream)
 * It computes the same reduction, in the same order, as igks_iterate does for its
 * status. Inputs and outputs belong to the caller; the only other memory used is a
 * fixed scratch array in the library's device data (IGKS_NOALLOC_MAX_CELLS / 256 * 2
 * doubles = 64 KiB, held on every GPU that loads the library until the process exits).
 * Its device address is looked up once per device, with that device current, by the
 * first call made on that device: make that first call before any stream capture.
 * Every call shares the scratch array and it keeps the last call's contents; each call
 * writes all it reads, but calls whose kernels overlap on the GPU race on it.
 * Asynchronous: returns after enqueueing; out is valid once the stream reaches it.
 * Errors: IGKS_EINVAL for null pointers, n_cells <= 0, n_cells > IGKS_NOALLOC_MAX_CELLS or
 * a current device ordinal of 64 or more (message in igks_last_error(NULL)), IGKS_ECUDA for
 * a CUDA error. */
#define IGKS_NOALLOC_MAX_CELLS (1 << 20)
int igks_residual_norms_noalloc(const double* m_rho, const double* area, int32_t n_cells,
                                double* out, void* stream);

/* Measured FP64 arithmetic rate of a device, for the roofline of the FP64-bound flux
 * kernel (measurement support; no counterpart in the paper): eight independent chains of
 * fused multiply-adds per thread over eight 256-thread blocks per SM, best of three timed
 * launches after a warm-up, in TFLOP/s (an FMA counts two flops). Takes about 30 ms.
 * Errors: IGKS_EINVAL (null tflops), IGKS_ECUDA. */
int igks_fp64_probe(int32_t device, double* tflops);

/* Message of the last error on this context (owned by the context; never NULL). */
const char* igks_last_error(igks_ctx* ctx);

/* ---------------------------------------------------------------------------------
 * Device memory accounting.
 * igks_footprint_bytes: upper bound of the device bytes one solve of this size takes in
 * a context (host only; nnz = cell_ptr[n_cells], the summed face count of the cells).
 * igks_device_bytes: device bytes the context holds now (0 before the first build). */
int igks_footprint_bytes(int32_t n_nodes, int32_t n_cells, int32_t n_faces, int32_t nnz, int64_t* out);
int igks_device_bytes(igks_ctx* ctx, int64_t* out);

/* ---------------------------------------------------------------------------------
 * Serving: continuous batching of steady solves (the paper solves one case at a time;
 * this layer has no counterpart there and adds no arithmetic: every solve runs the same
 * iteration as a context of its own and ends with bitwise the same fields).
 *
 * A server owns a FIFO queue of submitted requests and a set of resident cohorts. A
 * cohort is a context holding the solves admitted together, on its own CUDA stream, so
 * that the cohorts' iterations overlap on the GPU. igks_server_step
 *   1. retires the solves that stopped (converged, diverged or at the iteration cap):
 *      records the finish time, Cl/Cd/c on IGKS_BC_WALL faces and (keep_fields) the
 *      fields, and destroys a cohort once none of its solves is live;
 *   2. admits queued requests in arrival order while a slot is free (live solves <
 *      max_slots) and the HBM budget holds their igks_footprint_bytes, into one new
 *      cohort; cohorts whose live cells fell below repack_fraction of their cells move
 *      their live solves (fields and iteration state, bitwise) into that cohort too and
 *      are freed, so finished solves stop holding memory;
 *   3. enqueues iters_per_step iterations on every cohort with live solves, then waits
 *      for all of them. Solves stop on the device at their own iteration (a converged
 *      solve is skipped by every kernel), so a step never runs a solve past its stop.
 * Times are seconds of a steady host clock since igks_server_create. */
#define IGKS_MAXITER (-8)   /* result state: stopped at max_iters without converging */

typedef struct igks_server_options {
  int32_t precision;        /* IGKS_PREC_* of every solve */
  int32_t device;           /* CUDA device ordinal */
  int32_t max_slots;        /* live solves at most (>= 1) */
  int32_t max_cohort;       /* requests admitted into one new cohort at most (>= 1) */
  int32_t iters_per_step;   /* iterations per igks_server_step (>= 1) */
  int32_t max_iters;        /* iteration cap of a solve (>= 1) */
  int64_t hbm_budget;       /* device bytes the resident cohorts may hold; 0: 90% of the
                               free device memory at creation */
  double repack_fraction;   /* see step 2; 0 disables repacking */
  int32_t keep_fields;      /* keep the fields of finished solves for igks_server_take_fields */
  int32_t reserved[7];
} igks_server_options;

typedef struct igks_request {
  /* mesh, as for igks_mesh_upload (copied at submit) */
  int32_t n_nodes;
  const double* xy;
  int32_t n_cells;
  const int32_t* cell_ptr;
  const int32_t* cell_nodes;
  int32_t n_faces;
  const int32_t* face_nodes;
  const int32_t* face_cells;
  const int32_t* face_bc;
  igks_flow flow;
  int64_t tag;              /* caller's value, returned in the result */
  const double* W0;         /* nullable: starting state [5*n_cells] SoA as for igks_set_fields
                               (a warm start, copied at submit); NULL starts from the free stream */
} igks_request;

typedef struct igks_result {
  int64_t id, tag;
  int32_t state;            /* IGKS_CONVERGED, IGKS_DIVERGED or IGKS_MAXITER */
  int32_t iters;
  int32_t n_cells;
  int32_t cohort;           /* serial number of the cohort the solve finished in */
  double res_l2_rel;        /* final RMS(M_rho / Omega) over its first-iteration value */
  double t_submit, t_admit, t_finish;
  double forces[3];         /* igks_get_forces on IGKS_BC_WALL faces at the finish */
  int64_t footprint;        /* igks_footprint_bytes of the solve */
} igks_result;

typedef struct igks_server_status {
  int32_t queued;           /* submitted, not admitted */
  int32_t live;             /* admitted, still iterating */
  int32_t cohorts;          /* resident contexts */
  int32_t finished;         /* results waiting for igks_server_poll */
  int64_t bytes;            /* footprint of the resident cohorts */
  int64_t budget;           /* the HBM budget in force */
  int32_t admitted;         /* requests admitted by the last step */
  int32_t repacked;         /* live solves moved between cohorts by the last step */
  double step_s;            /* wall time of the last step */
} igks_server_status;

typedef struct igks_server igks_server;

/* Errors: IGKS_EINVAL (bad option), IGKS_ECUDA. */
int igks_server_create(const igks_server_options* opt, igks_server** out);
/* Queue one request; *id receives its id (ids count up from 0). The mesh is validated
 * here (IGKS_EMESH), the flow and a given W0 too (IGKS_EINVAL: non-positive density or
 * non-finite energy, as igks_set_fields). A request whose footprint exceeds the whole
 * budget is refused with IGKS_ENOMEM. A solve that diverges (non-positive density or
 * pressure, or a non-finite state, during an update) finishes with IGKS_DIVERGED. */
int igks_server_submit(igks_server* srv, const igks_request* req, int64_t* id);
/* One retire/admit/run round as described above. status (nullable) describes the
 * server after the step. Errors: IGKS_ECUDA, IGKS_ENOMEM (a cohort could not be
 * built: its requests go back to the queue head). */
int igks_server_step(igks_server* srv, igks_server_status* status);
/* Move up to cap finished results, in finish order, to out; *n receives the count. */
int igks_server_poll(igks_server* srv, igks_result* out, int32_t cap, int32_t* n);
/* Copy the fields ([5][n_cells] SoA, as igks_get_fields) of a finished solve and free
 * the server's copy. IGKS_EINVAL if the id has no kept fields. */
int igks_server_take_fields(igks_server* srv, int64_t id, double* W);
/* Seconds on the server clock. */
int igks_server_now(igks_server* srv, double* t);
int igks_server_get_status(igks_server* srv, igks_server_status* status);
int igks_server_destroy(igks_server* srv);
const char* igks_server_last_error(igks_server* srv);

#ifdef __cplusplus
}
#endif
#endif
