/*
 * mdl.h -- C ABI of the GB300 explicit local space-time adaptive monodomain library.
 *
 * The library advances the monodomain equations (Ogiermann, Balzani, Perotti,
 * "An Explicit Local Space-Time Adaptive Framework for Monodomain Models in
 * Cardiac Electrophysiology", Sec. 2, Eq. monodomain) on box slabs with a
 * symmetric interior penalty DG discretisation (Eq. monodomain-primal-formulation,
 * Eq. monodomain-numerical-flux) on GL-collocated Q1/Q2 elements (Sec. 2.1),
 * forest-of-trees h-adaptivity (Sec. 2.2), and synchronous local time stepping
 * (Sec. 2.3, Alg. 1).  Every part of a barrier step runs in CUDA kernels for sm_103a:
 * the sweep, both indicators, the level assignment and the forest adaptation
 * (refine/coarsen marks, 2:1 closure, coarsenable families, the new leaf list, face
 * tables and the solution transfer).  The host only validates uploads and reads
 * results.
 *
 * Conventions
 *   - Every function returns MDL_OK (0) or a negative MDL_E_* code; no C++
 *     exception crosses the ABI.  mdl_last_error() gives a message.
 *   - Units: cm, ms, mS/cm, uF/cm^2; V is the dimensionless Aliev-Panfilov potential.
 *   - The library copies every input; it never keeps a caller pointer.  All
 *     device memory is owned by the context and released by mdl_destroy().
 *   - Host buffers passed to mdl_read_* are caller-owned; `cap` is their capacity
 *     in elements; `*n` receives the number of elements the full answer needs
 *     (if cap < *n nothing is written and MDL_E_ARG is returned).
 *   - Element (leaf) order: ascending root id (x fastest over the base grid),
 *     then Morton order of the leaf's lower corner inside its root (x bit lowest).
 *     DOF order: element-blocked, local node index a0 + (p+1) a1 + (p+1)^2 a2.
 *   - A failing call leaves the context as it was, except mdl_step_to(), which
 *     stops at the last barrier that completed.
 *   - Calls on one context must not overlap (one host thread at a time).
 */
#ifndef MDL_H
#define MDL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MDL_OK            0
#define MDL_E_ARG        -1   /* invalid argument or size */
#define MDL_E_NOMEM      -2   /* device or host allocation failed */
#define MDL_E_NOSPACE    -3   /* batch: footprint does not fit the HBM budget */
#define MDL_E_CFL        -4   /* an element needs more LTS levels than n_lts_levels allows */
#define MDL_E_NONFINITE  -5   /* V or the state became NaN/Inf */
#define MDL_E_TIMEOUT    -6   /* a bounded wait gave up */
#define MDL_E_CUDA       -7   /* CUDA runtime error (message in mdl_last_error) */
#define MDL_E_STATE      -8   /* call not valid in the context's current state */

#define MDL_MAX_STIM      4
#define MDL_MAX_REFINE    7

/* Geometry (mdl_problem.geometry).  The forest lives on the reference box; the physical
 * domain is its image under x = Phi(X).  Element maps are x(xi) = Phi(X_c + (xi + 1) h / 2),
 * so elements are curved wherever Phi is; the SIPG terms (Eq. monodomain-primal-formulation,
 * Eq. monodomain-numerical-flux) take the Jacobian, area weight, normal and normal extent of
 * every GL point, and each element its own Gershgorin bound (Eq. cfl-monodomain).  A mapped
 * geometry adapts like a box slab (hanging faces integrated at the finer side's points; the
 * restriction weighted by the elements' own GL masses) but needs dt_barrier > 0 when it
 * adapts (MDL_E_ARG otherwise: an adapting curved mesh has no finite set of element classes
 * to bound the step by); it runs the thread-per-element sweep only and takes no
 * mdl_upload_mesh.  Its factors are recomputed on the device for every element whose face
 * kinds change.  Stimulus boxes and the fibre are in physical coordinates; probes stay the
 * GL nodes of the roots.
 *   MDL_GEOMETRY_BOX     Phi = identity (geo ignored)
 *   MDL_GEOMETRY_AFFINE  Phi(X) = A X + b, geo = (A row-major 3x3, b[3]); 2D: leading 2x2, b[0..1]
 *   MDL_GEOMETRY_SHELL   ellipsoidal shell sector, geo = (a_i, b_i, c_i, a_o, b_o, c_o, phi0,
 *                        dphi, theta0, dtheta): azimuth phi = phi0 + dphi X_0 / L_0; 3D polar
 *                        angle theta = theta0 + dtheta X_1 / L_1 inside (0, pi), transmural
 *                        u = X_2 / L_2, x = (a sin(theta) cos(phi), b sin(theta) sin(phi),
 *                        c cos(theta)); 2D u = X_1 / L_1, x = (a cos(phi), b sin(phi)); semi-axes
 *                        a = a_i + u (a_o - a_i) etc., all growing (or all shrinking). */
#define MDL_GEOMETRY_BOX    0
#define MDL_GEOMETRY_AFFINE 1
#define MDL_GEOMETRY_SHELL  2

/* Box stimulus: I_stim = -amplitude at nodes inside [lo, hi] (inclusive, 1e-12
 * slack) for t0 <= t < t1 (Sec. 2, I' = I_ion + I_stim). */
typedef struct mdl_stim {
    double lo[3], hi[3];
    double amplitude, t0, t1;
} mdl_stim;

/* One simulation (Sec. 2, Eq. monodomain with the parameters of Sec. 2.1-2.3).
 * Copied by mdl_create. */
typedef struct mdl_problem {
    int32_t dim;               /* 2 or 3 */
    int32_t order;             /* polynomial order p: 1 or 2 */
    double  extent[3];         /* slab size [cm] (extent[2] ignored in 2D) */
    int32_t base[3];           /* root grid (base[2] ignored in 2D) */
    double  sigma_l, sigma_t;  /* conductivity along / across the fibre [mS/cm] */
    double  fibre[3];          /* fibre direction (normalised by the library) */
    double  chi, cm;           /* surface-to-volume ratio [1/cm], capacitance [uF/cm^2] */
    double  gamma;             /* SIPG penalty factor, Eq. monodomain-numerical-flux */
    int32_t ionic_model;       /* 0 = Aliev-Panfilov, -1 = none (pure diffusion) */
    double  ionic_params[8];   /* AP: k, a, eps0, mu1, mu2, time_scale [ms per model unit] */
    int32_t n_stim;            /* 0 .. MDL_MAX_STIM */
    mdl_stim stim[MDL_MAX_STIM];
    double  dt_barrier;        /* barrier step [ms]; 0 = largest 2^-k ms such that every
                                  admissible element class needs <= n_lts_levels-1 levels */
    int32_t max_refine;        /* maximum refinement depth (0 .. MDL_MAX_REFINE) */
    int32_t n_lts_levels;      /* substeps per barrier are 2^b, b < n_lts_levels */
    double  tau_refine, tau_coarsen;   /* Alg. 1 thresholds on eta^s */
    double  tau_cell, dt_bar_cell;     /* Eq. num-substeps thresholds on eta^t (dt_bar_cell <= 0: off) */
    double  act_threshold;     /* activation threshold for LAT (Sec. 3.3) */
    int32_t state_integrator;  /* 0 forward Euler, 1 exponential (Rush-Larsen analogue) */
    int32_t precision;         /* 32 (FP32 bulk, FP64 reductions) or 64 */
    int32_t amr_enabled;       /* 0/1 */
    int32_t lts_enabled;       /* 0/1; 0 = every element takes one step per barrier */
    int32_t geometry;          /* MDL_GEOMETRY_*: the map x = Phi(X) from the reference box
                                  [0, extent] to the physical domain (curved meshes, Sec. 3.3) */
    int32_t fibre_ref;         /* 1: fibre along the image DPhi e_0 of the first reference axis */
    double  geo[12];           /* parameters of the map (see MDL_GEOMETRY_*) */
} mdl_problem;

typedef struct mdl_ctx mdl_ctx;

/* Per-context counters since creation (or since mdl_reset_stats). */
typedef struct mdl_stats {
    int64_t barriers;          /* barrier steps completed */
    int64_t dof_updates;       /* sum over element steps of (p+1)^d ("element evaluations") */
    int64_t element_updates;   /* element steps */
    int64_t tick_launches;     /* sweep kernel launches */
    int64_t kernel_launches;   /* all kernel launches of the library */
    int64_t amr_rebuilds;      /* barriers whose mesh changed */
    double  sweep_ms;          /* device time of the sweep kernels (CUDA events; 0 unless timing is on) */
    int64_t timed_barriers;    /* barriers whose sweep time is included in sweep_ms */
    double  indicator_ms;      /* device time of the eta^s kernel (timing on) */
    double  amr_host_ms;       /* always 0: the adaptation runs on the device (kept for layout) */
    double  transfer_ms;       /* always 0: the solution transfer runs on the device (kept for layout) */
    double  integral_V;        /* last FP64 integral of V over the domain */
    int64_t n_elements;        /* current leaf count */
    int64_t level_counts[8];   /* elements per LTS level b in the last barrier */
    int64_t factor_updates;    /* curved meshes: elements whose geometric factors were computed
                                  (at creation and after each adaptation; kept elements copy theirs) */
} mdl_stats;

/* Create a context: base grid of roots, V = v = 0 (rest), t = 0.
 * Validates the problem (MDL_E_ARG), allocates device memory (MDL_E_NOMEM) on the
 * current CUDA device, creates a private non-blocking stream. */
int mdl_create(const mdl_problem* prob, mdl_ctx** out);

/* Replace the mesh by the given leaves (any order; the library sorts them).
 * level[i] in 0..max_refine; coords[i*dim + k] is the leaf's integer cell
 * coordinate on the level-level[i] grid (0 <= c < base[k] 2^level[i]);
 * root[i] must equal the root id containing the leaf (checked).  The leaves
 * must tile the slab and be 2:1 face balanced (else MDL_E_ARG).  Resets V and
 * the state to 0 and the activation times to +INF; time is unchanged. */
int mdl_upload_mesh(mdl_ctx* ctx, int64_t n_leaves, const int32_t* root, const int8_t* level,
                    const int32_t* coords);

/* Set V and the state variable at every DOF (n_dof = n_elements (p+1)^d, leaf
 * order).  s may be NULL (state left unchanged).  Probes already above the
 * activation threshold get the current time as activation time. */
int mdl_set_initial(mdl_ctx* ctx, const double* V, const double* s, int64_t n_dof);

/* Replay: use these substep levels b_e (0 <= b_e < n_lts_levels) for the next
 * barrier instead of the library's own assignment (Eq. num-substeps). */
int mdl_set_levels(mdl_ctx* ctx, const int8_t* b_e, int64_t n_e);

/* Replay: use these indicators for the next barrier's refine/coarsen decision
 * (eta_s, Eq. dg-error-estimate) and level assignment (eta_t, Eq.
 * ratti-veroni-temporal).  Either pointer may be NULL (keep the library's own). */
int mdl_set_indicators(mdl_ctx* ctx, const double* eta_s, const double* eta_t, int64_t n_e);

/* Advance whole barrier steps until t >= t_end - 1e-9 dt (Alg. 1 per barrier). */
int mdl_step_to(mdl_ctx* ctx, double t_end);

/* Advance exactly n barrier steps. */
int mdl_step_barriers(mdl_ctx* ctx, int64_t n);

/* Current time t = barrier_tick * dt, the barrier count, and the barrier step dt. */
int mdl_get_time(const mdl_ctx* ctx, double* t, int64_t* barrier_tick, double* dt);

int mdl_get_sizes(const mdl_ctx* ctx, int64_t* n_e, int64_t* n_dof, int64_t* n_probe);

/* V, resp. the AP recovery variable, at every DOF (leaf order), as FP64. */
int mdl_read_V(mdl_ctx* ctx, double* out, int64_t cap, int64_t* n);
int mdl_read_state(mdl_ctx* ctx, double* out, int64_t cap, int64_t* n);

/* FP32 transfers of the fields, for callers that stage them in FP32 (the working
 * precision of FP32 contexts; half the bytes of the FP64 calls).  mdl_set_initial_f32
 * behaves as mdl_set_initial.  mdl_read_fields_f32 writes V and the state variable (either
 * pointer may be NULL) at every DOF in leaf order with one gather and one synchronisation;
 * cap and *n are counted in DOFs per field.  Page-locked host buffers mapped into the
 * device's address space (cudaHostAlloc / cudaMallocHost, e.g. pinned framework tensors) are
 * read or written by the layout kernel itself over the host link, with no staging copy;
 * other host memory goes through one device copy.  The buffers are not retained. */
int mdl_set_initial_f32(mdl_ctx* ctx, const float* V, const float* s, int64_t n_dof);
int mdl_read_fields_f32(mdl_ctx* ctx, float* V, float* s, int64_t cap, int64_t* n);

/* Activation time at each probe: the GL nodes of every root element, probe id =
 * root_id (p+1)^d + local node.  +INF = not activated (Sec. 3.3 LAT). */
int mdl_read_activation(mdl_ctx* ctx, double* out, int64_t cap, int64_t* n);

/* Mesh in leaf order: root id, level, integer coords [n*dim] on the leaf's level
 * grid, and the substep level b_e of the last barrier.  Any pointer may be NULL. */
int mdl_read_mesh(mdl_ctx* ctx, int32_t* root, int8_t* level, int32_t* coords, int8_t* b_e,
                  int64_t cap, int64_t* n);

/* Face table in leaf order: for element e and face f = 2 axis + (side > 0),
 * kind[e*2d+f] = 0 boundary, 1 same level, 2 coarser neighbour, 3 finer
 * neighbours; nbr[(e*2d+f)*2^(d-1) + j] = neighbour leaf index (j = 0 for kinds
 * 1, 2; j = tangential child bits for kind 3), -1 where unused; pos[e*2d+f] =
 * tangential position bits of e on a coarser neighbour's face (kind 2), else 0. */
int mdl_read_faces(mdl_ctx* ctx, int8_t* kind, int32_t* nbr, int8_t* pos, int64_t cap, int64_t* n);

/* eta^s of the last barrier's adapt step (its first n_e_before entries are valid, n_e_before
 * being the element count before that barrier's adaptation) and eta^t of the last completed
 * barrier on the current mesh. */
int mdl_read_indicators(mdl_ctx* ctx, double* eta_s, double* eta_t, int64_t cap, int64_t* n);

/* Counters; timing=1 records CUDA events around each barrier's sweep and indicator
 * kernels (inside the captured barrier graph) and adds their elapsed times to sweep_ms
 * and indicator_ms -- exactly for calls that step one barrier, for every barrier of a
 * call otherwise only when graphs are not used; 0 turns it off. */
int mdl_get_stats(const mdl_ctx* ctx, mdl_stats* out);
int mdl_reset_stats(mdl_ctx* ctx);
int mdl_set_timing(mdl_ctx* ctx, int on);

/* Device pointer to a resident array (valid until the next mutating call) and
 * the context's CUDA stream.  which: 0 V (the current values, normalised into slot 0),
 * 1 state, 2 activation times, 3 eta_t.  *n = element count of the array.  V and the
 * state are in the working precision and leaf/DOF order, (p+1)^d values per element;
 * Q2 3D contexts store their rows padded to 28 values, so for them the view is a compact
 * copy made by this call. */
int mdl_device_view(mdl_ctx* ctx, int which, void** dptr, int64_t* n, void** stream);

const char* mdl_last_error(const mdl_ctx* ctx);
void mdl_destroy(mdl_ctx* ctx);

/* Library build identifier (static string). */
const char* mdl_version(void);

/* Launch shape of the sweep kernel: threads per block in {64, 128, 256}, resident blocks
 * per SM with threads * blocks_per_sm <= 2048.  Results do not depend on it. */
int mdl_set_tick_shape(mdl_ctx* ctx, int32_t threads, int32_t blocks_per_sm);

/* Sweep kernel variant.  All follow Alg. 1 tick by tick; THREAD and COOP run the same
 * per-element arithmetic, GROUP sums the face terms in another order; they agree to the
 * working precision's rounding:
 *   MDL_SWEEP_THREAD  one thread per due element, one launch per tick; the default except
 *                     for Q2 3D FP32 contexts, whose default is MDL_SWEEP_TENSOR;
 *   MDL_SWEEP_GROUP   Q1 only: (p+1)^d lanes per element, one lane per face and per DOF,
 *                     one launch per tick (Q2 contexts use MDL_SWEEP_THREAD);
 *   MDL_SWEEP_COOP    every tick and the barrier epilogue in one cooperative launch with
 *                     grid-wide barriers between ticks (bounded waits: one that gives up
 *                     makes the stepping call return MDL_E_TIMEOUT);
 *   MDL_SWEEP_TENSOR  Q2 3D FP32 contexts only (their default): per tile of 64 due
 *                     elements the SIPG residual of elements with same-level neighbours is
 *                     one tcgen05 tensor-core product of the gathered element and face-
 *                     neighbour values with the level-0 operator (Sec. 2.1: box elements, so
 *                     every level is a power-of-two multiple of it), on values shifted by the
 *                     element mean, with both operands split into two FP16 terms and FP32
 *                     accumulation in tensor memory; other faces are added on the CUDA cores.
 *                     Two persistent blocks per SM walk the tiles.  Agrees with
 *                     THREAD within the FP32 tolerance, not bit for bit.  A bounded device
 *                     wait that gives up makes the stepping call return MDL_E_TIMEOUT.
 * Returns MDL_E_ARG for any other value, or for TENSOR on another kind of context. */
#define MDL_SWEEP_THREAD 0
#define MDL_SWEEP_GROUP 1
#define MDL_SWEEP_COOP 2
#define MDL_SWEEP_TENSOR 3
int mdl_set_sweep_variant(mdl_ctx* ctx, int32_t variant);

/* Upper bound on the number of thread blocks of the persistent tensor-core sweep
 * (MDL_SWEEP_TENSOR); 0 restores the library's default (two blocks per SM).  Results do
 * not depend on it: with a small bound every block walks many tiles of due elements, which
 * is how the tests exercise the kernel's tile-to-tile pipeline on meshes the FP64 oracle
 * can still run.  MDL_E_ARG if max_blocks < 0. */
int mdl_set_sweep_blocks(mdl_ctx* ctx, int32_t max_blocks);

/* ---- Batches: many resident simulations stepped together on one GPU ----
 * (The paper runs one simulation at a time on one CPU core, Sec. 3; batching many
 * resident simulations is this library's addition.)
 * Each slot is a context with its own stream.  Admission compares the slot's device-memory
 * footprint estimate (mdl_batch_footprint) with the budget.  mdl_batch_step steps in one
 * of two ways (mdl_batch_set_fused):
 *   fused (the default): in rounds, each advancing every running slot by one barrier step.
 *     Each slot runs its indicator, adaptation, level and ordering phases (Alg. 1) on its
 *     own stream; then ONE persistent sweep kernel per element class (2D/3D, Q1/Q2) and
 *     precision covers the due elements of all slots of the class, one launch per global
 *     tick (a slot with fewer LTS levels takes part in every 2^k-th), replayed from a CUDA
 *     graph captured for the batch's composition; then each slot's epilogue.  The rounds of
 *     one mdl_batch_step are issued back to back and waited for once.  With autotune the
 *     first rounds (one at a time) time, per class, every candidate launch shape of the
 *     fused kernel (threads per block, due elements per work item) and "own sweeps" (each
 *     slot's own sweep variant on its own stream) on the batch itself, and keep the fastest
 *     (mdl_batch_fused_info); without autotune the fused kernel runs at 128 threads and 256
 *     due elements per work item.  A fused element takes the step of the thread-per-element
 *     sweep (MDL_SWEEP_THREAD): an instance gives the values it gives alone with that sweep,
 *     up to the FP32 rounding of two compilations of the same arithmetic (meshes and levels
 *     identical); with own sweeps it gives the bits it gives alone.
 *   streams: every unfinished slot launches its own barriers (its own sweep variant)
 *     before any is waited for, so their kernels overlap on the device; with autotune a
 *     temporary copy of the first instance of each (precision, dim, order) class is stepped
 *     under a few sweep launch shapes and the fastest is used for the class.  Launch shapes
 *     do not change results: an instance gives the same bits alone and in the mix. */
#define MDL_SLOT_FREE    0
#define MDL_SLOT_RUNNING 1
#define MDL_SLOT_DONE    2
#define MDL_SLOT_FAILED  3
typedef struct mdl_batch mdl_batch;
/* hbm_budget_bytes <= 0: 90% of the current free device memory. */
int mdl_batch_create(int64_t hbm_budget_bytes, int autotune, mdl_batch** out);
int mdl_batch_footprint(const mdl_problem* prob, int64_t* bytes);
/* Create a slot for prob, optionally set its initial state on the base mesh (V0/s0 with
 * n_dof values, may be NULL), to run until t_end.  MDL_E_NOSPACE if it does not fit. */
int mdl_batch_admit(mdl_batch* b, const mdl_problem* prob, const double* V0, const double* s0, int64_t n_dof,
                    double t_end, int32_t* slot);
/* Advance every running slot by up to barriers_per_slot barriers, repeating rounds until
 * wall_budget_s seconds have passed (one round if <= 0) or nothing is left to run. */
int mdl_batch_step(mdl_batch* b, int64_t barriers_per_slot, double wall_budget_s, int64_t* barriers_done);
/* Slots that finished (reached t_end) or failed since the last poll. */
int mdl_batch_poll(mdl_batch* b, int32_t* done_slots, int32_t cap, int32_t* n);
/* The slot's context (for mdl_read_* / mdl_get_*), state (MDL_SLOT_*) and error code. */
int mdl_batch_slot(mdl_batch* b, int32_t slot, mdl_ctx** ctx, int32_t* state, int32_t* rc);
int mdl_batch_release(mdl_batch* b, int32_t slot);
int mdl_batch_usage(const mdl_batch* b, int64_t* used, int64_t* budget, int32_t* resident);
/* The autotuned sweep shape of prob's class in streams mode (MDL_E_STATE if not tuned yet). */
int mdl_batch_shape(const mdl_batch* b, const mdl_problem* prob, int32_t* threads, int32_t* blocks_per_sm);
/* on != 0: fused rounds (the default); 0: streams. */
int mdl_batch_set_fused(mdl_batch* b, int32_t on);
/* Fused rounds so far and fused sweep kernel launches (rounds, launches: always written);
 * for the group of (precision 32|64, dim 2|3, order 1|2): own = 1 if the tuner chose each
 * slot's own sweep, else the tuned launch shape of the fused kernel (threads per block, due
 * elements per work item); the mean sweep time per round of the fastest and the slowest
 * candidate and of own sweeps, as the tuner measured them (MDL_E_STATE until tuned).  Any
 * output pointer may be NULL. */
int mdl_batch_fused_info(const mdl_batch* b, int32_t precision, int32_t dim, int32_t order, int32_t* own,
                         int32_t* threads, int32_t* tile, double* best_ms, double* worst_ms, double* own_ms,
                         int64_t* rounds, int64_t* launches);
const char* mdl_batch_last_error(const mdl_batch* b);
void mdl_batch_destroy(mdl_batch* b);

/* ---- Allocation-free FP64 integral (the paper has no counterpart; a service for callers) ----
 *
 * Some callers cannot call cudaMalloc: code that runs while a stream is being captured
 * into a CUDA graph, a real-time loop that must not allocate, or a host application whose
 * device memory is fully pre-partitioned by its own allocator.  This entry point computes
 * the same FP64 integral as the barrier diagnostic (mdl_stats.integral_V),
 *   out = sum_e sum_q w_q prod_k (h_k(level_e) / 2) V[e (p+1)^d + q],
 *   h_k(l) = extent[k] / (base[k] 2^l),
 * of a caller-owned device field without allocating anything: its block partials live in
 * a file-scope static device array of MDL_NOALLOC_MAX_PARTIALS doubles (32 KiB) that every
 * GPU which loads the library keeps until the process exits.
 *   V_dev     device pointer, n_e (p+1)^d values, float (precision 32) or double (64)
 *   level_dev device pointer, n_e refinement levels (0..7); a level outside that range makes
 *             the result NaN (the levels are device data: they are checked by the kernel)
 *   out_dev   device pointer to one double, written on `stream`
 *   stream    cudaStream_t (NULL = legacy default stream); the call is asynchronous
 * The first call on a device looks up the array's device address (once per device, with
 * that device current); make that first call before any stream capture begins.  Every
 * call shares the one array: calls whose kernels overlap on a GPU race and give wrong
 * results, so serialise them (one stream, or events).  n_e above MDL_NOALLOC_MAX_ELEMENTS
 * is rejected with MDL_E_ARG; the message is in mdl_noalloc_last_error().  A CUDA error
 * already pending on the calling thread when the call starts is not cleared: the call
 * returns MDL_E_CUDA at once, with its own message, and launches nothing. */
#define MDL_NOALLOC_MAX_PARTIALS 4096
#define MDL_NOALLOC_MAX_ELEMENTS ((int64_t)1 << 30)
int mdl_integral_noalloc(int32_t dim, int32_t order, const double* extent, const int32_t* base,
                         int32_t precision, const void* V_dev, const int8_t* level_dev, int64_t n_e,
                         double* out_dev, void* stream);
const char* mdl_noalloc_last_error(void);

/* Self-test of the bounded device waits (failure detection without a GPU fault).  The
 * tensor-core sweep waits on an mbarrier for its MMAs and the cooperative sweep on a grid
 * barrier between ticks; a wait that runs out of polls records an error and returns, and the
 * stepping call reports MDL_E_TIMEOUT.  This runs one block of the same wait on a phase or a
 * count that nothing completes, on the current device: which = 0 the grid barrier (its
 * production limit, ~1 s), which = 1 the mbarrier wait (2^16 polls).  *status receives the code
 * a stepping call would return (MDL_E_TIMEOUT when the wait gave up as designed), *elapsed_ms
 * (may be null) the host time of the call.  Returns MDL_OK, MDL_E_ARG (which not 0 or 1, null
 * status) or MDL_E_CUDA; the device stays usable. */
int mdl_selftest_wait(int32_t which, int32_t* status, double* elapsed_ms);

#ifdef __cplusplus
}
#endif
#endif /* MDL_H */
