/*
 * mrlt.h -- C-ABI of the GB300 (sm_103a) library for adaptive cell-average
 * multiresolution finite volumes with local time-stepping by natural
 * continuous extension of Runge-Kutta methods (MRLT/NERK), after Lopes,
 * Domingues, Schneider and Mendes, "Local time-stepping for adaptive
 * multiresolution using natural extension of Runge-Kutta methods".
 *
 * One solver instance = one initial-value problem dq/dt = -div F(q) + S(q)
 * (Sec. 2, Eq. 1) on a box in d = 1, 2, 3 dimensions, discretised by finite
 * volumes (Eq. 2) on a dynamically adapted graded tree of nested dyadic grids
 * (Sec. 2) and advanced in time with compact RK2/RK3 stages (Sec. 3) either
 * with one global step (MR/RK) or with level-dependent steps dt_l = 2^{L-l} dt
 * (Eq. 13) synchronised through NERK values (Sec. 4, Algs. 3-9).
 *
 * Conventions for every call:
 *  - The solver owns all of its device memory; it is allocated by mr_create
 *    and released by mr_destroy.  Host buffers passed in are owned by the
 *    caller and only read/written during the call.
 *  - All device work is enqueued on the CUDA stream given to mr_create
 *    (NULL = legacy default stream).  Every call returns after its work has
 *    completed on that stream, except where stated.
 *  - Errors are returned as mr_status; no call aborts the process.  After an
 *    error, mr_last_error(h) gives a human-readable reason.  MR_E_CUDA means
 *    a CUDA runtime call failed; the handle should then be destroyed.
 *  - Not thread-safe per handle; distinct handles are independent.
 */
#ifndef MRLT_H
#define MRLT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mr_solver mr_solver; /* opaque */

typedef enum {
    MR_OK = 0,
    MR_E_INVALID = 1, /* bad argument or configuration                    */
    MR_E_NOMEM = 2,   /* device or host allocation failed                 */
    MR_E_CUDA = 3,    /* a CUDA runtime call failed                       */
    MR_E_TIMEOUT = 4, /* a bounded device wait (grid barrier) gave up      */
    MR_E_STATE = 5,   /* call not valid in the current state, or the tree
                         invariant was found broken on the device          */
    MR_E_NUMERIC = 6  /* a non-finite value appeared in the solution       */
} mr_status;

enum { MR_EQ_ADVECTION = 0, MR_EQ_BURGERS = 1, MR_EQ_EULER = 2, MR_EQ_REACTION_DIFFUSION = 3 };
/* Walls: periodic wrap; homogeneous Neumann (even mirror ghost cells); zero
 * Dirichlet (odd mirror: a ghost takes the negated value; scalar equations
 * only), the same rule on every level. */
enum { MR_BC_PERIODIC = 0, MR_BC_NEUMANN = 1, MR_BC_DIRICHLET0 = 2 };
enum { MR_TIME_GTS = 0, MR_TIME_LT_NERK = 1 };
enum { MR_ADAPT_NEVER = 0, MR_ADAPT_MACRO = 1, MR_ADAPT_EVERY = 2 };
/* Precision.  MR_PREC_MIXED stores the cell averages of every node in FP32
 * and does the stage arithmetic in FP32: exposures and NERK values, MUSCL
 * reconstruction, numerical fluxes, the compact RK updates and the
 * projections.  The conservative flux registers accumulate in FP64 (their
 * correction is rounded to FP32 once), and the detail norms and the
 * threshold test are evaluated in FP64 from the stored values (as are the
 * predictions of new nodes and the CFL reduction).  Host-side data
 * (mr_create, mr_read) stay double in both modes. */
enum { MR_PREC_FP64 = 0, MR_PREC_MIXED = 1 };
/* Numerical flux.  MR_FLUX_AUSM_PLUS (Euler only) is the advection upstream
 * splitting of Liou (1996), the flux the paper uses for its Euler cases
 * (Sec. 5); the default for Euler is HLL. */
enum { MR_FLUX_DEFAULT = 0, MR_FLUX_AUSM_PLUS = 1 };

/* Problem statement (Sec. 2, Eq. 1) and the method's parameters. */
typedef struct mr_config {
    int    dim;        /* d = 1, 2, 3                                               */
    int    equation;   /* MR_EQ_*: advection (centred flux, Sec. 4.5), inviscid
                          Burgers (MUSCL-minmod + Godunov), compressible Euler
                          (MUSCL-minmod on primitives + HLL), reaction-diffusion
                          u_t = D lap u + k u (1-u)(u-a) (two-point diffusion)  */
    int    max_level;  /* L: finest level, 2^L cells per direction (<= 16, d*L <= 30) */
    int    min_level;  /* coarsest leaf level; one macro step = 2^{L-min} fine steps */
    double eps;        /* threshold epsilon of Alg. 2; 0 disables coarsening       */
    int    eps_mode;   /* 0: eps on every level; 1: eps_l = 2^{d (l-L)} eps          */
    int    rk_order;   /* 2 or 3: compact RK2/RK3 of Sec. 3                          */
    int    time_mode;  /* MR_TIME_GTS (all leaves step dt) or MR_TIME_LT_NERK       */
    int    precision;  /* MR_PREC_FP64 or MR_PREC_MIXED                              */
    int    adapt_mode; /* MR_ADAPT_*: never (fixed tree), at each macro-step start,
                          or at every LT iteration on the synchronised levels      */
    int    reflux;     /* 1: conservative flux registers at coarse-fine faces (LT)  */
    double cfl;        /* Courant number sigma                                      */
    double lo[3], hi[3];/* box [lo, hi] per direction (unused entries ignored)      */
    int    bc[3];      /* MR_BC_* per direction                                     */
    double phys[8];    /* advection: a_x, a_y, a_z | Euler: gamma | RD: D, k, a     */
    int    flux;       /* MR_FLUX_DEFAULT (Euler: HLL) or MR_FLUX_AUSM_PLUS (Euler)  */
} mr_config;

/* Create a solver from the finest-level cell averages q0 (host, float64, layout
 * [var][cell], cell = i + 2^L (j + 2^L k), m = d+2 variables for Euler
 * (rho, rho u_1..u_d, E), else 1).  The nodes of all levels are formed by
 * projection (Eq. 3) and, unless adapt_mode == MR_ADAPT_NEVER, the tree is
 * adapted once (Algs. 1-2).  q0 is read only during the call.
 * Memory: each level keeps a status byte, a flag byte, a 4-byte node slot and
 * two 4-byte list entries per cell; the values (8 fields of m variables, and
 * for local time-stepping with reflux the flux registers, one per face) exist
 * only for the nodes of the tree, in node arrays.  A new tree keeps room for
 * every cell until the first macro-step boundary.  From there on (unless the
 * full arrays take at most 32 MB, or the launch mode is MR_LAUNCH_PERSISTENT)
 * the arrays hold 1.25 to 2 times the nodes in use: at each macro-step
 * boundary the first remesh of the macro step is flagged and counted before
 * its tree is installed, and the arrays are resized to fit that tree with a
 * margin; a remesh inside a macro step that would not fit halts the
 * solver's device work, and at the end of the macro step the host grows the
 * arrays and resumes at that remesh, so a growing tree never fails a step
 * while device memory lasts.  Results do not depend on the capacity.
 * Returns MR_E_INVALID for a bad configuration, MR_E_NOMEM when device memory
 * is insufficient: the footprint of the full tree is compared with the free
 * device memory before anything is allocated or q0 is read.  *out receives
 * the handle (NULL on failure). */
mr_status mr_create(const mr_config* cfg, const double* q0_finest, void* cuda_stream,
                    mr_solver** out);

/* Re-initialise an existing solver from new finest-level data (same layout as
 * mr_create): time, counters and tree are reset exactly as mr_create would set
 * them.  Like mr_create it rebuilds the node arrays (full tree, then compact);
 * they come from the library's memory pool, which keeps freed memory cached,
 * so a repeated reset does not call cudaMalloc. */
mr_status mr_reset(mr_solver* h, const double* q0_finest);

/* Replace the tree by a fixed graded tree given, for every finest cell (host,
 * uint8, 2^{dL} entries), the level of the leaf that covers it.  Values of the
 * new leaves are projections or predictions of the current ones (Sec. 2).
 * MR_E_INVALID if the map is not a graded partition into leaves.
 * Only allowed at a macro-step boundary. */
mr_status mr_set_tree(mr_solver* h, const unsigned char* leaf_level_finest);

/* Checkpoint / resume.  At a macro-step boundary every leaf is at the same
 * time t, the flux registers are applied and empty, and internal nodes are
 * projections of the leaves, so the leaves' keys and values (MR_READ_LEAF_KEYS,
 * MR_READ_LEAF_VALUES), t and the fine-iteration count (MR_READ_STATS) are the
 * whole state.  This creates a solver from such a state: keys int32
 * [n_leaves][4] and values double [n_leaves][m] (host, read during the call),
 * cfg as at the original creation.  The run then continues exactly as the
 * original one would (bit for bit on the same GPU).  MR_E_INVALID unless the
 * keys are a graded partition of the box into leaves; MR_E_STATE if iters is
 * not a multiple of the macro step 2^{L-min}.  The paper has no counterpart. */
mr_status mr_create_from_state(const mr_config* cfg, long long n_leaves, const int* keys, const double* values,
                               double t, long long iters, void* cuda_stream, mr_solver** out);

/* Full adaptation (Algs. 1-2) at the current synchronised time. */
mr_status mr_adapt(mr_solver* h);

/* Advance to t_target in whole macro steps of 2^{L-min} fine iterations; the
 * fine step follows the CFL rule once per macro step and the last macro step
 * is shortened to end exactly at t_target.  Must start at a macro-step
 * boundary.  *iters_out (may be NULL) receives the fine iterations done. */
mr_status mr_step(mr_solver* h, double t_target, long long* iters_out);

/* Run n_iters fine iterations (Alg. 3 in LT mode) with the given fine step dt.
 * May stop inside a macro step; dt may change only at a macro-step boundary. */
mr_status mr_iterate(mr_solver* h, double dt, long long n_iters, long long* iters_out);

/* Asynchronous mode (enable = 1): mr_iterate and mr_step return once their
 * work is enqueued on the solver's stream instead of after it has completed
 * (mr_step still waits for each macro step's CFL value, which sets its step;
 * a solver with compact node arrays and adaptation at every fine iteration
 * also waits at the end of each macro step, and of each call, for the check
 * that no remesh ran out of node slots -- see mr_create).
 * Errors found on the device, including the non-finite check after every
 * macro step, are reported by the next mr_sync (or by mr_set_async(h, 0),
 * which synchronises).  MR_E_STATE for an instance of a batch or server. */
mr_status mr_set_async(mr_solver* h, int enable);

/* Wait for all work of the solver and report any error it found. */
mr_status mr_sync(mr_solver* h);

/* Launch shape: at most `ctas` thread blocks per stage-kernel launch (0, the
 * default: the device's resident capacity for the kernel, which fills every
 * SM).  The blocks stride over the active tiles and each cell is written by
 * one thread, so the results are bitwise the same for every value; a smaller
 * grid leaves SMs to concurrent solvers (batches, servers).  Waits for the
 * solver's stream if a captured macro step must be replaced.  MR_E_INVALID
 * for a NULL handle or ctas < 0; MR_E_CUDA if that wait fails.  The paper has
 * no counterpart: it runs one problem on one CPU core. */
mr_status mr_set_grid_cap(mr_solver* h, int ctas);

/* How fine iterations are launched.  MR_LAUNCH_GRAPH (the default) launches
 * one kernel per phase of an iteration (projections, refreshes and stage
 * sweeps per level, the adaptation passes, compaction, reflux; Algs. 3-9),
 * whole macro steps replayed as a CUDA graph; batch instances and served
 * requests always use it, because they run concurrently on their own streams.
 * MR_LAUNCH_PERSISTENT runs the iterations of a macro step in one cooperative
 * launch of a persistent kernel whose CTAs all stay resident, the phases
 * separated by grid-wide barriers instead of kernel boundaries: two launches
 * per macro step instead of thousands.  Both modes run the same device code in
 * the same order; the compiler may contract a different set of multiply-adds
 * in the two kernels, so they agree to FP64 round-off rather than bit for bit.
 * A barrier wait is bounded (4 s): if it gives up, the call returns
 * MR_E_TIMEOUT and the solver should be destroyed.  The persistent kernel
 * installs trees without a host check, so switching to it gives the node
 * arrays room for every cell (MR_E_NOMEM if that does not fit).  Only at a
 * macro-step boundary (MR_E_STATE otherwise).  The paper has no counterpart. */
enum { MR_LAUNCH_PERSISTENT = 0, MR_LAUNCH_GRAPH = 1 };
mr_status mr_set_launch_mode(mr_solver* h, int mode);

/* Self-test of the bounded grid barrier used by MR_LAUNCH_PERSISTENT:
 * launches `ctas` (1..1024) small CTAs that meet at one barrier which expects
 * `missing` more CTAs than exist.  With missing = 0 the barrier completes and
 * the call returns MR_OK; with missing > 0 nobody releases it, every CTA gives
 * up after limit_s seconds (0 < limit_s <= 60), and the call returns
 * MR_E_TIMEOUT with the device still usable.  Allocates and frees 16 bytes of
 * device memory; synchronises cuda_stream.  The paper has no counterpart. */
mr_status mr_selftest_grid_wait(int ctas, int missing, double limit_s, void* cuda_stream);

/* Node arrays of at least `nodes` slots (the arrays are compacted and grown
 * by the capacity rule of mr_create otherwise).  Only at a macro-step boundary
 * (MR_E_STATE otherwise); MR_E_NOMEM if the device memory is insufficient.
 * The paper has no counterpart. */
mr_status mr_reserve_nodes(mr_solver* h, long long nodes);

/* What mr_read returns. */
enum {
    MR_READ_LEAF_KEYS = 0,   /* int32 [n_leaves][4]: level, i, j, k (ordered by
                                level, then cell index)                        */
    MR_READ_LEAF_VALUES = 1, /* double [n_leaves][m], same order, values at the
                                end of each leaf's latest step                 */
    MR_READ_UNIFORM = 2,     /* double [m][2^{dL}]: the adapted solution rebuilt
                                on the finest grid by the inverse MR transform  */
    MR_READ_STATS = 3,       /* double [64]: 0 t, 1 fine iterations, 2 macro steps,
                                3 dt, 4 leaves, 5 nodes, 6 near-threshold details,
                                7 leaf updates, 8..12 mass per variable,
                                13 node slots (capacity), 14 device bytes held,
                                15 position in the macro step, 16+l leaves on level l,
                                61 remeshes that halted to grow the node arrays,
                                62 free node slots */
    MR_READ_PROFILE = 4      /* double [64]: 0 stage-kernel launches timed since
                                mr_profile(h,1), 1 their summed device time (ms),
                                2..4 leaf-stages they processed for stages 1..3,
                                5 kernel launches of any kind in that window,
                                16+l leaf-stages processed on level l (all time),
                                40+l device time (ms) of the timed stage launches
                                on level l */
};

/* Copy a result into the caller's host buffer.  With buf == NULL only *used
 * is set to the size needed; MR_E_INVALID if cap_bytes is too small. */
mr_status mr_read(mr_solver* h, int what, void* buf, size_t cap_bytes, size_t* used);

/* Start (enable=1) or stop (enable=0) timing every stage-kernel launch with a
 * pair of CUDA events on the solver's stream; enabling clears the previous
 * totals.  Results are read with MR_READ_PROFILE.  Timing adds two event
 * records per stage launch and nothing else. */
mr_status mr_profile(mr_solver* h, int enable);

/* Total of every variable over a set of leaves, sum_i q_{i,v} |cell_i|, the
 * same quantity as the mass entries of MR_READ_STATS, for callers that cannot
 * allocate device memory: a process whose GPU memory is fully reserved by
 * another allocator (a caching allocator, a fixed serving budget), or a
 * latency-critical loop that must not pay for cudaMalloc and the device-wide
 * synchronisation it implies.  The paper has no counterpart; it is a utility
 * of this library.
 *   keys_dev   device int32 [n_leaves][4] (level, i, j, k), as MR_READ_LEAF_KEYS
 *   values_dev device float64 [n_leaves][m], as MR_READ_LEAF_VALUES
 *   lo, hi     host double[dim]: the box, |cell| = prod_k (hi_k - lo_k) / 2^{d level}
 *   mass_dev   device float64 [m], written
 *   msg        optional host buffer (msg_cap bytes) for a readable error
 * Limits: 1 <= m <= 5 variables, n_leaves <= INT_MAX; anything else returns
 * MR_E_INVALID with the reason in msg.  The call allocates nothing: its only
 * scratch is a fixed 10 KiB array in the library's device code, present on
 * every GPU that loads the library until the process exits.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress,
 * with the device current), so make the first call on each device before any
 * stream capture.  The looked-up address is cached per device (safely under
 * concurrent first calls from several host threads); a cudaDeviceReset
 * invalidates it, so do not call this after resetting a device in the same
 * process.  Work is only enqueued on cuda_stream: mass_dev is valid once the
 * stream reaches it.  Every call uses the same array, which keeps the previous
 * call's partial sums; calls that overlap on the GPU (other streams or other
 * threads) race on it and must be serialised by the caller. */
mr_status mr_leaf_mass_noalloc(int dim, const double* lo, const double* hi, const int* keys_dev,
                               const double* values_dev, long long n_leaves, int m, double* mass_dev,
                               void* cuda_stream, char* msg, size_t msg_cap);

/* Release everything owned by the handle (NULL is ignored). */
void mr_destroy(mr_solver* h);

/* Reason for the last failure on this handle (static string if h is NULL). */
const char* mr_last_error(const mr_solver* h);

/* Number of kernel launches issued by this handle since creation. */
long long mr_launch_count(const mr_solver* h);

/* Device memory of solvers comes from a library pool per device that keeps
 * freed memory reserved for the next solver (so that creating and destroying
 * solvers never synchronises the device).  This returns the reserved memory
 * that no live solver uses to the device, e.g. before handing the GPU's
 * memory to another allocator.  Memory that destroyed solvers' pending work
 * still uses is released once that work has completed. */
mr_status mr_release_cached_memory(void);

/* ---- Batched instances --------------------------------------------------
 * Many independent problems (each its own configuration, level range and
 * initial data) advanced together.  The paper treats one problem at a time;
 * batching is this library's way of filling a GPU with problems that are
 * each too small for it.  Every instance is an ordinary solver with its own
 * device memory and its own internal CUDA stream; one macro step of an
 * instance is a CUDA graph (captured once per instance), so the instances'
 * kernels overlap on the GPU while the host only picks each instance's CFL
 * step (Sec. 4, Eq. 13) and launches its graph. */
typedef struct mr_batch mr_batch;

/* Create n >= 1 instances from cfgs[i] and the finest-level data q0s[i] (each
 * as for mr_create).  The batch orders its work after the work already
 * enqueued on cuda_stream at each call, and each call returns after all of its
 * work has completed.  On failure nothing is left allocated and *out is NULL;
 * *failed_index (may be NULL) receives the instance that failed, or -1. */
mr_status mr_batch_create(int n, const mr_config* cfgs, const double* const* q0s, void* cuda_stream,
                          mr_batch** out, int* failed_index);

/* Advance every instance to t_target as mr_step does (whole macro steps of its
 * own CFL step, the last shortened), all instances concurrently, each at the
 * pace of its own stream (the host queues an instance's next macro step as
 * soon as its CFL value has arrived).  Every
 * instance must be at a macro-step boundary.  *iters_out (may be NULL)
 * receives the fine iterations done, summed over instances.  On an error the
 * failing instance is reported by mr_batch_last_error. */
mr_status mr_batch_step(mr_batch* b, double t_target, long long* iters_out);

/* mr_set_grid_cap on every instance: the stage-kernel launches of each
 * instance use at most `ctas` thread blocks, so that more instances run on the
 * GPU at once.  Results are unchanged.  Call between steps.  MR_E_INVALID for
 * a NULL batch or ctas < 0; otherwise the first failing instance's status,
 * named by mr_batch_last_error. */
mr_status mr_batch_set_grid_cap(mr_batch* b, int ctas);

/* Instance i (0 <= i < n), owned by the batch: use it with mr_read,
 * mr_last_error and mr_launch_count; NULL if i is out of range.  Do not destroy
 * it, and do not step it while the batch is stepping. */
mr_solver* mr_batch_instance(mr_batch* b, int i);

/* Reason for the last failure of a batch call. */
const char* mr_batch_last_error(const mr_batch* b);

/* Release the batch and all its instances (NULL is ignored). */
void mr_batch_destroy(mr_batch* b);

/* ---- Serving -------------------------------------------------------------
 * Problems that arrive over time, each with its own end time, served by
 * continuous batching: every admitted problem advances by whole macro steps
 * at the pace of its own stream (as in mr_batch_step); queued problems join
 * at macro-step boundaries, first come first served, while their
 * device footprint fits the memory budget and fewer than max_active problems
 * are in flight; a problem leaves when it reaches its end time.  The paper has
 * no counterpart.  A request is admitted by its projected footprint: the
 * per-cell arrays plus node arrays for a projected node count, which models an
 * adapted tree as fronts of codimension one, min(all cells, 64 x 2^{(d-1) L})
 * nodes with the compact margin of mr_create; once created, the request counts
 * the larger of that and its actual footprint, which is the full tree until
 * its first macro-step boundary and compact from there on.  Results stay on
 * the device until released. */
typedef struct mr_server mr_server;

/* mem_budget_bytes: device bytes all admitted problems may hold together;
 * max_active >= 1: problems in flight at once.  Work is ordered after the
 * work on cuda_stream at creation. */
mr_status mr_server_create(size_t mem_budget_bytes, int max_active, void* cuda_stream, mr_server** out);

/* Queue a problem (cfg and finest data q0 as for mr_create; q0 is copied) to
 * be advanced from t = 0 to t_end.  *id receives its request id.  MR_E_NOMEM
 * if the problem alone exceeds the budget, MR_E_INVALID for a bad config. */
mr_status mr_server_submit(mr_server* s, const mr_config* cfg, const double* q0, double t_end, long long* id);

/* Admit what fits, then queue the next macro step of every active problem
 * whose previous one has completed.  Never waits for the GPU: call it in a
 * loop.  *n_active (problems admitted and not yet reported) and *n_queued
 * may be NULL. */
mr_status mr_server_advance(mr_server* s, int* n_active, int* n_queued);

/* Ids of up to cap problems that finished since the last poll (in the order
 * they were found finished); *n_done receives how many were written. */
mr_status mr_server_poll(mr_server* s, long long* ids, int cap, int* n_done);

/* Outcome of a finished request (MR_E_STATE while it is not finished,
 * MR_E_INVALID for an unknown id). */
mr_status mr_server_status(mr_server* s, long long id);

/* The solver of a finished request, for mr_read; NULL otherwise.  Owned by the
 * server until mr_server_release. */
mr_solver* mr_server_result(mr_server* s, long long id);

/* Free a finished request and its device memory. */
mr_status mr_server_release(mr_server* s, long long id);

/* Device bytes held by admitted, not yet released requests. */
size_t mr_server_memory(const mr_server* s);

/* mr_set_grid_cap for every request admitted after this call (requests
 * already running keep their launch shape).  Results are unchanged.
 * MR_E_INVALID for a NULL server or ctas < 0. */
mr_status mr_server_set_grid_cap(mr_server* s, int ctas);

/* Reason for the last failure of a server call. */
const char* mr_server_last_error(const mr_server* s);

/* Release the server and every request it holds (NULL is ignored). */
void mr_server_destroy(mr_server* s);

#ifdef __cplusplus
}
#endif
#endif
