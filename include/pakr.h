/*
 * pakr.h -- C ABI of the GB300 PAKR planner.
 *
 * PAKR (Parallel Asymptotically Optimal Kinodynamic RRT) grows a kinodynamic
 * RRT in batches and wraps it in the AO-x meta-algorithm (Algorithm 1 of
 * "Fast Asymptotically Optimal Kinodynamic Planning via Vectorization").  This
 * library runs one batched expansion iteration (SampleStates, cost-pruned
 * NearestNeighbor, SampleControls, RK4 Propagate with a collision check at
 * every substep, goal test, insert) as hand-written sm_103a CUDA kernels, and
 * the AO-x loop as a device-resident CUDA graph.
 *
 * Conventions for every entry point:
 *  - Host pointers are plain host memory; the library copies what it keeps.
 *  - Device memory is either allocated by the library (cudaMalloc) or carved
 *    from a caller buffer given in pakr_problem_desc.workspace.
 *  - Every call returns a pakr_status; nothing is thrown or aborted across the
 *    ABI.  A negative status is an error; pakr_last_error() returns a message
 *    for the calling thread.
 *  - Work is queued on the CUDA stream given at create (NULL = the legacy
 *    default stream).  Calls that return data to host buffers synchronise
 *    that stream; the others only enqueue.
 *  - A planner is not thread-safe: one host thread drives it at a time.
 *
 * Layout on the device (Sec. IV-A "structure of arrays"): the tree is stored
 * dimension-major, states[k * cap + i] for state coordinate k of node i, with
 * controls, parent indices, costs-to-come, cached f-costs and edge durations in
 * their own arrays, and a device-resident node counter.
 */
#ifndef PAKR_H
#define PAKR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  Non-negative values are outcomes, negative values errors. */
typedef enum pakr_status {
    PAKR_OK = 0,                /* the call did its work */
    PAKR_GOAL_REACHED = 1,      /* an appended child lies in the goal region (Algorithm 1, goal test) */
    PAKR_TREE_FULL = 2,         /* some surviving children did not fit under tree_cap and were dropped */
    PAKR_NO_ELIGIBLE = 3,       /* no tree node has f-cost below the bound; nothing was expanded */
    PAKR_BUDGET_EXPIRED = 4,    /* pakr_plan ran out of time / iterations without any solution */
    PAKR_ERR_INVALID_ARG = -1,  /* a bad argument (NULL, out of range, NaN, inconsistent sizes) */
    PAKR_ERR_CUDA = -2,         /* a CUDA runtime call failed; the message names it */
    PAKR_ERR_OOM = -3,          /* device allocation failed or the workspace is too small */
    PAKR_ERR_TIMEOUT = -4,      /* a bounded device wait gave up */
    PAKR_ERR_UNIMPLEMENTED = -5,/* the requested combination is not built */
    PAKR_ERR_DEVICE = -6        /* a kernel reported an internal consistency failure */
} pakr_status;

/* System dynamics x' = f(x, u) (Eq. 1).  State / control / position sizes:
 *   PAKR_DI2       planar double integrator [x,y,vx,vy] / [ax,ay]         d=4  m=2 p=2
 *   PAKR_DI3       double integrator [x,y,z,vx,vy,vz] / [ax,ay,az]        d=6  m=3 p=3  (Sec. V-A item 1)
 *   PAKR_QUAD12    quadcopter [x,y,z,phi,theta,psi,u,v,w,p,q,r] /
 *                  [thrust, tau_x, tau_y, tau_z], body-frame velocities   d=12 m=4 p=3  (Sec. V-A item 3)
 *   PAKR_DUBINS3D  Dubins airplane [x,y,z,yaw,pitch,v] / [yaw', pitch', v'] d=6 m=3 p=3 (Sec. V-A item 2)
 *   PAKR_UNICYCLE1 [x,y,theta] / [v,omega]                                 d=3  m=2 p=2  (Sec. V-C item 1)
 *   PAKR_UNICYCLE2 [x,y,theta,v,omega] / [a,alpha]                         d=5  m=2 p=2  (Sec. V-C item 2)
 * The first p state coordinates are the position used by obstacles, goal and
 * path-length cost. */
typedef enum pakr_dynamics {
    PAKR_DI2 = 0,
    PAKR_DI3 = 1,
    PAKR_QUAD12 = 2,
    PAKR_DUBINS3D = 3,
    PAKR_UNICYCLE1 = 4,
    PAKR_UNICYCLE2 = 5
} pakr_dynamics;

/* Trajectory cost J (Sec. III: additive, e.g. path length or duration). */
typedef enum pakr_cost {
    PAKR_COST_PATH_LENGTH = 0,  /* sum over substeps of |p_s - p_{s-1}| */
    PAKR_COST_DURATION = 1      /* substeps * dt */
} pakr_cost;

/* Heuristic h of the f-cost f = g + h used by the cost-bounded pruning (Sec. IV). */
typedef enum pakr_heuristic {
    PAKR_H_POSITION = 0,        /* max(0, |p - p_goal| - r_goal); divided by heuristic_speed for duration cost */
    PAKR_H_FULLSTATE = 1        /* |x - x_goal| over the whole state, the formula as printed in Sec. IV */
} pakr_heuristic;

/* Per-rollout outcome of the last expansion (pakr_debug_last_expand). */
/* Nearest-neighbour kernel choice.  Both give the same result (the exact FP32
 * argmin, lowest index on a tie).  The tensor-core kernel needs a packed
 * FP16 operand copy of the tree: 2 * (2d + 2 rounded up to 16) bytes per node for
 * d = 5, 6 and 12, and 2 * (3d + 2 rounded up to 16) for d = 3 and 4. */
typedef enum pakr_nn_mode {
    PAKR_NN_AUTO = 0,           /* tensor cores for trees of >= 28672 nodes when n_parents >= 256, FP32 otherwise */
    PAKR_NN_FP32 = 1,           /* FP32 kernel only; no packed copy is kept */
    PAKR_NN_TENSOR = 2          /* tensor-core kernel at every tree size */
} pakr_nn_mode;

typedef enum pakr_outcome {
    PAKR_ROLLOUT_APPENDED = 0,  /* inserted into the tree */
    PAKR_ROLLOUT_PRUNED = 1,    /* f-cost not below the bound */
    PAKR_ROLLOUT_COLLIDED = 2,  /* some substep left the state box or entered an obstacle */
    PAKR_ROLLOUT_NO_PARENT = 3, /* no eligible parent */
    PAKR_ROLLOUT_DROPPED = 4    /* survived but the tree was full */
} pakr_outcome;

/* Problem and batch description (Sec. III problem statement; Algorithm 1
 * inputs: batch size B = n_parents * branching, branching factor A).
 * All host arrays are read during pakr_create only. */
typedef struct pakr_problem_desc {
    int32_t dynamics;           /* pakr_dynamics */
    const float *x_lo, *x_hi;   /* d each: closed state box; a state outside it is invalid */
    const float *u_lo, *u_hi;   /* m each: control box sampled uniformly */
    float dt;                   /* RK4 step (s), > 0 */
    int32_t steps_min, steps_max; /* control held for a uniform number of substeps in [min, max], 1 <= min <= max */
    int32_t n_boxes;            /* >= 0 */
    const float *boxes;         /* n_boxes x (lo[p], hi[p]); a position inside a closed box is invalid */
    int32_t n_spheres;          /* >= 0 */
    const float *spheres;       /* n_spheres x (c[p], r); a position inside a closed ball is invalid */
    float goal_radius;          /* goal region: closed ball of this radius around the goal position */
    int32_t cost;               /* pakr_cost */
    int32_t heuristic;          /* pakr_heuristic */
    float heuristic_speed;      /* speed bound for PAKR_COST_DURATION with PAKR_H_POSITION; <= 0 gives h = 0 */
    const float *nn_weights;    /* d per-coordinate weights of the squared NN distance, NULL = all ones */
    const float *model_params;  /* PAKR_QUAD12: mass, Ixx, Iyy, Izz, g; NULL = 1, 0.01, 0.01, 0.02, 9.81 */
    int32_t n_parents;          /* K = nearest-neighbour queries per iteration, >= 1 */
    int32_t branching;          /* A = controls propagated per parent, >= 1 */
    int64_t tree_cap;           /* N = maximum tree size, >= 1, <= 2^31 - 2^20 (32-bit node indices with room
                                   for the kernels' rounding of node chunks and tiles) */
    int32_t device;             /* CUDA device ordinal */
    void *cuda_stream;          /* cudaStream_t to queue work on; NULL = default stream */
    void *workspace;            /* optional device buffer the library carves all its memory from; NULL = cudaMalloc */
    uint64_t workspace_bytes;   /* size of workspace; see pakr_workspace_size */
    int32_t path_cap;           /* maximum solution path length in edges kept on the device; 0 = 4096 */
    int32_t history_cap;        /* maximum AO-x solutions recorded per plan; 0 = 1024 */
    int32_t nn_mode;            /* pakr_nn_mode */
} pakr_problem_desc;

typedef struct pakr_planner pakr_planner;

/* Result of one expansion.  Filled only when the caller passes a pointer. */
typedef struct pakr_expand_info {
    int64_t n_start;            /* tree size the batch saw (the frozen snapshot, Sec. IV-B) */
    int64_t n_appended;
    int64_t n_pruned;
    int64_t n_collided;
    int64_t n_no_parent;
    int64_t n_dropped;
    int32_t goal_found;
    int32_t reserved;
    int64_t goal_idx;           /* cheapest appended goal child (lowest index on a tie), -1 if none */
    float goal_cost;            /* its cost-to-come */
    uint32_t iteration;         /* expansion counter value this batch used (Philox counter word 0) */
} pakr_expand_info;

/* Tree snapshot in host memory, node-major rows.  Caller-owned buffers. */
typedef struct pakr_tree_host {
    int64_t capacity;           /* rows available in each array */
    int64_t count;              /* nodes (out for export, in for import) */
    uint32_t iteration;         /* expansion counter */
    float *states;              /* capacity x d */
    float *controls;            /* capacity x m (row 0, the root, is zero) */
    int32_t *parents;           /* capacity; root = -1 */
    float *costs;               /* capacity; cost-to-come */
    int32_t *steps;             /* capacity; substeps of the edge into each node */
} pakr_tree_host;

/* Best path and AO-x history of pakr_plan.  Caller-owned buffers with
 * capacities; outputs after the separator. */
typedef struct pakr_path {
    int32_t max_edges;          /* capacity of controls / steps; states holds max_edges + 1 rows */
    float *states;              /* (n_edges + 1) x d, root first */
    float *controls;            /* n_edges x m */
    int32_t *steps;             /* n_edges */
    int32_t max_history;        /* capacity of the history arrays */
    double *history_time_s;     /* device time of each solution since the plan started */
    float *history_cost;        /* c_best after each solution (strictly decreasing) */
    int64_t *history_iteration; /* expansion iteration of each solution */
    /* ---- outputs ---- */
    int32_t n_edges;            /* edges of the best path; if it exceeds max_edges nothing is copied */
    float cost;                 /* best cost found (c_best), +inf if none */
    int32_t n_solutions;        /* AO-x solutions found */
    int32_t n_restarts;         /* fresh trees started because the tree filled without a solution */
    double t_first_solution_s;  /* device time to the first solution, < 0 if none */
    double t_total_s;           /* device time of the whole plan */
    int64_t iterations;         /* expansion iterations run */
    int64_t nodes_first_solution;      /* tree size when the first solution was found, -1 if none */
    int64_t iterations_first_solution; /* expansion iterations up to the first solution, -1 if none */
} pakr_path;

/* Plan flags. */
#define PAKR_PLAN_STOP_AT_FIRST 1u  /* return after the first solution (no AO-x refinement) */

/* Bytes of device memory the planner needs for this description (tree, batch
 * workspace, path / history buffers).  Does not touch the GPU. */
pakr_status pakr_workspace_size(const pakr_problem_desc *desc, uint64_t *bytes_out);

/* Validate the description, copy its host arrays, take device memory and build
 * the kernels' launch configuration.  *out receives the planner (NULL on
 * error).  The tree starts empty; call pakr_tree_reset or pakr_tree_import
 * before pakr_expand. */
pakr_status pakr_create(const pakr_problem_desc *desc, pakr_planner **out);

/* Release device memory the library allocated, graphs and events.  A NULL
 * planner is ignored. */
void pakr_destroy(pakr_planner *planner);

/* Message for the last error of the calling thread ("" if none). */
const char *pakr_last_error(void);

/* T <- {(x_init, -, 0)} (Algorithm 1, fresh tree): one root node with cost 0,
 * the expansion counter set to 0, and the goal set to x_goal (d floats; its
 * position is the centre of the goal ball, the whole state is the target of
 * PAKR_H_FULLSTATE).  Synchronises the stream.  Returns
 * PAKR_ERR_INVALID_ARG if x_init is not a valid state. */
pakr_status pakr_tree_reset(pakr_planner *planner, const float *x_init, const float *x_goal);

/* One batched expansion iteration (Algorithm 1 inner loop body):
 *   1. SampleStates: n_parents states uniform in the state box, Philox4x32-10
 *      keyed by seed with counter (iteration, i, 0xFFFFFFFF, block);
 *   2. NearestNeighbor: for each sample the nearest node among those present at
 *      the start of the call whose f-cost is below cost_bound (lowest index on
 *      a tie of the FP32 squared distance);
 *   3. SampleControls: branching controls per parent, uniform in the control
 *      box, and a duration in [steps_min, steps_max], counter (iteration, i, j, block);
 *   4. Propagate: RK4 with step dt for that many substeps, validity checked at
 *      every substep;
 *   5. prune children with f = g + h not below cost_bound (strict), drop
 *      invalid ones, append the rest in ascending rollout order i*branching+j
 *      (truncated at tree_cap), test the goal, and advance the counter.
 * cost_bound may be +inf.  If info is NULL the call only enqueues the kernels
 * and returns PAKR_OK; otherwise it synchronises the stream, fills *info and
 * returns PAKR_NO_ELIGIBLE, PAKR_GOAL_REACHED, PAKR_TREE_FULL or PAKR_OK (in
 * that order of precedence). */
pakr_status pakr_expand(pakr_planner *planner, float cost_bound, uint64_t seed, pakr_expand_info *info);

/* Algorithm 1 in full: AO-x replanning from x_init towards the goal ball
 * around x_goal until budget_s of device time has passed or max_iterations
 * expansion iterations have run (<= 0, or above 10^7: 10^7, a hard bound on the device loop).  c_best starts at
 * +inf; each solution sets c_best to its cost, records it, extracts its path
 * and restarts from a fresh tree, so c_best strictly decreases.  A tree that
 * fills without a solution is restarted; a bound no node can beat ends the run.
 * The loop runs on the device as one CUDA graph with a conditional while node
 * (no host round trip per iteration).  Synchronises the stream and fills *out.
 * Returns PAKR_GOAL_REACHED if any solution was found, else
 * PAKR_BUDGET_EXPIRED (or PAKR_NO_ELIGIBLE); PAKR_ERR_INVALID_ARG for an
 * invalid start or a path longer than out->max_edges (out->n_edges then holds
 * the required size). */
pakr_status pakr_plan(pakr_planner *planner, const float *x_init, const float *x_goal, double budget_s,
                      int64_t max_iterations, uint64_t seed, uint32_t flags, pakr_path *out);

/* pakr_plan starting from c_best = initial_bound instead of +inf: only
 * solutions cheaper than the bound are found (AO-x continued from an earlier
 * or refined solution).  initial_bound = +inf is pakr_plan. */
pakr_status pakr_plan_bounded(pakr_planner *planner, const float *x_init, const float *x_goal, double budget_s,
                              int64_t max_iterations, uint64_t seed, uint32_t flags, float initial_bound,
                              pakr_path *out);

/* Lower the AO-x bound c_best of a pakr_plan / pakr_plan_bounded run that is
 * in progress on this planner to *cost_dev (device memory, one float read on
 * the device) if that is smaller: AO-x continued from a cheaper path found
 * outside the loop, such as a gradient-refined path (the paper has no
 * counterpart; the loop itself is Algorithm 1).  Only enqueues one small
 * kernel on cuda_stream (NULL = default stream), which should be another
 * stream than the planner's, so that it runs while the plan's graph runs; the
 * loop picks the bound up at its next iteration: an offer that lowers the bound
 * counts as a new solution of the loop, which restarts its tree from the root
 * with the lower bound, as after one of its own (Algorithm 1; the restart is
 * not counted in pakr_path.n_restarts).  It may be made from another
 * host thread while pakr_plan runs on this planner.
 * The kernel's GPU code is loaded at pakr_create, so the call loads nothing
 * (a first, lazy load could wait for the running plan); the caller should
 * likewise allocate cost_dev, and launch once any kernel of its own that
 * writes it, before the plan starts.  An offer that lands before the plan's first iteration is
 * overwritten by its start (pass such a bound as initial_bound instead); one that lands
 * after the plan ended is kept until the next plan starts.  A non-finite or
 * negative cost is ignored.  pakr_path.cost stays the cost of the run's own
 * best path.  PAKR_ERR_INVALID_ARG for NULL arguments.  Besides
 * pakr_plan_snapshot, this is the one call that may be made while the plan
 * runs. */
pakr_status pakr_plan_offer_bound(pakr_planner *planner, const float *cost_dev, void *cuda_stream);

/* Copy the current best path of a pakr_plan / pakr_plan_bounded run on this
 * planner, which may still be running, into caller device buffers: states
 * ((n_edges + 1) x d), controls (n_edges x m), steps (n_edges), capacities
 * for max_edges edges, and info (4 int32): info[0] = 1 if the copy is one
 * whole path (0 if there is none yet, it has more than max_edges edges, or a
 * newer path replaced it while it was copied: the AO-x step marks the path's
 * rows as being written with a sequence number), info[1] = n_edges,
 * info[2] = the sequence number (it grows with every new best path of the
 * run), info[3] = the path's cost as float bits.  For refining AO-x solutions
 * beside the running loop (the paper has no counterpart).  Only enqueues one
 * small kernel on cuda_stream (another stream than the planner's, so that it
 * runs while the plan does); like pakr_plan_offer_bound it may be called from
 * another host thread while the plan runs, its code is loaded at pakr_create,
 * and the caller's buffers should exist before the plan starts.
 * PAKR_ERR_INVALID_ARG for NULL buffers or max_edges < 1. */
pakr_status pakr_plan_snapshot(pakr_planner *planner, float *states_dev, float *controls_dev, int32_t *steps_dev,
                               int32_t max_edges, int32_t *info_dev, void *cuda_stream);

/* Current node count of the tree (and the expansion counter, if iteration is
 * not NULL).  Synchronises the stream; reads two words, not the tree.
 * PAKR_ERR_INVALID_ARG if planner or count is NULL. */
pakr_status pakr_tree_size(pakr_planner *planner, int64_t *count, uint32_t *iteration);

/* Copy the tree to host memory (node-major).  Synchronises the stream.
 * PAKR_ERR_INVALID_ARG if tree->capacity < the node count (tree->count then
 * holds the count). */
pakr_status pakr_tree_export(pakr_planner *planner, pakr_tree_host *tree);

/* Keep only the first count nodes of the tree (1 <= count <= tree_cap; a
 * count above the current size leaves the tree unchanged).  The expansion
 * counter is not touched.  Only enqueues a one-thread kernel. */
pakr_status pakr_tree_truncate(pakr_planner *planner, int64_t count);

/* Replace the tree with a host snapshot (for resuming AO-x runs and parity
 * checks) and set the goal to x_goal; f-costs are recomputed on the device.
 * Synchronises the stream.  PAKR_ERR_INVALID_ARG if count is outside
 * [1, tree_cap] or a parent index is not smaller than its node's index. */
pakr_status pakr_tree_import(pakr_planner *planner, const pakr_tree_host *tree, const float *x_goal);

/* Per-query and per-rollout records of the last pakr_expand, for parity
 * checks: samples (n_parents x d, node-major), near (n_parents nearest-node
 * indices, -1 if none), outcome (R = n_parents*branching pakr_outcome codes),
 * goal (R flags: 1 if the rollout's child survived the prune and the
 * validity checks -- appended or dropped at a full tree -- and its end
 * position lies in the goal ball, Algorithm 1 goal test; 0 otherwise),
 * controls (R x m) and steps (R).  Any pointer may be NULL.  Synchronises. */
pakr_status pakr_debug_last_expand(pakr_planner *planner, float *samples, int32_t *near, int8_t *outcome,
                                   int8_t *goal, float *controls, int32_t *steps);

/* Per-kernel device time accumulated since profiling was last enabled, in
 * milliseconds, measured with CUDA events on the planner's stream around each
 * launch.  pakr_set_profiling(p, 1) clears and starts, 0 stops.  names_out
 * (optional) receives a static string per slot.  Slots: 0 sample, 1 nearest
 * neighbour (FP32 kernel), 2 propagate, 3 append, 4 nearest neighbour (tensor-core
 * kernel).  launches_out counts launches per slot.  While profiling, pakr_expand
 * launches its kernels one by one (both nearest-neighbour kernels, the one not
 * taken returning at once); otherwise it launches one CUDA graph per expansion. */
pakr_status pakr_set_profiling(pakr_planner *planner, int32_t enable);
pakr_status pakr_kernel_times(pakr_planner *planner, double *ms_out, int64_t *launches_out, const char **names_out,
                              int32_t n_slots);

/* Device-side Philox4x32-10 (Salmon et al., SC'11) for n counters: out[4*t..]
 * = Philox(ctr[4*t..], key).  Host buffers; synchronises.  Exposes the
 * generator the kernels use so that it can be checked word for word. */
pakr_status pakr_philox4x32_10(pakr_planner *planner, const uint32_t *ctr, const uint32_t key[2], uint32_t *out,
                               int64_t n);

/* ---------------------------------------------------------------------------
 * Batched planning: many independent queries, one persistent launch.
 *
 * Each query is a full Algorithm 1 run (its own tree, c_best and AO-x state)
 * with its own start, goal, obstacles and tree cap; dynamics, bounds, step,
 * durations, goal radius, cost, heuristic, K and A are shared.  One
 * cooperative kernel runs every query's expansions phase by phase
 * (SampleStates, NearestNeighbor, Propagate, insert, AO-x step) with
 * grid-wide barriers in between, spreading each phase's work items over all
 * SMs; the launch is captured once into a CUDA graph.  Query q seeds its
 * Philox stream with seed + q.
 * ------------------------------------------------------------------------- */
typedef struct pakr_batch pakr_batch;

typedef struct pakr_batch_query {
    const float *x_init;        /* d */
    const float *x_goal;        /* d */
    int32_t n_boxes;
    const float *boxes;         /* n_boxes x (lo[p], hi[p]) */
    int32_t n_spheres;
    const float *spheres;       /* n_spheres x (c[p], r) */
    int64_t tree_cap;           /* >= 1, <= 2^31 - 2^20 */
} pakr_batch_query;

/* Launch shape of the persistent kernel: threads per block (128 or 256; a
 * nearest-neighbour work item covers 4 x block_threads queries) and tree
 * nodes per nearest-neighbour work item (a multiple of 8, >= 64). */
typedef struct pakr_batch_tuning {
    int32_t block_threads;
    int32_t nn_chunk;
    /* outputs of pakr_batch_autotune */
    int32_t n_tried;
    double best_ms;             /* time of the chosen shape on the tuning run */
} pakr_batch_tuning;

typedef struct pakr_batch_result {
    int32_t status;             /* PAKR_GOAL_REACHED, PAKR_BUDGET_EXPIRED, PAKR_NO_ELIGIBLE or PAKR_ERR_INVALID_ARG (bad start) */
    int32_t n_solutions;
    float cost;                 /* best cost, +inf if none */
    int32_t n_edges;            /* edges of the best path (-1 if it exceeded path_cap) */
    int64_t iterations;         /* expansion iterations of this query */
    double t_first_solution_s;  /* device time to the first solution, < 0 if none */
    int32_t n_restarts;
    int32_t reserved;
    int64_t nodes_first_solution;      /* tree size when the first solution was found, -1 if none */
    int64_t iterations_first_solution; /* expansion iterations up to the first solution, -1 if none */
} pakr_batch_result;

/* base: the shared problem (its obstacles and tree_cap are ignored; path_cap
 * bounds each query's stored best path, 0 = 1024).  queries: n_queries
 * entries, copied.  Allocates device memory for every query's tree. */
pakr_status pakr_batch_create(const pakr_problem_desc *base, const pakr_batch_query *queries, int32_t n_queries,
                              pakr_batch **out);
void pakr_batch_destroy(pakr_batch *batch);

/* Run every query's AO-x loop (as pakr_plan, flags PAKR_PLAN_STOP_AT_FIRST
 * allowed) in one graph launch; results holds n_queries entries.
 * Synchronises the stream.  Returns PAKR_OK when the launch completed. */
pakr_status pakr_batch_plan(pakr_batch *batch, double budget_s, int64_t max_iterations, uint64_t seed, uint32_t flags,
                            pakr_batch_result *results);

/* Best path of query q after pakr_batch_plan (rows as in pakr_path). */
pakr_status pakr_batch_path(pakr_batch *batch, int32_t query, float *states, float *controls, int32_t *steps,
                            int32_t max_edges);

/* Launch-shape autotuner: times pakr_batch_plan with every candidate shape
 * (block_threads in {128, 256} x nn_chunk in {512, 1024, 2048, 4096, 8192})
 * for `iterations` expansion iterations per query without stopping at
 * solutions, keeps the fastest, and reports it. */
pakr_status pakr_batch_autotune(pakr_batch *batch, int64_t iterations, uint64_t seed, pakr_batch_tuning *out);

/* Set the launch shape directly (for example, a cached autotuner result). */
pakr_status pakr_batch_set_tuning(pakr_batch *batch, const pakr_batch_tuning *tuning);

/* ---------------------------------------------------------------------------
 * Smooth trajectory cost and its gradient (adjoint RK4), for refining AO-x
 * solutions by gradient descent.  The paper has no counterpart: it is a
 * refinement step around Algorithm 1, not part of it.
 *
 * A trajectory t starts at x0[t*d..] and applies control
 * controls[(t*n_steps + n)*m + j] during RK4 step n (n = 0..n_steps-1) of the
 * planner's dt.  Cost
 *   J = w_duration n_steps dt + w_control sum_n |u_n|^2 dt
 *     + w_obstacle sum_{n=1..N} sum_obstacles softplus_beta(margin - sdf(p_n)) dt
 *     + w_goal |p_N - p_goal|^2 + w_length sum_n sqrt(|p_{n+1} - p_n|^2 + length_eps^2)
 * with softplus_beta(z) = log(1 + exp(beta z)) / beta, the exact box signed
 * distance and |p - c| - r for spheres, over the planner's obstacles.  The
 * duration term is constant in the controls (the step count is fixed).
 * All arrays are device memory; x_goal is host memory (d floats).  The calls
 * enqueue on the planner's stream.
 * ------------------------------------------------------------------------- */
typedef struct pakr_traj_params {
    float w_duration, w_control, w_obstacle, beta, margin, w_goal, w_length, length_eps;
} pakr_traj_params;

/* cost[t] (and x_final[t*d..] if not NULL) for n_traj trajectories. */
pakr_status pakr_traj_cost(pakr_planner *planner, const float *x0, const float *controls, int32_t n_traj,
                           int32_t n_steps, const float *x_goal, const pakr_traj_params *params, float *cost,
                           float *x_final);

/* controls_grad = cost_grad[t] * dJ_t/dU (cost_grad NULL = 1) and, if not
 * NULL, x0_grad = cost_grad[t] * dJ_t/dx0, by a forward sweep that keeps the
 * state every 16 steps in checkpoints (pakr_traj_checkpoint_floats floats,
 * caller-owned device scratch) and a backward sweep that recomputes each
 * 16-step segment and pulls the adjoint back through every RK4 stage. */
pakr_status pakr_traj_grad(pakr_planner *planner, const float *x0, const float *controls, int32_t n_traj,
                           int32_t n_steps, const float *x_goal, const pakr_traj_params *params,
                           const float *cost_grad, float *controls_grad, float *x0_grad, float *checkpoints);

/* Size in floats of the checkpoint scratch pakr_traj_grad needs (-1 on a bad argument). */
int64_t pakr_traj_checkpoint_floats(const pakr_planner *planner, int32_t n_traj, int32_t n_steps);

/* The planner's rules on control sequences: valid[t] = 1 if every state after
 * a step lies in the state box and no obstacle; in_goal[t] = 1 if the final
 * position lies in the goal ball; path_length[t] = sum of |p_{n+1} - p_n|.
 * in_goal, path_length and x_final may be NULL. */
pakr_status pakr_traj_check(pakr_planner *planner, const float *x0, const float *controls, int32_t n_traj,
                            int32_t n_steps, const float *x_goal, int32_t *valid, int32_t *in_goal,
                            float *path_length, float *x_final);

/* Refinement of one path by projected gradient steps on its per-edge controls,
 * in one kernel launch (a 64-thread CTA, small enough to run beside the
 * search kernels of a plan on another stream).  A refinement step of the
 * AO-x solutions, not a step of the paper's method.
 *   x0             device, d floats: the path's start state;
 *   edge_controls  device, n_edges x m floats, row-major: the control of each
 *                  edge, updated in place when a shorter path is accepted;
 *   steps          device, n_edges int32: RK4 steps of each edge, summing to
 *                  n_steps (the step counts stay fixed);
 *   x_goal         host, d floats; params: the smooth cost whose gradient
 *                  gives the descent direction (as pakr_traj_cost);
 *   iters          iterations; each takes the gradient of the cost with
 *                  respect to the edge controls, normalises it to d, tries the
 *                  n_candidates (1..32) candidates clamp(u - step 2^-c d,
 *                  u_lo, u_hi), c = 0, 1, ..., and keeps the shortest one (the
 *                  lowest c on a tie) that the planner's rules accept (valid
 *                  after every step as pakr_traj_check, the end in the goal
 *                  ball and within goal_radius * (1 - goal_margin) of the
 *                  goal), if it is shorter than the current path;
 *   scratch        device, pakr_traj_refine_scratch_floats floats, caller-owned;
 *   lengths        device, 2 floats: the starting path length (+inf if the
 *                  start is not accepted) and the final one; both NaN if the
 *                  step counts are negative or do not sum to n_steps.
 * Enqueues on the planner's stream; nothing is read back to the host. */
pakr_status pakr_traj_refine(pakr_planner *planner, const float *x0, float *edge_controls, const int32_t *steps,
                             int32_t n_edges, int32_t n_steps, const float *x_goal, const pakr_traj_params *params,
                             int32_t iters, int32_t n_candidates, float step, float goal_margin, float *scratch,
                             float *lengths);

/* Size in floats of the scratch pakr_traj_refine needs (-1 on a bad argument). */
int64_t pakr_traj_refine_scratch_floats(const pakr_planner *planner, int32_t n_edges, int32_t n_steps);

/* Cost-pruned nearest neighbour that allocates no device memory.
 *
 * The paper has no counterpart of this call: it exists for callers that
 * cannot allocate device memory where they need the search, such as
 * real-time loops that forbid allocation (and the device-wide
 * synchronisation cudaFree can bring) after start-up, or plugins confined to
 * another framework's memory pool.  It runs the same search kernel as
 * pakr_expand's NearestNeighbor step, but its per-query scratch lives in one
 * static device array built into the library (about 512 KB, held on every
 * GPU that loads the library until the process exits) instead of planner
 * memory.
 *
 * For each query i it writes nearest[i] = the index j < n with fcost[j] <
 * bound that minimises the FP32 squared distance sum_k (queries[k*n_queries +
 * i] - states[k*ld + j])^2, the lowest j on a tie, or -1 if no node is
 * eligible; dist2[i] (optional) gets that squared distance (+inf if none).
 * (pakr_expand ranks the same distances on coordinates centred on the state
 * box, which round differently: the two can pick different nodes only where
 * two candidates' distances are within rounding of each other.)
 *   states   device, d x ld floats, coordinate k of node j at states[k*ld + j]
 *   ld, n    row stride and node count, 0 <= n <= 2^31 - 2^20, n <= ld < 2^31
 *   d        3, 4, 5, 6 or 12
 *   fcost    device, n floats (node j is eligible iff fcost[j] < bound)
 *   queries  device, d x n_queries floats, coordinate k of query i at
 *            queries[k*n_queries + i]
 *   n_queries 0..65536; more is PAKR_ERR_INVALID_ARG (the static scratch limit)
 *   nearest  device, n_queries int32; dist2 device, n_queries floats or NULL
 *   cuda_stream  stream to enqueue on (NULL = default stream)
 * Runs on the calling thread's current device and only enqueues work; no
 * cudaMalloc, cudaFree or allocating library call is made.  Every call looks
 * up the scratch array's device address (that lookup allocates nothing once
 * the library's GPU code is loaded).  The first call on a device also loads
 * the GPU code of every search variant for every supported d (the set-up
 * step); make that first call before any stream capture.  All calls share the
 * one scratch array, which keeps the last call's contents; each call clears
 * what it uses, but calls whose kernels overlap on the GPU (different streams
 * with no ordering between them) race and give wrong results: order them on
 * one stream or with events. */
pakr_status pakr_nearest_static(const float *states, int64_t ld, int64_t n, int32_t d, const float *fcost,
                                float bound, const float *queries, int32_t n_queries, int32_t *nearest,
                                float *dist2, void *cuda_stream);

/* Library version string. */
const char *pakr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PAKR_H */
