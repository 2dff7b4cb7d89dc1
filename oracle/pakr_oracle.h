/*
 * pakr_oracle.h -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of one PAKR expansion
 * iteration and of the AO-x outer loop (Algorithm 1 and Sec. IV of "Fast
 * Asymptotically Optimal Kinodynamic Planning via Vectorization").  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline / reference arm
 * may load it.  It shares no source, header, table or helper with the CUDA
 * library; the two meet only through the seeded input generators.
 *
 * Readings of points the paper leaves open are stated beside each function.
 * Parity of the quadrotor model against the paper is unpinned (the paper
 * prints no equations); it is pinned to rigid-body invariants instead.
 */
#ifndef PAKR_ORACLE_H
#define PAKR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORA_MAX_D 16
#define ORA_MAX_M 8

enum { ORA_DI2 = 0, ORA_DI3 = 1, ORA_QUAD12 = 2, ORA_DUBINS3D = 3, ORA_UNICYCLE1 = 4, ORA_UNICYCLE2 = 5 };
enum { ORA_COST_PATH_LENGTH = 0, ORA_COST_DURATION = 1 };
enum { ORA_H_POSITION = 0, ORA_H_FULLSTATE = 1 };
enum { ORA_OUT_APPENDED = 0, ORA_OUT_PRUNED = 1, ORA_OUT_COLLIDED = 2, ORA_OUT_NO_PARENT = 3, ORA_OUT_DROPPED = 4 };
enum { ORA_OK = 0, ORA_GOAL_REACHED = 1, ORA_TREE_FULL = 2, ORA_NO_ELIGIBLE = 3, ORA_BUDGET_EXPIRED = 4,
       ORA_ERR_INVALID_ARG = -1 };

/* The planning problem (Sec. III): dynamics, state / control boxes, fixed RK4
 * step, duration range, obstacles, goal ball, cost and heuristic.  Obstacles:
 * boxes are n x (lo[pdim], hi[pdim]); spheres are n x (c[pdim], r). */
typedef struct {
    int dyn, d, m, pdim;
    double x_lo[ORA_MAX_D], x_hi[ORA_MAX_D];
    double u_lo[ORA_MAX_M], u_hi[ORA_MAX_M];
    double dt;
    int s_min, s_max;
    int n_boxes;
    const double *boxes;
    int n_spheres;
    const double *spheres;
    double x_goal[ORA_MAX_D];
    double goal_r;
    int cost, heuristic;
    double h_speed;           /* speed bound for the duration-cost heuristic */
    double nn_w[ORA_MAX_D];   /* per-dimension NN weights (all ones = plain) */
    double model[8];          /* QUAD12: mass, Ixx, Iyy, Izz, g */
    int K, k;                 /* parents per iteration, controls per parent */
} ora_problem;

/* Structure-of-arrays tree (Sec. IV-A), node-major rows here. */
typedef struct {
    int64_t cap, count;
    uint32_t iteration;       /* expansion counter, the Philox counter's first word */
    double *states;           /* cap x d */
    double *controls;         /* cap x m */
    int32_t *parents;         /* cap, root = -1 */
    double *costs;            /* cap, cost-to-come */
    int32_t *steps;           /* cap, substeps of the edge into the node */
} ora_tree;

/* Per-query nearest-neighbour report. */
typedef struct {
    int64_t idx;              /* argmin, -1 if no node is eligible */
    double d1, d2;            /* best and second-best Euclidean distance (inf if absent) */
    int fragile_elig;         /* 1 if a node whose f lies within tol of the bound could change the answer */
} ora_nn_result;

/* Per-rollout propagation report. */
typedef struct {
    double x_end[ORA_MAX_D];
    double cost_end;          /* cost-to-come of the child */
    double f_end;             /* cost_end + h(x_end) */
    int collided;             /* some substep invalid */
    int first_invalid;        /* 1-based substep, 0 if none */
    double face_margin;       /* min |distance to a face| over substeps 1..stop */
    int in_goal;
    double goal_margin;       /* | |p_end - p_goal| - r | */
} ora_rollout;

/* Everything one expansion produced; arrays are caller-owned (K, R = K*k). */
typedef struct {
    double *samples;          /* K x d */
    int64_t *near;            /* K */
    double *nn_d1, *nn_d2;    /* K */
    int32_t *nn_fragile;      /* K */
    double *u;                /* R x m */
    int32_t *S;               /* R */
    int32_t *outcome;         /* R */
    double *x_end;            /* R x d */
    double *cost_end, *f_end, *face_margin, *goal_margin; /* R */
    int32_t *in_goal;         /* R */
    int64_t *node;            /* R: node index of appended rollouts, else -1 */
    /* scalars */
    int64_t n_start, n_appended, n_pruned, n_collided, n_no_parent, n_dropped;
    int goal_found;
    int64_t goal_idx;
    double goal_cost;
    uint32_t iteration;
} ora_expand_out;

/* --- counter-based RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) --- */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double ora_u01(uint32_t w);
void ora_sample_state(const ora_problem *P, uint64_t seed, uint32_t iter, uint32_t i, double *x);
void ora_sample_control(const ora_problem *P, uint64_t seed, uint32_t iter, uint32_t i, uint32_t j,
                        double *u, int *S);

/* --- problem model (Sec. III) --- */
void ora_dynamics(const ora_problem *P, const double *x, const double *u, double *xdot);
void ora_rk4_step(const ora_problem *P, const double *x, const double *u, double h, double *out);
int ora_state_valid(const ora_problem *P, const double *x);
double ora_face_margin(const ora_problem *P, const double *x);
double ora_heuristic(const ora_problem *P, const double *x);

/* --- method steps (Algorithm 1) --- */
void ora_fcosts(const ora_problem *P, const ora_tree *T, int64_t n, double *f);
void ora_nearest(const ora_problem *P, const ora_tree *T, int64_t n, const double *f,
                 const double *q, double bound, double tol, ora_nn_result *out);
void ora_propagate(const ora_problem *P, const double *x0, double g0, const double *u, int S,
                   double bound, ora_rollout *out);
int ora_tree_reset(const ora_problem *P, ora_tree *T, const double *x_init);
int ora_expand(const ora_problem *P, ora_tree *T, double bound, uint64_t seed, ora_expand_out *o);
int64_t ora_extract_path(const ora_tree *T, int64_t node, int64_t *nodes_out, int64_t cap);

/* --- AO-x outer loop, budgeted in expansion iterations for determinism --- */
typedef struct {
    int64_t max_iterations;
    int stop_at_first;
    /* outputs */
    int64_t iterations;
    int n_solutions, n_restarts;
    double best_cost;
    int64_t best_path_len;    /* nodes on the best path, root..goal */
    int64_t *best_path;       /* caller buffer, capacity path_cap */
    int64_t path_cap;
    double *best_states;      /* path_cap x d copy of the best path's states */
    double *best_controls;    /* path_cap x m (entry 0 unused) */
    int32_t *best_steps;      /* path_cap (entry 0 unused) */
    double *hist_cost;        /* history capacity hist_cap */
    int64_t *hist_iter;
    int64_t hist_cap;
    int status;
    int64_t fragile_iteration; /* first iteration with an exemption-class event, -1 if none */
} ora_plan_out;
int ora_plan(const ora_problem *P, ora_tree *T, const double *x_init, uint64_t seed, ora_plan_out *o);

/* --- smooth trajectory cost and its reverse-mode gradient (adjoint RK4) ---
 * Trajectory: x_{n+1} = RK4(x_n, u_n, dt), n = 0..N-1, controls row-major
 * U[n*m + j].  Cost
 *   J = w_dur N dt + w_u sum_n |u_n|^2 dt + w_obs sum_{n=1..N} sum_obstacles softplus_beta(margin - sdf(p_n)) dt
 *       + w_goal |p_N - p_goal|^2 + w_len sum_n sqrt(|p_{n+1} - p_n|^2 + eps^2),
 * softplus_beta(z) = log(1 + exp(beta z)) / beta.  Not part of the paper. */
typedef struct {
    double w_dur, w_u, w_obs, beta, margin, w_goal, w_len, len_eps;
} ora_traj_params;
double ora_traj_cost(const ora_problem *P, const double *x0, const double *U, int N, const ora_traj_params *w,
                     double *x_final);
double ora_traj_grad(const ora_problem *P, const double *x0, const double *U, int N, const ora_traj_params *w,
                     double *dU, double *dx0);
void ora_dynamics_vjp(const ora_problem *P, const double *x, const double *u, const double *a, double *gx,
                      double *gu);

/* --- validation-only dense re-checks (Sec. IV-A checks validity at the
 * integration substeps only; these look between them) ---
 * ora_recheck_edge_dense: re-integrates the edge with RK4 at dt/sub and
 * returns 1 if any of the S*sub fine states is invalid (sub = 1 is the
 * planner's own substep check).
 * ora_di_edge_hits_exact: double integrator only; 1 if the continuous
 * closed-form edge p(t) = p0 + v0 t + u t^2/2, t in (0, S dt], touches an
 * obstacle box or leaves the state box (spheres: dense check at dt/64). */
int ora_recheck_edge_dense(const ora_problem *P, const double *x0, const double *u, int S, int sub);
int ora_di_edge_hits_exact(const ora_problem *P, const double *x0, const double *u, int S);

#ifdef __cplusplus
}
#endif
#endif
