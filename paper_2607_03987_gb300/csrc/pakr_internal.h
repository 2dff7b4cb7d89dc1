// pakr_internal.h -- types shared by the host runtime (pakr_api.cu) and the
// kernels (pakr_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pakr.h"

namespace pakr {

constexpr int kMaxD = 16;
constexpr int kMaxM = 8;
constexpr uint64_t kNoKey = ~0ull;  // empty packed (distance | index) or (cost | index) key

enum Dyn { DI2 = 0, DI3 = 1, QUAD12 = 2, DUBINS3D = 3, UNICYCLE1 = 4, UNICYCLE2 = 5, kNumDyn = 6 };
enum Outcome { OUT_APPENDED = 0, OUT_PRUNED = 1, OUT_COLLIDED = 2, OUT_NO_PARENT = 3, OUT_DROPPED = 4 };
enum { COST_PATH_LENGTH = 0, COST_DURATION = 1 };
enum { H_POSITION = 0, H_FULLSTATE = 1 };
enum { MODE_EXPAND = 0, MODE_PLAN = 1 };
enum { ERR_PATH_CYCLE = 1, ERR_BAD_PARENT = 2, ERR_TC_TIMEOUT = 4 };
#ifndef PAKR_TC_ONE_CTA
#define PAKR_TC_ONE_CTA 0
#endif
constexpr int kTcCtasPerSm = PAKR_TC_ONE_CTA ? 1 : 2;  // resident tensor-core nearest-neighbour CTAs per SM
constexpr int kMaxPropLanes = 16;  // lanes per rollout in k_propagate at most
// Largest tree (and nearest-neighbour node count) the kernels take: their node indices and
// chunk arithmetic are 32-bit, and rounding a chunk or a tile up past the last node adds at
// most a few thousand, so 2^20 below 2^31 leaves room for every rounding.
constexpr long long kMaxTreeNodes = (1LL << 31) - (1LL << 20);

// Problem constants, passed to every kernel by value.
struct DevProblem {
    int dyn, d, m, pdim;
    float x_lo[kMaxD], x_hi[kMaxD];
    float u_lo[kMaxM], u_hi[kMaxM];
    float sw[kMaxD];      // square roots of the NN weights
    float model[8];       // QUAD12: mass, Ixx, Iyy, Izz, g
    float dt, goal_r, h_speed;
    int s_min, s_max;
    int n_boxes, n_spheres;
    const float4 *boxes;  // n_boxes x 2 float4: (lo.xyz, 0), (hi.xyz, 0); unused coordinates zero
    const float4 *spheres;// n_spheres x float4: (c.xyz, r)
    int cost, heuristic;
    int K, k;             // parents per iteration, controls per parent
    int cap;              // tree capacity
    // tensor-core nearest neighbour: centre of the weighted state box, bound on |x_w - c|^2,
    // smallest tree size that takes the tensor-core kernel (INT_MAX: never)
    float tc_c[kMaxD];
    float tc_xbox2;
    float tc_s = 1.f;     // power of two the FP16 filter scales centred coordinates by (box radius to [2^7, 2^8))
    // > 0: the tensor-core grid is one full wave of two CTAs per SM, and the CTA of each pair
    // that is launched first takes this share of the pair's node tiles (0: equal chunks)
    float tc_pair_share = 0.f;
    int tc_min_n = 0x7FFFFFFF;
    // obstacle grid over the position box (grid_g = 0: none, every obstacle is tested): cell
    // index per position axis a is obstacle_cell(p_a, grid_lo[a], grid_inv[a], grid_g), cells
    // numbered (z * g + y) * g + x; cell c lists obstacles grid_items[grid_start[c] ..
    // grid_start[c + 1]) (box b as b, sphere s as n_boxes + s), every obstacle that can hold a
    // point of that cell
    int grid_g = 0, grid_cells = 0, grid_n_items = 0;
    float grid_lo[3] = {0.f, 0.f, 0.f}, grid_inv[3] = {0.f, 0.f, 0.f};
    const int *grid_start = nullptr;
    const unsigned short *grid_items = nullptr;
};

// Shared memory k_propagate stages: the obstacles, the goal and the obstacle grid.
__host__ __device__ inline int propagate_smem_bytes(int n_boxes, int n_spheres, int grid_cells, int grid_n_items)
{
    int b = 16 * (2 * n_boxes + n_spheres) + 4 * kMaxD;
    if (grid_cells > 0)
        b += 4 * (grid_cells + 1) + 2 * ((grid_n_items + 1) / 2 * 2);
    return b;
}

// Cell index of coordinate v on one axis of the obstacle grid: fl(fl(v - lo) * inv) truncated
// and clamped to [0, g - 1].  Every step is monotone in v, so a point inside an obstacle's
// bounding box [b_lo, b_hi] always falls in a cell between cell(b_lo) and cell(b_hi): the host
// lists each obstacle in exactly that range with this same function, and the device test of a
// point against its cell's list gives the same answer as testing every obstacle.
__host__ __device__ __forceinline__ int obstacle_cell(float v, float lo, float inv, int g)
{
#ifdef __CUDA_ARCH__
    const float t = __fmul_rn(__fsub_rn(v, lo), inv);
#else
    const float d = v - lo;
    const float t = d * inv;
#endif
    if (!(t >= 0.f))
        return 0;
    if (t >= (float)g)
        return g - 1;
    return (int)t;
}

// Dimension-major tree arrays.
struct DevTree {
    float *X;       // d x cap
    float *U;       // m x cap
    float *cost;    // cap
    float *fcost;   // cap, cost + h(x)
    int *parent;    // cap
    int *steps;     // cap
    float *XT = nullptr;  // packed tensor-core operand rows, 256-node tiles (nullptr: not kept)
};

// Per-batch workspace.
struct DevWork {
    float *xr;                  // d x K samples
    unsigned long long *nn_key; // K packed (dist bits << 32 | node)
    float *st_x;                // d x R child states
    float *st_u;                // m x R controls
    float *st_cost;             // R
    float *st_f;                // R
    int *st_steps;              // R
    int *st_parent;             // R
    int8_t *outcome;            // R
    int8_t *goal;               // R
    int *block_count;           // one per propagate block
    unsigned *nn_amin = nullptr;  // K: smallest tensor-core filter value per query over node chunks
                                  // (order-preserving unsigned encoding; all ones = none yet)
};

// Device control block: tree counter, per-batch scalars and AO-x state.
struct Ctl {
    int count;               // nodes in the tree
    unsigned int iteration;  // expansion counter (Philox counter word 0)
    int n_start;             // snapshot of count for the current batch
    float bound;             // cost bound of the current batch
    unsigned long long seed;
    unsigned long long goal_key;  // packed (cost bits << 32 | node) of the best appended goal child
    int n_appended, n_pruned, n_collided, n_no_parent, n_dropped;
    int err;
    int status;              // tree_reset: 1 valid root, 0 invalid
    unsigned tc_flag;        // a tree node lies outside the box bound of the tensor-core filter
    float x_goal[kMaxD];
    // AO-x plan state
    float c_best;            // the AO-x bound: own solutions and bounds offered from outside (a minimum)
    float sol_best;          // cost of this run's own best solution (+inf if none)
    int plan_stop;
    long long iterations_done;
    unsigned long long t0_ns;
    unsigned long long t_first_ns;
    long long nodes_first;   // tree size when the first solution was recorded
    long long iterations_first;
    unsigned long long t_end_ns;
    int n_solutions;
    int n_restarts;
    int path_len;            // nodes on the best path (edges + 1); negative = required length when too long
    unsigned path_seq;       // odd while the AO-x step writes a new best path, even otherwise
    int plan_status;         // 0 running/budget, 1 goal at stop_at_first, 3 no eligible, -1 invalid start
    int offer_restart;       // an offered bound lowered c_best: the AO-x step restarts the tree
};

struct PlanParams {
    float x_init[kMaxD];
    float x_goal[kMaxD];
    unsigned long long seed;
    unsigned long long budget_ns;
    long long max_iterations;
    int stop_at_first;
    float c_best_init;   // AO-x bound the run starts from (+inf for a fresh run)
};

struct DevPlanBufs {
    int *path_nodes;        // path_cap + 1
    float *path_x;          // (path_cap + 1) x d, node-major
    float *path_u;          // (path_cap + 1) x m
    int *path_steps;        // path_cap + 1
    int path_cap;           // edges
    unsigned long long *hist_t;  // history_cap, ns since t0
    float *hist_cost;
    long long *hist_iter;
    int hist_cap;
};

// Launch configuration chosen at create.
struct LaunchCfg {
    int nn_variant;     // 0: 64 threads x 2 queries, 1: 128 x 2, 2: 256 x 4
    int nn_threads, nn_qpt, nn_qgroups, nn_chunks;
    int prop_threads, prop_blocks;
    int prop_lanes;     // lanes per rollout in k_propagate (1, 2, 4, 8 or 16, at most kMaxPropLanes)
    int sample_threads, sample_blocks;
    int obs_smem_bytes; // shared memory for obstacles + goal
    int tc_chunks, tc_qblocks;  // tensor-core nearest neighbour grid (node chunks x query blocks)
};

// Kernel launchers (pakr_kernels.cu).  Each returns the launch error.
cudaError_t launch_sample(const DevProblem &P, Ctl *ctl, const DevWork &W, const LaunchCfg &L, float bound,
                          unsigned long long seed, int mode, cudaStream_t s);
// Index of the bound and seed arguments of k_sample (for updating them in a graph).
constexpr int kSampleArgBound = 3, kSampleArgSeed = 4, kSampleArgs = 6;
cudaError_t launch_nn(const DevProblem &P, const Ctl *ctl, const DevTree &T, const DevWork &W, const LaunchCfg &L,
                      cudaStream_t s);
// k_nn alone (it still returns at once for trees of P.tc_min_n nodes or more).
cudaError_t launch_nn_fp32(const DevProblem &P, const Ctl *ctl, const DevTree &T, const DevWork &W,
                           const LaunchCfg &L, cudaStream_t s);
cudaError_t launch_nn_tc(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W, const LaunchCfg &L,
                         cudaStream_t s);
cudaError_t launch_tc_pack(const DevProblem &P, Ctl *ctl, const DevTree &T, int count, cudaStream_t s);
int tc_operand_floats(int d);  // 4-byte words per packed node row (pakr_tc.cuh: TcShape<D>::KT operand elements)
float tc_scale(float xbox2);   // the FP16 filter's coordinate scale for a box of squared radius xbox2
cudaError_t tc_configure(const DevProblem &P);
cudaError_t launch_propagate(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W, const LaunchCfg &L,
                             cudaStream_t s);
cudaError_t launch_append(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W, const LaunchCfg &L,
                          cudaStream_t s);
cudaError_t launch_tree_reset(const DevProblem &P, Ctl *ctl, const DevTree &T, const float *x_init_dev,
                              cudaStream_t s);
cudaError_t launch_import_fcost(const DevProblem &P, Ctl *ctl, const DevTree &T, int count, cudaStream_t s);
cudaError_t launch_plan_init(const DevProblem &P, Ctl *ctl, const DevTree &T, const PlanParams *pp,
                             cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_plan_cont(const Ctl *ctl, cudaGraphConditionalHandle h, cudaStream_t s);
// inner: the handles of the FP32 and tensor-core inner loops of a nested AO-x graph, or nullptr.
cudaError_t launch_plan_step(const DevProblem &P, Ctl *ctl, const DevTree &T, const PlanParams *pp,
                             const DevPlanBufs &B, cudaGraphConditionalHandle h, cudaStream_t s,
                             const cudaGraphConditionalHandle *inner = nullptr);
cudaError_t launch_truncate(Ctl *ctl, int count, cudaStream_t s);
cudaError_t launch_offer_bound(Ctl *ctl, const float *cost, cudaStream_t s);
cudaError_t preload_offer_bound();
// Copy of the best path of a running plan (pakr_plan_snapshot; pakr_kernels.cu).
cudaError_t launch_plan_snapshot(const Ctl *ctl, const DevPlanBufs &B, int d, int m, float *states,
                                 float *controls, int *steps, int max_edges, int *info, cudaStream_t s);
cudaError_t preload_plan_snapshot();
cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int64_t n, cudaStream_t s);

// Sets the calling thread's pakr_last_error() message (pakr_api.cu).
void record_error(const char *msg);

// Planner internals for the other translation units (pakr_api.cu).
const DevProblem *planner_problem(const pakr_planner *p);
cudaStream_t planner_stream(const pakr_planner *p);
int planner_device(const pakr_planner *p);

// Validates the problem part of a description (not obstacles or tree size)
// and fills the kernel constants (pakr_api.cu).
pakr_status fill_problem(const pakr_problem_desc *desc, DevProblem *P, int *d, int *m, int *pdim);

// Occupancy-derived sizes (pakr_kernels.cu).
int nn_blocks_per_sm(int d, int variant);
// Loads every k_nn instantiation's GPU code on the current device (pakr_kernels.cu).
cudaError_t nn_preload_all();

}  // namespace pakr
