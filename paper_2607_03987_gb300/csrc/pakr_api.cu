// pakr_api.cu -- host runtime behind include/pakr.h: argument checks, device
// memory layout, kernel sequencing, the AO-x CUDA graph, tree import / export
// and per-kernel timing.  Every compute step runs in pakr_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pakr.h"
#include "pakr_internal.h"

using namespace pakr;

namespace {

thread_local std::string g_last_error;

pakr_status fail(pakr_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

}  // namespace

// Error message sink shared with the other translation units of the library.
void pakr::record_error(const char *msg) { g_last_error = msg ? msg : ""; }

namespace {

#define CUDA_TRY(expr)                                                                                                 \
    do {                                                                                                               \
        cudaError_t e_ = (expr);                                                                                       \
        if (e_ != cudaSuccess)                                                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? PAKR_ERR_OOM : PAKR_ERR_CUDA, "%s failed: %s (%s:%d)",      \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                                            \
    } while (0)

struct DimInfo {
    int d, m, pdim;
};

bool dims_of(int dyn, DimInfo *out)
{
    switch (dyn) {
    case PAKR_DI2: *out = {4, 2, 2}; return true;
    case PAKR_DI3: *out = {6, 3, 3}; return true;
    case PAKR_QUAD12: *out = {12, 4, 3}; return true;
    case PAKR_DUBINS3D: *out = {6, 3, 3}; return true;
    case PAKR_UNICYCLE1: *out = {3, 2, 2}; return true;
    case PAKR_UNICYCLE2: *out = {5, 2, 2}; return true;
    default: return false;
    }
}

constexpr int kPropThreads = 256;
constexpr int kSampleThreads = 128;
constexpr int kMaxObstacleRecords = 3000;  // float4 records staged in 48 KB of shared memory
constexpr int64_t kMaxPlanIterations = 10000000;  // hard bound on the device-resident AO-x loop

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Uniform grid over the position box for the per-substep obstacle test: each cell lists the
// obstacles whose bounding box reaches it (cell ranges from obstacle_cell, the function the
// device applies to points, so the lists are exact), and a substep tests only its cell's list.
// Chosen among a few resolutions for the fewest expected tests per point (list entries per
// cell), within the shared memory k_propagate stages; none when it would not save at least half
// of the tests (few obstacles, or obstacles as large as the box).
struct ObstacleGrid {
    int g = 0, cells = 0;
    float lo[3] = {0.f, 0.f, 0.f}, inv[3] = {0.f, 0.f, 0.f};
    std::vector<int> start;
    std::vector<unsigned short> items;
};

constexpr int kPropSmemBudget = 46 * 1024;  // dynamic shared memory of k_propagate (default limit 48 KB)
// k_nn_tc, one full wave: the share of each pair's node tiles that the CTA launched first takes
// (bench, 1M-node tree: 0.50 88.2 us, 0.52 87.0, 0.54 89.1, 0.56 91.6)
constexpr float kTcPairShare = 0.52f;

ObstacleGrid build_obstacle_grid(const pakr_problem_desc *d, const DimInfo &di)
{
    ObstacleGrid best;
    const int pd = di.pdim, nb = d->n_boxes, ns = d->n_spheres, n_obs = nb + ns;
    if (n_obs < 4 || pd < 2 || pd > 3)
        return best;
    // bounding boxes: boxes as given; spheres widened by a margin that covers the rounding of
    // the device's FP32 test |p - c|^2 <= r^2
    std::vector<float> blo((size_t)n_obs * pd), bhi((size_t)n_obs * pd);
    for (int i = 0; i < nb; ++i)
        for (int a = 0; a < pd; ++a) {
            blo[(size_t)i * pd + a] = d->boxes[(size_t)i * 2 * pd + a];
            bhi[(size_t)i * pd + a] = d->boxes[(size_t)i * 2 * pd + pd + a];
        }
    for (int i = 0; i < ns; ++i) {
        const float *sp = d->spheres + (size_t)i * (pd + 1);
        const float r = std::fabs(sp[pd]) * (1.f + 1e-4f) + 1e-6f;
        for (int a = 0; a < pd; ++a) {
            blo[(size_t)(nb + i) * pd + a] = sp[a] - r;
            bhi[(size_t)(nb + i) * pd + a] = sp[a] + r;
        }
    }
    float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < pd; ++a) {
        lo[a] = d->x_lo[a];
        hi[a] = d->x_hi[a];
        if (!(hi[a] > lo[a]))
            return best;
    }
    const int cand3[] = {10, 8, 6, 4}, cand2[] = {32, 24, 16, 8};
    double best_tests = 0.5 * n_obs;
    for (int ci = 0; ci < 4; ++ci) {
        const int g = pd == 3 ? cand3[ci] : cand2[ci];
        ObstacleGrid G;
        G.g = g;
        G.cells = pd == 3 ? g * g * g : g * g;
        for (int a = 0; a < pd; ++a) {
            G.lo[a] = lo[a];
            G.inv[a] = (float)((double)g / ((double)hi[a] - (double)lo[a]));
        }
        std::vector<int> count((size_t)G.cells + 1, 0);
        std::vector<int> r0((size_t)n_obs * 3, 0), r1((size_t)n_obs * 3, 0);
        size_t items = 0;
        for (int o = 0; o < n_obs; ++o) {
            size_t vol = 1;
            for (int a = 0; a < pd; ++a) {
                r0[(size_t)o * 3 + a] = obstacle_cell(blo[(size_t)o * pd + a], G.lo[a], G.inv[a], g);
                r1[(size_t)o * 3 + a] = obstacle_cell(bhi[(size_t)o * pd + a], G.lo[a], G.inv[a], g);
                vol *= (size_t)(r1[(size_t)o * 3 + a] - r0[(size_t)o * 3 + a] + 1);
            }
            items += vol;
        }
        const double tests = (double)items / G.cells;
        if (items > 65535 ||
            propagate_smem_bytes(nb, ns, G.cells, (int)items) > kPropSmemBudget || !(tests < best_tests))
            continue;
        // lists in obstacle order (boxes, then spheres), cells in (z, y, x) order
        for (int o = 0; o < n_obs; ++o)
            for (int z = pd == 3 ? r0[(size_t)o * 3 + 2] : 0; z <= (pd == 3 ? r1[(size_t)o * 3 + 2] : 0); ++z)
                for (int y = r0[(size_t)o * 3 + 1]; y <= r1[(size_t)o * 3 + 1]; ++y)
                    for (int x = r0[(size_t)o * 3]; x <= r1[(size_t)o * 3]; ++x)
                        ++count[(size_t)(z * g + y) * g + x + 1];
        G.start.assign((size_t)G.cells + 1, 0);
        for (int c = 0; c < G.cells; ++c)
            G.start[c + 1] = G.start[c] + count[c + 1];
        G.items.assign(items, 0);
        std::vector<int> fill(G.start.begin(), G.start.end() - 1);
        for (int o = 0; o < n_obs; ++o)
            for (int z = pd == 3 ? r0[(size_t)o * 3 + 2] : 0; z <= (pd == 3 ? r1[(size_t)o * 3 + 2] : 0); ++z)
                for (int y = r0[(size_t)o * 3 + 1]; y <= r1[(size_t)o * 3 + 1]; ++y)
                    for (int x = r0[(size_t)o * 3]; x <= r1[(size_t)o * 3]; ++x)
                        G.items[fill[(size_t)(z * g + y) * g + x]++] = (unsigned short)o;
        best_tests = tests;
        best = std::move(G);
    }
    return best;
}

// Pinned staging of a plan's result: the first kStageHist history entries and kStageEdges path
// edges, copied right behind the control block.
constexpr int kStageHist = 64, kStageEdges = 128;
struct PlanStage {
    unsigned long long t[kStageHist];
    float cost[kStageHist];
    long long iter[kStageHist];
    float x[(kStageEdges + 1) * kMaxD];
    float u[kStageEdges * kMaxM];
    int steps[kStageEdges];
};

// Byte offsets of every device buffer inside one allocation.
struct Layout {
    size_t X, U, cost, fcost, parent, steps, XT;
    size_t xr, nn_key, nn_amin, st_x, st_u, st_cost, st_f, st_steps, st_parent, outcome, goal, block_count;
    size_t boxes, spheres, grid_start, grid_items, ctl, pp;
    size_t path_nodes, path_x, path_u, path_steps, hist_t, hist_cost, hist_iter;
    size_t total;
};

Layout make_layout(const DimInfo &di, int64_t cap, int K, int k, int nb, int ns, int path_cap, int hist_cap,
                   int tc_row_floats, const ObstacleGrid &grid)
{
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + std::max<size_t>(bytes, 1), 256);
        return at;
    };
    const size_t R = (size_t)K * k;
    const size_t nblk = (R * kMaxPropLanes + kPropThreads - 1) / kPropThreads;  // blocks at the largest lane count
    const size_t c = (size_t)cap;
    L.X = take(sizeof(float) * di.d * c);
    L.U = take(sizeof(float) * di.m * c);
    L.cost = take(sizeof(float) * c);
    L.fcost = take(sizeof(float) * (c + 4));  // bulk copies of f-costs round up to 16 bytes
    L.parent = take(sizeof(int) * c);
    L.steps = take(sizeof(int) * c);
    // packed tensor-core operand rows, whole 256-node tiles
    L.XT = take(tc_row_floats > 0 ? sizeof(float) * (size_t)tc_row_floats * ((c + 255) / 256 * 256) : 0);
    L.xr = take(sizeof(float) * di.d * (size_t)K);
    L.nn_key = take(sizeof(unsigned long long) * (size_t)K);
    L.nn_amin = take(sizeof(unsigned) * (size_t)K);
    L.st_x = take(sizeof(float) * di.d * R);
    L.st_u = take(sizeof(float) * di.m * R);
    L.st_cost = take(sizeof(float) * R);
    L.st_f = take(sizeof(float) * R);
    L.st_steps = take(sizeof(int) * R);
    L.st_parent = take(sizeof(int) * R);
    L.outcome = take(R);
    L.goal = take(R);
    L.block_count = take(sizeof(int) * nblk);
    L.boxes = take(sizeof(float4) * 2 * (size_t)nb);
    L.spheres = take(sizeof(float4) * (size_t)ns);
    L.grid_start = take(sizeof(int) * grid.start.size());
    L.grid_items = take(sizeof(unsigned short) * grid.items.size());
    L.ctl = take(sizeof(Ctl));
    L.pp = take(sizeof(PlanParams));
    L.path_nodes = take(sizeof(int) * (size_t)(path_cap + 1));
    L.path_x = take(sizeof(float) * di.d * (size_t)(path_cap + 1));
    L.path_u = take(sizeof(float) * di.m * (size_t)(path_cap + 1));
    L.path_steps = take(sizeof(int) * (size_t)(path_cap + 1));
    L.hist_t = take(sizeof(unsigned long long) * (size_t)hist_cap);
    L.hist_cost = take(sizeof(float) * (size_t)hist_cap);
    L.hist_iter = take(sizeof(long long) * (size_t)hist_cap);
    L.total = off;
    return L;
}

bool finite_all(const float *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i]))
            return false;
    return true;
}

pakr_status check_desc(const pakr_problem_desc *d, DimInfo *di)
{
    if (!d)
        return fail(PAKR_ERR_INVALID_ARG, "desc is NULL");
    if (!dims_of(d->dynamics, di))
        return fail(PAKR_ERR_INVALID_ARG, "unknown dynamics %d", d->dynamics);
    if (!d->x_lo || !d->x_hi || !d->u_lo || !d->u_hi)
        return fail(PAKR_ERR_INVALID_ARG, "state / control bounds must be given");
    if (!finite_all(d->x_lo, di->d) || !finite_all(d->x_hi, di->d) || !finite_all(d->u_lo, di->m) ||
        !finite_all(d->u_hi, di->m))
        return fail(PAKR_ERR_INVALID_ARG, "bounds must be finite");
    for (int a = 0; a < di->d; ++a)
        if (!(d->x_lo[a] <= d->x_hi[a]))
            return fail(PAKR_ERR_INVALID_ARG, "x_lo[%d] > x_hi[%d]", a, a);
    for (int a = 0; a < di->m; ++a)
        if (!(d->u_lo[a] <= d->u_hi[a]))
            return fail(PAKR_ERR_INVALID_ARG, "u_lo[%d] > u_hi[%d]", a, a);
    if (!(d->dt > 0.f) || !std::isfinite(d->dt))
        return fail(PAKR_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (d->steps_min < 1 || d->steps_max < d->steps_min)
        return fail(PAKR_ERR_INVALID_ARG, "need 1 <= steps_min <= steps_max");
    if (d->n_boxes < 0 || d->n_spheres < 0 || (d->n_boxes > 0 && !d->boxes) || (d->n_spheres > 0 && !d->spheres))
        return fail(PAKR_ERR_INVALID_ARG, "bad obstacle arrays");
    if (2 * (int64_t)d->n_boxes + d->n_spheres > kMaxObstacleRecords)
        return fail(PAKR_ERR_INVALID_ARG, "too many obstacles: 2*n_boxes + n_spheres must be <= %d",
                    kMaxObstacleRecords);
    if (d->n_boxes > 0 && !finite_all(d->boxes, d->n_boxes * 2 * di->pdim))
        return fail(PAKR_ERR_INVALID_ARG, "boxes must be finite");
    if (d->n_spheres > 0 && !finite_all(d->spheres, d->n_spheres * (di->pdim + 1)))
        return fail(PAKR_ERR_INVALID_ARG, "spheres must be finite");
    if (!(d->goal_radius >= 0.f) || !std::isfinite(d->goal_radius))
        return fail(PAKR_ERR_INVALID_ARG, "goal_radius must be finite and >= 0");
    if (d->cost != PAKR_COST_PATH_LENGTH && d->cost != PAKR_COST_DURATION)
        return fail(PAKR_ERR_INVALID_ARG, "unknown cost %d", d->cost);
    if (d->heuristic != PAKR_H_POSITION && d->heuristic != PAKR_H_FULLSTATE)
        return fail(PAKR_ERR_INVALID_ARG, "unknown heuristic %d", d->heuristic);
    if (!std::isfinite(d->heuristic_speed))
        return fail(PAKR_ERR_INVALID_ARG, "heuristic_speed must be finite");
    if (d->nn_weights) {
        for (int a = 0; a < di->d; ++a)
            if (!(d->nn_weights[a] >= 0.f) || !std::isfinite(d->nn_weights[a]))
                return fail(PAKR_ERR_INVALID_ARG, "nn_weights must be finite and >= 0");
    }
    if (d->model_params && !finite_all(d->model_params, 5))
        return fail(PAKR_ERR_INVALID_ARG, "model_params must be finite");
    if (d->model_params && d->dynamics == PAKR_QUAD12) {
        for (int a = 0; a < 4; ++a)
            if (!(d->model_params[a] > 0.f))
                return fail(PAKR_ERR_INVALID_ARG, "mass and inertia must be > 0");
    }
    if (d->n_parents < 1 || d->branching < 1)
        return fail(PAKR_ERR_INVALID_ARG, "n_parents and branching must be >= 1");
    if ((int64_t)d->n_parents * d->branching > (int64_t)1 << 30)
        return fail(PAKR_ERR_INVALID_ARG, "n_parents * branching too large");
    if (d->tree_cap < 1 || d->tree_cap > kMaxTreeNodes)
        return fail(PAKR_ERR_INVALID_ARG, "tree_cap must be in [1, 2^31 - 2^20]");
    if (d->path_cap < 0 || d->history_cap < 0)
        return fail(PAKR_ERR_INVALID_ARG, "path_cap / history_cap must be >= 0");
    if (d->nn_mode < PAKR_NN_AUTO || d->nn_mode > PAKR_NN_TENSOR)
        return fail(PAKR_ERR_INVALID_ARG, "nn_mode %d is not a pakr_nn_mode", d->nn_mode);
    return PAKR_OK;
}

// Smallest tree size the tensor-core nearest neighbour takes (0x7FFFFFFF: never), and
// the floats per packed node row it needs (0: no packed copy).  Below about 28k nodes, or
// with fewer than two query blocks, the FP32 kernel in its 128-query blocks is faster
// (d = 6, 1024 queries: 20.3 vs 25.1 us at 16k nodes, 30.8 vs 28.5 us at 32k).
constexpr int kTcAutoMinNodes = 28672;
constexpr int kTcAutoMinQueries = 256;
int tc_min_nodes(const pakr_problem_desc *d)
{
    if (d->nn_mode == PAKR_NN_TENSOR)
        return 0;
    if (d->nn_mode == PAKR_NN_AUTO && d->n_parents >= kTcAutoMinQueries)
        return kTcAutoMinNodes;
    return 0x7FFFFFFF;
}
int tc_floats(const pakr_problem_desc *d, const DimInfo &di)
{
    return tc_min_nodes(d) < 0x7FFFFFFF ? tc_operand_floats(di.d) : 0;
}

struct EventPair {
    cudaEvent_t a, b;
};

// Per-kernel timing slots of pakr_kernel_times.
constexpr int kTimeSlots = 5;

}  // namespace

struct pakr_planner {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    DimInfo di{};
    DevProblem P{};
    DevTree T{};
    DevWork W{};
    DevPlanBufs B{};
    LaunchCfg L{};
    Layout lay{};
    Ctl *ctl = nullptr;
    PlanParams *pp = nullptr;
    char *base = nullptr;
    bool owns_base = false;
    Ctl *ctl_host = nullptr;        // pinned
    PlanParams *pp_host = nullptr;  // pinned
    PlanStage *stage_host = nullptr;  // pinned
    int64_t cap = 0;
    int K = 0, k = 0;
    int path_cap = 0, hist_cap = 0;
    cudaGraphExec_t plan_exec = nullptr;
    cudaGraph_t plan_graph = nullptr;
    // one expansion as a graph (pakr_expand without profiling), one per nearest-neighbour
    // kernel ([0] k_nn, [1] k_nn_tc): its sample node takes the bound and seed of each call
    cudaGraphExec_t expand_exec[2] = {nullptr, nullptr};
    cudaGraph_t expand_graph[2] = {nullptr, nullptr};
    cudaGraphNode_t expand_sample[2] = {nullptr, nullptr};
    // an upper bound on the device-side tree size, for choosing the nearest-neighbour kernel
    // on the host: exact after every read of the control block and every host-side tree
    // operation, raised by K * k per expansion in between
    int64_t n_upper = 0;
    // profiling
    bool profiling = false;
    std::vector<EventPair> pool;
    std::vector<std::pair<int, EventPair>> pending;
    double ms[kTimeSlots] = {0, 0, 0, 0, 0};
    int64_t launches[kTimeSlots] = {0, 0, 0, 0, 0};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

EventPair take_pair(pakr_planner *p)
{
    if (!p->pool.empty()) {
        EventPair e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    EventPair e{};
    cudaEventCreate(&e.a);
    cudaEventCreate(&e.b);
    return e;
}

template <class F>
pakr_status timed(pakr_planner *p, int slot, F &&launch, const char *what)
{
    EventPair ev{};
    if (p->profiling) {
        ev = take_pair(p);
        cudaEventRecord(ev.a, p->stream);
    }
    cudaError_t e = launch();
    if (e != cudaSuccess)
        return fail(PAKR_ERR_CUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    if (p->profiling) {
        cudaEventRecord(ev.b, p->stream);
        p->pending.push_back({slot, ev});
    }
    return PAKR_OK;
}

// The nearest-neighbour kernel for the next expansion, chosen on the host: the tensor-core one
// once the tree can hold tc_min_n nodes (by the upper bound; either kernel gives the same
// result at any size, the choice only decides the speed).
bool use_tc_nn(const pakr_planner *p)
{
    return p->T.XT != nullptr && p->P.tc_min_n < 0x7FFFFFFF && p->n_upper >= p->P.tc_min_n;
}

// P for a nearest-neighbour kernel launched for any tree size (its device-side range check
// then always passes).
DevProblem nn_problem(const pakr_planner *p, bool tc)
{
    DevProblem P = p->P;
    P.tc_min_n = tc ? 0 : 0x7FFFFFFF;
    return P;
}

pakr_status enqueue_expand(pakr_planner *p, float bound, uint64_t seed, bool tc)
{
    pakr_status st;
    st = timed(p, 0, [&] { return launch_sample(p->P, p->ctl, p->W, p->L, bound, seed, MODE_EXPAND, p->stream); },
               "sample");
    if (st != PAKR_OK)
        return st;
    const DevProblem Pn = nn_problem(p, tc);
    if (tc)
        st = timed(p, 4, [&] { return launch_nn_tc(Pn, p->ctl, p->T, p->W, p->L, p->stream); }, "nearest (tc)");
    else
        st = timed(p, 1, [&] { return launch_nn_fp32(Pn, p->ctl, p->T, p->W, p->L, p->stream); }, "nearest");
    if (st != PAKR_OK)
        return st;
    st = timed(p, 2, [&] { return launch_propagate(p->P, p->ctl, p->T, p->W, p->L, p->stream); }, "propagate");
    if (st != PAKR_OK)
        return st;
    return timed(p, 3, [&] { return launch_append(p->P, p->ctl, p->T, p->W, p->L, p->stream); }, "append");
}

// The nodes of g that are not in `before`.
std::vector<cudaGraphNode_t> new_nodes(cudaGraph_t g, const std::vector<cudaGraphNode_t> &before)
{
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> all(n), out;
    if (n)
        cudaGraphGetNodes(g, all.data(), &n);
    for (cudaGraphNode_t x : all)
        if (std::find(before.begin(), before.end(), x) == before.end())
            out.push_back(x);
    return out;
}

std::vector<cudaGraphNode_t> graph_nodes(cudaGraph_t g)
{
    return new_nodes(g, {});
}

// Capture `launch` into graph g after the node `dep` (none if nullptr); returns the
// single node it adds in *node.
template <class F>
pakr_status capture_one(pakr_planner *p, cudaGraph_t g, cudaGraphNode_t dep, F &&launch, cudaGraphNode_t *node)
{
    const std::vector<cudaGraphNode_t> before = graph_nodes(g);
    CUDA_TRY(cudaStreamBeginCaptureToGraph(p->capture_stream, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0,
                                           cudaStreamCaptureModeThreadLocal));
    cudaError_t le = launch(p->capture_stream);
    cudaGraph_t tmp = nullptr;
    CUDA_TRY(cudaStreamEndCapture(p->capture_stream, &tmp));
    CUDA_TRY(le);
    const std::vector<cudaGraphNode_t> added = new_nodes(g, before);
    if (added.size() != 1)
        return fail(PAKR_ERR_CUDA, "unexpected graph shape (%zu nodes captured)", added.size());
    *node = added[0];
    return PAKR_OK;
}

// Which nearest-neighbour kernel an expansion graph runs.
enum NnKind { NN_ONLY_FP32 = 1, NN_ONLY_TC = 2 };

// Append one expansion to graph g after `dep`: sample, nearest neighbour (the one kernel of
// `kind`, launched for any tree size: the graph's owner has chosen it), propagate, append.
// No conditional node: a device-side IF node costs about 10 us of the step on GB300.
pakr_status add_expansion(pakr_planner *p, cudaGraph_t g, cudaGraphNode_t dep, float bound, uint64_t seed, int mode,
                          NnKind kind, cudaGraphNode_t *sample_node, cudaGraphNode_t *last)
{
    pakr_status st = capture_one(
        p, g, dep, [&](cudaStream_t s) { return launch_sample(p->P, p->ctl, p->W, p->L, bound, seed, mode, s); },
        sample_node);
    if (st != PAKR_OK)
        return st;
    cudaGraphNode_t at = *sample_node;
    const DevProblem Pn = nn_problem(p, kind == NN_ONLY_TC);
    if (kind == NN_ONLY_TC)
        st = capture_one(p, g, at, [&](cudaStream_t s) { return launch_nn_tc(Pn, p->ctl, p->T, p->W, p->L, s); },
                         &at);
    else
        st = capture_one(p, g, at, [&](cudaStream_t s) { return launch_nn_fp32(Pn, p->ctl, p->T, p->W, p->L, s); },
                         &at);
    if (st != PAKR_OK)
        return st;
    st = capture_one(p, g, at, [&](cudaStream_t s) { return launch_propagate(p->P, p->ctl, p->T, p->W, p->L, s); },
                     &at);
    if (st != PAKR_OK)
        return st;
    st = capture_one(p, g, at, [&](cudaStream_t s) { return launch_append(p->P, p->ctl, p->T, p->W, p->L, s); }, &at);
    *last = at;
    return st;
}

// Add a WHILE node on handle h after `dep` (none if nullptr); *body receives its body graph.
pakr_status add_while(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h, cudaGraphNode_t *node,
                      cudaGraph_t *body)
{
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CUDA_TRY(cudaGraphAddNode(node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &cp));
    *body = cp.conditional.phGraph_out[0];
    return PAKR_OK;
}

// The AO-x graph: k_plan_init, then a WHILE loop of expansions, each followed by
// k_plan_step.  With both nearest-neighbour kernels in play the loop body holds two inner
// WHILE loops, FP32 while the tree is below tc_min_n nodes and tensor-core from there;
// k_plan_step opens the one the next iteration needs (no IF node per iteration).
pakr_status build_plan_graph(pakr_planner *p)
{
    if (p->plan_exec)
        return PAKR_OK;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h{};
    CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t init_node = nullptr;
    pakr_status st = capture_one(
        p, g, nullptr, [&](cudaStream_t s) { return launch_plan_init(p->P, p->ctl, p->T, p->pp, h, s); }, &init_node);
    if (st != PAKR_OK)
        return st;
    cudaGraphNode_t wnode = nullptr;
    cudaGraph_t body = nullptr;
    st = add_while(g, init_node, h, &wnode, &body);
    if (st != PAKR_OK)
        return st;
    const bool has_tc = p->T.XT != nullptr && p->P.tc_min_n < 0x7FFFFFFF;
    const bool nested = has_tc && p->P.tc_min_n > 1;
    cudaGraphNode_t sample_node = nullptr, last = nullptr, step = nullptr;
    if (!nested) {
        st = add_expansion(p, body, nullptr, 0.f, 0ull, MODE_PLAN, has_tc ? NN_ONLY_TC : NN_ONLY_FP32, &sample_node,
                           &last);
        if (st != PAKR_OK)
            return st;
        st = capture_one(
            p, body, last, [&](cudaStream_t s) { return launch_plan_step(p->P, p->ctl, p->T, p->pp, p->B, h, s); },
            &step);
    } else {
        // every run starts (and restarts) from a one-node tree: the FP32 loop first
        cudaGraphConditionalHandle inner[2]{};
        CUDA_TRY(cudaGraphConditionalHandleCreate(&inner[0], body, 1, cudaGraphCondAssignDefault));
        CUDA_TRY(cudaGraphConditionalHandleCreate(&inner[1], body, 0, cudaGraphCondAssignDefault));
        cudaGraphNode_t wa = nullptr, wb = nullptr;
        cudaGraph_t body_a = nullptr, body_b = nullptr;
        st = add_while(body, nullptr, inner[0], &wa, &body_a);
        if (st == PAKR_OK)
            st = add_while(body, wa, inner[1], &wb, &body_b);
        for (int k = 0; k < 2 && st == PAKR_OK; ++k) {
            cudaGraph_t bg = k == 0 ? body_a : body_b;
            st = add_expansion(p, bg, nullptr, 0.f, 0ull, MODE_PLAN, k == 0 ? NN_ONLY_FP32 : NN_ONLY_TC,
                               &sample_node, &last);
            if (st == PAKR_OK)
                st = capture_one(
                    p, bg, last,
                    [&](cudaStream_t s) { return launch_plan_step(p->P, p->ctl, p->T, p->pp, p->B, h, s, inner); },
                    &step);
        }
        // the outer loop's condition is set at its own level, after both inner loops
        cudaGraphNode_t cont = nullptr;
        if (st == PAKR_OK)
            st = capture_one(p, body, wb, [&](cudaStream_t s) { return launch_plan_cont(p->ctl, h, s); }, &cont);
    }
    if (st != PAKR_OK)
        return st;
    cudaGraphExec_t exec = nullptr;
    CUDA_TRY(cudaGraphInstantiate(&exec, g, 0));
    p->plan_graph = g;
    p->plan_exec = exec;
    return PAKR_OK;
}

pakr_status build_expand_graph(pakr_planner *p, bool tc)
{
    if (p->expand_exec[tc])
        return PAKR_OK;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphNode_t sample_node = nullptr, last = nullptr;
    pakr_status st = add_expansion(p, g, nullptr, 0.f, 0ull, MODE_EXPAND, tc ? NN_ONLY_TC : NN_ONLY_FP32, &sample_node,
                                   &last);
    if (st != PAKR_OK) {
        cudaGraphDestroy(g);
        return st;
    }
    cudaGraphExec_t exec = nullptr;
    CUDA_TRY(cudaGraphInstantiate(&exec, g, 0));
    p->expand_graph[tc] = g;
    p->expand_exec[tc] = exec;
    p->expand_sample[tc] = sample_node;
    return PAKR_OK;
}

// One expansion through the graph of the chosen nearest-neighbour kernel: the sample node's
// bound and seed arguments are replaced (a host-side update of the instantiated graph), then
// one graph launch.
pakr_status launch_expand_graph(pakr_planner *p, float bound, uint64_t seed, bool tc)
{
    pakr_status st = build_expand_graph(p, tc);
    if (st != PAKR_OK)
        return st;
    cudaKernelNodeParams kp{};
    CUDA_TRY(cudaGraphKernelNodeGetParams(p->expand_sample[tc], &kp));
    void *args[kSampleArgs];
    unsigned long long seed_arg = seed;
    for (int i = 0; i < kSampleArgs; ++i)
        args[i] = kp.kernelParams[i];
    args[kSampleArgBound] = &bound;
    args[kSampleArgSeed] = &seed_arg;
    kp.kernelParams = args;
    kp.extra = nullptr;
    CUDA_TRY(cudaGraphExecKernelNodeSetParams(p->expand_exec[tc], p->expand_sample[tc], &kp));
    CUDA_TRY(cudaGraphLaunch(p->expand_exec[tc], p->stream));
    return PAKR_OK;
}

pakr_status read_ctl(pakr_planner *p)
{
    CUDA_TRY(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    p->n_upper = p->ctl_host->count;
    return PAKR_OK;
}

}  // namespace

// Checks the problem part of a description (everything but obstacles and
// tree size) and fills the matching kernel constants; obstacles, counts and
// the tree capacity are left for the caller.  Shared with the batched planner.
pakr_status pakr::fill_problem(const pakr_problem_desc *desc, DevProblem *P, int *d_out, int *m_out, int *pdim_out)
{
    if (!desc || !P)
        return fail(PAKR_ERR_INVALID_ARG, "NULL argument");
    pakr_problem_desc d = *desc;
    d.n_boxes = 0;
    d.boxes = nullptr;
    d.n_spheres = 0;
    d.spheres = nullptr;
    d.tree_cap = 1;
    DimInfo di;
    pakr_status st = check_desc(&d, &di);
    if (st != PAKR_OK)
        return st;
    *P = DevProblem{};
    P->dyn = d.dynamics;
    P->d = di.d;
    P->m = di.m;
    P->pdim = di.pdim;
    for (int a = 0; a < kMaxD; ++a) {
        P->x_lo[a] = a < di.d ? d.x_lo[a] : 0.f;
        P->x_hi[a] = a < di.d ? d.x_hi[a] : 0.f;
        P->sw[a] = (a < di.d && d.nn_weights) ? std::sqrt(d.nn_weights[a]) : 1.f;
    }
    for (int a = 0; a < kMaxM; ++a) {
        P->u_lo[a] = a < di.m ? d.u_lo[a] : 0.f;
        P->u_hi[a] = a < di.m ? d.u_hi[a] : 0.f;
    }
    const float quad_default[5] = {1.f, 0.01f, 0.01f, 0.02f, 9.81f};
    for (int a = 0; a < 8; ++a)
        P->model[a] = a < 5 ? (d.model_params ? d.model_params[a] : quad_default[a]) : 0.f;
    P->dt = d.dt;
    P->goal_r = d.goal_radius;
    P->h_speed = d.heuristic_speed;
    P->s_min = d.steps_min;
    P->s_max = d.steps_max;
    P->cost = d.cost;
    P->heuristic = d.heuristic;
    P->K = d.n_parents;
    P->k = d.branching;
    for (int a = 0; a < kMaxD; ++a)  // nearest-neighbour coordinates are centred on the state box
        P->tc_c[a] = a < di.d ? 0.5f * (d.x_lo[a] + d.x_hi[a]) * P->sw[a] : 0.f;
    *d_out = di.d;
    *m_out = di.m;
    *pdim_out = di.pdim;
    return PAKR_OK;
}

const DevProblem *pakr::planner_problem(const pakr_planner *p) { return &p->P; }
cudaStream_t pakr::planner_stream(const pakr_planner *p) { return p->stream; }
int pakr::planner_device(const pakr_planner *p) { return p->device; }

extern "C" {

const char *pakr_version(void) { return "pakr-gb300 0.1 (sm_103a)"; }

const char *pakr_last_error(void) { return g_last_error.c_str(); }

pakr_status pakr_workspace_size(const pakr_problem_desc *desc, uint64_t *bytes_out)
{
    DimInfo di;
    pakr_status st = check_desc(desc, &di);
    if (st != PAKR_OK)
        return st;
    if (!bytes_out)
        return fail(PAKR_ERR_INVALID_ARG, "bytes_out is NULL");
    const int pc = desc->path_cap ? desc->path_cap : 4096;
    const int hc = desc->history_cap ? desc->history_cap : 1024;
    Layout L = make_layout(di, desc->tree_cap, desc->n_parents, desc->branching, desc->n_boxes, desc->n_spheres, pc,
                           hc, tc_floats(desc, di), build_obstacle_grid(desc, di));
    *bytes_out = L.total + 256;  // slack for aligning the caller's base pointer
    return PAKR_OK;
}

pakr_status pakr_create(const pakr_problem_desc *desc, pakr_planner **out)
{
    if (!out)
        return fail(PAKR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    DimInfo di;
    pakr_status st = check_desc(desc, &di);
    if (st != PAKR_OK)
        return st;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (desc->device < 0 || desc->device >= ndev)
        return fail(PAKR_ERR_INVALID_ARG, "device %d out of range (%d devices)", desc->device, ndev);
    DeviceGuard guard(desc->device);

    pakr_planner *p = new pakr_planner();
    p->device = desc->device;
    p->stream = (cudaStream_t)desc->cuda_stream;
    p->di = di;
    p->cap = desc->tree_cap;
    p->K = desc->n_parents;
    p->k = desc->branching;
    p->path_cap = desc->path_cap ? desc->path_cap : 4096;
    p->hist_cap = desc->history_cap ? desc->history_cap : 1024;
    const ObstacleGrid grid = build_obstacle_grid(desc, di);
    p->lay = make_layout(di, p->cap, p->K, p->k, desc->n_boxes, desc->n_spheres, p->path_cap, p->hist_cap,
                         tc_floats(desc, di), grid);

    auto cleanup = [&](pakr_status s) {
        pakr_destroy(p);
        return s;
    };

    if (desc->workspace) {
        uintptr_t b = (uintptr_t)desc->workspace;
        uintptr_t aligned = (b + 255) & ~(uintptr_t)255;
        if (desc->workspace_bytes < p->lay.total + (aligned - b))
            return cleanup(fail(PAKR_ERR_OOM, "workspace too small: need %zu bytes (+256 for alignment), got %llu",
                                p->lay.total, (unsigned long long)desc->workspace_bytes));
        p->base = (char *)aligned;
        p->owns_base = false;
    } else {
        cudaError_t e = cudaMalloc(&p->base, p->lay.total);
        if (e != cudaSuccess)
            return cleanup(fail(PAKR_ERR_OOM, "cudaMalloc(%zu) failed: %s", p->lay.total, cudaGetErrorString(e)));
        p->owns_base = true;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return cleanup(fail(PAKR_ERR_CUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e)));
    e = cudaMallocHost(&p->ctl_host, sizeof(Ctl));
    if (e == cudaSuccess)
        e = cudaMallocHost(&p->pp_host, sizeof(PlanParams));
    if (e == cudaSuccess)
        e = cudaMallocHost(&p->stage_host, sizeof(PlanStage));
    if (e != cudaSuccess)
        return cleanup(fail(PAKR_ERR_OOM, "cudaMallocHost failed: %s", cudaGetErrorString(e)));

    char *b = p->base;
    const Layout &L = p->lay;
    p->T = DevTree{(float *)(b + L.X), (float *)(b + L.U), (float *)(b + L.cost), (float *)(b + L.fcost),
                   (int *)(b + L.parent), (int *)(b + L.steps),
                   tc_floats(desc, di) > 0 ? (float *)(b + L.XT) : nullptr};
    p->W = DevWork{(float *)(b + L.xr),       (unsigned long long *)(b + L.nn_key),
                   (float *)(b + L.st_x),     (float *)(b + L.st_u),
                   (float *)(b + L.st_cost),  (float *)(b + L.st_f),
                   (int *)(b + L.st_steps),   (int *)(b + L.st_parent),
                   (int8_t *)(b + L.outcome), (int8_t *)(b + L.goal),
                   (int *)(b + L.block_count), (unsigned *)(b + L.nn_amin)};
    p->ctl = (Ctl *)(b + L.ctl);
    p->pp = (PlanParams *)(b + L.pp);
    p->B = DevPlanBufs{(int *)(b + L.path_nodes), (float *)(b + L.path_x), (float *)(b + L.path_u),
                       (int *)(b + L.path_steps), p->path_cap, (unsigned long long *)(b + L.hist_t),
                       (float *)(b + L.hist_cost), (long long *)(b + L.hist_iter), p->hist_cap};

    DevProblem &P = p->P;
    P.dyn = desc->dynamics;
    P.d = di.d;
    P.m = di.m;
    P.pdim = di.pdim;
    for (int a = 0; a < kMaxD; ++a) {
        P.x_lo[a] = a < di.d ? desc->x_lo[a] : 0.f;
        P.x_hi[a] = a < di.d ? desc->x_hi[a] : 0.f;
        P.sw[a] = (a < di.d && desc->nn_weights) ? std::sqrt(desc->nn_weights[a]) : 1.f;
    }
    for (int a = 0; a < kMaxM; ++a) {
        P.u_lo[a] = a < di.m ? desc->u_lo[a] : 0.f;
        P.u_hi[a] = a < di.m ? desc->u_hi[a] : 0.f;
    }
    const float quad_default[5] = {1.f, 0.01f, 0.01f, 0.02f, 9.81f};
    for (int a = 0; a < 8; ++a)
        P.model[a] = a < 5 ? (desc->model_params ? desc->model_params[a] : quad_default[a]) : 0.f;
    P.dt = desc->dt;
    P.goal_r = desc->goal_radius;
    P.h_speed = desc->heuristic_speed;
    P.s_min = desc->steps_min;
    P.s_max = desc->steps_max;
    P.n_boxes = desc->n_boxes;
    P.n_spheres = desc->n_spheres;
    P.boxes = (const float4 *)(b + L.boxes);
    P.spheres = (const float4 *)(b + L.spheres);
    P.cost = desc->cost;
    P.heuristic = desc->heuristic;
    P.K = desc->n_parents;
    P.k = desc->branching;
    P.cap = (int)desc->tree_cap;
    // tensor-core filter: centre and radius of the weighted state box (rounded up)
    {
        double r2 = 0.0;
        for (int a = 0; a < kMaxD; ++a) {
            P.tc_c[a] = a < di.d ? 0.5f * (desc->x_lo[a] + desc->x_hi[a]) * P.sw[a] : 0.f;
            if (a < di.d) {
                const double h = 0.5 * ((double)desc->x_hi[a] - (double)desc->x_lo[a]) * P.sw[a];
                r2 += h * h;
            }
        }
        P.tc_xbox2 = (float)(r2 * 1.0001 + 1e-30);
        P.tc_s = tc_scale(P.tc_xbox2);
        P.tc_min_n = p->T.XT ? tc_min_nodes(desc) : 0x7FFFFFFF;
        if (p->T.XT) {
            e = tc_configure(P);
            if (e != cudaSuccess)
                return cleanup(fail(PAKR_ERR_CUDA, "tensor-core kernel setup failed: %s", cudaGetErrorString(e)));
        }
    }

    // Obstacles as padded float4 records.
    std::vector<float4> box4(2 * (size_t)desc->n_boxes), sph4((size_t)desc->n_spheres);
    const int pd = di.pdim;
    for (int i = 0; i < desc->n_boxes; ++i) {
        const float *r = desc->boxes + (size_t)i * 2 * pd;
        box4[2 * i] = make_float4(r[0], r[1], pd > 2 ? r[2] : 0.f, 0.f);
        box4[2 * i + 1] = make_float4(r[pd], r[pd + 1], pd > 2 ? r[pd + 2] : 0.f, 0.f);
    }
    for (int i = 0; i < desc->n_spheres; ++i) {
        const float *r = desc->spheres + (size_t)i * (pd + 1);
        sph4[i] = make_float4(r[0], r[1], pd > 2 ? r[2] : 0.f, r[pd]);
    }
    if (!box4.empty()) {
        e = cudaMemcpy(b + L.boxes, box4.data(), sizeof(float4) * box4.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return cleanup(fail(PAKR_ERR_CUDA, "obstacle upload failed: %s", cudaGetErrorString(e)));
    }
    if (!sph4.empty()) {
        e = cudaMemcpy(b + L.spheres, sph4.data(), sizeof(float4) * sph4.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return cleanup(fail(PAKR_ERR_CUDA, "obstacle upload failed: %s", cudaGetErrorString(e)));
    }
    if (grid.g > 0) {
        e = cudaMemcpy(b + L.grid_start, grid.start.data(), sizeof(int) * grid.start.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b + L.grid_items, grid.items.data(), sizeof(unsigned short) * grid.items.size(),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return cleanup(fail(PAKR_ERR_CUDA, "obstacle grid upload failed: %s", cudaGetErrorString(e)));
        P.grid_g = grid.g;
        P.grid_cells = grid.cells;
        P.grid_n_items = (int)grid.items.size();
        for (int a = 0; a < 3; ++a) {
            P.grid_lo[a] = grid.lo[a];
            P.grid_inv[a] = grid.inv[a];
        }
        P.grid_start = (const int *)(b + L.grid_start);
        P.grid_items = (const unsigned short *)(b + L.grid_items);
    }
    e = preload_offer_bound();
    if (e == cudaSuccess)
        e = preload_plan_snapshot();
    if (e != cudaSuccess)
        return cleanup(fail(PAKR_ERR_CUDA, "loading the bound-offer kernel failed: %s", cudaGetErrorString(e)));
    e = cudaMemset(p->ctl, 0, sizeof(Ctl));
    // The tensor-core filter stages whole 128-node halves of the packed copy: rows past the
    // tree are masked by their norm column, but their coordinate columns still enter the
    // products, so they must hold finite values (zeros here, or rows of earlier nodes after a
    // truncation), never a stale bit pattern that reads as an infinity.
    if (e == cudaSuccess && p->T.XT)
        e = cudaMemset(p->T.XT, 0, L.xr - L.XT);
    if (e != cudaSuccess)
        return cleanup(fail(PAKR_ERR_CUDA, "cudaMemset failed: %s", cudaGetErrorString(e)));

    // Launch configuration.
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    LaunchCfg &C = p->L;
    C.sample_threads = kSampleThreads;
    C.sample_blocks = (p->K + kSampleThreads - 1) / kSampleThreads;
    // With the tensor-core kernel on, the FP32 kernel only sees trees below its switch
    // (28672 nodes): there, blocks of 1024 queries leave most SMs idle (a 4096-node tree fills
    // 64 of 456 blocks), so the 128-query blocks are used instead (4096 nodes: 12.6 vs
    // 16.4 us; 16384: 20.3 vs 25.3 us).
    const bool nn_small_trees_only = tc_min_nodes(desc) < 0x7FFFFFFF;
    if (p->K >= 1024 && !nn_small_trees_only) {
        C.nn_variant = 2;
        C.nn_threads = 256;
        C.nn_qpt = 4;
    } else if (p->K >= 256 && !nn_small_trees_only) {
        C.nn_variant = 1;
        C.nn_threads = 128;
        C.nn_qpt = 2;
    } else {
        C.nn_variant = 0;
        C.nn_threads = 64;
        C.nn_qpt = 2;
    }
    const int per_block = C.nn_threads * C.nn_qpt;
    C.nn_qgroups = (p->K + per_block - 1) / per_block;
    const int occ = std::max(1, nn_blocks_per_sm(di.d, C.nn_variant));
    C.nn_chunks = std::max(1, sms * occ / C.nn_qgroups);
    // tensor-core grid: kTcCtasPerSm CTAs per SM; node chunks x query blocks in near-full waves
    C.tc_qblocks = (p->K + 127) / 128;  // 128 queries per tensor-core CTA
    const int tc_slots = sms * kTcCtasPerSm;
    C.tc_chunks = std::max(1, tc_slots / C.tc_qblocks);
    for (int w = 1; w <= 16; ++w) {
        const int c = (w * tc_slots + C.tc_qblocks - 1) / C.tc_qblocks;
        const int items = c * C.tc_qblocks;
        const int waves = (items + tc_slots - 1) / tc_slots;
        if ((double)items / ((double)waves * tc_slots) >= 0.95) {
            C.tc_chunks = c;
            break;
        }
    }
    // one full wave with an even number of chunks: pair the CTAs launched first and second
    // (k_nn_tc), the first taking kTcPairShare of each pair's tiles
    p->P.tc_pair_share =
        (C.tc_chunks * C.tc_qblocks == tc_slots && C.tc_chunks % 2 == 0 && kTcCtasPerSm == 2) ? kTcPairShare : 0.f;
    const int64_t R = (int64_t)p->K * p->k;
    // Lanes per rollout: as many as fit one resident wave of k_propagate on every SM (six
    // 256-thread blocks, its register limit), but no more lanes than there are obstacle tests
    // per substep to split between them (all obstacles, or with the obstacle grid the mean
    // length of a cell's list).  More lanes shorten each substep's obstacle tests, the
    // kernel's latency chain; one lane needs no ballot per substep.
    const double tests = grid.g > 0 ? (double)grid.items.size() / grid.cells : (double)(desc->n_boxes + desc->n_spheres);
    int lanes = 1;
    while (lanes < kMaxPropLanes && R * lanes * 2 <= (int64_t)sms * 1536 && lanes * 2 <= std::max(1.0, tests))
        lanes *= 2;
    C.prop_lanes = lanes;
    // 256-thread blocks at every lane count (measured at one lane per rollout: 128- and
    // 64-thread blocks, which spread the rollouts over more SMs, took 22.8 and 27.0 us for di3
    // and 57.3 and 65.1 us for the quadrotor, against 20.9 and 54.2 us)
    C.prop_threads = kPropThreads;
    const int64_t rollouts_per_block = C.prop_threads / lanes;
    C.prop_blocks = (int)((R + rollouts_per_block - 1) / rollouts_per_block);
    C.obs_smem_bytes = propagate_smem_bytes(desc->n_boxes, desc->n_spheres, P.grid_cells, P.grid_n_items);
    *out = p;
    g_last_error.clear();
    return PAKR_OK;
}

void pakr_destroy(pakr_planner *p)
{
    if (!p)
        return;
    DeviceGuard guard(p->device);
    if (p->stream || true)
        cudaStreamSynchronize(p->stream);
    if (p->plan_exec)
        cudaGraphExecDestroy(p->plan_exec);
    if (p->plan_graph)
        cudaGraphDestroy(p->plan_graph);
    for (int k = 0; k < 2; ++k) {
        if (p->expand_exec[k])
            cudaGraphExecDestroy(p->expand_exec[k]);
        if (p->expand_graph[k])
            cudaGraphDestroy(p->expand_graph[k]);
    }
    for (auto &pe : p->pending)
        p->pool.push_back(pe.second);
    for (auto &ev : p->pool) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    if (p->owns_base && p->base)
        cudaFree(p->base);
    if (p->ctl_host)
        cudaFreeHost(p->ctl_host);
    if (p->pp_host)
        cudaFreeHost(p->pp_host);
    if (p->stage_host)
        cudaFreeHost(p->stage_host);
    if (p->capture_stream)
        cudaStreamDestroy(p->capture_stream);
    delete p;
}

pakr_status pakr_tree_reset(pakr_planner *p, const float *x_init, const float *x_goal)
{
    if (!p || !x_init || !x_goal)
        return fail(PAKR_ERR_INVALID_ARG, "NULL argument");
    if (!finite_all(x_init, p->di.d) || !finite_all(x_goal, p->di.d))
        return fail(PAKR_ERR_INVALID_ARG, "x_init / x_goal must be finite");
    DeviceGuard guard(p->device);
    PlanParams *h = p->pp_host;
    memset(h, 0, sizeof(PlanParams));
    memcpy(h->x_init, x_init, sizeof(float) * p->di.d);
    memcpy(h->x_goal, x_goal, sizeof(float) * p->di.d);
    CUDA_TRY(cudaMemcpyAsync(p->pp, h, sizeof(PlanParams), cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(cudaMemcpyAsync(p->ctl->x_goal, p->pp->x_goal, sizeof(float) * kMaxD, cudaMemcpyDeviceToDevice,
                             p->stream));
    CUDA_TRY(launch_tree_reset(p->P, p->ctl, p->T, p->pp->x_init, p->stream));
    pakr_status st = read_ctl(p);
    if (st != PAKR_OK)
        return st;
    if (!p->ctl_host->status)
        return fail(PAKR_ERR_INVALID_ARG, "x_init is not a valid state (outside the state box or in an obstacle)");
    return PAKR_OK;
}

pakr_status pakr_expand(pakr_planner *p, float cost_bound, uint64_t seed, pakr_expand_info *info)
{
    if (!p)
        return fail(PAKR_ERR_INVALID_ARG, "planner is NULL");
    if (std::isnan(cost_bound))
        return fail(PAKR_ERR_INVALID_ARG, "cost_bound is NaN");
    DeviceGuard guard(p->device);
    // per-kernel timing needs events between the launches: plain launches then
    const bool tc = use_tc_nn(p);
    pakr_status st = p->profiling ? enqueue_expand(p, cost_bound, seed, tc) : launch_expand_graph(p, cost_bound, seed, tc);
    if (st != PAKR_OK)
        return st;
    p->n_upper = std::min<int64_t>(p->cap, p->n_upper + (int64_t)p->K * p->k);
    if (!info)
        return st;
    st = read_ctl(p);
    if (st != PAKR_OK)
        return st;
    const Ctl &c = *p->ctl_host;
    info->n_start = c.n_start;
    info->n_appended = c.n_appended;
    info->n_pruned = c.n_pruned;
    info->n_collided = c.n_collided;
    info->n_no_parent = c.n_no_parent;
    info->n_dropped = c.n_dropped;
    info->goal_found = c.goal_key != kNoKey;
    info->reserved = 0;
    info->goal_idx = info->goal_found ? (int64_t)(uint32_t)(c.goal_key & 0xFFFFFFFFull) : -1;
    uint32_t bits = (uint32_t)(c.goal_key >> 32);
    float gc;
    memcpy(&gc, &bits, sizeof(gc));
    info->goal_cost = info->goal_found ? gc : INFINITY;
    info->iteration = c.iteration - 1u;
    if (c.err)
        return fail(PAKR_ERR_DEVICE, "device error flags 0x%x", c.err);
    if (c.n_no_parent >= (int64_t)p->K * p->k)
        return PAKR_NO_ELIGIBLE;
    if (info->goal_found)
        return PAKR_GOAL_REACHED;
    if (c.n_dropped > 0)
        return PAKR_TREE_FULL;
    return PAKR_OK;
}

pakr_status pakr_plan(pakr_planner *p, const float *x_init, const float *x_goal, double budget_s,
                      int64_t max_iterations, uint64_t seed, uint32_t flags, pakr_path *out)
{
    return pakr_plan_bounded(p, x_init, x_goal, budget_s, max_iterations, seed, flags, INFINITY, out);
}

pakr_status pakr_plan_bounded(pakr_planner *p, const float *x_init, const float *x_goal, double budget_s,
                              int64_t max_iterations, uint64_t seed, uint32_t flags, float initial_bound,
                              pakr_path *out)
{
    if (std::isnan(initial_bound))
        return fail(PAKR_ERR_INVALID_ARG, "initial_bound is NaN");
    if (!p || !x_init || !x_goal || !out)
        return fail(PAKR_ERR_INVALID_ARG, "NULL argument");
    if (!finite_all(x_init, p->di.d) || !finite_all(x_goal, p->di.d))
        return fail(PAKR_ERR_INVALID_ARG, "x_init / x_goal must be finite");
    if (std::isnan(budget_s) || budget_s < 0)
        return fail(PAKR_ERR_INVALID_ARG, "budget_s must be >= 0");
    if (out->max_edges < 0 || out->max_history < 0 ||
        (out->max_edges > 0 && (!out->states || !out->controls || !out->steps)) ||
        (out->max_history > 0 && (!out->history_time_s || !out->history_cost || !out->history_iteration)))
        return fail(PAKR_ERR_INVALID_ARG, "path buffers missing for the given capacities");
    DeviceGuard guard(p->device);
    pakr_status st = build_plan_graph(p);
    if (st != PAKR_OK)
        return st;
    PlanParams *h = p->pp_host;
    memset(h, 0, sizeof(PlanParams));
    memcpy(h->x_init, x_init, sizeof(float) * p->di.d);
    memcpy(h->x_goal, x_goal, sizeof(float) * p->di.d);
    h->seed = seed;
    const double ns = budget_s * 1e9;
    h->budget_ns = ns >= 1.8e19 ? ~0ull : (unsigned long long)ns;
    h->max_iterations = max_iterations > 0 ? std::min<int64_t>(max_iterations, kMaxPlanIterations) : kMaxPlanIterations;
    h->stop_at_first = (flags & PAKR_PLAN_STOP_AT_FIRST) ? 1 : 0;
    h->c_best_init = initial_bound;
    CUDA_TRY(cudaMemcpyAsync(p->pp, h, sizeof(PlanParams), cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(cudaGraphLaunch(p->plan_exec, p->stream));
    // the control block, then the first kStageHist history entries and kStageEdges path edges
    // into pinned staging, and one synchronization: a result that fits needs no second one
    PlanStage *sg = p->stage_host;
    const int d = p->di.d, m = p->di.m;
    const int sh = std::min(kStageHist, p->hist_cap), se = std::min(kStageEdges, p->path_cap);
    CUDA_TRY(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, p->stream));
    if (sh > 0) {
        CUDA_TRY(cudaMemcpyAsync(sg->t, p->B.hist_t, sizeof(unsigned long long) * sh, cudaMemcpyDeviceToHost,
                                 p->stream));
        CUDA_TRY(cudaMemcpyAsync(sg->cost, p->B.hist_cost, sizeof(float) * sh, cudaMemcpyDeviceToHost, p->stream));
        CUDA_TRY(cudaMemcpyAsync(sg->iter, p->B.hist_iter, sizeof(long long) * sh, cudaMemcpyDeviceToHost,
                                 p->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(sg->x, p->B.path_x, sizeof(float) * d * (size_t)(se + 1), cudaMemcpyDeviceToHost,
                             p->stream));
    if (se > 0) {
        CUDA_TRY(cudaMemcpyAsync(sg->u, p->B.path_u + m, sizeof(float) * m * (size_t)se, cudaMemcpyDeviceToHost,
                                 p->stream));
        CUDA_TRY(cudaMemcpyAsync(sg->steps, p->B.path_steps + 1, sizeof(int) * (size_t)se, cudaMemcpyDeviceToHost,
                                 p->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    p->n_upper = p->ctl_host->count;
    const Ctl &c = *p->ctl_host;
    out->cost = c.n_solutions > 0 ? c.sol_best : INFINITY;
    out->n_solutions = c.n_solutions;
    out->n_restarts = c.n_restarts;
    out->iterations = c.iterations_done;
    out->t_first_solution_s = c.t_first_ns == ~0ull ? -1.0 : (double)c.t_first_ns * 1e-9;
    out->nodes_first_solution = c.n_solutions > 0 ? c.nodes_first : -1;
    out->iterations_first_solution = c.n_solutions > 0 ? c.iterations_first : -1;
    out->t_total_s = (double)(c.t_end_ns - c.t0_ns) * 1e-9;
    out->n_edges = 0;
    if (c.err)
        return fail(PAKR_ERR_DEVICE, "device error flags 0x%x", c.err);
    if (c.plan_status == -1)
        return fail(PAKR_ERR_INVALID_ARG, "x_init is not a valid state (outside the state box or in an obstacle)");
    const int nh = std::min(std::min(c.n_solutions, p->hist_cap), out->max_history);
    if (nh > 0 && nh <= sh) {
        for (int i = 0; i < nh; ++i) {
            out->history_time_s[i] = (double)sg->t[i] * 1e-9;
            out->history_cost[i] = sg->cost[i];
            out->history_iteration[i] = sg->iter[i];
        }
    } else if (nh > 0) {
        std::vector<unsigned long long> ht(nh);
        CUDA_TRY(cudaMemcpyAsync(ht.data(), p->B.hist_t, sizeof(unsigned long long) * nh, cudaMemcpyDeviceToHost,
                                 p->stream));
        CUDA_TRY(cudaMemcpyAsync(out->history_cost, p->B.hist_cost, sizeof(float) * nh, cudaMemcpyDeviceToHost,
                                 p->stream));
        CUDA_TRY(cudaMemcpyAsync(out->history_iteration, p->B.hist_iter, sizeof(long long) * nh,
                                 cudaMemcpyDeviceToHost, p->stream));
        CUDA_TRY(cudaStreamSynchronize(p->stream));
        for (int i = 0; i < nh; ++i)
            out->history_time_s[i] = (double)ht[i] * 1e-9;
    }
    if (c.n_solutions > 0) {
        if (c.path_len < 0) {
            out->n_edges = -c.path_len - 1;
            return fail(PAKR_ERR_INVALID_ARG, "best path has %d edges, more than path_cap %d", out->n_edges,
                        p->path_cap);
        }
        const int edges = c.path_len - 1;
        out->n_edges = edges;
        if (edges > out->max_edges)
            return fail(PAKR_ERR_INVALID_ARG, "best path has %d edges, more than max_edges %d", edges,
                        out->max_edges);
        if (edges <= se) {
            if (out->states)
                memcpy(out->states, sg->x, sizeof(float) * d * (size_t)(edges + 1));
            if (edges > 0) {
                memcpy(out->controls, sg->u, sizeof(float) * m * (size_t)edges);
                memcpy(out->steps, sg->steps, sizeof(int) * (size_t)edges);
            }
            return PAKR_GOAL_REACHED;
        }
        CUDA_TRY(cudaMemcpyAsync(out->states, p->B.path_x, sizeof(float) * d * (size_t)(edges + 1),
                                 cudaMemcpyDeviceToHost, p->stream));
        if (edges > 0) {
            CUDA_TRY(cudaMemcpyAsync(out->controls, p->B.path_u + m, sizeof(float) * m * (size_t)edges,
                                     cudaMemcpyDeviceToHost, p->stream));
            CUDA_TRY(cudaMemcpyAsync(out->steps, p->B.path_steps + 1, sizeof(int) * (size_t)edges,
                                     cudaMemcpyDeviceToHost, p->stream));
        }
        CUDA_TRY(cudaStreamSynchronize(p->stream));
        return PAKR_GOAL_REACHED;
    }
    if (c.plan_status == 3)
        return PAKR_NO_ELIGIBLE;
    return PAKR_BUDGET_EXPIRED;
}

pakr_status pakr_plan_offer_bound(pakr_planner *p, const float *cost_dev, void *cuda_stream)
{
    if (!p || !cost_dev)
        return fail(PAKR_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(p->device);
    CUDA_TRY(launch_offer_bound(p->ctl, cost_dev, (cudaStream_t)cuda_stream));
    return PAKR_OK;
}

pakr_status pakr_plan_snapshot(pakr_planner *p, float *states_dev, float *controls_dev, int32_t *steps_dev,
                               int32_t max_edges, int32_t *info_dev, void *cuda_stream)
{
    if (!p || !states_dev || !controls_dev || !steps_dev || !info_dev || max_edges < 1)
        return fail(PAKR_ERR_INVALID_ARG, "NULL buffer or max_edges < 1");
    DeviceGuard guard(p->device);
    CUDA_TRY(launch_plan_snapshot(p->ctl, p->B, p->di.d, p->di.m, states_dev, controls_dev, steps_dev,
                                  std::min(max_edges, p->path_cap), info_dev, (cudaStream_t)cuda_stream));
    return PAKR_OK;
}

pakr_status pakr_tree_size(pakr_planner *p, int64_t *count, uint32_t *iteration)
{
    if (!p || !count)
        return fail(PAKR_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(p->device);
    pakr_status st = read_ctl(p);
    if (st != PAKR_OK)
        return st;
    *count = p->ctl_host->count;
    if (iteration)
        *iteration = p->ctl_host->iteration;
    return PAKR_OK;
}

pakr_status pakr_tree_export(pakr_planner *p, pakr_tree_host *t)
{
    if (!p || !t)
        return fail(PAKR_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(p->device);
    pakr_status st = read_ctl(p);
    if (st != PAKR_OK)
        return st;
    const int64_t n = p->ctl_host->count;
    t->iteration = p->ctl_host->iteration;
    if (t->capacity < n) {
        t->count = n;
        return fail(PAKR_ERR_INVALID_ARG, "tree has %lld nodes, capacity %lld", (long long)n,
                    (long long)t->capacity);
    }
    t->count = n;
    if (n == 0)
        return PAKR_OK;
    if (!t->states || !t->controls || !t->parents || !t->costs || !t->steps)
        return fail(PAKR_ERR_INVALID_ARG, "tree buffers missing");
    const int d = p->di.d, m = p->di.m;
    std::vector<float> row((size_t)n);
    for (int a = 0; a < d; ++a) {
        CUDA_TRY(cudaMemcpy(row.data(), p->T.X + (size_t)a * p->cap, sizeof(float) * n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i)
            t->states[i * d + a] = row[i];
    }
    for (int a = 0; a < m; ++a) {
        CUDA_TRY(cudaMemcpy(row.data(), p->T.U + (size_t)a * p->cap, sizeof(float) * n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i)
            t->controls[i * m + a] = row[i];
    }
    CUDA_TRY(cudaMemcpy(t->parents, p->T.parent, sizeof(int) * n, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(t->costs, p->T.cost, sizeof(float) * n, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(t->steps, p->T.steps, sizeof(int) * n, cudaMemcpyDeviceToHost));
    return PAKR_OK;
}

pakr_status pakr_tree_truncate(pakr_planner *p, int64_t count)
{
    if (!p)
        return fail(PAKR_ERR_INVALID_ARG, "planner is NULL");
    if (count < 1 || count > p->cap)
        return fail(PAKR_ERR_INVALID_ARG, "count %lld outside [1, tree_cap]", (long long)count);
    DeviceGuard guard(p->device);
    CUDA_TRY(launch_truncate(p->ctl, (int)count, p->stream));
    p->n_upper = std::min<int64_t>(p->n_upper, count);
    return PAKR_OK;
}

pakr_status pakr_tree_import(pakr_planner *p, const pakr_tree_host *t, const float *x_goal)
{
    if (!p || !t || !x_goal)
        return fail(PAKR_ERR_INVALID_ARG, "NULL argument");
    const int64_t n = t->count;
    if (n < 1 || n > p->cap || t->capacity < n)
        return fail(PAKR_ERR_INVALID_ARG, "count %lld outside [1, tree_cap=%lld]", (long long)n, (long long)p->cap);
    if (!t->states || !t->controls || !t->parents || !t->costs || !t->steps)
        return fail(PAKR_ERR_INVALID_ARG, "tree buffers missing");
    if (!finite_all(x_goal, p->di.d))
        return fail(PAKR_ERR_INVALID_ARG, "x_goal must be finite");
    if (t->parents[0] != -1)
        return fail(PAKR_ERR_INVALID_ARG, "node 0 must be the root (parent -1)");
    for (int64_t i = 1; i < n; ++i)
        if (t->parents[i] < 0 || t->parents[i] >= i)
            return fail(PAKR_ERR_INVALID_ARG, "parent of node %lld is %d, must be in [0, %lld)", (long long)i,
                        t->parents[i], (long long)i);
    for (int64_t i = 0; i < n; ++i)
        if (!(t->costs[i] >= 0.f) || !std::isfinite(t->costs[i]))
            return fail(PAKR_ERR_INVALID_ARG, "cost of node %lld must be finite and >= 0", (long long)i);
    const int d = p->di.d, m = p->di.m;
    if (!finite_all(t->states, (int)std::min<int64_t>(n * d, 0x7FFFFFFF)))
        return fail(PAKR_ERR_INVALID_ARG, "states must be finite");
    DeviceGuard guard(p->device);
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    std::vector<float> row((size_t)n);
    for (int a = 0; a < d; ++a) {
        for (int64_t i = 0; i < n; ++i)
            row[i] = t->states[i * d + a];
        CUDA_TRY(cudaMemcpy(p->T.X + (size_t)a * p->cap, row.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    for (int a = 0; a < m; ++a) {
        for (int64_t i = 0; i < n; ++i)
            row[i] = t->controls[i * m + a];
        CUDA_TRY(cudaMemcpy(p->T.U + (size_t)a * p->cap, row.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(p->T.parent, t->parents, sizeof(int) * n, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->T.cost, t->costs, sizeof(float) * n, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->T.steps, t->steps, sizeof(int) * n, cudaMemcpyHostToDevice));
    Ctl *h = p->ctl_host;
    memset(h, 0, sizeof(Ctl));
    h->count = (int)n;
    h->iteration = t->iteration;
    for (int a = 0; a < d; ++a)
        h->x_goal[a] = x_goal[a];
    h->c_best = INFINITY;
    h->status = 1;
    CUDA_TRY(cudaMemcpyAsync(p->ctl, h, sizeof(Ctl), cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(launch_import_fcost(p->P, p->ctl, p->T, (int)n, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    p->n_upper = n;
    return PAKR_OK;
}

pakr_status pakr_debug_last_expand(pakr_planner *p, float *samples, int32_t *near, int8_t *outcome,
                                   int8_t *goal, float *controls, int32_t *steps)
{
    if (!p)
        return fail(PAKR_ERR_INVALID_ARG, "planner is NULL");
    DeviceGuard guard(p->device);
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    const int K = p->K, d = p->di.d, m = p->di.m;
    const size_t R = (size_t)K * p->k;
    if (samples) {
        std::vector<float> v((size_t)K * d);
        CUDA_TRY(cudaMemcpy(v.data(), p->W.xr, sizeof(float) * v.size(), cudaMemcpyDeviceToHost));
        for (int i = 0; i < K; ++i)
            for (int a = 0; a < d; ++a)
                samples[(size_t)i * d + a] = v[(size_t)a * K + i];
    }
    if (near) {
        std::vector<unsigned long long> v(K);
        CUDA_TRY(cudaMemcpy(v.data(), p->W.nn_key, sizeof(unsigned long long) * K, cudaMemcpyDeviceToHost));
        for (int i = 0; i < K; ++i)
            near[i] = v[i] == kNoKey ? -1 : (int32_t)(uint32_t)(v[i] & 0xFFFFFFFFull);
    }
    if (outcome)
        CUDA_TRY(cudaMemcpy(outcome, p->W.outcome, R, cudaMemcpyDeviceToHost));
    if (goal)
        CUDA_TRY(cudaMemcpy(goal, p->W.goal, R, cudaMemcpyDeviceToHost));
    if (controls) {
        std::vector<float> v(R * m);
        CUDA_TRY(cudaMemcpy(v.data(), p->W.st_u, sizeof(float) * v.size(), cudaMemcpyDeviceToHost));
        for (size_t r = 0; r < R; ++r)
            for (int a = 0; a < m; ++a)
                controls[r * m + a] = v[(size_t)a * R + r];
    }
    if (steps)
        CUDA_TRY(cudaMemcpy(steps, p->W.st_steps, sizeof(int) * R, cudaMemcpyDeviceToHost));
    return PAKR_OK;
}

pakr_status pakr_set_profiling(pakr_planner *p, int32_t enable)
{
    if (!p)
        return fail(PAKR_ERR_INVALID_ARG, "planner is NULL");
    DeviceGuard guard(p->device);
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    for (auto &pe : p->pending)
        p->pool.push_back(pe.second);
    p->pending.clear();
    for (int s = 0; s < kTimeSlots; ++s) {
        p->ms[s] = 0;
        p->launches[s] = 0;
    }
    p->profiling = enable != 0;
    return PAKR_OK;
}

pakr_status pakr_kernel_times(pakr_planner *p, double *ms_out, int64_t *launches_out, const char **names_out,
                              int32_t n_slots)
{
    static const char *names[kTimeSlots] = {"k_sample", "k_nn", "k_propagate", "k_append", "k_nn_tc"};
    if (!p || n_slots < 0)
        return fail(PAKR_ERR_INVALID_ARG, "bad argument");
    DeviceGuard guard(p->device);
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    for (auto &pe : p->pending) {
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, pe.second.a, pe.second.b));
        p->ms[pe.first] += t;
        p->launches[pe.first] += 1;
        p->pool.push_back(pe.second);
    }
    p->pending.clear();
    for (int s = 0; s < n_slots && s < kTimeSlots; ++s) {
        if (ms_out)
            ms_out[s] = p->ms[s];
        if (launches_out)
            launches_out[s] = p->launches[s];
        if (names_out)
            names_out[s] = names[s];
    }
    return PAKR_OK;
}

pakr_status pakr_philox4x32_10(pakr_planner *p, const uint32_t *ctr, const uint32_t key[2], uint32_t *out,
                               int64_t n)
{
    if (!p || !ctr || !key || !out || n < 0)
        return fail(PAKR_ERR_INVALID_ARG, "bad argument");
    if (n == 0)
        return PAKR_OK;
    DeviceGuard guard(p->device);
    uint32_t *dc = nullptr, *dout = nullptr;
    CUDA_TRY(cudaMalloc(&dc, sizeof(uint32_t) * 4 * n));
    cudaError_t e = cudaMalloc(&dout, sizeof(uint32_t) * 4 * n);
    if (e == cudaSuccess)
        e = cudaMemcpy(dc, ctr, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_philox(dc, key[0], key[1], dout, n, p->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, dout, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    if (dout)
        cudaFree(dout);
    if (e != cudaSuccess)
        return fail(PAKR_ERR_CUDA, "philox batch failed: %s", cudaGetErrorString(e));
    return PAKR_OK;
}

}  // extern "C"
