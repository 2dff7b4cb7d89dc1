// pakr_batch.cu -- batched planning: many independent PAKR queries (each its
// own Algorithm 1 run, with its own obstacles, tree cap, start and goal)
// advanced together by one persistent cooperative kernel.
//
// Each loop pass runs five phases over all still-active queries, separated
// by grid-wide barriers (a cooperative launch keeps every block resident, so
// the barriers cannot wait on an unscheduled block):
//   A  SampleStates for every query; one block lays out the nearest-neighbour
//      work items (query, node chunk, query group) with a block scan
//   B  NearestNeighbor work items spread over all blocks
//   C  Propagate work items (query, rollout block)
//   D  insert work items (query, rollout block)
//   E  AO-x step per query (solution bookkeeping, restart, stop)
// The phase bodies are the same device functions the single-query kernels
// run (pakr_device.cuh).  The launch is captured once into a CUDA graph per
// launch shape; a small autotuner picks the shape.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "pakr_device.cuh"

namespace cg = cooperative_groups;

namespace pakr {
namespace {

struct BatchQueryDev {
    DevProblem P;
    DevTree T;
    DevWork W;
    DevPlanBufs B;
    Ctl *ctl;
    float x_init[kMaxD];
    float x_goal[kMaxD];
};

struct BatchGlobal {
    unsigned long long seed;
    unsigned long long budget_ns;
    long long max_iterations;
    int stop_at_first;
    int n_active[2];  // active queries after each pass, double-buffered across passes
    int passes;
    unsigned long long t0_ns, t_end_ns;
};

constexpr int kBatchNnTile = 256;
constexpr int kBatchNnGroup = 8;
constexpr int kBatchQP = 2;  // query pairs per thread in the NN phase

// Exclusive prefix of v over the block; *total receives the block sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int *s_warp, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o)
                w += y;
        }
        if (lane < nw)
            s_warp[lane] = w;
    }
    __syncthreads();
    const int before = wid > 0 ? s_warp[wid - 1] : 0;
    *total = s_warp[nw - 1];
    __syncthreads();
    return before + x - v;
}

template <int DYN, int NT>
__global__ void __launch_bounds__(NT, (NnMinBlocks<Dims<DYN>::D, NT>::value))
    k_batch_plan(const BatchQueryDev *__restrict__ Q, int nq, BatchGlobal *G, int *nn_prefix, int nn_chunk)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M;
    cg::grid_group grid = cg::this_grid();
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    __shared__ int s_tmp[32];
    __shared__ int s_warp[32];
    __shared__ int s_len, s_found;

    const int nthreads = gridDim.x * NT;
    const int gtid = blockIdx.x * NT + threadIdx.x;
    const int K = Q[0].P.K;
    const int R = K * Q[0].P.k;
    const int qgroups = (K + NT * 2 * kBatchQP - 1) / (NT * 2 * kBatchQP);
    const int nblk = (R + NT - 1) / NT;

    for (int q = gtid; q < nq; q += nthreads) {
        const BatchQueryDev &qd = Q[q];
        aox_init_one<DYN>(qd.P, qd.ctl, qd.T, qd.x_init, qd.x_goal, G->seed + (unsigned long long)q,
                          G->max_iterations, G->budget_ns, __int_as_float(0x7f800000));
    }
    if (gtid == 0) {
        G->t0_ns = globaltimer_ns();
        G->n_active[0] = 0;
        G->n_active[1] = 0;
        G->passes = 0;
    }
    grid.sync();

    for (int pass = 0;; ++pass) {
        const int slot = pass & 1;
        // ---- A: samples, batch start, nearest-neighbour work layout
        for (long long idx = gtid; idx < (long long)nq * K; idx += nthreads) {
            const int q = (int)(idx / K);
            const int i = (int)(idx - (long long)q * K);
            const BatchQueryDev &qd = Q[q];
            if (!qd.ctl->plan_stop)
                sample_state<D>(qd.P, qd.W, i, qd.ctl->iteration, qd.ctl->seed);
        }
        for (int q = gtid; q < nq; q += nthreads) {
            Ctl *c = Q[q].ctl;
            if (!c->plan_stop)
                begin_batch(c, c->c_best);
        }
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0)
                G->n_active[slot] = 0;
            const int per = (nq + NT - 1) / NT;
            const int q0 = min(nq, (int)threadIdx.x * per), q1 = min(nq, q0 + per);
            int local = 0;
            for (int q = q0; q < q1; ++q) {
                const Ctl *c = Q[q].ctl;
                local += c->plan_stop ? 0 : ((c->count + nn_chunk - 1) / nn_chunk) * qgroups;
            }
            int total = 0;
            int run = block_exclusive_scan(local, s_tmp, &total);
            for (int q = q0; q < q1; ++q) {
                nn_prefix[q] = run;
                const Ctl *c = Q[q].ctl;
                run += c->plan_stop ? 0 : ((c->count + nn_chunk - 1) / nn_chunk) * qgroups;
            }
            if (threadIdx.x == 0)
                nn_prefix[nq] = total;
        }
        grid.sync();

        // ---- B: nearest neighbours
        const int total_nn = nn_prefix[nq];
        for (int w = blockIdx.x; w < total_nn; w += gridDim.x) {
            int lo = 0, hi = nq;  // last q with nn_prefix[q] <= w
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (nn_prefix[mid] <= w)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const BatchQueryDev &qd = Q[lo];
            const int local = w - nn_prefix[lo];
            const int chunk = local / qgroups, qg = local - chunk * qgroups;
            const int n = qd.ctl->n_start;
            const int start = chunk * nn_chunk;
            const int end = min(n, start + nn_chunk);
            nn_scan<D, kBatchQP, NT, kBatchNnTile, kBatchNnGroup>(qd.P, qd.T, qd.W, qd.ctl->bound,
                                                                       qg * NT * 2 * kBatchQP, start, end, smem);
        }
        grid.sync();

        // ---- C: propagate
        for (int w = blockIdx.x; w < nq * nblk; w += gridDim.x) {
            const int q = w / nblk, vb = w - q * nblk;
            const BatchQueryDev &qd = Q[q];
            if (qd.ctl->plan_stop)
                continue;
            propagate_block<DYN, 1>(qd.P, qd.ctl, qd.T, qd.W, vb, smem4);
        }
        grid.sync();

        // ---- D: insert
        for (int w = blockIdx.x; w < nq * nblk; w += gridDim.x) {
            const int q = w / nblk, vb = w - q * nblk;
            const BatchQueryDev &qd = Q[q];
            if (qd.ctl->plan_stop)
                continue;
            append_block<D, M>(qd.P, qd.ctl, qd.T, qd.W, vb, nblk, NT, 1, s_tmp, s_warp);
        }
        grid.sync();

        // ---- E: AO-x step of every active query
        if (threadIdx.x < 32) {
            for (int q = blockIdx.x; q < nq; q += gridDim.x) {
                const BatchQueryDev &qd = Q[q];
                if (qd.ctl->plan_stop)
                    continue;
                const bool stop = aox_step_warp<D, M>(qd.P, qd.ctl, qd.T, qd.B, G->stop_at_first, G->budget_ns,
                                                      G->max_iterations, &s_len, &s_found);
                if (threadIdx.x == 0 && !stop)
                    atomicAdd(&G->n_active[slot], 1);
            }
        }
        if (gtid == 0)
            G->passes = pass + 1;
        grid.sync();
        if (G->n_active[slot] == 0)
            break;
    }
    if (gtid == 0)
        G->t_end_ns = globaltimer_ns();
}

#define PAKR_BATCH_DISPATCH(dyn, nt, BODY)                                                                             \
    switch ((dyn) * 1000 + (nt)) {                                                                                     \
    case DI2 * 1000 + 128: { constexpr int DYN_ = DI2, NT_ = 128; BODY; } break;                                      \
    case DI2 * 1000 + 256: { constexpr int DYN_ = DI2, NT_ = 256; BODY; } break;                                      \
    case DI3 * 1000 + 128: { constexpr int DYN_ = DI3, NT_ = 128; BODY; } break;                                      \
    case DI3 * 1000 + 256: { constexpr int DYN_ = DI3, NT_ = 256; BODY; } break;                                      \
    case QUAD12 * 1000 + 128: { constexpr int DYN_ = QUAD12, NT_ = 128; BODY; } break;                                \
    case QUAD12 * 1000 + 256: { constexpr int DYN_ = QUAD12, NT_ = 256; BODY; } break;                                \
    case DUBINS3D * 1000 + 128: { constexpr int DYN_ = DUBINS3D, NT_ = 128; BODY; } break;                            \
    case DUBINS3D * 1000 + 256: { constexpr int DYN_ = DUBINS3D, NT_ = 256; BODY; } break;                            \
    case UNICYCLE1 * 1000 + 128: { constexpr int DYN_ = UNICYCLE1, NT_ = 128; BODY; } break;                          \
    case UNICYCLE1 * 1000 + 256: { constexpr int DYN_ = UNICYCLE1, NT_ = 256; BODY; } break;                          \
    case UNICYCLE2 * 1000 + 128: { constexpr int DYN_ = UNICYCLE2, NT_ = 128; BODY; } break;                          \
    case UNICYCLE2 * 1000 + 256: { constexpr int DYN_ = UNICYCLE2, NT_ = 256; BODY; } break;                          \
    default: return cudaErrorInvalidValue;                                                                             \
    }

cudaError_t batch_occupancy(int dyn, int nt, size_t smem, int *blocks)
{
    PAKR_BATCH_DISPATCH(dyn, nt,
                        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch_plan<DYN_, NT_>, NT_, smem));
    return cudaSuccess;
}

cudaError_t batch_launch(int dyn, int nt, int grid, size_t smem, cudaStream_t s, const BatchQueryDev *Q, int nq,
                         BatchGlobal *G, int *nn_prefix, int nn_chunk)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PAKR_BATCH_DISPATCH(dyn, nt, return cudaLaunchKernelEx(&cfg, k_batch_plan<DYN_, NT_>, Q, nq, G, nn_prefix, nn_chunk));
    return cudaSuccess;
}

cudaError_t batch_set_smem(int dyn, int nt, size_t smem)
{
    PAKR_BATCH_DISPATCH(dyn, nt,
                        return cudaFuncSetAttribute(k_batch_plan<DYN_, NT_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem));
    return cudaSuccess;
}

pakr_status bfail(pakr_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    record_error(buf);
    return st;
}

#define BCUDA(expr)                                                                                                    \
    do {                                                                                                               \
        cudaError_t e_ = (expr);                                                                                       \
        if (e_ != cudaSuccess)                                                                                         \
            return bfail(e_ == cudaErrorMemoryAllocation ? PAKR_ERR_OOM : PAKR_ERR_CUDA, "%s failed: %s", #expr,        \
                         cudaGetErrorString(e_));                                                                      \
    } while (0)

size_t aup(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace pakr

using namespace pakr;

struct pakr_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    int dyn = 0, d = 0, m = 0, pdim = 0, nq = 0, K = 0, k = 0, R = 0;
    int path_cap = 0;
    char *base = nullptr;
    BatchQueryDev *qdev = nullptr;
    Ctl *ctls = nullptr;
    BatchGlobal *G = nullptr;
    int *nn_prefix = nullptr;
    std::vector<BatchQueryDev> qhost;
    std::vector<Ctl> ctl_host;
    BatchGlobal *G_host = nullptr;  // pinned
    size_t smem = 0;
    int sms = 0;
    pakr_batch_tuning tuning{256, 2048, 0, 0.0};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_threads = 0, exec_chunk = 0, exec_grid = 0;
};

namespace {

struct BatchDeviceGuard {
    int prev = -1;
    explicit BatchDeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~BatchDeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

pakr_status check_tuning(const pakr_batch_tuning *t)
{
    if (!t)
        return bfail(PAKR_ERR_INVALID_ARG, "tuning is NULL");
    if (t->block_threads != 128 && t->block_threads != 256)
        return bfail(PAKR_ERR_INVALID_ARG, "block_threads must be 128 or 256");
    if (t->nn_chunk < 64 || t->nn_chunk % 8 != 0)
        return bfail(PAKR_ERR_INVALID_ARG, "nn_chunk must be a multiple of 8, at least 64");
    return PAKR_OK;
}

// Instantiate the cooperative launch for the current tuning as a CUDA graph.
pakr_status ensure_graph(pakr_batch *b)
{
    const int nt = b->tuning.block_threads, chunk = b->tuning.nn_chunk;
    if (b->exec && b->exec_threads == nt && b->exec_chunk == chunk)
        return PAKR_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    BCUDA(batch_set_smem(b->dyn, nt, b->smem));
    int occ = 0;
    BCUDA(batch_occupancy(b->dyn, nt, b->smem, &occ));
    if (occ < 1)
        return bfail(PAKR_ERR_CUDA, "batched kernel does not fit on an SM (%zu bytes of shared memory)", b->smem);
    const int grid = occ * b->sms;
    BCUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = batch_launch(b->dyn, nt, grid, b->smem, b->capture_stream, b->qdev, b->nq, b->G, b->nn_prefix,
                                  chunk);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->capture_stream, &g);
    if (le != cudaSuccess || ee != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        return bfail(PAKR_ERR_CUDA, "capturing the cooperative batched launch failed: %s",
                     cudaGetErrorString(le != cudaSuccess ? le : ee));
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        return bfail(PAKR_ERR_CUDA, "instantiating the batched graph failed: %s", cudaGetErrorString(ie));
    }
    b->graph = g;
    b->exec = ex;
    b->exec_threads = nt;
    b->exec_chunk = chunk;
    b->exec_grid = grid;
    return PAKR_OK;
}

pakr_status run_plan(pakr_batch *b, double budget_s, int64_t max_iterations, uint64_t seed, uint32_t flags,
                     float *ms_out)
{
    pakr_status st = ensure_graph(b);
    if (st != PAKR_OK)
        return st;
    BatchGlobal *h = b->G_host;
    memset(h, 0, sizeof(BatchGlobal));
    h->seed = seed;
    const double ns = budget_s * 1e9;
    h->budget_ns = ns >= 1.8e19 ? ~0ull : (unsigned long long)ns;
    const int64_t cap = 10000000;
    h->max_iterations = max_iterations > 0 ? std::min<int64_t>(max_iterations, cap) : cap;
    h->stop_at_first = (flags & PAKR_PLAN_STOP_AT_FIRST) ? 1 : 0;
    BCUDA(cudaMemcpyAsync(b->G, h, sizeof(BatchGlobal), cudaMemcpyHostToDevice, b->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        BCUDA(cudaEventCreate(&e0));
        BCUDA(cudaEventCreate(&e1));
        BCUDA(cudaEventRecord(e0, b->stream));
    }
    BCUDA(cudaGraphLaunch(b->exec, b->stream));
    if (ms_out)
        BCUDA(cudaEventRecord(e1, b->stream));
    BCUDA(cudaMemcpyAsync(b->ctl_host.data(), b->ctls, sizeof(Ctl) * b->nq, cudaMemcpyDeviceToHost, b->stream));
    BCUDA(cudaMemcpyAsync(h, b->G, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    if (ms_out) {
        BCUDA(cudaEventElapsedTime(ms_out, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    return PAKR_OK;
}

}  // namespace

extern "C" {

pakr_status pakr_batch_create(const pakr_problem_desc *base, const pakr_batch_query *queries, int32_t n_queries,
                              pakr_batch **out)
{
    if (!out)
        return bfail(PAKR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!base || !queries || n_queries < 1)
        return bfail(PAKR_ERR_INVALID_ARG, "need a base description and at least one query");
    DevProblem P{};
    int d = 0, m = 0, pdim = 0;
    pakr_status st = fill_problem(base, &P, &d, &m, &pdim);
    if (st != PAKR_OK)
        return st;
    const int K = base->n_parents, k = base->branching;
    const int64_t R = (int64_t)K * k;
    if (R > (1 << 24))
        return bfail(PAKR_ERR_INVALID_ARG, "n_parents * branching too large for the batched planner");
    int max_obs = 0;
    for (int q = 0; q < n_queries; ++q) {
        const pakr_batch_query &qq = queries[q];
        if (!qq.x_init || !qq.x_goal)
            return bfail(PAKR_ERR_INVALID_ARG, "query %d: x_init / x_goal missing", q);
        for (int a = 0; a < d; ++a)
            if (!std::isfinite(qq.x_init[a]) || !std::isfinite(qq.x_goal[a]))
                return bfail(PAKR_ERR_INVALID_ARG, "query %d: x_init / x_goal must be finite", q);
        if (qq.tree_cap < 1 || qq.tree_cap > kMaxTreeNodes)
            return bfail(PAKR_ERR_INVALID_ARG, "query %d: tree_cap out of range", q);
        if (qq.n_boxes < 0 || qq.n_spheres < 0 || (qq.n_boxes && !qq.boxes) || (qq.n_spheres && !qq.spheres))
            return bfail(PAKR_ERR_INVALID_ARG, "query %d: bad obstacle arrays", q);
        for (int i = 0; i < qq.n_boxes * 2 * pdim; ++i)
            if (!std::isfinite(qq.boxes[i]))
                return bfail(PAKR_ERR_INVALID_ARG, "query %d: boxes must be finite", q);
        for (int i = 0; i < qq.n_spheres * (pdim + 1); ++i)
            if (!std::isfinite(qq.spheres[i]))
                return bfail(PAKR_ERR_INVALID_ARG, "query %d: spheres must be finite", q);
        max_obs = std::max(max_obs, 2 * qq.n_boxes + qq.n_spheres);
    }
    if (max_obs > 3000)
        return bfail(PAKR_ERR_INVALID_ARG, "too many obstacles in a query: 2*n_boxes + n_spheres must be <= 3000");
    int ndev = 0;
    BCUDA(cudaGetDeviceCount(&ndev));
    if (base->device < 0 || base->device >= ndev)
        return bfail(PAKR_ERR_INVALID_ARG, "device %d out of range", base->device);
    BatchDeviceGuard guard(base->device);

    pakr_batch *b = new pakr_batch();
    b->device = base->device;
    b->stream = (cudaStream_t)base->cuda_stream;
    b->dyn = base->dynamics;
    b->d = d;
    b->m = m;
    b->pdim = pdim;
    b->nq = n_queries;
    b->K = K;
    b->k = k;
    b->R = (int)R;
    b->path_cap = base->path_cap ? base->path_cap : 1024;
    auto cleanup = [&](pakr_status s) {
        pakr_batch_destroy(b);
        return s;
    };

    // Layout: per query tree, batch workspace, path buffers, obstacles; then the globals.
    const size_t nblk = (size_t)(R + 127) / 128;  // propagate blocks at the smallest block size
    const int pc = b->path_cap;
    std::vector<size_t> q_off(n_queries);
    size_t off = 0;
    for (int q = 0; q < n_queries; ++q) {
        const size_t c = (size_t)queries[q].tree_cap;
        q_off[q] = off;
        off += aup(4 * d * c) + aup(4 * m * c) + 4 * aup(4 * c);
        off += aup(4 * d * (size_t)K) + aup(8 * (size_t)K) + aup(4 * d * (size_t)R) + aup(4 * m * (size_t)R) +
               4 * aup(4 * (size_t)R) + 2 * aup((size_t)R) + aup(4 * nblk);
        off += aup(4 * (size_t)(pc + 1)) * 2 + aup(4 * d * (size_t)(pc + 1)) + aup(4 * m * (size_t)(pc + 1)) +
               aup(8) * 3;
        off += aup(16 * (size_t)(2 * queries[q].n_boxes + queries[q].n_spheres));
    }
    const size_t qdev_off = off;
    off += aup(sizeof(BatchQueryDev) * n_queries);
    const size_t ctl_off = off;
    off += aup(sizeof(Ctl) * n_queries);
    const size_t g_off = off;
    off += aup(sizeof(BatchGlobal));
    const size_t pre_off = off;
    off += aup(sizeof(int) * (n_queries + 1));
    cudaError_t e = cudaMalloc(&b->base, off);
    if (e != cudaSuccess)
        return cleanup(bfail(PAKR_ERR_OOM, "cudaMalloc(%zu) for the batch failed: %s", off, cudaGetErrorString(e)));
    e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMallocHost(&b->G_host, sizeof(BatchGlobal));
    if (e != cudaSuccess)
        return cleanup(bfail(PAKR_ERR_CUDA, "batch set-up failed: %s", cudaGetErrorString(e)));
    b->qdev = (BatchQueryDev *)(b->base + qdev_off);
    b->ctls = (Ctl *)(b->base + ctl_off);
    b->G = (BatchGlobal *)(b->base + g_off);
    b->nn_prefix = (int *)(b->base + pre_off);
    b->qhost.resize(n_queries);
    b->ctl_host.resize(n_queries);
    for (int q = 0; q < n_queries; ++q) {
        const pakr_batch_query &qq = queries[q];
        const size_t c = (size_t)qq.tree_cap;
        char *p = b->base + q_off[q];
        auto take = [&](size_t bytes) {
            char *at = p;
            p += aup(bytes);
            return at;
        };
        BatchQueryDev &h = b->qhost[q];
        memset(&h, 0, sizeof(h));
        h.P = P;
        h.P.cap = (int)c;
        h.T.X = (float *)take(4 * d * c);
        h.T.U = (float *)take(4 * m * c);
        h.T.cost = (float *)take(4 * c);
        h.T.fcost = (float *)take(4 * c);
        h.T.parent = (int *)take(4 * c);
        h.T.steps = (int *)take(4 * c);
        h.W.xr = (float *)take(4 * d * (size_t)K);
        h.W.nn_key = (unsigned long long *)take(8 * (size_t)K);
        h.W.st_x = (float *)take(4 * d * (size_t)R);
        h.W.st_u = (float *)take(4 * m * (size_t)R);
        h.W.st_cost = (float *)take(4 * (size_t)R);
        h.W.st_f = (float *)take(4 * (size_t)R);
        h.W.st_steps = (int *)take(4 * (size_t)R);
        h.W.st_parent = (int *)take(4 * (size_t)R);
        h.W.outcome = (int8_t *)take((size_t)R);
        h.W.goal = (int8_t *)take((size_t)R);
        h.W.block_count = (int *)take(4 * nblk);
        h.B.path_nodes = (int *)take(4 * (size_t)(pc + 1));
        h.B.path_steps = (int *)take(4 * (size_t)(pc + 1));
        h.B.path_x = (float *)take(4 * d * (size_t)(pc + 1));
        h.B.path_u = (float *)take(4 * m * (size_t)(pc + 1));
        h.B.path_cap = pc;
        h.B.hist_t = (unsigned long long *)take(8);
        h.B.hist_cost = (float *)take(8);
        h.B.hist_iter = (long long *)take(8);
        h.B.hist_cap = 1;
        float4 *obs = (float4 *)take(16 * (size_t)(2 * qq.n_boxes + qq.n_spheres));
        std::vector<float4> o4(2 * (size_t)qq.n_boxes + qq.n_spheres);
        for (int i = 0; i < qq.n_boxes; ++i) {
            const float *r = qq.boxes + (size_t)i * 2 * pdim;
            o4[2 * i] = make_float4(r[0], r[1], pdim > 2 ? r[2] : 0.f, 0.f);
            o4[2 * i + 1] = make_float4(r[pdim], r[pdim + 1], pdim > 2 ? r[pdim + 2] : 0.f, 0.f);
        }
        for (int i = 0; i < qq.n_spheres; ++i) {
            const float *r = qq.spheres + (size_t)i * (pdim + 1);
            o4[2 * qq.n_boxes + i] = make_float4(r[0], r[1], pdim > 2 ? r[2] : 0.f, r[pdim]);
        }
        if (!o4.empty()) {
            e = cudaMemcpy(obs, o4.data(), 16 * o4.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess)
                return cleanup(bfail(PAKR_ERR_CUDA, "obstacle upload failed: %s", cudaGetErrorString(e)));
        }
        h.P.n_boxes = qq.n_boxes;
        h.P.n_spheres = qq.n_spheres;
        h.P.boxes = obs;
        h.P.spheres = obs + 2 * qq.n_boxes;
        h.ctl = b->ctls + q;
        for (int a = 0; a < kMaxD; ++a) {
            h.x_init[a] = a < d ? qq.x_init[a] : 0.f;
            h.x_goal[a] = a < d ? qq.x_goal[a] : 0.f;
        }
    }
    e = cudaMemcpy(b->qdev, b->qhost.data(), sizeof(BatchQueryDev) * n_queries, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(b->ctls, 0, sizeof(Ctl) * n_queries);
    if (e != cudaSuccess)
        return cleanup(bfail(PAKR_ERR_CUDA, "batch upload failed: %s", cudaGetErrorString(e)));
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    const size_t nn_tile = (size_t)kBatchNnTile * ((2 * d + 2 + 3) / 4 * 4) * sizeof(float);
    const size_t obs_bytes = (size_t)max_obs * sizeof(float4) + kMaxD * sizeof(float);
    b->smem = std::max(nn_tile, obs_bytes);
    *out = b;
    return PAKR_OK;
}

void pakr_batch_destroy(pakr_batch *b)
{
    if (!b)
        return;
    BatchDeviceGuard guard(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    if (b->base)
        cudaFree(b->base);
    if (b->G_host)
        cudaFreeHost(b->G_host);
    if (b->capture_stream)
        cudaStreamDestroy(b->capture_stream);
    delete b;
}

pakr_status pakr_batch_set_tuning(pakr_batch *b, const pakr_batch_tuning *t)
{
    if (!b)
        return bfail(PAKR_ERR_INVALID_ARG, "batch is NULL");
    pakr_status st = check_tuning(t);
    if (st != PAKR_OK)
        return st;
    b->tuning.block_threads = t->block_threads;
    b->tuning.nn_chunk = t->nn_chunk;
    return PAKR_OK;
}

pakr_status pakr_batch_plan(pakr_batch *b, double budget_s, int64_t max_iterations, uint64_t seed, uint32_t flags,
                            pakr_batch_result *results)
{
    if (!b || !results)
        return bfail(PAKR_ERR_INVALID_ARG, "NULL argument");
    if (std::isnan(budget_s) || budget_s < 0)
        return bfail(PAKR_ERR_INVALID_ARG, "budget_s must be >= 0");
    BatchDeviceGuard guard(b->device);
    pakr_status st = run_plan(b, budget_s, max_iterations, seed, flags, nullptr);
    if (st != PAKR_OK)
        return st;
    int err = 0;
    for (int q = 0; q < b->nq; ++q) {
        const Ctl &c = b->ctl_host[q];
        pakr_batch_result &r = results[q];
        memset(&r, 0, sizeof(r));
        r.n_solutions = c.n_solutions;
        r.cost = c.n_solutions > 0 ? c.sol_best : INFINITY;
        r.n_edges = c.n_solutions > 0 ? (c.path_len > 0 ? c.path_len - 1 : -1) : 0;
        r.iterations = c.iterations_done;
        r.t_first_solution_s = c.t_first_ns == ~0ull ? -1.0 : (double)c.t_first_ns * 1e-9;
        r.nodes_first_solution = c.n_solutions > 0 ? c.nodes_first : -1;
        r.iterations_first_solution = c.n_solutions > 0 ? c.iterations_first : -1;
        r.n_restarts = c.n_restarts;
        if (c.plan_status == -1)
            r.status = PAKR_ERR_INVALID_ARG;
        else if (c.n_solutions > 0)
            r.status = PAKR_GOAL_REACHED;
        else if (c.plan_status == 3)
            r.status = PAKR_NO_ELIGIBLE;
        else
            r.status = PAKR_BUDGET_EXPIRED;
        err |= c.err;
    }
    if (err)
        return bfail(PAKR_ERR_DEVICE, "device error flags 0x%x", err);
    return PAKR_OK;
}

pakr_status pakr_batch_path(pakr_batch *b, int32_t query, float *states, float *controls, int32_t *steps,
                            int32_t max_edges)
{
    if (!b || query < 0 || query >= b->nq)
        return bfail(PAKR_ERR_INVALID_ARG, "bad query index");
    const Ctl &c = b->ctl_host[query];
    if (c.n_solutions == 0 || c.path_len < 1)
        return bfail(PAKR_ERR_INVALID_ARG, "query %d has no stored path", query);
    const int edges = c.path_len - 1;
    if (edges > max_edges || !states || (edges > 0 && (!controls || !steps)))
        return bfail(PAKR_ERR_INVALID_ARG, "path of %d edges does not fit (max_edges %d)", edges, max_edges);
    BatchDeviceGuard guard(b->device);
    const BatchQueryDev &h = b->qhost[query];
    BCUDA(cudaMemcpy(states, h.B.path_x, sizeof(float) * b->d * (size_t)(edges + 1), cudaMemcpyDeviceToHost));
    if (edges > 0) {
        BCUDA(cudaMemcpy(controls, h.B.path_u + b->m, sizeof(float) * b->m * (size_t)edges, cudaMemcpyDeviceToHost));
        BCUDA(cudaMemcpy(steps, h.B.path_steps + 1, sizeof(int) * (size_t)edges, cudaMemcpyDeviceToHost));
    }
    return PAKR_OK;
}

pakr_status pakr_batch_autotune(pakr_batch *b, int64_t iterations, uint64_t seed, pakr_batch_tuning *out)
{
    if (!b || !out || iterations < 1)
        return bfail(PAKR_ERR_INVALID_ARG, "bad argument");
    BatchDeviceGuard guard(b->device);
    const int threads[2] = {128, 256};
    const int chunks[5] = {512, 1024, 2048, 4096, 8192};
    pakr_batch_tuning best = b->tuning;
    double best_ms = 1e30;
    int tried = 0;
    for (int t : threads) {
        for (int c : chunks) {
            b->tuning.block_threads = t;
            b->tuning.nn_chunk = c;
            float ms = 0.f;
            pakr_status st = run_plan(b, 1e6, iterations, seed, 0, &ms);
            if (st != PAKR_OK)
                return st;
            ++tried;
            if (ms < best_ms) {
                best_ms = ms;
                best.block_threads = t;
                best.nn_chunk = c;
            }
        }
    }
    b->tuning.block_threads = best.block_threads;
    b->tuning.nn_chunk = best.nn_chunk;
    best.n_tried = tried;
    best.best_ms = best_ms;
    b->tuning.n_tried = tried;
    b->tuning.best_ms = best_ms;
    *out = best;
    return ensure_graph(b);
}

}  // extern "C"
