// pakr_kernels.cu -- sm_103a kernels of one PAKR expansion iteration
// (Algorithm 1 inner loop) and of the device-resident AO-x loop.  The block
// bodies live in pakr_device.cuh.
//
//   k_sample     SampleStates: Philox4x32-10 uniform states, clears the NN keys,
//                snapshots the tree size (the frozen snapshot of Sec. IV-B).
//   k_nn         NearestNeighbor among nodes with f-cost below the bound.
//   k_propagate  SampleControls + RK4 Propagate + per-substep validity +
//                cost-bounded pruning + goal test.
//   k_append     insert survivors in ascending rollout order, truncate at the
//                cap, cheapest goal child.
//   k_plan_*     AO-x bookkeeping inside a conditional-while CUDA graph.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pakr_device.cuh"

namespace pakr {

// ---------------------------------------------------------------------------
// Expansion kernels.
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_sample(DevProblem P, Ctl *ctl, DevWork W, float bound, unsigned long long seed_arg, int mode)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long seed = (mode == MODE_EXPAND) ? seed_arg : ctl->seed;
    if (i < P.K)
        sample_state<D>(P, W, i, ctl->iteration, seed);
    if (i == 0) {
        if (mode == MODE_EXPAND)
            ctl->seed = seed_arg;
        begin_batch(ctl, (mode == MODE_EXPAND) ? bound : ctl->c_best);
    }
}

template <int D, int QP, int NT, int TILE, int G>
__global__ void __launch_bounds__(NT, (NnMinBlocks<D, NT>::value))
    k_nn(DevProblem P, const Ctl *__restrict__ ctl, DevTree T, DevWork W)
{
    constexpr int RW = (2 * D + 2 + 3) / 4 * 4;
    __shared__ __align__(16) float s_node[TILE * RW];
    const int n = ctl->n_start;
    if (n >= P.tc_min_n)
        return;  // large trees take k_nn_tc
    const int per = nn_chunk_nodes<G>(n, gridDim.x);
    const int start = blockIdx.x * per;
    const int end = min(n, start + per);
    nn_scan<D, QP, NT, TILE, G>(P, T, W, ctl->bound, blockIdx.y * NT * 2 * QP, start, end, s_node);
}

template <int DYN, int LG>
__global__ void __launch_bounds__(256) k_propagate(DevProblem P, Ctl *ctl, DevTree T, DevWork W)
{
    extern __shared__ float4 s_obs[];
    propagate_block<DYN, LG>(P, ctl, T, W, blockIdx.x, s_obs);
}

template <int D, int M>
__global__ void __launch_bounds__(256) k_append(DevProblem P, Ctl *ctl, DevTree T, DevWork W, int nblk, int rpb)
{
    __shared__ int s_tmp[32];
    __shared__ int s_warp[32];
    append_block<D, M>(P, ctl, T, W, blockIdx.x, nblk, rpb, (int)blockDim.x / rpb, s_tmp, s_warp);
}

// ---------------------------------------------------------------------------
// Tree reset / import / AO-x graph kernels.
// ---------------------------------------------------------------------------
template <int DYN>
__global__ void k_tree_reset(DevProblem P, Ctl *ctl, DevTree T, const float *x_init)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    float x[D], goal[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = x_init[a];
        goal[a] = ctl->x_goal[a];
        T.X[(size_t)a * P.cap] = x[a];
    }
#pragma unroll
    for (int a = 0; a < M; ++a)
        T.U[(size_t)a * P.cap] = 0.f;
    T.cost[0] = 0.f;
    T.fcost[0] = heuristic<D, PD>(x, P, goal);
    T.parent[0] = -1;
    T.steps[0] = 0;
    ctl->tc_flag = 0u;
    tc_pack_node<D>(P, T, ctl, 0, x);
    ctl->count = 1;
    ctl->iteration = 0u;
    ctl->err = 0;
    ctl->status = state_valid<D, PD>(x, P, P.boxes, P.n_boxes, P.spheres, P.n_spheres) ? 1 : 0;
}

template <int DYN>
__global__ void k_import_fcost(DevProblem P, Ctl *ctl, DevTree T, int count)
{
    constexpr int D = Dims<DYN>::D, PD = Dims<DYN>::PD;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count)
        return;
    float x[D], goal[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = T.X[(size_t)a * P.cap + j];
        goal[a] = ctl->x_goal[a];
    }
    T.fcost[j] = T.cost[j] + heuristic<D, PD>(x, P, goal);
    tc_pack_node<D>(P, T, ctl, j, x);
}

// Fresh AO-x run: goal, root, c_best = +inf, clock start.  Closes the while
// loop before its first pass when the start is invalid or the budget is zero.
template <int DYN>
__global__ void k_plan_init(DevProblem P, Ctl *ctl, DevTree T, const PlanParams *pp, cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    const bool run =
        aox_init_one<DYN>(P, ctl, T, pp->x_init, pp->x_goal, pp->seed, pp->max_iterations, pp->budget_ns,
                          pp->c_best_init);
    cudaGraphSetConditional(h, run ? 1u : 0u);
}

// End of one AO-x loop pass: record a solution (c_best, history, path) and
// restart from the root, restart a full tree, stop on budget / iterations /
// no eligible node.  One warp: lane 0 chases parents, the warp gathers rows.
// Without nested loops h is the AO-x loop.  With them (nested != 0) h_fp32 and h_tc
// are two inner loops, for iterations whose tree is below P.tc_min_n nodes (FP32
// nearest neighbour) and for the rest: unless the run stops exactly one is opened,
// chosen by the tree size the next iteration will see; stopping closes both, and
// k_plan_cont then closes the AO-x loop.
template <int D, int M>
__global__ void k_plan_step(DevProblem P, Ctl *ctl, DevTree T, const PlanParams *pp, DevPlanBufs B,
                            cudaGraphConditionalHandle h, cudaGraphConditionalHandle h_fp32,
                            cudaGraphConditionalHandle h_tc, int nested)
{
    __shared__ int s_len;
    __shared__ int s_found;
    const bool stop = aox_step_warp<D, M>(P, ctl, T, B, pp->stop_at_first, pp->budget_ns, pp->max_iterations, &s_len,
                                          &s_found);
    if (threadIdx.x == 0) {
        if (nested) {
            const bool next_tc = ctl->count >= P.tc_min_n;
            cudaGraphSetConditional(h_fp32, (!stop && !next_tc) ? 1u : 0u);
            cudaGraphSetConditional(h_tc, (!stop && next_tc) ? 1u : 0u);
        } else {
            cudaGraphSetConditional(h, stop ? 0u : 1u);
        }
    }
}

// End of one pass of the outer AO-x loop of a nested graph: continue unless the last
// k_plan_step stopped the run.
__global__ void k_plan_cont(const Ctl *ctl, cudaGraphConditionalHandle h)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        cudaGraphSetConditional(h, ctl->plan_stop ? 0u : 1u);
}

// Lowers the AO-x bound to *cost if that is smaller (a finite, non-negative cost; the bit
// patterns of such floats order like the values).
__global__ void k_offer_bound(Ctl *ctl, const float *cost)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const float c = *cost;
        if (c >= 0.f && c < __int_as_float(0x7f800000)) {
            const int old = atomicMin(reinterpret_cast<int *>(&ctl->c_best), __float_as_int(c));
            // a cheaper path than the loop's bound is a new AO-x solution: the loop restarts its
            // tree at its next step, as after one of its own (Algorithm 1)
            if (old > __float_as_int(c))
                atomicExch(&ctl->offer_restart, 1);
        }
    }
}

// One warp copies the best path of a plan that may be running on another stream, under the
// path sequence: info = (1 if the copy is whole, edges, sequence, cost bits); a copy that a new
// path overwrote meanwhile, or an empty or oversized path, gives info[0] = 0.
__global__ void k_plan_snapshot(const Ctl *ctl, DevPlanBufs B, int d, int m, float *states, float *controls,
                                int *steps, int max_edges, int *info)
{
    const int lane = threadIdx.x;
    __shared__ unsigned s_seq;
    __shared__ int s_len;
    __shared__ float s_cost;
    if (lane == 0) {
        s_seq = __ldcg(&ctl->path_seq);
        __threadfence();
        s_len = __ldcg(&ctl->path_len);
        s_cost = __ldcg(&ctl->sol_best);
    }
    __syncwarp();
    const unsigned seq = s_seq;
    const int len = s_len;
    const bool ok = !(seq & 1u) && len > 0 && len - 1 <= max_edges;
    if (ok) {
        for (int t = lane; t < len; t += 32) {
            for (int a = 0; a < d; ++a)
                states[(size_t)t * d + a] = __ldcg(B.path_x + (size_t)t * d + a);
            if (t > 0) {
                for (int a = 0; a < m; ++a)
                    controls[(size_t)(t - 1) * m + a] = __ldcg(B.path_u + (size_t)t * m + a);
                steps[t - 1] = __ldcg(B.path_steps + t);
            }
        }
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        const unsigned seq2 = __ldcg(&ctl->path_seq);
        info[0] = (ok && seq2 == seq) ? 1 : 0;
        info[1] = len - 1;
        info[2] = (int)seq;
        info[3] = __float_as_int(s_cost);
    }
}

cudaError_t launch_plan_snapshot(const Ctl *ctl, const DevPlanBufs &B, int d, int m, float *states,
                                 float *controls, int *steps, int max_edges, int *info, cudaStream_t s)
{
    k_plan_snapshot<<<1, 32, 0, s>>>(ctl, B, d, m, states, controls, steps, max_edges, info);
    return cudaGetLastError();
}

cudaError_t preload_plan_snapshot()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, k_plan_snapshot);
}

__global__ void k_truncate(Ctl *ctl, int count)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && count < ctl->count)
        ctl->count = count;
}

__global__ void k_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int64_t n)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n)
        return;
    const Words4 w = philox(ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3], k0, k1);
#pragma unroll
    for (int a = 0; a < 4; ++a)
        out[4 * t + a] = w.w[a];
}

// ---------------------------------------------------------------------------
// Launchers and dispatch.
// ---------------------------------------------------------------------------
constexpr int kNnTile = 256;
constexpr int kNnGroup = 8;

cudaError_t launch_sample(const DevProblem &P, Ctl *ctl, const DevWork &W, const LaunchCfg &L, float bound,
                          unsigned long long seed, int mode, cudaStream_t s)
{
    PAKR_DISPATCH_DYN(P.dyn, (k_sample<Dims<DYN_>::D><<<L.sample_blocks, L.sample_threads, 0, s>>>(
                                 P, ctl, W, bound, seed, mode)));
    return cudaGetLastError();
}

template <int D>
static cudaError_t launch_nn_d(const DevProblem &P, const Ctl *ctl, const DevTree &T, const DevWork &W,
                               const LaunchCfg &L, cudaStream_t s)
{
    const dim3 grid(L.nn_chunks, L.nn_qgroups);
    switch (L.nn_variant) {
    case 0: k_nn<D, 1, 64, kNnTile, kNnGroup><<<grid, 64, 0, s>>>(P, ctl, T, W); break;
    case 1: k_nn<D, 1, 128, kNnTile, kNnGroup><<<grid, 128, 0, s>>>(P, ctl, T, W); break;
    default: k_nn<D, 2, 256, kNnTile, kNnGroup><<<grid, 256, 0, s>>>(P, ctl, T, W); break;
    }
    return cudaGetLastError();
}

// k_nn returns at once when the device-side tree size is P.tc_min_n or more, k_nn_tc when it
// is below: a caller that picks one kernel for any tree size passes P with tc_min_n set past
// (k_nn: INT_MAX) or below (k_nn_tc: 0) every size.
cudaError_t launch_nn_fp32(const DevProblem &P, const Ctl *ctl, const DevTree &T, const DevWork &W,
                           const LaunchCfg &L, cudaStream_t s)
{
    PAKR_DISPATCH_DYN(P.dyn, return launch_nn_d<Dims<DYN_>::D>(P, ctl, T, W, L, s));
    return cudaSuccess;
}

cudaError_t launch_nn(const DevProblem &P, const Ctl *ctl, const DevTree &T, const DevWork &W, const LaunchCfg &L,
                      cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (P.tc_min_n > 0) {
        PAKR_DISPATCH_DYN(P.dyn, e = launch_nn_d<Dims<DYN_>::D>(P, ctl, T, W, L, s));
        if (e != cudaSuccess)
            return e;
    }
    if (T.XT && P.tc_min_n < 0x7FFFFFFF)
        e = launch_nn_tc(P, const_cast<Ctl *>(ctl), T, W, L, s);
    return e;
}

template <int DYN>
static cudaError_t launch_propagate_dyn(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W,
                                        const LaunchCfg &L, cudaStream_t s)
{
    switch (L.prop_lanes) {
    case 1: k_propagate<DYN, 1><<<L.prop_blocks, L.prop_threads, L.obs_smem_bytes, s>>>(P, ctl, T, W); break;
    case 2: k_propagate<DYN, 2><<<L.prop_blocks, L.prop_threads, L.obs_smem_bytes, s>>>(P, ctl, T, W); break;
    case 4: k_propagate<DYN, 4><<<L.prop_blocks, L.prop_threads, L.obs_smem_bytes, s>>>(P, ctl, T, W); break;
    case 8: k_propagate<DYN, 8><<<L.prop_blocks, L.prop_threads, L.obs_smem_bytes, s>>>(P, ctl, T, W); break;
    case 16: k_propagate<DYN, 16><<<L.prop_blocks, L.prop_threads, L.obs_smem_bytes, s>>>(P, ctl, T, W); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_propagate(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W, const LaunchCfg &L,
                             cudaStream_t s)
{
    PAKR_DISPATCH_DYN(P.dyn, return launch_propagate_dyn<DYN_>(P, ctl, T, W, L, s));
    return cudaSuccess;
}

cudaError_t launch_append(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W, const LaunchCfg &L,
                          cudaStream_t s)
{
    // one thread per rollout, at least a warp per block (the scans are warp-wide): with more
    // than 8 lanes per rollout an append block covers several propagate blocks
    const int rollouts_per_block = L.prop_threads / L.prop_lanes;
    const int threads = rollouts_per_block < 32 ? 32 : rollouts_per_block;
    const int pbs = threads / rollouts_per_block;
    PAKR_DISPATCH_DYN(P.dyn, (k_append<Dims<DYN_>::D, Dims<DYN_>::M><<<(L.prop_blocks + pbs - 1) / pbs, threads, 0, s>>>(
                                 P, ctl, T, W, L.prop_blocks, rollouts_per_block)));
    return cudaGetLastError();
}

cudaError_t launch_tree_reset(const DevProblem &P, Ctl *ctl, const DevTree &T, const float *x_init_dev,
                              cudaStream_t s)
{
    PAKR_DISPATCH_DYN(P.dyn, (k_tree_reset<DYN_><<<1, 32, 0, s>>>(P, ctl, T, x_init_dev)));
    return cudaGetLastError();
}

cudaError_t launch_import_fcost(const DevProblem &P, Ctl *ctl, const DevTree &T, int count, cudaStream_t s)
{
    const int blocks = (count + 255) / 256;
    PAKR_DISPATCH_DYN(P.dyn, (k_import_fcost<DYN_><<<blocks, 256, 0, s>>>(P, ctl, T, count)));
    return cudaGetLastError();
}

cudaError_t launch_plan_init(const DevProblem &P, Ctl *ctl, const DevTree &T, const PlanParams *pp,
                             cudaGraphConditionalHandle h, cudaStream_t s)
{
    PAKR_DISPATCH_DYN(P.dyn, (k_plan_init<DYN_><<<1, 32, 0, s>>>(P, ctl, T, pp, h)));
    return cudaGetLastError();
}

cudaError_t launch_plan_step(const DevProblem &P, Ctl *ctl, const DevTree &T, const PlanParams *pp,
                             const DevPlanBufs &B, cudaGraphConditionalHandle h, cudaStream_t s,
                             const cudaGraphConditionalHandle *inner)
{
    const cudaGraphConditionalHandle h0 = inner ? inner[0] : cudaGraphConditionalHandle{};
    const cudaGraphConditionalHandle h1 = inner ? inner[1] : cudaGraphConditionalHandle{};
    PAKR_DISPATCH_DYN(P.dyn, (k_plan_step<Dims<DYN_>::D, Dims<DYN_>::M><<<1, 32, 0, s>>>(P, ctl, T, pp, B, h, h0, h1,
                                                                                           inner ? 1 : 0)));
    return cudaGetLastError();
}

cudaError_t launch_plan_cont(const Ctl *ctl, cudaGraphConditionalHandle h, cudaStream_t s)
{
    k_plan_cont<<<1, 32, 0, s>>>(ctl, h);
    return cudaGetLastError();
}

// Loads k_offer_bound's GPU code now: a first launch would load it lazily, and loading code can
// wait for kernels that are running, such as the AO-x graph the offer is meant for.
cudaError_t preload_offer_bound()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, k_offer_bound);
}

cudaError_t launch_offer_bound(Ctl *ctl, const float *cost, cudaStream_t s)
{
    k_offer_bound<<<1, 32, 0, s>>>(ctl, cost);
    return cudaGetLastError();
}

cudaError_t launch_truncate(Ctl *ctl, int count, cudaStream_t s)
{
    k_truncate<<<1, 32, 0, s>>>(ctl, count);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int64_t n, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    k_philox<<<(unsigned)blocks, 256, 0, s>>>(ctr, k0, k1, out, n);
    return cudaGetLastError();
}

template <int D>
static int nn_occ(int variant)
{
    int nb = 0;
    switch (variant) {
    case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_nn<D, 1, 64, kNnTile, kNnGroup>, 64, 0); break;
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_nn<D, 1, 128, kNnTile, kNnGroup>, 128, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_nn<D, 2, 256, kNnTile, kNnGroup>, 256, 0); break;
    }
    return nb;
}

// Loads the GPU code of every k_nn instantiation (three variants for each supported state
// dimension) by querying its attributes, so that a later first launch of any of them loads
// nothing.
template <int D>
static cudaError_t nn_preload_d()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_nn<D, 1, 64, kNnTile, kNnGroup>);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&a, k_nn<D, 1, 128, kNnTile, kNnGroup>);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&a, k_nn<D, 2, 256, kNnTile, kNnGroup>);
    return e;
}

cudaError_t nn_preload_all()
{
    cudaError_t e = nn_preload_d<3>();
    if (e == cudaSuccess)
        e = nn_preload_d<4>();
    if (e == cudaSuccess)
        e = nn_preload_d<5>();
    if (e == cudaSuccess)
        e = nn_preload_d<6>();
    if (e == cudaSuccess)
        e = nn_preload_d<12>();
    return e;
}

int nn_blocks_per_sm(int d, int variant)
{
    switch (d) {
    case 3: return nn_occ<3>(variant);
    case 4: return nn_occ<4>(variant);
    case 5: return nn_occ<5>(variant);
    case 6: return nn_occ<6>(variant);
    case 12: return nn_occ<12>(variant);
    default: return 0;
    }
}

}  // namespace pakr
