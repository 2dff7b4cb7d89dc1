// pakr_device.cuh -- device functions of one PAKR expansion iteration
// (Algorithm 1 inner loop), shared by the single-query kernels
// (pakr_kernels.cu) and the batched persistent planner (pakr_batch.cu):
// Philox4x32-10, the dynamics and RK4, validity and heuristic, and the block
// bodies of SampleStates, NearestNeighbor, Propagate and insert.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pakr_internal.h"
#include "pakr_tc.cuh"

namespace pakr {


// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products, Weyl key schedule.
// ---------------------------------------------------------------------------
struct Words4 {
    uint32_t w[4];
};

__device__ __forceinline__ Words4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                         uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    Words4 r;
    r.w[0] = c0;
    r.w[1] = c1;
    r.w[2] = c2;
    r.w[3] = c3;
    return r;
}

// Top 24 bits as a uniform in [0, 1): exact in FP32.
__device__ __forceinline__ float u01(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

__device__ __forceinline__ float lerp_box(float lo, float hi, uint32_t w) { return __fmaf_rn(hi - lo, u01(w), lo); }

// Squared distance of the first N coordinates of a and b as a chain of fused multiply-adds
// (the library compiles without implicit contraction, so it is written out).
template <int N>
__device__ __forceinline__ float sq_dist(const float *a, const float *b)
{
    const float d0 = a[0] - b[0];
    float dd = __fmul_rn(d0, d0);
#pragma unroll
    for (int k = 1; k < N; ++k) {
        const float dk = a[k] - b[k];
        dd = __fmaf_rn(dk, dk, dd);
    }
    return dd;
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// Dynamics x' = f(x, u) (Eq. 1) per model, FP32.
// ---------------------------------------------------------------------------
template <int DYN> struct Dims;
template <> struct Dims<DI2> { static constexpr int D = 4, M = 2, PD = 2; };
template <> struct Dims<DI3> { static constexpr int D = 6, M = 3, PD = 3; };
template <> struct Dims<QUAD12> { static constexpr int D = 12, M = 4, PD = 3; };
template <> struct Dims<DUBINS3D> { static constexpr int D = 6, M = 3, PD = 3; };
template <> struct Dims<UNICYCLE1> { static constexpr int D = 3, M = 2, PD = 2; };
template <> struct Dims<UNICYCLE2> { static constexpr int D = 5, M = 2, PD = 2; };

template <int DYN>
__device__ __forceinline__ void deriv(const float *x, const float *u, float *xd, const DevProblem &P);

// Double integrator: position' = velocity, velocity' = control.
template <>
__device__ __forceinline__ void deriv<DI2>(const float *x, const float *u, float *xd, const DevProblem &)
{
    xd[0] = x[2];
    xd[1] = x[3];
    xd[2] = u[0];
    xd[3] = u[1];
}

template <>
__device__ __forceinline__ void deriv<DI3>(const float *x, const float *u, float *xd, const DevProblem &)
{
    xd[0] = x[3];
    xd[1] = x[4];
    xd[2] = x[5];
    xd[3] = u[0];
    xd[4] = u[1];
    xd[5] = u[2];
}

// Quadcopter, Z-Y-X Euler angles, body-frame linear / angular velocity, thrust
// along body z, gravity -g along world z: p' = R v, eta' = W(eta) omega,
// v' = v x omega + R^T g + T/m e3, omega' = I^-1 (tau - omega x I omega).
template <>
__device__ __forceinline__ void deriv<QUAD12>(const float *x, const float *u, float *xd, const DevProblem &P)
{
    const float mass = P.model[0], Ixx = P.model[1], Iyy = P.model[2], Izz = P.model[3], g = P.model[4];
    float sf, cf, st, ct, sp, cp;
    sincosf(x[3], &sf, &cf);
    sincosf(x[4], &st, &ct);
    sincosf(x[5], &sp, &cp);
    const float r00 = cp * ct, r01 = cp * st * sf - sp * cf, r02 = cp * st * cf + sp * sf;
    const float r10 = sp * ct, r11 = sp * st * sf + cp * cf, r12 = sp * st * cf - cp * sf;
    const float r20 = -st, r21 = ct * sf, r22 = ct * cf;
    const float vu = x[6], vv = x[7], vw = x[8];
    const float wp = x[9], wq = x[10], wr = x[11];
    xd[0] = r00 * vu + r01 * vv + r02 * vw;
    xd[1] = r10 * vu + r11 * vv + r12 * vw;
    xd[2] = r20 * vu + r21 * vv + r22 * vw;
    const float tt = st / ct;
    xd[3] = wp + sf * tt * wq + cf * tt * wr;
    xd[4] = cf * wq - sf * wr;
    xd[5] = (sf * wq + cf * wr) / ct;
    xd[6] = (vv * wr - vw * wq) + (-g * r20);
    xd[7] = (vw * wp - vu * wr) + (-g * r21);
    xd[8] = (vu * wq - vv * wp) + (-g * r22) + u[0] / mass;
    const float Ip = Ixx * wp, Iq = Iyy * wq, Ir = Izz * wr;
    xd[9] = (u[1] - (wq * Ir - wr * Iq)) / Ixx;
    xd[10] = (u[2] - (wr * Ip - wp * Ir)) / Iyy;
    xd[11] = (u[3] - (wp * Iq - wq * Ip)) / Izz;
}

// Dubins airplane: speed v along the heading given by yaw and pitch.
template <>
__device__ __forceinline__ void deriv<DUBINS3D>(const float *x, const float *u, float *xd, const DevProblem &)
{
    float sy, cy, sp, cp;
    sincosf(x[3], &sy, &cy);
    sincosf(x[4], &sp, &cp);
    xd[0] = x[5] * cp * cy;
    xd[1] = x[5] * cp * sy;
    xd[2] = x[5] * sp;
    xd[3] = u[0];
    xd[4] = u[1];
    xd[5] = u[2];
}

template <>
__device__ __forceinline__ void deriv<UNICYCLE1>(const float *x, const float *u, float *xd, const DevProblem &)
{
    float s, c;
    sincosf(x[2], &s, &c);
    xd[0] = u[0] * c;
    xd[1] = u[0] * s;
    xd[2] = u[1];
}

template <>
__device__ __forceinline__ void deriv<UNICYCLE2>(const float *x, const float *u, float *xd, const DevProblem &)
{
    float s, c;
    sincosf(x[2], &s, &c);
    xd[0] = x[3] * c;
    xd[1] = x[3] * s;
    xd[2] = x[4];
    xd[3] = u[0];
    xd[4] = u[1];
}

// Classical RK4 step with the control held (Sec. IV-A).  The stage sum is
// accumulated in the order k1 + 2 k2 + 2 k3 + k4; the stage points and the
// update are explicit fused multiply-adds.
template <int DYN>
__device__ __forceinline__ void rk4_step(float *x, const float *u, float h, const DevProblem &P)
{
    constexpr int D = Dims<DYN>::D;
    float k[D], t[D], acc[D];
    const float hh = 0.5f * h;
    deriv<DYN>(x, u, k, P);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        acc[a] = k[a];
        t[a] = __fmaf_rn(hh, k[a], x[a]);
    }
    deriv<DYN>(t, u, k, P);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        acc[a] = __fmaf_rn(2.0f, k[a], acc[a]);
        t[a] = __fmaf_rn(hh, k[a], x[a]);
    }
    deriv<DYN>(t, u, k, P);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        acc[a] = __fmaf_rn(2.0f, k[a], acc[a]);
        t[a] = __fmaf_rn(h, k[a], x[a]);
    }
    deriv<DYN>(t, u, k, P);
    const float h6 = h / 6.0f;
#pragma unroll
    for (int a = 0; a < D; ++a)
        x[a] = __fmaf_rn(h6, acc[a] + k[a], x[a]);
}

// ---------------------------------------------------------------------------
// Validity (point robot): closed state box is valid, closed boxes and balls
// are obstacles.  Obstacles come as padded float4 records.
// ---------------------------------------------------------------------------
template <int D, int PD>
__device__ __forceinline__ bool state_valid(const float *x, const DevProblem &P, const float4 *boxes, int nb,
                                            const float4 *spheres, int ns)
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a)
        ok = ok && (x[a] >= P.x_lo[a]) && (x[a] <= P.x_hi[a]);
    if (!ok)
        return false;
    for (int b = 0; b < nb; ++b) {
        const float4 lo = boxes[2 * b], hi = boxes[2 * b + 1];
        bool inside = (x[0] >= lo.x) & (x[0] <= hi.x) & (x[1] >= lo.y) & (x[1] <= hi.y);
        if (PD > 2)
            inside = inside & (x[2] >= lo.z) & (x[2] <= hi.z);
        if (inside)
            return false;
    }
    for (int s = 0; s < ns; ++s) {
        const float4 c = spheres[s];
        const float cc[3] = {c.x, c.y, c.z};
        if (sq_dist<PD>(x, cc) <= c.w * c.w)
            return false;
    }
    return true;
}

// h of the f-cost (Sec. IV): distance of the position to the goal ball
// (duration cost: divided by the speed bound), or the whole-state Euclidean
// distance to the goal state when the full-state formula is selected.
template <int D, int PD>
__device__ __forceinline__ float heuristic(const float *x, const DevProblem &P, const float *goal)
{
    if (P.heuristic == H_FULLSTATE)
        return sqrtf(sq_dist<D>(x, goal));
    const float h = fmaxf(0.f, sqrtf(sq_dist<PD>(x, goal)) - P.goal_r);
    if (P.cost == COST_DURATION)
        return P.h_speed > 0.f ? h / P.h_speed : 0.f;
    return h;
}

template <int PD>
__device__ __forceinline__ bool in_goal(const float *x, const DevProblem &P, const float *goal)
{
    return sq_dist<PD>(x, goal) <= P.goal_r * P.goal_r;
}

// ---------------------------------------------------------------------------
// k_sample: SampleStates and per-batch reset of the control block.
// ---------------------------------------------------------------------------
// Sample i of this batch into xr and clear its NN key.
template <int D>
__device__ __forceinline__ void sample_state(const DevProblem &P, const DevWork &W, int i, uint32_t it,
                                             unsigned long long seed)
{
    constexpr int NB = (D + 3) / 4;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const Words4 w = philox(it, (uint32_t)i, 0xFFFFFFFFu, (uint32_t)b, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int dim = 4 * b + t;
            if (dim < D)
                W.xr[(size_t)dim * P.K + i] = lerp_box(P.x_lo[dim], P.x_hi[dim], w.w[t]);
        }
    }
    W.nn_key[i] = kNoKey;
    if (W.nn_amin)
        W.nn_amin[i] = 0xFFFFFFFFu;
}

// Per-batch reset of a control block: the bound, the frozen tree size and the counters.
__device__ __forceinline__ void begin_batch(Ctl *ctl, float bound)
{
    ctl->bound = bound;
    ctl->n_start = ctl->count;
    ctl->goal_key = kNoKey;
    ctl->n_appended = 0;
    ctl->n_pruned = 0;
    ctl->n_collided = 0;
    ctl->n_no_parent = 0;
    ctl->n_dropped = 0;
}

// Instantiate BODY for the runtime dynamics id (DYN_ names the model).
#define PAKR_DISPATCH_DYN(dyn, BODY)                                                                                   \
    switch (dyn) {                                                                                                     \
    case DI2: { constexpr int DYN_ = DI2; BODY; } break;                                                               \
    case DI3: { constexpr int DYN_ = DI3; BODY; } break;                                                               \
    case QUAD12: { constexpr int DYN_ = QUAD12; BODY; } break;                                                         \
    case DUBINS3D: { constexpr int DYN_ = DUBINS3D; BODY; } break;                                                     \
    case UNICYCLE1: { constexpr int DYN_ = UNICYCLE1; BODY; } break;                                                   \
    case UNICYCLE2: { constexpr int DYN_ = UNICYCLE2; BODY; } break;                                                   \
    default: return cudaErrorInvalidValue;                                                                             \
    }

// ---------------------------------------------------------------------------
// k_nn: cost-pruned brute-force nearest neighbour.
//
// Result: for each query the eligible node (f-cost below the bound) with the
// smallest exact FP32 squared distance  e = sum_a fl(q_a - x_a)^2  (FADD then
// FMA per coordinate, in coordinate order), the lowest index on a tie.  The
// coordinates are the weighted states centred on the state box:
// q_a = fl(fl(q_a sw_a) - c_a), the same values the tensor-core kernel keeps
// in its packed copy (P.tc_c = c; zero where no box is known).
//
// Scan: block (chunk c, query group g) holds 2*QP queries per thread as QP
// float2 pairs and streams its node range in TILE-node tiles through shared
// memory.  The scan ranks nodes by the expanded form
//     a = (|q|^2 + |x|^2) + sum_a q_a (-2 x_a),
// one packed FFMA2 per coordinate for two queries (a tile row holds
// (|x|^2, |x|^2, -2x_0, -2x_0, ...)), about half the FP32 work of the exact
// form.  For every group of G consecutive nodes it keeps a running minimum
// (one FMNMX per pair) and per query the two smallest group minima m1 <= m2
// with their groups.  Ineligible nodes and padding carry |x|^2 = +inf.
//
// Exactness: rounding error analysis bounds |a - e| <= B = 2 gamma_{3D+3}
// (|q| + X)^2 with gamma_k = k u / (1 - k u), u = 2^-24, X the largest node
// norm of the chunk.  After the scan each query recomputes the exact form on
// its best group (first node of the group minimum on a tie).  Every node of
// another group has e >= m2 - B, so if m2 - B exceeds that exact minimum the
// exact argmin of the chunk lies in the best group; otherwise the second group
// is recomputed too, and if m2 - B still does not exceed the best exact value
// the whole block rescans the chunk exactly for that query (nodes spread over
// the threads, a warp minimum of the packed keys).  The answer is therefore
// the exact argmin, bit for bit.  Across threads and chunks the key
// (distance bits << 32 | index) is merged with atomicMin, ordering by
// distance and then by index (non-negative floats order like their bits).
// ---------------------------------------------------------------------------
// Resident blocks per SM the register budget is set for: about 80 registers
// per thread for D <= 6, 128 for D = 12.
template <int D, int NT>
struct NnMinBlocks {
    static constexpr int value = 65536 / (NT * (D <= 6 ? 80 : 128));
};

// Exact FP32 squared distance of node j to query qv, or +inf if ineligible.
template <int D>
__device__ __forceinline__ float exact_dist2(const DevProblem &P, const DevTree &T, int j, float bound, const float *qv)
{
    if (!(T.fcost[j] < bound))
        return __int_as_float(0x7f800000);
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float nx = -__fsub_rn(__fmul_rn(T.X[(size_t)a * P.cap + j], P.sw[a]), P.tc_c[a]);
        const float diff = __fadd_rn(qv[a], nx);
        acc = (a == 0) ? __fmul_rn(diff, diff) : __fmaf_rn(diff, diff, acc);
    }
    return acc;
}

// Exact minimum over the group [j0, j0 + G) (nodes below end): smallest
// distance, lowest index on a tie; all loads issued before the comparisons.
template <int D, int G>
__device__ __forceinline__ void exact_min_group(const DevProblem &P, const DevTree &T, int j0, int end, float bound,
                                                const float *qv, float &best, int &bidx)
{
    float e[G];
#pragma unroll
    for (int g = 0; g < G; ++g)
        e[g] = (j0 + g < end) ? exact_dist2<D>(P, T, j0 + g, bound, qv) : __int_as_float(0x7f800000);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = j0 + g;
        if (e[g] < best || (e[g] == best && j < bidx)) {
            best = e[g];
            bidx = j;
        }
    }
}

// Queries per block whose chunk is rescanned cooperatively (more fall back to a per-thread scan).
constexpr int kNnFlagCap = 64;

// gamma_k of rounding error analysis for FP32 (u = 2^-24).
__host__ __device__ constexpr float nn_gamma(int k) { return (k * 5.9604645e-8f) / (1.f - k * 5.9604645e-8f); }

// One block's scan: 2*QP queries per thread starting at query qbase, nodes
// [start, end) in tiles; merges each query's result into W.nn_key.  All
// threads of the block must call it (it synchronises the block).
template <int D, int QP, int NT, int TILE, int G>
__device__ __forceinline__ void nn_scan(const DevProblem &P, const DevTree &T, const DevWork &W, float bound,
                                        int qbase, int start, int end, float *s_node)
{
    constexpr int NQ = 2 * QP;                     // queries per thread
    constexpr int RW = (2 * D + 2 + 3) / 4 * 4;    // floats per tile row
    constexpr int RV = RW / 4;
    static_assert(TILE % G == 0, "tile must hold whole groups");
    __shared__ float s_xmax[NT / 32];
    __shared__ int s_nflag;
    __shared__ int s_flag_qid[kNnFlagCap];
    __shared__ float s_flag_q[kNnFlagCap][D];
    const int K = P.K;
    const int cap = P.cap;
    const int tid = threadIdx.x;
    const float inf = __int_as_float(0x7f800000);

    // query qi of this thread is qbase + qi * NT + tid; packed pair p holds queries 2p and 2p+1
    float qs[NQ][D], qn[NQ];
#pragma unroll
    for (int qi = 0; qi < NQ; ++qi) {
        const int qid = qbase + qi * NT + tid;
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            qs[qi][a] = (qid < K) ? __fsub_rn(__fmul_rn(W.xr[(size_t)a * K + qid], P.sw[a]), P.tc_c[a]) : 0.f;
            s = __fmaf_rn(qs[qi][a], qs[qi][a], s);
        }
        qn[qi] = s;
    }
    float m1[NQ], m2[NQ];
    int g1[NQ], g2[NQ];
#pragma unroll
    for (int qi = 0; qi < NQ; ++qi) {
        m1[qi] = inf;
        m2[qi] = inf;
        g1[qi] = -1;
        g2[qi] = -1;
    }
    float xmax2 = 0.f;  // largest eligible node norm this thread staged
    const float4 *s4 = reinterpret_cast<const float4 *>(s_node);

    for (int t0 = start; t0 < end; t0 += TILE) {
        const int tile_len = min(TILE, (end - t0 + G - 1) / G * G);  // whole groups; the tail is +inf padding
        __syncthreads();
        for (int e = tid; e < tile_len; e += NT) {
            const int j = t0 + e;
            const bool in = j < end;
            const bool ok = in && (T.fcost[j] < bound);
            float row[RW];
#pragma unroll
            for (int a = 0; a < RW; ++a)
                row[a] = 0.f;
            float xn = 0.f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float v = in ? __fsub_rn(__fmul_rn(T.X[(size_t)a * cap + j], P.sw[a]), P.tc_c[a]) : 0.f;
                xn = __fmaf_rn(v, v, xn);
                row[2 + 2 * a] = -2.f * v;
                row[3 + 2 * a] = -2.f * v;
            }
            if (ok)
                xmax2 = fmaxf(xmax2, xn);
            else
                xn = inf;
            row[0] = xn;
            row[1] = xn;
            float4 *dst = reinterpret_cast<float4 *>(&s_node[e * RW]);
#pragma unroll
            for (int c = 0; c < RV; ++c)
                dst[c] = make_float4(row[4 * c], row[4 * c + 1], row[4 * c + 2], row[4 * c + 3]);
        }
        __syncthreads();
        for (int e0 = 0; e0 < tile_len; e0 += G) {
            float m[NQ];
#pragma unroll
            for (int qi = 0; qi < NQ; ++qi)
                m[qi] = inf;
#pragma unroll 2
            for (int g = 0; g < G; ++g) {
                const float4 *src = s4 + (e0 + g) * RV;
                float nx[RW];
#pragma unroll
                for (int c = 0; c < RV; ++c) {
                    const float4 t = src[c];
                    nx[4 * c] = t.x;
                    nx[4 * c + 1] = t.y;
                    nx[4 * c + 2] = t.z;
                    nx[4 * c + 3] = t.w;
                }
#pragma unroll
                for (int p = 0; p < QP; ++p) {
                    float2 acc = __fadd2_rn(make_float2(qn[2 * p], qn[2 * p + 1]), make_float2(nx[0], nx[1]));
#pragma unroll
                    for (int a = 0; a < D; ++a)
                        acc = __ffma2_rn(make_float2(qs[2 * p][a], qs[2 * p + 1][a]),
                                         make_float2(nx[2 + 2 * a], nx[3 + 2 * a]), acc);
                    m[2 * p] = fminf(m[2 * p], acc.x);
                    m[2 * p + 1] = fminf(m[2 * p + 1], acc.y);
                }
            }
            const int grp = t0 + e0;
#pragma unroll
            for (int qi = 0; qi < NQ; ++qi) {
                const bool c1 = m[qi] < m1[qi];
                const bool c2 = m[qi] < m2[qi];
                m2[qi] = c1 ? m1[qi] : (c2 ? m[qi] : m2[qi]);
                g2[qi] = c1 ? g1[qi] : (c2 ? grp : g2[qi]);
                m1[qi] = c1 ? m[qi] : m1[qi];
                g1[qi] = c1 ? grp : g1[qi];
            }
        }
    }
    // largest node norm of the chunk (a block-wide maximum)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        xmax2 = fmaxf(xmax2, __shfl_xor_sync(0xFFFFFFFFu, xmax2, o));
    __syncthreads();
    if ((tid & 31) == 0)
        s_xmax[tid >> 5] = xmax2;
    if (tid == 0)
        s_nflag = 0;
    __syncthreads();
    float X2 = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w)
        X2 = fmaxf(X2, s_xmax[w]);
    const float X = sqrtf(X2);
    constexpr float kGamma = nn_gamma(3 * D + 3);
#pragma unroll
    for (int qi = 0; qi < NQ; ++qi) {
        const int qid = qbase + qi * NT + tid;
        if (qid >= K || g1[qi] < 0 || !(m1[qi] < inf))
            continue;
        const float r = sqrtf(qn[qi]) + X;
        const float B = 2.f * kGamma * r * r * 1.0001f;
        float best = inf;
        int bidx = 0x7FFFFFFF;
        exact_min_group<D, G>(P, T, g1[qi], end, bound, qs[qi], best, bidx);
        bool certain = m2[qi] - B > best;
        if (!certain && g2[qi] >= 0) {
            exact_min_group<D, G>(P, T, g2[qi], end, bound, qs[qi], best, bidx);
            certain = m2[qi] - B > best;
        }
        if (certain) {
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(best) << 32) | (unsigned long long)(uint32_t)bidx;
            atomicMin(&W.nn_key[qid], key);
        } else {
            // a third group may be as close: the block rescans the chunk for this query below
            const int slot = atomicAdd(&s_nflag, 1);
            if (slot < kNnFlagCap) {
                s_flag_qid[slot] = qid;
#pragma unroll
                for (int a = 0; a < D; ++a)
                    s_flag_q[slot][a] = qs[qi][a];
            } else {
                float b2 = inf;
                int i2 = 0x7FFFFFFF;
                for (int j = start; j < end; ++j) {
                    const float e = exact_dist2<D>(P, T, j, bound, qs[qi]);
                    if (e < b2) {
                        b2 = e;
                        i2 = j;
                    }
                }
                if (b2 < inf)
                    atomicMin(&W.nn_key[qid],
                              ((unsigned long long)__float_as_uint(b2) << 32) | (unsigned long long)(uint32_t)i2);
            }
        }
    }
    __syncthreads();
    // exact rescans of the flagged queries by the whole block (coalesced nodes, warp minimum)
    const int nflag = min(s_nflag, kNnFlagCap);
    for (int f = 0; f < nflag; ++f) {
        float qv[D];
#pragma unroll
        for (int a = 0; a < D; ++a)
            qv[a] = s_flag_q[f][a];
        unsigned long long key = kNoKey;
        for (int j = start + tid; j < end; j += NT) {
            const float e = exact_dist2<D>(P, T, j, bound, qv);
            if (e < inf) {
                const unsigned long long k =
                    ((unsigned long long)__float_as_uint(e) << 32) | (unsigned long long)(uint32_t)j;
                key = k < key ? k : key;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, key, o);
            key = other < key ? other : key;
        }
        if ((tid & 31) == 0 && key != kNoKey)
            atomicMin(&W.nn_key[s_flag_qid[f]], key);
    }
}

// Node chunk of a block: an even share of the n nodes, a multiple of the
// group size and at least 64 nodes, so a small tree spreads over as many
// blocks as it fills.
template <int G>
__device__ __forceinline__ int nn_chunk_nodes(int n, int nchunks)
{
    const int per = (n + nchunks - 1) / nchunks;
    return max(64, (per + G - 1) / G * G);
}

// ---------------------------------------------------------------------------
// k_propagate: LG lanes per rollout r = i*k + j (LG divides 32).
//
// Every lane of a rollout's group samples the same control (counter-based
// Philox) and integrates the same RK4 steps, so their states are identical;
// the obstacle tests of each substep are split across the group's lanes and
// combined with a warp ballot (LG > 1; then the substep loop runs to the
// warp's longest rollout so that every lane reaches each ballot).  The
// obstacle tests of a substep are those of the position's cell of the
// obstacle grid when the planner keeps one (every obstacle otherwise), which
// gives the same answer with a few tests instead of all.  With path-length
// cost and the position heuristic, f = g + h never decreases along an edge (h
// is 1-Lipschitz in position), so a partial f at or above a finite bound
// already decides the prune.
// ---------------------------------------------------------------------------
template <int D, int PD>
__device__ __forceinline__ bool in_state_box(const float *x, const DevProblem &P)
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a)
        ok = ok & (x[a] >= P.x_lo[a]) & (x[a] <= P.x_hi[a]);
    return ok;
}

template <int PD>
__device__ __forceinline__ bool in_box(const float *x, const float4 *boxes, int b)
{
    const float4 lo = boxes[2 * b], hi = boxes[2 * b + 1];
    bool inside = (x[0] >= lo.x) & (x[0] <= hi.x) & (x[1] >= lo.y) & (x[1] <= hi.y);
    if (PD > 2)
        inside = inside & (x[2] >= lo.z) & (x[2] <= hi.z);
    return inside;
}

template <int PD>
__device__ __forceinline__ bool in_sphere(const float *x, const float4 *spheres, int s)
{
    const float4 c = spheres[s];
    const float cc[3] = {c.x, c.y, c.z};
    return sq_dist<PD>(x, cc) <= c.w * c.w;
}

// Obstacle test of position x on this lane's share (first, first + stride, ...) of the
// obstacles: all of them, or with the obstacle grid only those listed in x's cell.
template <int PD>
__device__ __forceinline__ bool hits_obstacle(const float *x, const DevProblem &P, const float4 *boxes, int nb,
                                              const float4 *spheres, int ns, const int *g_start,
                                              const unsigned short *g_items, int first, int stride)
{
    if (P.grid_g > 0) {
        const int g = P.grid_g;
        int c = obstacle_cell(x[0], P.grid_lo[0], P.grid_inv[0], g) + g * obstacle_cell(x[1], P.grid_lo[1], P.grid_inv[1], g);
        if (PD > 2)
            c += g * g * obstacle_cell(x[2], P.grid_lo[2], P.grid_inv[2], g);
        const int k1 = g_start[c + 1];
        for (int k = g_start[c] + first; k < k1; k += stride) {
            const int o = g_items[k];
            if (o < nb ? in_box<PD>(x, boxes, o) : in_sphere<PD>(x, spheres, o - nb))
                return true;
        }
        return false;
    }
    for (int b = first; b < nb; b += stride)
        if (in_box<PD>(x, boxes, b))
            return true;
    for (int s = first; s < ns; s += stride)
        if (in_sphere<PD>(x, spheres, s))
            return true;
    return false;
}

// Block-wide copy of n elements from global to shared memory with every thread's loads (up to
// four) issued before its stores, so that a block staging a few KB pays about one memory round
// trip instead of one per loop pass.
template <typename T>
__device__ __forceinline__ void stage_to_shared(T *dst, const T *src, int n)
{
    const int nt = blockDim.x;
    for (int t0 = threadIdx.x; t0 < n; t0 += 4 * nt) {
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t0 + k * nt < n)
                v[k] = src[t0 + k * nt];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t0 + k * nt < n)
                dst[t0 + k * nt] = v[k];
    }
}

// Rollouts of propagate block vb (blockDim.x / LG rollouts) with the obstacles staged into
// s_obs (2 n_boxes + n_spheres float4, then the goal, then the obstacle grid's cell offsets and
// lists).
template <int DYN, int LG>
__device__ __forceinline__ void propagate_block(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W,
                                                int vb, float4 *s_obs)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    float4 *s_box = s_obs;
    float4 *s_sph = s_obs + 2 * P.n_boxes;
    float *s_goal = reinterpret_cast<float *>(s_sph + P.n_spheres);
    int *s_gstart = reinterpret_cast<int *>(s_goal + kMaxD);
    unsigned short *s_gitems = reinterpret_cast<unsigned short *>(s_gstart + P.grid_cells + 1);

    const int R = P.K * P.k;
    const int lane = threadIdx.x & 31;
    const int sub = lane % LG;
    const unsigned gmask = (LG == 32 ? 0xFFFFFFFFu : ((1u << LG) - 1u)) << (lane - sub);
    const int r = (int)(((long long)vb * blockDim.x + threadIdx.x) / LG);
    const bool have = r < R;
    const float bound = ctl->bound;
    // with path-length cost and the position heuristic f never decreases along an edge, so a
    // partial f at or above a finite bound already decides the prune
    const bool early = (P.cost == COST_PATH_LENGTH) && (P.heuristic == H_POSITION) &&
                       (bound < __int_as_float(0x7f800000));

    // SampleControls and the parent's state first: their global loads are in flight while the
    // block stages the obstacles below
    int out = -1;
    bool alive = false;
    float u[M];
    float x[D];
    float g = 0.f, f = 0.f;
    int S = 0, par = -1;
    if (have) {
        const int i = r / P.k;
        const int j = r - i * P.k;
        const uint32_t it = ctl->iteration;
        const unsigned long long seed = ctl->seed;
        // words 0..M-1 the control, word M the duration
        constexpr int NB = (M + 1 + 3) / 4;
        uint32_t words[4 * NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const Words4 w = philox(it, (uint32_t)i, (uint32_t)j, (uint32_t)b, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
            for (int t = 0; t < 4; ++t)
                words[4 * b + t] = w.w[t];
        }
#pragma unroll
        for (int a = 0; a < M; ++a)
            u[a] = lerp_box(P.u_lo[a], P.u_hi[a], words[a]);
        const uint64_t span = (uint64_t)(P.s_max - P.s_min + 1);
        S = P.s_min + (int)(((uint64_t)words[M] * span) >> 32);
        const unsigned long long key = W.nn_key[i];
        if (key == kNoKey) {
            out = OUT_NO_PARENT;
        } else {
            par = (int)(uint32_t)(key & 0xFFFFFFFFull);
#pragma unroll
            for (int a = 0; a < D; ++a)
                x[a] = T.X[(size_t)a * P.cap + par];
            g = T.cost[par];
            alive = true;
            if (P.cost == COST_DURATION) {
                g = g + (float)S * P.dt;
                if (!(g < bound)) {  // h >= 0
                    out = OUT_PRUNED;
                    alive = false;
                }
            }
        }
    }
    stage_to_shared(s_box, P.boxes, 2 * P.n_boxes);
    stage_to_shared(s_sph, P.spheres, P.n_spheres);
    if (threadIdx.x < D)
        s_goal[threadIdx.x] = ctl->x_goal[threadIdx.x];
    if (P.grid_g > 0) {
        stage_to_shared(s_gstart, P.grid_start, P.grid_cells + 1);
        stage_to_shared(s_gitems, P.grid_items, P.grid_n_items);
    }
    // outcome counters: cleared by thread 0 alone, the thread that read them at the end of the
    // block's previous call (the batched planner calls this body once per work item)
    __shared__ int s_cnt[4];
    if (threadIdx.x == 0) {
        s_cnt[0] = 0;
        s_cnt[1] = 0;
        s_cnt[2] = 0;
        s_cnt[3] = 0;
    }
    __syncthreads();

    // one lane per rollout: each lane runs its own substeps; with several lanes per rollout
    // every lane of the warp reaches each substep's ballot
    const int s_last = (LG == 1) ? (alive ? S : 0) : __reduce_max_sync(0xFFFFFFFFu, alive ? S : 0);
    for (int s = 1; s <= s_last; ++s) {
        const bool act = alive && s <= S;
        bool inb = true;
        if (act) {
            float xp[PD];
#pragma unroll
            for (int a = 0; a < PD; ++a)
                xp[a] = x[a];
            rk4_step<DYN>(x, u, P.dt, P);
            if (P.cost == COST_PATH_LENGTH)
                g += sqrtf(sq_dist<PD>(x, xp));
            inb = in_state_box<D, PD>(x, P);
        }
        const bool hit = act && inb &&
                         hits_obstacle<PD>(x, P, s_box, P.n_boxes, s_sph, P.n_spheres, s_gstart, s_gitems, sub, LG);
        bool any_hit = hit;
        if constexpr (LG > 1)
            any_hit = (__ballot_sync(0xFFFFFFFFu, hit) & gmask) != 0u;
        if (act) {
            if (!inb || any_hit) {
                out = OUT_COLLIDED;
                alive = false;
            } else if (early && !(g + heuristic<D, PD>(x, P, s_goal) < bound)) {
                out = OUT_PRUNED;
                alive = false;
            }
        }
    }
    if (alive) {
        f = g + heuristic<D, PD>(x, P, s_goal);
        out = (f < bound) ? OUT_APPENDED : OUT_PRUNED;
    }
    const bool leader = have && sub == 0;
    if (leader) {
#pragma unroll
        for (int a = 0; a < M; ++a)
            W.st_u[(size_t)a * R + r] = u[a];
        W.st_steps[r] = S;
        if (out == OUT_APPENDED) {
#pragma unroll
            for (int a = 0; a < D; ++a)
                W.st_x[(size_t)a * R + r] = x[a];
            W.st_cost[r] = g;
            W.st_f[r] = f;
            W.st_parent[r] = par;
        }
        // goal flag of every rollout: 1 only for a surviving child in the goal ball
        W.goal[r] = (out == OUT_APPENDED && in_goal<PD>(x, P, s_goal)) ? 1 : 0;
        W.outcome[r] = (int8_t)out;
    }
    // the four outcome counts of the block: warp ballots into the shared counters, one barrier
    const unsigned c_app = __ballot_sync(0xFFFFFFFFu, leader && out == OUT_APPENDED);
    const unsigned c_pr = __ballot_sync(0xFFFFFFFFu, leader && out == OUT_PRUNED);
    const unsigned c_col = __ballot_sync(0xFFFFFFFFu, leader && out == OUT_COLLIDED);
    const unsigned c_np = __ballot_sync(0xFFFFFFFFu, leader && out == OUT_NO_PARENT);
    if (lane == 0) {
        if (c_app)
            atomicAdd(&s_cnt[0], __popc(c_app));
        if (c_pr)
            atomicAdd(&s_cnt[1], __popc(c_pr));
        if (c_col)
            atomicAdd(&s_cnt[2], __popc(c_col));
        if (c_np)
            atomicAdd(&s_cnt[3], __popc(c_np));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        W.block_count[vb] = s_cnt[0];
        if (s_cnt[1])
            atomicAdd(&ctl->n_pruned, s_cnt[1]);
        if (s_cnt[2])
            atomicAdd(&ctl->n_collided, s_cnt[2]);
        if (s_cnt[3])
            atomicAdd(&ctl->n_no_parent, s_cnt[3]);
    }
}

// ---------------------------------------------------------------------------
// k_append: survivors of block b go to n_start + (survivors of blocks < b) +
// (rank inside the block), i.e. ascending rollout order; positions at or past
// the cap are dropped.  Goal children compete through atomicMin on the packed
// (cost bits << 32 | node) key: the cheapest wins, the lowest node on a tie.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_sum(int v, int *s_tmp)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
        s_tmp[wid] = v;
    __syncthreads();
    int tot = 0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w)
        tot += s_tmp[w];
    return tot;
}

// Append the survivors of propagate blocks vb * pbs .. vb * pbs + pbs - 1 (rpb rollouts each),
// handled by the first rpb * pbs threads (the rest take part in the scans only).  blockDim.x is a
// multiple of 32: the scans are warp-wide.
template <int D, int M>
__device__ __forceinline__ void append_block(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W, int vb,
                                             int nblk, int rpb, int pbs, int *s_tmp, int *s_warp)
{
    const int R = P.K * P.k;
    const int rpa = rpb * pbs;
    const int r = vb * rpa + threadIdx.x;
    const bool cand = ((int)threadIdx.x < rpa) && (r < R) && (W.outcome[r] == OUT_APPENDED);
    // the candidate's staged child is loaded before the prefix below, so that both round trips
    // to memory overlap
    float xs[D], us[M];
    float c = 0.f, fv = 0.f;
    int parent = 0, steps = 0;
    bool goal = false;
    if (cand) {
#pragma unroll
        for (int a = 0; a < D; ++a)
            xs[a] = W.st_x[(size_t)a * R + r];
#pragma unroll
        for (int a = 0; a < M; ++a)
            us[a] = W.st_u[(size_t)a * R + r];
        c = W.st_cost[r];
        fv = W.st_f[r];
        parent = W.st_parent[r];
        steps = W.st_steps[r];
        goal = W.goal[r] != 0;
    }
    // survivors of the blocks before this one, and of all: eight independent loads in flight
    int part = 0, tot = 0;
    for (int b0 = threadIdx.x; b0 < nblk; b0 += 8 * (int)blockDim.x) {
        int cnt[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = b0 + u * (int)blockDim.x;
            cnt[u] = b < nblk ? W.block_count[b] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            tot += cnt[u];
            if (b0 + u * (int)blockDim.x < vb * pbs)
                part += cnt[u];
        }
    }
    part = block_sum(part, s_tmp);
    tot = block_sum(tot, s_tmp);

    const int n_start = ctl->n_start;
    const int cap = P.cap;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, cand);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        s_warp[wid] = __popc(bal);
    __syncthreads();
    int warp_off = 0;
    for (int w = 0; w < wid; ++w)
        warp_off += s_warp[w];
    const long long pos = (long long)n_start + part + warp_off + __popc(bal & ((1u << lane) - 1u));
    if (cand) {
        if (pos < cap) {
            const int p = (int)pos;
#pragma unroll
            for (int a = 0; a < D; ++a)
                T.X[(size_t)a * cap + p] = xs[a];
            tc_pack_node<D>(P, T, ctl, p, xs);
#pragma unroll
            for (int a = 0; a < M; ++a)
                T.U[(size_t)a * cap + p] = us[a];
            T.cost[p] = c;
            T.fcost[p] = fv;
            T.parent[p] = parent;
            T.steps[p] = steps;
            if (goal)
                atomicMin(&ctl->goal_key, ((unsigned long long)__float_as_uint(c) << 32) | (unsigned long long)p);
        } else {
            W.outcome[r] = OUT_DROPPED;
        }
    }
    if (vb == 0 && threadIdx.x == 0) {
        long long room = (long long)cap - n_start;
        if (room < 0)
            room = 0;
        const int app = (int)min((long long)tot, room);
        ctl->n_appended = app;
        ctl->n_dropped = tot - app;
        ctl->count = n_start + app;
        ctl->iteration = ctl->iteration + 1u;
    }
}

// ---------------------------------------------------------------------------
// End of one AO-x loop pass for one tree (Algorithm 1): a goal child found by
// this batch becomes the new solution (c_best, history entry, best path via
// ExtractPath) and the tree restarts from its root; a tree that filled
// without a solution restarts too; the run stops at the first solution if
// asked, when no node can beat c_best, or when the device-clock budget or
// the iteration cap is spent.  c_best is only ever lowered (a minimum), so a
// bound offered by another stream while the loop runs is kept.  Called by all 32 lanes of one warp (lane 0
// chases parents, the warp gathers the path rows); returns, on lane 0,
// whether the run stops.
// ---------------------------------------------------------------------------
template <int D, int M>
__device__ __forceinline__ bool aox_step_warp(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevPlanBufs &B,
                                              int stop_at_first, unsigned long long budget_ns,
                                              long long max_iterations, int *s_len, int *s_found)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        const unsigned long long now = globaltimer_ns();
        ctl->iterations_done += 1;
        const unsigned long long key = ctl->goal_key;
        *s_found = 0;
        *s_len = 0;
        // a bound offered from outside during this iteration (pakr_plan_offer_bound) may already
        // be below the child's cost: then the child improves nothing and the tree goes on
        const float cur = *reinterpret_cast<volatile float *>(&ctl->c_best);
        if (key != kNoKey && __uint_as_float((uint32_t)(key >> 32)) < cur) {
            const float c = __uint_as_float((uint32_t)(key >> 32));
            const int node = (int)(uint32_t)(key & 0xFFFFFFFFull);
            // a new best path and its cost are being written: the sequence turns odd
            // (pakr_plan_snapshot discards what it copies meanwhile) and even again once the
            // rows are out
            ctl->path_seq = ctl->path_seq + 1u;
            __threadfence();
            // costs are non-negative, so their bit patterns order like the values: the minimum
            // keeps an offer that lands in between
            atomicMin(reinterpret_cast<int *>(&ctl->c_best), __float_as_int(c));
            ctl->sol_best = c;
            const int ns = ctl->n_solutions;
            if (ns < B.hist_cap) {
                B.hist_t[ns] = now - ctl->t0_ns;
                B.hist_cost[ns] = c;
                B.hist_iter[ns] = ctl->iterations_done - 1;
            }
            if (ns == 0) {
                ctl->t_first_ns = now - ctl->t0_ns;
                ctl->nodes_first = ctl->count;
                ctl->iterations_first = ctl->iterations_done;
            }
            ctl->n_solutions = ns + 1;
            // ExtractPath: length first, bounded by the node count.
            int len = 0;
            const int limit = ctl->count + 1;
            for (int v = node; v >= 0 && len <= limit; v = T.parent[v])
                ++len;
            if (len > limit) {
                ctl->err |= ERR_PATH_CYCLE;
                ctl->path_len = 0;
            } else if (len > B.path_cap + 1) {
                ctl->path_len = -len;
            } else {
                int at = len - 1;
                for (int v = node; v >= 0; v = T.parent[v])
                    B.path_nodes[at--] = v;
                ctl->path_len = len;
                *s_len = len;
            }
            *s_found = 1;
        }
    }
    __syncwarp();
    const int len = *s_len;
    for (int t = lane; t < len; t += 32) {
        const int v = B.path_nodes[t];
#pragma unroll
        for (int a = 0; a < D; ++a)
            B.path_x[(size_t)t * D + a] = T.X[(size_t)a * P.cap + v];
#pragma unroll
        for (int a = 0; a < M; ++a)
            B.path_u[(size_t)t * M + a] = T.U[(size_t)a * P.cap + v];
        B.path_steps[t] = T.steps[v];
    }
    __threadfence();
    __syncwarp();
    bool stop = false;
    if (lane == 0) {
        const unsigned long long now = globaltimer_ns();
        bool restart = false;
        const bool found = *s_found != 0;
        // a bound offered from outside that lowered c_best is a solution too: restart
        const bool offered = atomicExch(&ctl->offer_restart, 0) != 0;
        if (found)
            ctl->path_seq = ctl->path_seq + 1u;
        if (found || offered)
            restart = true;
        if (found) {
            if (stop_at_first) {
                stop = true;
                ctl->plan_status = 1;
            }
        } else if (ctl->count >= P.cap) {
            restart = true;
            ctl->n_restarts += 1;
        }
        if (!found && ctl->n_no_parent >= P.K * P.k) {
            stop = true;
            ctl->plan_status = 3;
        }
        if (now - ctl->t0_ns >= budget_ns || ctl->iterations_done >= max_iterations)
            stop = true;
        if (restart)
            ctl->count = 1;
        ctl->plan_stop = stop ? 1 : 0;
        ctl->t_end_ns = now;
    }
    __syncwarp();
    return stop;
}

// Fresh AO-x run for one tree (Algorithm 1): the goal, the root
// {(x_init, -, 0)}, c_best = c_best_init (+inf for a fresh run), the
// expansion counter at 0 and the device clock started.  One thread.  Returns whether the loop should run (a valid
// start, a positive budget and iteration cap).
template <int DYN>
__device__ __forceinline__ bool aox_init_one(const DevProblem &P, Ctl *ctl, const DevTree &T, const float *x_init,
                                             const float *x_goal, unsigned long long seed, long long max_iterations,
                                             unsigned long long budget_ns, float c_best_init)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    float x[D], goal[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = x_init[a];
        goal[a] = x_goal[a];
        ctl->x_goal[a] = goal[a];
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
    ctl->seed = seed;
    ctl->c_best = c_best_init;
    ctl->sol_best = __int_as_float(0x7f800000);
    ctl->iterations_done = 0;
    ctl->n_solutions = 0;
    ctl->n_restarts = 0;
    ctl->path_len = 0;
    ctl->path_seq = 0u;
    ctl->offer_restart = 0;
    ctl->err = 0;
    ctl->t_first_ns = ~0ull;
    ctl->nodes_first = -1;
    ctl->iterations_first = -1;
    const bool valid = state_valid<D, PD>(x, P, P.boxes, P.n_boxes, P.spheres, P.n_spheres);
    ctl->plan_status = valid ? 0 : -1;
    const bool run = valid && max_iterations > 0 && budget_ns > 0;
    ctl->plan_stop = run ? 0 : 1;
    const unsigned long long now = globaltimer_ns();
    ctl->t0_ns = now;
    ctl->t_end_ns = now;
    return run;
}

}  // namespace pakr
