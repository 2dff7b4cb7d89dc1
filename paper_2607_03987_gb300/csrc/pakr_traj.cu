// pakr_traj.cu -- smooth trajectory cost, its gradient with respect to the
// controls (a hand-written discrete adjoint of RK4 with checkpoints every 16
// steps), and a planner-rule validity check of control sequences.  Used to
// refine AO-x solutions by gradient descent; not part of the paper's method.
//
// Trajectory: x_{n+1} = RK4(x_n, u_n, dt) for n = 0..N-1, controls row-major
// U[(t*N + n)*m + j].  Cost
//   J = w_dur N dt + w_u sum_n |u_n|^2 dt
//     + w_obs sum_{n=1..N} sum_obstacles softplus_beta(margin - sdf(p_n)) dt
//     + w_goal |p_N - p_goal|^2 + w_len sum_n sqrt(|p_{n+1} - p_n|^2 + eps^2),
// softplus_beta(z) = log(1 + exp(beta z)) / beta.
//
// One warp per trajectory: every lane integrates the same steps, the
// obstacle terms are split across the lanes and summed with shuffles.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "pakr_device.cuh"

namespace pakr {
namespace {

constexpr int kCkpt = 16;  // checkpoint interval of the adjoint sweep
constexpr int kTrajWarpsPerBlock = 4;
constexpr int kRefineWarps = 2;     // warps of the refinement CTA: it fits beside the search kernels on an SM
constexpr int kRefineMaxCand = 32;  // line-search candidates per refinement iteration at most

struct TrajWeights {
    float w_dur, w_u, w_obs, beta, margin, w_goal, w_len, len_eps;
    float goal[kMaxD];
};

// ---------------------------------------------------------------------------
// Vector-Jacobian products a^T df/dx, a^T df/du of each model (FP32).
// ---------------------------------------------------------------------------
template <int DYN>
__device__ __forceinline__ void vjp(const float *x, const float *u, const float *a, float *gx, float *gu,
                                    const DevProblem &P);

template <>
__device__ __forceinline__ void vjp<DI2>(const float *, const float *, const float *a, float *gx, float *gu,
                                         const DevProblem &)
{
    gx[0] = 0.f;
    gx[1] = 0.f;
    gx[2] = a[0];
    gx[3] = a[1];
    gu[0] = a[2];
    gu[1] = a[3];
}

template <>
__device__ __forceinline__ void vjp<DI3>(const float *, const float *, const float *a, float *gx, float *gu,
                                         const DevProblem &)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gx[i] = 0.f;
        gx[3 + i] = a[i];
        gu[i] = a[3 + i];
    }
}

template <>
__device__ __forceinline__ void vjp<QUAD12>(const float *x, const float *, const float *a, float *gx, float *gu,
                                            const DevProblem &P)
{
    const float mass = P.model[0], Ixx = P.model[1], Iyy = P.model[2], Izz = P.model[3], g = P.model[4];
    float sf, cf, st, ct, sp, cp;
    sincosf(x[3], &sf, &cf);
    sincosf(x[4], &st, &ct);
    sincosf(x[5], &sp, &cp);
    const float tt = st / ct, ic = 1.f / ct, ic2 = ic * ic;
    const float v0 = x[6], v1 = x[7], v2 = x[8], w0 = x[9], w1 = x[10], w2 = x[11];
    const float ap0 = a[0], ap1 = a[1], ap2 = a[2], ae0 = a[3], ae1 = a[4], ae2 = a[5];
    const float av0 = a[6], av1 = a[7], av2 = a[8], aw0 = a[9], aw1 = a[10], aw2 = a[11];
    // rotation R = Rz(psi) Ry(theta) Rx(phi) and its partial derivatives
    const float R00 = cp * ct, R01 = cp * st * sf - sp * cf, R02 = cp * st * cf + sp * sf;
    const float R10 = sp * ct, R11 = sp * st * sf + cp * cf, R12 = sp * st * cf - cp * sf;
    const float R20 = -st, R21 = ct * sf, R22 = ct * cf;
    // d/dphi (column 0 is zero)
    const float F01 = cp * st * cf + sp * sf, F02 = -cp * st * sf + sp * cf;
    const float F11 = sp * st * cf - cp * sf, F12 = -sp * st * sf - cp * cf;
    const float F21 = ct * cf, F22 = -ct * sf;
    // d/dtheta
    const float T00 = -cp * st, T01 = cp * ct * sf, T02 = cp * ct * cf;
    const float T10 = -sp * st, T11 = sp * ct * sf, T12 = sp * ct * cf;
    const float T20 = -ct, T21 = -st * sf, T22 = -st * cf;
    // d/dpsi (row 2 is zero)
    const float P00 = -sp * ct, P01 = -sp * st * sf - cp * cf, P02 = -sp * st * cf + cp * sf;
    const float P10 = cp * ct, P11 = cp * st * sf - sp * cf, P12 = cp * st * cf + sp * sf;
    // p' = R v
    gx[0] = 0.f;
    gx[1] = 0.f;
    gx[2] = 0.f;
    gx[6] = R00 * ap0 + R10 * ap1 + R20 * ap2;
    gx[7] = R01 * ap0 + R11 * ap1 + R21 * ap2;
    gx[8] = R02 * ap0 + R12 * ap1 + R22 * ap2;
    float gphi = ap0 * (F01 * v1 + F02 * v2) + ap1 * (F11 * v1 + F12 * v2) + ap2 * (F21 * v1 + F22 * v2);
    float gth = ap0 * (T00 * v0 + T01 * v1 + T02 * v2) + ap1 * (T10 * v0 + T11 * v1 + T12 * v2) +
                ap2 * (T20 * v0 + T21 * v1 + T22 * v2);
    const float gpsi = ap0 * (P00 * v0 + P01 * v1 + P02 * v2) + ap1 * (P10 * v0 + P11 * v1 + P12 * v2);
    // eta' = W omega, W = [[1, sf tt, cf tt], [0, cf, -sf], [0, sf/ct, cf/ct]]
    gx[9] = ae0;
    gx[10] = ae0 * sf * tt + ae1 * cf + ae2 * sf * ic;
    gx[11] = ae0 * cf * tt - ae1 * sf + ae2 * cf * ic;
    gphi += ae0 * (cf * tt * w1 - sf * tt * w2) + ae1 * (-sf * w1 - cf * w2) + ae2 * (cf * ic * w1 - sf * ic * w2);
    gth += ae0 * (sf * ic2 * w1 + cf * ic2 * w2) + ae2 * (sf * st * ic2 * w1 + cf * st * ic2 * w2);
    // v' = v x omega - g (third row of R) + T/m e3
    gx[6] += w1 * av2 - w2 * av1;
    gx[7] += w2 * av0 - w0 * av2;
    gx[8] += w0 * av1 - w1 * av0;
    gx[9] += av1 * v2 - av2 * v1;
    gx[10] += av2 * v0 - av0 * v2;
    gx[11] += av0 * v1 - av1 * v0;
    gphi += -g * (av1 * F21 + av2 * F22);
    gth += -g * (av0 * T20 + av1 * T21 + av2 * T22);
    gu[0] = av2 / mass;
    // omega' = I^-1 (tau - omega x I omega)
    gu[1] = aw0 / Ixx;
    gu[2] = aw1 / Iyy;
    gu[3] = aw2 / Izz;
    gx[9] += -(Ixx - Izz) * w2 * aw1 / Iyy - (Iyy - Ixx) * w1 * aw2 / Izz;
    gx[10] += -(Izz - Iyy) * w2 * aw0 / Ixx - (Iyy - Ixx) * w0 * aw2 / Izz;
    gx[11] += -(Izz - Iyy) * w1 * aw0 / Ixx - (Ixx - Izz) * w0 * aw1 / Iyy;
    gx[3] = gphi;
    gx[4] = gth;
    gx[5] = gpsi;
}

template <>
__device__ __forceinline__ void vjp<DUBINS3D>(const float *x, const float *, const float *a, float *gx, float *gu,
                                              const DevProblem &)
{
    float sy, cy, sp, cp;
    sincosf(x[3], &sy, &cy);
    sincosf(x[4], &sp, &cp);
    const float v = x[5];
    gx[0] = 0.f;
    gx[1] = 0.f;
    gx[2] = 0.f;
    gx[3] = a[0] * (-v * cp * sy) + a[1] * (v * cp * cy);
    gx[4] = a[0] * (-v * sp * cy) + a[1] * (-v * sp * sy) + a[2] * (v * cp);
    gx[5] = a[0] * cp * cy + a[1] * cp * sy + a[2] * sp;
    gu[0] = a[3];
    gu[1] = a[4];
    gu[2] = a[5];
}

template <>
__device__ __forceinline__ void vjp<UNICYCLE1>(const float *x, const float *u, const float *a, float *gx, float *gu,
                                               const DevProblem &)
{
    float s, c;
    sincosf(x[2], &s, &c);
    gx[0] = 0.f;
    gx[1] = 0.f;
    gx[2] = a[0] * (-u[0] * s) + a[1] * (u[0] * c);
    gu[0] = a[0] * c + a[1] * s;
    gu[1] = a[2];
}

template <>
__device__ __forceinline__ void vjp<UNICYCLE2>(const float *x, const float *, const float *a, float *gx, float *gu,
                                               const DevProblem &)
{
    float s, c;
    sincosf(x[2], &s, &c);
    gx[0] = 0.f;
    gx[1] = 0.f;
    gx[2] = a[0] * (-x[3] * s) + a[1] * (x[3] * c);
    gx[3] = a[0] * c + a[1] * s;
    gx[4] = a[2];
    gu[0] = a[3];
    gu[1] = a[4];
}

// ---------------------------------------------------------------------------
// Obstacle penalty over the warp: sum_obstacles softplus_beta(margin - sdf(p))
// and its gradient in p; every lane returns the totals.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float softplus_beta(float z, float beta)
{
    const float bz = beta * z;
    return (fmaxf(bz, 0.f) + log1pf(expf(-fabsf(bz)))) / beta;
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.f / (1.f + expf(-z)); }

template <int PD>
__device__ __forceinline__ float warp_penalty(const float *p, const DevProblem &P, const TrajWeights &w, float *grad)
{
    const int lane = threadIdx.x & 31;
    float total = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    for (int b = lane; b < P.n_boxes; b += 32) {
        const float4 lo = P.boxes[2 * b], hi = P.boxes[2 * b + 1];
        const float los[3] = {lo.x, lo.y, lo.z}, his[3] = {hi.x, hi.y, hi.z};
        float q[3], sg[3], out2 = 0.f, qmax = -INFINITY;
        int amax = 0;
#pragma unroll
        for (int a = 0; a < PD; ++a) {
            const float ql = los[a] - p[a], qh = p[a] - his[a];
            q[a] = fmaxf(ql, qh);
            sg[a] = ql > qh ? -1.f : 1.f;
            if (q[a] > 0.f)
                out2 += q[a] * q[a];
            if (q[a] > qmax) {
                qmax = q[a];
                amax = a;
            }
        }
        float sdf, gs[3] = {0.f, 0.f, 0.f};
        if (out2 > 0.f) {
            sdf = sqrtf(out2);
#pragma unroll
            for (int a = 0; a < PD; ++a)
                gs[a] = q[a] > 0.f ? sg[a] * q[a] / sdf : 0.f;
        } else {
            sdf = qmax;
#pragma unroll
            for (int a = 0; a < PD; ++a)
                gs[a] = a == amax ? sg[a] : 0.f;
        }
        const float z = w.margin - sdf;
        total += softplus_beta(z, w.beta);
        const float s = sigmoidf(w.beta * z);
        g0 -= s * gs[0];
        g1 -= s * gs[1];
        if (PD > 2)
            g2 -= s * gs[2];
    }
    for (int sidx = lane; sidx < P.n_spheres; sidx += 32) {
        const float4 c = P.spheres[sidx];
        const float d0 = p[0] - c.x, d1 = p[1] - c.y, d2 = PD > 2 ? p[2] - c.z : 0.f;
        const float dist = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        const float z = w.margin - (dist - c.w);
        total += softplus_beta(z, w.beta);
        const float s = dist > 0.f ? sigmoidf(w.beta * z) / dist : 0.f;
        g0 -= s * d0;
        g1 -= s * d1;
        g2 -= s * d2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        total += __shfl_xor_sync(0xFFFFFFFFu, total, o);
        g0 += __shfl_xor_sync(0xFFFFFFFFu, g0, o);
        g1 += __shfl_xor_sync(0xFFFFFFFFu, g1, o);
        g2 += __shfl_xor_sync(0xFFFFFFFFu, g2, o);
    }
    grad[0] = g0;
    grad[1] = g1;
    if (PD > 2)
        grad[2] = g2;
    return total;
}

// ---------------------------------------------------------------------------
// Kernels.
// ---------------------------------------------------------------------------
template <int DYN>
__global__ void __launch_bounds__(32 * kTrajWarpsPerBlock)
    k_traj_cost(DevProblem P, TrajWeights w, const float *__restrict__ x0, const float *__restrict__ U, int n_traj,
                int N, float *__restrict__ cost, float *__restrict__ x_final)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= n_traj)
        return;
    const int lane = threadIdx.x & 31;
    float x[D], u[M], gp[3];
#pragma unroll
    for (int a = 0; a < D; ++a)
        x[a] = x0[(size_t)t * D + a];
    const float h = P.dt;
    float J = w.w_dur * (float)N * h;
    for (int n = 0; n < N; ++n) {
        float uu = 0.f;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            u[j] = U[((size_t)t * N + n) * M + j];
            uu += u[j] * u[j];
        }
        J += w.w_u * uu * h;
        float xp[PD];
#pragma unroll
        for (int a = 0; a < PD; ++a)
            xp[a] = x[a];
        rk4_step<DYN>(x, u, h, P);
        float dd = 0.f;
#pragma unroll
        for (int a = 0; a < PD; ++a)
            dd += (x[a] - xp[a]) * (x[a] - xp[a]);
        J += w.w_len * sqrtf(dd + w.len_eps * w.len_eps);
        if (w.w_obs != 0.f)
            J += w.w_obs * warp_penalty<PD>(x, P, w, gp) * h;
    }
    float e2 = 0.f;
#pragma unroll
    for (int a = 0; a < PD; ++a)
        e2 += (x[a] - w.goal[a]) * (x[a] - w.goal[a]);
    J += w.w_goal * e2;
    if (lane == 0) {
        cost[t] = J;
        if (x_final) {
#pragma unroll
            for (int a = 0; a < D; ++a)
                x_final[(size_t)t * D + a] = x[a];
        }
    }
}

// Pull the adjoint lam of x' = RK4(x, u) back to x (xb) and u (ub, added).
template <int DYN>
__device__ __forceinline__ void rk4_vjp(const float *x, const float *u, float h, const DevProblem &P,
                                        const float *lam, float *xb, float *ub)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M;
    float k[D], y2[D], y3[D], y4[D];
    const float hh = 0.5f * h;
    deriv<DYN>(x, u, k, P);
#pragma unroll
    for (int a = 0; a < D; ++a)
        y2[a] = __fmaf_rn(hh, k[a], x[a]);
    deriv<DYN>(y2, u, k, P);
#pragma unroll
    for (int a = 0; a < D; ++a)
        y3[a] = __fmaf_rn(hh, k[a], x[a]);
    deriv<DYN>(y3, u, k, P);
#pragma unroll
    for (int a = 0; a < D; ++a)
        y4[a] = __fmaf_rn(h, k[a], x[a]);
    float a1[D], a2[D], a3[D], a4[D], gx[D], gu[M];
    const float h6 = h / 6.f, h3 = h / 3.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        xb[a] = lam[a];
        a1[a] = h6 * lam[a];
        a2[a] = h3 * lam[a];
        a3[a] = h3 * lam[a];
        a4[a] = h6 * lam[a];
    }
    vjp<DYN>(y4, u, a4, gx, gu, P);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        xb[a] += gx[a];
        a3[a] = __fmaf_rn(h, gx[a], a3[a]);
    }
#pragma unroll
    for (int j = 0; j < M; ++j)
        ub[j] += gu[j];
    vjp<DYN>(y3, u, a3, gx, gu, P);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        xb[a] += gx[a];
        a2[a] = __fmaf_rn(hh, gx[a], a2[a]);
    }
#pragma unroll
    for (int j = 0; j < M; ++j)
        ub[j] += gu[j];
    vjp<DYN>(y2, u, a2, gx, gu, P);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        xb[a] += gx[a];
        a1[a] = __fmaf_rn(hh, gx[a], a1[a]);
    }
#pragma unroll
    for (int j = 0; j < M; ++j)
        ub[j] += gu[j];
    vjp<DYN>(x, u, a1, gx, gu, P);
#pragma unroll
    for (int a = 0; a < D; ++a)
        xb[a] += gx[a];
#pragma unroll
    for (int j = 0; j < M; ++j)
        ub[j] += gu[j];
}

// Gradient of one trajectory's cost by one warp: a forward sweep keeps x every kCkpt steps in
// ck ((N / kCkpt + 1) rows of D), then each segment is recomputed from its checkpoint and the
// adjoint is pulled back through it.  u_at(n, j) is control j of step n; lane 0 calls
// grad_out(n, ub) with dJ/du_n, from the last step to the first; lam receives dJ/dx0.
template <int DYN, class UAt, class GradOut>
__device__ __forceinline__ void traj_adjoint_warp(const DevProblem &P, const TrajWeights &w, const float *x0, int N,
                                                  float *ck, UAt u_at, GradOut grad_out, float *lam)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    const int lane = threadIdx.x & 31;
    const float h = P.dt;
    const int nseg = (N + kCkpt - 1) / kCkpt;
    float x[D], u[M], gp[3];
#pragma unroll
    for (int a = 0; a < D; ++a)
        x[a] = x0[a];
    // forward sweep: checkpoints at n = 0, 16, 32, ...
    for (int n = 0; n < N; ++n) {
        if (n % kCkpt == 0 && lane == 0) {
#pragma unroll
            for (int a = 0; a < D; ++a)
                ck[(size_t)(n / kCkpt) * D + a] = x[a];
        }
#pragma unroll
        for (int j = 0; j < M; ++j)
            u[j] = u_at(n, j);
        rk4_step<DYN>(x, u, h, P);
    }
    __syncwarp();
    // adjoint of x_N: goal error and the obstacle penalty at x_N
#pragma unroll
    for (int a = 0; a < D; ++a)
        lam[a] = 0.f;
#pragma unroll
    for (int a = 0; a < PD; ++a)
        lam[a] = 2.f * w.w_goal * (x[a] - w.goal[a]);
    // (a zero obstacle weight skips the penalty's sum over every obstacle)
    if (w.w_obs != 0.f) {
        warp_penalty<PD>(x, P, w, gp);
#pragma unroll
        for (int a = 0; a < PD; ++a)
            lam[a] += w.w_obs * gp[a] * h;
    }
    float xs[kCkpt + 1][D];
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int s = seg * kCkpt;
        const int L = min(kCkpt, N - s);
#pragma unroll
        for (int a = 0; a < D; ++a)
            xs[0][a] = ck[(size_t)seg * D + a];
        for (int i = 0; i < L; ++i) {
#pragma unroll
            for (int j = 0; j < M; ++j)
                u[j] = u_at(s + i, j);
#pragma unroll
            for (int a = 0; a < D; ++a)
                xs[i + 1][a] = xs[i][a];
            rk4_step<DYN>(xs[i + 1], u, h, P);
        }
        for (int i = L - 1; i >= 0; --i) {
            const int n = s + i;
            float uu[M], ub[M], xb[D];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                uu[j] = u_at(n, j);
                ub[j] = 2.f * w.w_u * uu[j] * h;
            }
            // path-length segment n -> n+1
            float dd = 0.f, dl[PD];
#pragma unroll
            for (int a = 0; a < PD; ++a) {
                dl[a] = xs[i + 1][a] - xs[i][a];
                dd += dl[a] * dl[a];
            }
            const float Ls = sqrtf(dd + w.len_eps * w.len_eps);
#pragma unroll
            for (int a = 0; a < PD; ++a)
                lam[a] += w.w_len * dl[a] / Ls;
            rk4_vjp<DYN>(xs[i], uu, h, P, lam, xb, ub);
            if (lane == 0)
                grad_out(n, ub);
#pragma unroll
            for (int a = 0; a < D; ++a)
                lam[a] = xb[a];
#pragma unroll
            for (int a = 0; a < PD; ++a)
                lam[a] -= w.w_len * dl[a] / Ls;
            if (n >= 1 && w.w_obs != 0.f) {
                warp_penalty<PD>(xs[i], P, w, gp);
#pragma unroll
                for (int a = 0; a < PD; ++a)
                    lam[a] += w.w_obs * gp[a] * h;
            }
        }
    }
}

// Gradient of the cost of each trajectory (one warp each), per-step controls U[(t N + n) M + j].
template <int DYN>
__global__ void __launch_bounds__(32 * kTrajWarpsPerBlock)
    k_traj_grad(DevProblem P, TrajWeights w, const float *__restrict__ x0, const float *__restrict__ U, int n_traj,
                int N, const float *__restrict__ cost_grad, float *__restrict__ dU, float *__restrict__ dx0,
                float *__restrict__ ckpt)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M;
    const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= n_traj)
        return;
    const int lane = threadIdx.x & 31;
    const int nseg = (N + kCkpt - 1) / kCkpt;
    const float scale = cost_grad ? cost_grad[t] : 1.f;
    const float *Ut = U + (size_t)t * N * M;
    float *dUt = dU + (size_t)t * N * M;
    float lam[D];
    traj_adjoint_warp<DYN>(
        P, w, x0 + (size_t)t * D, N, ckpt + (size_t)t * (nseg + 1) * D,
        [&](int n, int j) { return Ut[(size_t)n * M + j]; },
        [&](int n, const float *ub) {
#pragma unroll
            for (int j = 0; j < M; ++j)
                dUt[(size_t)n * M + j] = scale * ub[j];
        },
        lam);
    if (lane == 0 && dx0) {
#pragma unroll
        for (int a = 0; a < D; ++a)
            dx0[(size_t)t * D + a] = scale * lam[a];
    }
}

// The planner's own rules on one control sequence, by one warp: validity after every step (in
// the state box, no obstacle), the path length of the substep polyline, the final state in x.
template <int DYN, class UAt>
__device__ __forceinline__ bool traj_check_warp(const DevProblem &P, const float *x0, int N, UAt u_at, float *x,
                                                float &len)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    const int lane = threadIdx.x & 31;
    float u[M];
#pragma unroll
    for (int a = 0; a < D; ++a)
        x[a] = x0[a];
    bool ok = true;
    len = 0.f;
    for (int n = 0; n < N; ++n) {
#pragma unroll
        for (int j = 0; j < M; ++j)
            u[j] = u_at(n, j);
        float xp[PD];
#pragma unroll
        for (int a = 0; a < PD; ++a)
            xp[a] = x[a];
        rk4_step<DYN>(x, u, P.dt, P);
        len += sqrtf(sq_dist<PD>(x, xp));  // the planner's path-length increment, rounded the same way
        bool inb = true;
#pragma unroll
        for (int a = 0; a < D; ++a)
            inb = inb && (x[a] >= P.x_lo[a]) && (x[a] <= P.x_hi[a]);
        const bool hit = inb && hits_obstacle<PD>(x, P, P.boxes, P.n_boxes, P.spheres, P.n_spheres, P.grid_start,
                                                  P.grid_items, lane, 32);
        if (!inb || __any_sync(0xFFFFFFFFu, hit))
            ok = false;
    }
    return ok;
}

// The same rules on one control sequence by one thread (the obstacle tests of a step in turn),
// for checking one candidate per lane.
template <int DYN, class UAt>
__device__ __forceinline__ bool traj_check_thread(const DevProblem &P, const float *x0, int N, UAt u_at, float *x,
                                                  float &len)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    float u[M];
#pragma unroll
    for (int a = 0; a < D; ++a)
        x[a] = x0[a];
    bool ok = true;
    len = 0.f;
    for (int n = 0; n < N && ok; ++n) {
#pragma unroll
        for (int j = 0; j < M; ++j)
            u[j] = u_at(n, j);
        float xp[PD];
#pragma unroll
        for (int a = 0; a < PD; ++a)
            xp[a] = x[a];
        rk4_step<DYN>(x, u, P.dt, P);
        len += sqrtf(sq_dist<PD>(x, xp));
        bool inb = true;
#pragma unroll
        for (int a = 0; a < D; ++a)
            inb = inb && (x[a] >= P.x_lo[a]) && (x[a] <= P.x_hi[a]);
        ok = inb && !hits_obstacle<PD>(x, P, P.boxes, P.n_boxes, P.spheres, P.n_spheres, P.grid_start, P.grid_items,
                                       0, 1);
    }
    return ok;
}

template <int DYN>
__global__ void __launch_bounds__(32 * kTrajWarpsPerBlock)
    k_traj_check(DevProblem P, TrajWeights w, const float *__restrict__ x0, const float *__restrict__ U, int n_traj,
                 int N, int *__restrict__ valid, int *__restrict__ in_goal_out, float *__restrict__ length,
                 float *__restrict__ x_final)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= n_traj)
        return;
    const int lane = threadIdx.x & 31;
    const float *Ut = U + (size_t)t * N * M;
    float x[D], len;
    const bool ok =
        traj_check_warp<DYN>(P, x0 + (size_t)t * D, N, [&](int n, int j) { return Ut[(size_t)n * M + j]; }, x, len);
    if (lane == 0) {
        valid[t] = ok ? 1 : 0;
        if (in_goal_out)
            in_goal_out[t] = in_goal<PD>(x, P, w.goal) ? 1 : 0;
        if (length)
            length[t] = len;
        if (x_final) {
#pragma unroll
            for (int a = 0; a < D; ++a)
                x_final[(size_t)t * D + a] = x[a];
        }
    }
}

// One refinement of one path, all of it on the device (one CTA of kRefineWarps warps): the
// per-edge controls Ue (E x M, updated in place) with per-edge step counts steps[E] (summing to
// N).  Each of `iters` iterations: warp 0 takes dJ/dUe (the adjoint sweep, per-step gradients
// summed over each edge's steps) and normalises it to d; the warps check the n_cand candidates
// clamp(Ue - step 2^-c d, u_lo, u_hi) under the planner's rules (valid after every step, the end
// in the goal ball and within sqrt(r_in2) of the goal); the shortest accepted candidate (the
// lowest c on a tie) replaces Ue if it is shorter than the current path.  Candidate c is
// checked by thread c (kRefineMaxCand <= 32 * kRefineWarps).  out[0] receives the
// starting length (+inf if the start is not accepted), out[1] the final one; both NaN if the
// step counts do not sum to N.  Scratch: edge_of[N] (int), ck ((N / kCkpt + 1) x D), gE (E x M).
template <int DYN>
__global__ void __launch_bounds__(32 * kRefineWarps)
    k_traj_refine(DevProblem P, TrajWeights w, const float *__restrict__ x0, float *__restrict__ Ue,
                  const int *__restrict__ steps, int E, int N, int iters, int n_cand, float step, float r_in2,
                  int *__restrict__ edge_of, float *__restrict__ ck, float *__restrict__ gE, float *__restrict__ out)
{
    constexpr int D = Dims<DYN>::D, M = Dims<DYN>::M, PD = Dims<DYN>::PD;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ float s_res[kRefineMaxCand];
    __shared__ float s_cur;
    __shared__ int s_ok, s_acc;
    if (tid == 0) {
        int n = 0;
        bool ok = true;
        for (int e = 0; e < E && ok; ++e) {
            const int se = steps[e];
            if (se < 0 || se > N - n) {
                ok = false;
                break;
            }
            for (int k = 0; k < se; ++k)
                edge_of[n++] = e;
        }
        s_ok = ok && n == N;
    }
    __syncthreads();
    if (!s_ok) {
        if (tid == 0)
            out[0] = out[1] = __int_as_float(0x7fc00000);
        return;
    }
    float x0r[D];
#pragma unroll
    for (int a = 0; a < D; ++a)
        x0r[a] = x0[a];
    // the end rule: valid, in the goal ball, and inside it by the caller's margin; one candidate
    // per thread
    auto accepted_length = [&](float alpha) {
        float x[D], len;
        const bool ok = traj_check_thread<DYN>(
            P, x0r, N,
            [&](int n, int j) {
                const int e = edge_of[n];
                const float v = Ue[e * M + j];
                return alpha > 0.f ? fminf(fmaxf(v - alpha * gE[e * M + j], P.u_lo[j]), P.u_hi[j]) : v;
            },
            x, len);
        return (ok && in_goal<PD>(x, P, w.goal) && sq_dist<PD>(x, w.goal) <= r_in2) ? len
                                                                                   : __int_as_float(0x7f800000);
    };
    if (tid == 0) {
        const float L0 = accepted_length(0.f);
        s_cur = L0;
        out[0] = L0;
    }
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        if (warp == 0) {
            for (int k = lane; k < E * M; k += 32)
                gE[k] = 0.f;
            __syncwarp();
            float lam[D];
            traj_adjoint_warp<DYN>(
                P, w, x0r, N, ck, [&](int n, int j) { return Ue[edge_of[n] * M + j]; },
                [&](int n, const float *ub) {
                    const int e = edge_of[n];
#pragma unroll
                    for (int j = 0; j < M; ++j)
                        gE[e * M + j] += ub[j];
                },
                lam);
            __syncwarp();
            float g2 = 0.f;
            for (int k = lane; k < E * M; k += 32)
                g2 = fmaf(gE[k], gE[k], g2);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                g2 += __shfl_xor_sync(0xFFFFFFFFu, g2, o);
            const float inv = 1.f / (sqrtf(g2) + 1e-12f);
            for (int k = lane; k < E * M; k += 32)
                gE[k] *= inv;
        }
        __syncthreads();
        if (tid < n_cand)
            s_res[tid] = accepted_length(ldexpf(step, -tid));
        __syncthreads();
        if (tid == 0) {
            int best = 0;
            for (int c = 1; c < n_cand; ++c)
                if (s_res[c] < s_res[best])
                    best = c;
            s_acc = s_res[best] < s_cur ? best : -1;
            if (s_acc >= 0)
                s_cur = s_res[best];
        }
        __syncthreads();
        if (s_acc >= 0) {
            const float alpha = ldexpf(step, -s_acc);
            for (int k = tid; k < E * M; k += 32 * kRefineWarps)
                Ue[k] = fminf(fmaxf(Ue[k] - alpha * gE[k], P.u_lo[k % M]), P.u_hi[k % M]);
        }
        __syncthreads();
    }
    if (tid == 0)
        out[1] = s_cur;
}

#define PAKR_TRAJ_DISPATCH(dyn, BODY)                                                                                  \
    switch (dyn) {                                                                                                     \
    case DI2: { constexpr int DYN_ = DI2; BODY; } break;                                                               \
    case DI3: { constexpr int DYN_ = DI3; BODY; } break;                                                               \
    case QUAD12: { constexpr int DYN_ = QUAD12; BODY; } break;                                                         \
    case DUBINS3D: { constexpr int DYN_ = DUBINS3D; BODY; } break;                                                     \
    case UNICYCLE1: { constexpr int DYN_ = UNICYCLE1; BODY; } break;                                                   \
    case UNICYCLE2: { constexpr int DYN_ = UNICYCLE2; BODY; } break;                                                   \
    default: return cudaErrorInvalidValue;                                                                             \
    }

pakr_status tfail(pakr_status st, const char *msg)
{
    record_error(msg);
    return st;
}

pakr_status make_weights(const pakr_planner *p, const pakr_traj_params *params, const float *x_goal, TrajWeights *w)
{
    if (!params || !x_goal)
        return tfail(PAKR_ERR_INVALID_ARG, "params / x_goal missing");
    const DevProblem &P = *planner_problem(p);
    w->w_dur = params->w_duration;
    w->w_u = params->w_control;
    w->w_obs = params->w_obstacle;
    w->beta = params->beta;
    w->margin = params->margin;
    w->w_goal = params->w_goal;
    w->w_len = params->w_length;
    w->len_eps = params->length_eps;
    if (!(w->beta > 0.f) || !std::isfinite(w->beta))
        return tfail(PAKR_ERR_INVALID_ARG, "beta must be finite and > 0");
    for (int a = 0; a < kMaxD; ++a)
        w->goal[a] = a < P.d ? x_goal[a] : 0.f;
    return PAKR_OK;
}

struct TrajGuard {
    int prev = -1;
    explicit TrajGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~TrajGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace pakr

using namespace pakr;

extern "C" {

pakr_status pakr_traj_cost(pakr_planner *planner, const float *x0, const float *controls, int32_t n_traj,
                           int32_t n_steps, const float *x_goal, const pakr_traj_params *params, float *cost,
                           float *x_final)
{
    if (!planner || !x0 || !controls || !cost || n_traj < 0 || n_steps < 0)
        return tfail(PAKR_ERR_INVALID_ARG, "pakr_traj_cost: bad argument");
    if (n_traj == 0)
        return PAKR_OK;
    TrajWeights w;
    pakr_status st = make_weights(planner, params, x_goal, &w);
    if (st != PAKR_OK)
        return st;
    TrajGuard guard(planner_device(planner));
    const DevProblem &P = *planner_problem(planner);
    const int threads = 32 * kTrajWarpsPerBlock;
    const int blocks = (n_traj + kTrajWarpsPerBlock - 1) / kTrajWarpsPerBlock;
    cudaStream_t s = planner_stream(planner);
    cudaError_t e = cudaSuccess;
    [&]() -> cudaError_t {
        PAKR_TRAJ_DISPATCH(P.dyn, (k_traj_cost<DYN_><<<blocks, threads, 0, s>>>(P, w, x0, controls, n_traj, n_steps,
                                                                                cost, x_final)));
        return cudaSuccess;
    }();
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return tfail(PAKR_ERR_CUDA, cudaGetErrorString(e));
    return PAKR_OK;
}

pakr_status pakr_traj_grad(pakr_planner *planner, const float *x0, const float *controls, int32_t n_traj,
                           int32_t n_steps, const float *x_goal, const pakr_traj_params *params,
                           const float *cost_grad, float *controls_grad, float *x0_grad, float *checkpoints)
{
    if (!planner || !x0 || !controls || !controls_grad || !checkpoints || n_traj < 0 || n_steps < 0)
        return tfail(PAKR_ERR_INVALID_ARG, "pakr_traj_grad: bad argument");
    if (n_traj == 0)
        return PAKR_OK;
    TrajWeights w;
    pakr_status st = make_weights(planner, params, x_goal, &w);
    if (st != PAKR_OK)
        return st;
    TrajGuard guard(planner_device(planner));
    const DevProblem &P = *planner_problem(planner);
    const int threads = 32 * kTrajWarpsPerBlock;
    const int blocks = (n_traj + kTrajWarpsPerBlock - 1) / kTrajWarpsPerBlock;
    cudaStream_t s = planner_stream(planner);
    [&]() -> cudaError_t {
        PAKR_TRAJ_DISPATCH(P.dyn, (k_traj_grad<DYN_><<<blocks, threads, 0, s>>>(
                                      P, w, x0, controls, n_traj, n_steps, cost_grad, controls_grad, x0_grad,
                                      checkpoints)));
        return cudaSuccess;
    }();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return tfail(PAKR_ERR_CUDA, cudaGetErrorString(e));
    return PAKR_OK;
}

int64_t pakr_traj_checkpoint_floats(const pakr_planner *planner, int32_t n_traj, int32_t n_steps)
{
    if (!planner || n_traj < 0 || n_steps < 0)
        return -1;
    const int nseg = (n_steps + kCkpt - 1) / kCkpt;
    return (int64_t)n_traj * (nseg + 1) * planner_problem(planner)->d;
}

pakr_status pakr_traj_check(pakr_planner *planner, const float *x0, const float *controls, int32_t n_traj,
                            int32_t n_steps, const float *x_goal, int32_t *valid, int32_t *in_goal,
                            float *path_length, float *x_final)
{
    if (!planner || !x0 || !controls || !valid || !x_goal || n_traj < 0 || n_steps < 0)
        return tfail(PAKR_ERR_INVALID_ARG, "pakr_traj_check: bad argument");
    if (n_traj == 0)
        return PAKR_OK;
    pakr_traj_params dummy{0, 0, 0, 1, 0, 0, 0, 0};
    TrajWeights w;
    pakr_status st = make_weights(planner, &dummy, x_goal, &w);
    if (st != PAKR_OK)
        return st;
    TrajGuard guard(planner_device(planner));
    const DevProblem &P = *planner_problem(planner);
    const int threads = 32 * kTrajWarpsPerBlock;
    const int blocks = (n_traj + kTrajWarpsPerBlock - 1) / kTrajWarpsPerBlock;
    cudaStream_t s = planner_stream(planner);
    [&]() -> cudaError_t {
        PAKR_TRAJ_DISPATCH(P.dyn, (k_traj_check<DYN_><<<blocks, threads, 0, s>>>(
                                      P, w, x0, controls, n_traj, n_steps, valid, in_goal, path_length, x_final)));
        return cudaSuccess;
    }();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return tfail(PAKR_ERR_CUDA, cudaGetErrorString(e));
    return PAKR_OK;
}

int64_t pakr_traj_refine_scratch_floats(const pakr_planner *planner, int32_t n_edges, int32_t n_steps)
{
    if (!planner || n_edges < 1 || n_steps < 0)
        return -1;
    const DevProblem &P = *planner_problem(planner);
    const int nseg = (n_steps + kCkpt - 1) / kCkpt;
    return (int64_t)n_steps + (int64_t)(nseg + 1) * P.d + (int64_t)n_edges * P.m;
}

pakr_status pakr_traj_refine(pakr_planner *planner, const float *x0, float *edge_controls, const int32_t *steps,
                             int32_t n_edges, int32_t n_steps, const float *x_goal, const pakr_traj_params *params,
                             int32_t iters, int32_t n_candidates, float step, float goal_margin, float *scratch,
                             float *lengths)
{
    if (!planner || !x0 || !edge_controls || !steps || !scratch || !lengths || n_edges < 1 || n_steps < 0 ||
        iters < 0 || n_candidates < 1 || n_candidates > kRefineMaxCand || !(step > 0.f) || !std::isfinite(step) ||
        !(goal_margin >= 0.f && goal_margin < 1.f))
        return tfail(PAKR_ERR_INVALID_ARG, "pakr_traj_refine: bad argument");
    TrajWeights w;
    pakr_status st = make_weights(planner, params, x_goal, &w);
    if (st != PAKR_OK)
        return st;
    TrajGuard guard(planner_device(planner));
    const DevProblem &P = *planner_problem(planner);
    const float r_in = P.goal_r * (1.f - goal_margin);
    const int nseg = (n_steps + kCkpt - 1) / kCkpt;
    int *edge_of = reinterpret_cast<int *>(scratch);
    float *ck = scratch + n_steps;
    float *gE = ck + (size_t)(nseg + 1) * P.d;
    cudaStream_t s = planner_stream(planner);
    [&]() -> cudaError_t {
        PAKR_TRAJ_DISPATCH(P.dyn, (k_traj_refine<DYN_><<<1, 32 * kRefineWarps, 0, s>>>(
                                      P, w, x0, edge_controls, steps, n_edges, n_steps, iters, n_candidates, step,
                                      r_in * r_in, edge_of, ck, gE, lengths)));
        return cudaSuccess;
    }();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return tfail(PAKR_ERR_CUDA, cudaGetErrorString(e));
    return PAKR_OK;
}

}  // extern "C"
