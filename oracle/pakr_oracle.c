/*
 * pakr_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain FP64, single-threaded restatement of the PAKR expansion iteration
 * (Algorithm 1, Sec. IV, Sec. IV-A) and of the AO-x outer loop.  Every step
 * is written as its definition, in the algorithm's order, with no blocking,
 * fusion or reordering.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this code.
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vectors, the closed-form
 * double-integrator solution, rigid-body invariants of the quadrotor,
 * brute-force nearest neighbours against a k-d tree library routine, tree
 * invariants and the AO-x monotone bound.  The quadrotor equations are not
 * printed in the paper: parity of that model against the paper is unpinned.
 */
#include "pakr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from its published definition (Salmon et al., SC'11):       */
/* ten rounds of two 32x32->64 multiplies with a Weyl-sequence key schedule.   */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Uniform in [0,1) from the top 24 bits of a word: exact in FP32 and FP64. */
double ora_u01(uint32_t w)
{
    return (double)(w >> 8) * (1.0 / 16777216.0);
}

static void seed_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
}

/* SampleStates (Algorithm 1): uniform over the state box; the paper states no
 * other distribution and no goal bias.  Counter = (iteration, i, 0xFFFFFFFF,
 * block); words 0..d-1 feed dimensions 0..d-1 in order. */
void ora_sample_state(const ora_problem *P, uint64_t seed, uint32_t iter, uint32_t i, double *x)
{
    uint32_t key[2];
    seed_key(seed, key);
    int nblocks = (P->d + 3) / 4;
    for (int b = 0; b < nblocks; ++b) {
        uint32_t ctr[4] = {iter, i, 0xFFFFFFFFu, (uint32_t)b};
        uint32_t w[4];
        ora_philox4x32_10(ctr, key, w);
        for (int t = 0; t < 4; ++t) {
            int dim = 4 * b + t;
            if (dim < P->d)
                x[dim] = P->x_lo[dim] + (P->x_hi[dim] - P->x_lo[dim]) * ora_u01(w[t]);
        }
    }
}

/* SampleControls (Algorithm 1): each of the A controls of parent i is uniform
 * over the control box (Sec. II-A, random propagation), and is held for a
 * duration drawn uniformly from {s_min..s_max} substeps.  Counter =
 * (iteration, i, j, block); words 0..m-1 are the control, word m the duration. */
void ora_sample_control(const ora_problem *P, uint64_t seed, uint32_t iter, uint32_t i, uint32_t j,
                        double *u, int *S)
{
    uint32_t key[2];
    seed_key(seed, key);
    uint32_t words[ORA_MAX_M + 4];
    int nwords = P->m + 1;
    int nblocks = (nwords + 3) / 4;
    for (int b = 0; b < nblocks; ++b) {
        uint32_t ctr[4] = {iter, i, j, (uint32_t)b};
        ora_philox4x32_10(ctr, key, &words[4 * b]);
    }
    for (int a = 0; a < P->m; ++a)
        u[a] = P->u_lo[a] + (P->u_hi[a] - P->u_lo[a]) * ora_u01(words[a]);
    uint64_t span = (uint64_t)(P->s_max - P->s_min + 1);
    *S = P->s_min + (int)(((uint64_t)words[P->m] * span) >> 32);
}

/* ------------------------------------------------------------------------- */
/* Dynamics x' = f(x, u) (Eq. 1).                                              */
/* ------------------------------------------------------------------------- */

/* Double integrator (Sec. V-A item 1, and its planar analogue): the first half
 * of the state is position, the second half velocity, the control is the
 * acceleration. */
static void f_double_integrator(int pdim, const double *x, const double *u, double *xd)
{
    for (int a = 0; a < pdim; ++a) {
        xd[a] = x[pdim + a];
        xd[pdim + a] = u[a];
    }
}

/* 12D quadcopter (Sec. V-A item 3): state [x,y,z, phi,theta,psi, u,v,w, p,q,r]
 * with body-frame linear and angular velocity, control [T, tau_x, tau_y,
 * tau_z].  The paper prints no equations; this is the textbook rigid body with
 * Z-Y-X Euler angles, z up, thrust along body z:
 *   p_world' = R v,  R = Rz(psi) Ry(theta) Rx(phi)
 *   [phi',theta',psi'] = W(phi,theta) omega
 *   v' = v x omega + R^T (0,0,-g) + (0,0,T/m)
 *   omega' = I^{-1} (tau - omega x I omega). */
static void f_quadrotor(const double *model, const double *x, const double *u, double *xd)
{
    double mass = model[0], Ixx = model[1], Iyy = model[2], Izz = model[3], g = model[4];
    double phi = x[3], th = x[4], psi = x[5];
    double vb[3] = {x[6], x[7], x[8]};
    double w[3] = {x[9], x[10], x[11]};
    double cf = cos(phi), sf = sin(phi), ct = cos(th), st = sin(th), cp = cos(psi), sp = sin(psi);
    double R[3][3] = {
        {cp * ct, cp * st * sf - sp * cf, cp * st * cf + sp * sf},
        {sp * ct, sp * st * sf + cp * cf, sp * st * cf - cp * sf},
        {-st, ct * sf, ct * cf},
    };
    for (int r = 0; r < 3; ++r)
        xd[r] = R[r][0] * vb[0] + R[r][1] * vb[1] + R[r][2] * vb[2];
    double tt = st / ct;
    xd[3] = w[0] + sf * tt * w[1] + cf * tt * w[2];
    xd[4] = cf * w[1] - sf * w[2];
    xd[5] = (sf * w[1] + cf * w[2]) / ct;
    /* v x omega */
    double vxw[3] = {vb[1] * w[2] - vb[2] * w[1], vb[2] * w[0] - vb[0] * w[2], vb[0] * w[1] - vb[1] * w[0]};
    /* R^T (0,0,-g) = -g * (third row of R) */
    double gb[3] = {-g * R[2][0], -g * R[2][1], -g * R[2][2]};
    xd[6] = vxw[0] + gb[0];
    xd[7] = vxw[1] + gb[1];
    xd[8] = vxw[2] + gb[2] + u[0] / mass;
    double Iw[3] = {Ixx * w[0], Iyy * w[1], Izz * w[2]};
    double wxIw[3] = {w[1] * Iw[2] - w[2] * Iw[1], w[2] * Iw[0] - w[0] * Iw[2], w[0] * Iw[1] - w[1] * Iw[0]};
    xd[9] = (u[1] - wxIw[0]) / Ixx;
    xd[10] = (u[2] - wxIw[1]) / Iyy;
    xd[11] = (u[3] - wxIw[2]) / Izz;
}

/* 6D Dubins airplane (Sec. V-A item 2): [x,y,z, yaw, pitch, speed], control
 * [yaw rate, pitch rate, acceleration]; equations not printed in the paper,
 * the standard kinematic model is used. */
static void f_dubins3d(const double *x, const double *u, double *xd)
{
    double yaw = x[3], pitch = x[4], v = x[5];
    xd[0] = v * cos(pitch) * cos(yaw);
    xd[1] = v * cos(pitch) * sin(yaw);
    xd[2] = v * sin(pitch);
    xd[3] = u[0];
    xd[4] = u[1];
    xd[5] = u[2];
}

/* Unicycles (Sec. V-C items 1-2): velocity-controlled [x,y,theta] / [v,omega]
 * and acceleration-controlled [x,y,theta,v,omega] / [a,alpha]. */
static void f_unicycle1(const double *x, const double *u, double *xd)
{
    xd[0] = u[0] * cos(x[2]);
    xd[1] = u[0] * sin(x[2]);
    xd[2] = u[1];
}

static void f_unicycle2(const double *x, const double *u, double *xd)
{
    xd[0] = x[3] * cos(x[2]);
    xd[1] = x[3] * sin(x[2]);
    xd[2] = x[4];
    xd[3] = u[0];
    xd[4] = u[1];
}

void ora_dynamics(const ora_problem *P, const double *x, const double *u, double *xd)
{
    switch (P->dyn) {
    case ORA_DI2:
    case ORA_DI3:
        f_double_integrator(P->pdim, x, u, xd);
        break;
    case ORA_QUAD12:
        f_quadrotor(P->model, x, u, xd);
        break;
    case ORA_DUBINS3D:
        f_dubins3d(x, u, xd);
        break;
    case ORA_UNICYCLE1:
        f_unicycle1(x, u, xd);
        break;
    case ORA_UNICYCLE2:
        f_unicycle2(x, u, xd);
        break;
    default:
        for (int a = 0; a < P->d; ++a)
            xd[a] = NAN;
    }
}

/* Classical fourth-order Runge-Kutta step with the control held (Sec. IV-A). */
void ora_rk4_step(const ora_problem *P, const double *x, const double *u, double h, double *out)
{
    int d = P->d;
    double k1[ORA_MAX_D], k2[ORA_MAX_D], k3[ORA_MAX_D], k4[ORA_MAX_D], tmp[ORA_MAX_D];
    ora_dynamics(P, x, u, k1);
    for (int a = 0; a < d; ++a)
        tmp[a] = x[a] + 0.5 * h * k1[a];
    ora_dynamics(P, tmp, u, k2);
    for (int a = 0; a < d; ++a)
        tmp[a] = x[a] + 0.5 * h * k2[a];
    ora_dynamics(P, tmp, u, k3);
    for (int a = 0; a < d; ++a)
        tmp[a] = x[a] + h * k3[a];
    ora_dynamics(P, tmp, u, k4);
    for (int a = 0; a < d; ++a)
        out[a] = x[a] + h / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
}

/* ------------------------------------------------------------------------- */
/* Validity, heuristic (Sec. III, Sec. IV).                                    */
/* ------------------------------------------------------------------------- */

/* A point robot is valid when every state coordinate lies in the closed state
 * box and its position lies in no closed box and no closed ball. */
int ora_state_valid(const ora_problem *P, const double *x)
{
    for (int a = 0; a < P->d; ++a) {
        if (!(x[a] >= P->x_lo[a] && x[a] <= P->x_hi[a]))
            return 0;
    }
    int pd = P->pdim;
    for (int b = 0; b < P->n_boxes; ++b) {
        const double *lo = P->boxes + (size_t)b * 2 * pd;
        const double *hi = lo + pd;
        int inside = 1;
        for (int a = 0; a < pd; ++a)
            if (!(x[a] >= lo[a] && x[a] <= hi[a]))
                inside = 0;
        if (inside)
            return 0;
    }
    for (int s = 0; s < P->n_spheres; ++s) {
        const double *c = P->spheres + (size_t)s * (pd + 1);
        double r = c[pd], dd = 0.0;
        for (int a = 0; a < pd; ++a)
            dd += (x[a] - c[a]) * (x[a] - c[a]);
        if (dd <= r * r)
            return 0;
    }
    return 1;
}

/* Smallest distance from the state to any face that decides validity (state
 * box faces, box surfaces, sphere surfaces).  Reporting only: tells the parity
 * checks when a validity decision is too close to call across precisions. */
double ora_face_margin(const ora_problem *P, const double *x)
{
    double m = INFINITY;
    for (int a = 0; a < P->d; ++a) {
        m = fmin(m, fabs(x[a] - P->x_lo[a]));
        m = fmin(m, fabs(x[a] - P->x_hi[a]));
    }
    int pd = P->pdim;
    for (int b = 0; b < P->n_boxes; ++b) {
        const double *lo = P->boxes + (size_t)b * 2 * pd;
        const double *hi = lo + pd;
        double out2 = 0.0, qmax = -INFINITY;
        for (int a = 0; a < pd; ++a) {
            double q = fmax(lo[a] - x[a], x[a] - hi[a]);
            if (q > 0)
                out2 += q * q;
            qmax = fmax(qmax, q);
        }
        double sdf = sqrt(out2) + fmin(qmax, 0.0);
        m = fmin(m, fabs(sdf));
    }
    for (int s = 0; s < P->n_spheres; ++s) {
        const double *c = P->spheres + (size_t)s * (pd + 1);
        double dd = 0.0;
        for (int a = 0; a < pd; ++a)
            dd += (x[a] - c[a]) * (x[a] - c[a]);
        m = fmin(m, fabs(sqrt(dd) - c[pd]));
    }
    return m;
}

static double pos_dist_to_goal(const ora_problem *P, const double *x)
{
    double dd = 0.0;
    for (int a = 0; a < P->pdim; ++a)
        dd += (x[a] - P->x_goal[a]) * (x[a] - P->x_goal[a]);
    return sqrt(dd);
}

/* h(n) of the f-cost f = g + h (Sec. IV).  The paper writes the Euclidean
 * distance of the state to the goal state; ORA_H_FULLSTATE is that formula
 * over all state coordinates.  ORA_H_POSITION (default) is the distance of
 * the position to the goal ball, which never overestimates a path-length
 * cost; with the duration cost it is divided by a speed bound. */
double ora_heuristic(const ora_problem *P, const double *x)
{
    if (P->heuristic == ORA_H_FULLSTATE) {
        double dd = 0.0;
        for (int a = 0; a < P->d; ++a)
            dd += (x[a] - P->x_goal[a]) * (x[a] - P->x_goal[a]);
        return sqrt(dd);
    }
    double h = fmax(0.0, pos_dist_to_goal(P, x) - P->goal_r);
    if (P->cost == ORA_COST_DURATION)
        return P->h_speed > 0.0 ? h / P->h_speed : 0.0;
    return h;
}

/* f = g + h of the first n nodes (the quantity the prune compares, Sec. IV). */
void ora_fcosts(const ora_problem *P, const ora_tree *T, int64_t n, double *f)
{
    for (int64_t j = 0; j < n; ++j)
        f[j] = T->costs[j] + ora_heuristic(P, T->states + (size_t)j * P->d);
}

/* ------------------------------------------------------------------------- */
/* NearestNeighbor (Algorithm 1) over the frozen tree prefix [0, n), among     */
/* nodes whose f-cost is below the bound; lowest index wins a tie.             */
/* ------------------------------------------------------------------------- */
static double weighted_dist(const ora_problem *P, const double *q, const double *x)
{
    double s = 0.0;
    for (int a = 0; a < P->d; ++a)
        s += P->nn_w[a] * (q[a] - x[a]) * (q[a] - x[a]);
    return sqrt(s);
}

void ora_nearest(const ora_problem *P, const ora_tree *T, int64_t n, const double *f, const double *q,
                 double bound, double tol, ora_nn_result *out)
{
    int64_t best = -1;
    double d1 = INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        if (!(f[j] < bound))
            continue;
        double dj = weighted_dist(P, q, T->states + (size_t)j * P->d);
        if (dj < d1) {
            d1 = dj;
            best = j;
        }
    }
    double d2 = INFINITY, dfrag = INFINITY;
    int best_fragile = 0;
    for (int64_t j = 0; j < n; ++j) {
        int eligible = f[j] < bound;
        int fragile = fabs(f[j] - bound) < tol;
        if (!eligible && !fragile)
            continue;
        double dj = weighted_dist(P, q, T->states + (size_t)j * P->d);
        if (eligible && j != best && dj < d2)
            d2 = dj;
        if (fragile) {
            if (j == best)
                best_fragile = 1;
            else if (!eligible && dj < dfrag)
                dfrag = dj;
        }
    }
    out->idx = best;
    out->d1 = d1;
    out->d2 = d2;
    out->fragile_elig = best_fragile || (dfrag <= d1 + 1e-6);
}

/* ------------------------------------------------------------------------- */
/* Propagate (Algorithm 1, Sec. IV-A): S classical RK4 steps of length dt with */
/* the control held; validity is checked after every step (the parent state is */
/* not re-checked).  Path-length cost accumulates the distance between         */
/* successive substep positions; duration cost is S*dt.                        */
/* ------------------------------------------------------------------------- */
void ora_propagate(const ora_problem *P, const double *x0, double g0, const double *u, int S, double bound,
                   ora_rollout *out)
{
    (void)bound;
    int d = P->d;
    double x[ORA_MAX_D], xn[ORA_MAX_D];
    memcpy(x, x0, sizeof(double) * (size_t)d);
    double g = g0;
    double margin = INFINITY;
    int first_invalid = 0;
    for (int s = 1; s <= S; ++s) {
        ora_rk4_step(P, x, u, P->dt, xn);
        if (P->cost == ORA_COST_PATH_LENGTH) {
            double dd = 0.0;
            for (int a = 0; a < P->pdim; ++a)
                dd += (xn[a] - x[a]) * (xn[a] - x[a]);
            g += sqrt(dd);
        }
        memcpy(x, xn, sizeof(double) * (size_t)d);
        if (first_invalid == 0) {
            margin = fmin(margin, ora_face_margin(P, x));
            if (!ora_state_valid(P, x))
                first_invalid = s;
        }
    }
    if (P->cost == ORA_COST_DURATION)
        g = g0 + (double)S * P->dt;
    memcpy(out->x_end, x, sizeof(double) * (size_t)d);
    out->cost_end = g;
    out->f_end = g + ora_heuristic(P, x);
    out->collided = first_invalid > 0;
    out->first_invalid = first_invalid;
    out->face_margin = margin;
    double dg = pos_dist_to_goal(P, x);
    out->in_goal = dg <= P->goal_r;
    out->goal_margin = fabs(dg - P->goal_r);
}

/* ------------------------------------------------------------------------- */
/* Tree (Sec. IV-A) and one expansion iteration (Algorithm 1 inner loop).      */
/* ------------------------------------------------------------------------- */
int ora_tree_reset(const ora_problem *P, ora_tree *T, const double *x_init)
{
    if (T->cap < 1)
        return ORA_ERR_INVALID_ARG;
    memcpy(T->states, x_init, sizeof(double) * (size_t)P->d);
    for (int a = 0; a < P->m; ++a)
        T->controls[a] = 0.0;
    T->parents[0] = -1;
    T->costs[0] = 0.0;
    T->steps[0] = 0;
    T->count = 1;
    T->iteration = 0;
    return ora_state_valid(P, x_init) ? ORA_OK : ORA_ERR_INVALID_ARG;
}

int ora_expand(const ora_problem *P, ora_tree *T, double bound, uint64_t seed, ora_expand_out *o)
{
    int d = P->d, m = P->m, K = P->K, k = P->k;
    int64_t R = (int64_t)K * k;
    int64_t n = T->count; /* the frozen snapshot every query of this batch sees (Sec. IV-B) */
    uint32_t it = T->iteration;
    if (n < 1 || K < 1 || k < 1)
        return ORA_ERR_INVALID_ARG;

    /* f-cost of every existing node; eligibility for expansion is f < bound. */
    double *f = (double *)malloc(sizeof(double) * (size_t)n);
    ora_fcosts(P, T, n, f);
    double tol = 1e-5 * fmax(1.0, fabs(bound));

    /* SampleStates + NearestNeighbor */
    int any_parent = 0;
    for (int i = 0; i < K; ++i) {
        double *q = o->samples + (size_t)i * d;
        ora_sample_state(P, seed, it, (uint32_t)i, q);
        ora_nn_result r;
        ora_nearest(P, T, n, f, q, bound, tol, &r);
        o->near[i] = r.idx;
        o->nn_d1[i] = r.d1;
        o->nn_d2[i] = r.d2;
        o->nn_fragile[i] = r.fragile_elig;
        if (r.idx >= 0)
            any_parent = 1;
    }

    /* SampleControls + Propagate + prune + CollisionFree + insert, in
     * ascending rollout order r = i*k + j. */
    int64_t pos = n;
    int64_t n_app = 0, n_pr = 0, n_col = 0, n_np = 0, n_dr = 0;
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j < k; ++j) {
            int64_t r = (int64_t)i * k + j;
            double *u = o->u + (size_t)r * m;
            int S;
            ora_sample_control(P, seed, it, (uint32_t)i, (uint32_t)j, u, &S);
            o->S[r] = S;
            o->node[r] = -1;
            int64_t par = o->near[i];
            if (par < 0) {
                o->outcome[r] = ORA_OUT_NO_PARENT;
                o->cost_end[r] = NAN;
                o->f_end[r] = NAN;
                o->face_margin[r] = INFINITY;
                o->goal_margin[r] = INFINITY;
                o->in_goal[r] = 0;
                for (int a = 0; a < d; ++a)
                    o->x_end[(size_t)r * d + a] = NAN;
                ++n_np;
                continue;
            }
            ora_rollout ro;
            ora_propagate(P, T->states + (size_t)par * d, T->costs[par], u, S, bound, &ro);
            memcpy(o->x_end + (size_t)r * d, ro.x_end, sizeof(double) * (size_t)d);
            o->cost_end[r] = ro.cost_end;
            o->f_end[r] = ro.f_end;
            o->face_margin[r] = ro.face_margin;
            o->goal_margin[r] = ro.goal_margin;
            o->in_goal[r] = ro.in_goal;
            if (!(ro.f_end < bound)) {
                o->outcome[r] = ORA_OUT_PRUNED;
                ++n_pr;
            } else if (ro.collided) {
                o->outcome[r] = ORA_OUT_COLLIDED;
                ++n_col;
            } else if (pos < T->cap) {
                memcpy(T->states + (size_t)pos * d, ro.x_end, sizeof(double) * (size_t)d);
                memcpy(T->controls + (size_t)pos * m, u, sizeof(double) * (size_t)m);
                T->parents[pos] = (int32_t)par;
                T->costs[pos] = ro.cost_end;
                T->steps[pos] = S;
                o->outcome[r] = ORA_OUT_APPENDED;
                o->node[r] = pos;
                ++pos;
                ++n_app;
            } else {
                o->outcome[r] = ORA_OUT_DROPPED;
                ++n_dr;
            }
        }
    }
    T->count = pos;

    /* Goal test over the appended children: the cheapest one is the solution,
     * the lowest node index breaks a tie. */
    int goal_found = 0;
    int64_t goal_idx = -1;
    double goal_cost = INFINITY;
    for (int64_t r = 0; r < R; ++r) {
        if (o->outcome[r] != ORA_OUT_APPENDED || !o->in_goal[r])
            continue;
        double c = o->cost_end[r];
        if (!goal_found || c < goal_cost || (c == goal_cost && o->node[r] < goal_idx)) {
            goal_found = 1;
            goal_cost = c;
            goal_idx = o->node[r];
        }
    }
    o->n_start = n;
    o->n_appended = n_app;
    o->n_pruned = n_pr;
    o->n_collided = n_col;
    o->n_no_parent = n_np;
    o->n_dropped = n_dr;
    o->goal_found = goal_found;
    o->goal_idx = goal_idx;
    o->goal_cost = goal_cost;
    o->iteration = it;
    T->iteration = it + 1;
    free(f);

    if (!any_parent)
        return ORA_NO_ELIGIBLE;
    if (goal_found)
        return ORA_GOAL_REACHED;
    if (n_dr > 0)
        return ORA_TREE_FULL;
    return ORA_OK;
}

/* ExtractPath (Algorithm 1): parent pointers from the node back to the root;
 * written root first.  Returns the number of nodes, or -1 if cap is short. */
int64_t ora_extract_path(const ora_tree *T, int64_t node, int64_t *nodes_out, int64_t cap)
{
    int64_t len = 0;
    for (int64_t v = node; v >= 0; v = T->parents[v]) {
        ++len;
        if (len > T->count)
            return -1;
    }
    if (len > cap)
        return -1;
    int64_t at = len - 1;
    for (int64_t v = node; v >= 0; v = T->parents[v])
        nodes_out[at--] = v;
    return len;
}

/* ------------------------------------------------------------------------- */
/* AO-x outer loop (Algorithm 1): c_best starts at infinity; each goal found   */
/* lowers it to that child's cost and restarts from a fresh tree, so c_best    */
/* strictly decreases.  The budget is an iteration count here.  A full tree    */
/* without a solution restarts too; no eligible node (the root's f-cost has    */
/* reached c_best) ends the run.                                               */
/* ------------------------------------------------------------------------- */
static int iteration_is_fragile(const ora_problem *P, const ora_expand_out *o, double bound)
{
    int64_t R = (int64_t)P->K * P->k;
    double tol = 1e-5 * fmax(1.0, fabs(bound));
    for (int i = 0; i < P->K; ++i) {
        if (o->near[i] < 0)
            continue;
        if (o->nn_fragile[i] || o->nn_d2[i] - o->nn_d1[i] < 1e-6)
            return 1;
    }
    for (int64_t r = 0; r < R; ++r) {
        if (o->outcome[r] == ORA_OUT_NO_PARENT)
            continue;
        if (fabs(o->f_end[r] - bound) < tol)
            return 1;
        if (o->outcome[r] != ORA_OUT_PRUNED && o->face_margin[r] < 1e-5)
            return 1;
        if ((o->outcome[r] == ORA_OUT_APPENDED || o->outcome[r] == ORA_OUT_DROPPED) && o->goal_margin[r] < 1e-5)
            return 1;
    }
    return 0;
}

int ora_plan(const ora_problem *P, ora_tree *T, const double *x_init, uint64_t seed, ora_plan_out *o)
{
    int d = P->d, m = P->m, K = P->K;
    int64_t R = (int64_t)K * P->k;
    o->iterations = 0;
    o->n_solutions = 0;
    o->n_restarts = 0;
    o->best_cost = INFINITY;
    o->best_path_len = 0;
    o->fragile_iteration = -1;
    if (ora_tree_reset(P, T, x_init) != ORA_OK) {
        o->status = ORA_ERR_INVALID_ARG;
        return o->status;
    }
    ora_expand_out e;
    e.samples = (double *)malloc(sizeof(double) * (size_t)K * d);
    e.near = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    e.nn_d1 = (double *)malloc(sizeof(double) * (size_t)K);
    e.nn_d2 = (double *)malloc(sizeof(double) * (size_t)K);
    e.nn_fragile = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    e.u = (double *)malloc(sizeof(double) * (size_t)R * m);
    e.S = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
    e.outcome = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
    e.x_end = (double *)malloc(sizeof(double) * (size_t)R * d);
    e.cost_end = (double *)malloc(sizeof(double) * (size_t)R);
    e.f_end = (double *)malloc(sizeof(double) * (size_t)R);
    e.face_margin = (double *)malloc(sizeof(double) * (size_t)R);
    e.goal_margin = (double *)malloc(sizeof(double) * (size_t)R);
    e.in_goal = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
    e.node = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);

    double c_best = INFINITY;
    int status = ORA_BUDGET_EXPIRED;
    while (o->iterations < o->max_iterations) {
        int st = ora_expand(P, T, c_best, seed, &e);
        if (o->fragile_iteration < 0 && iteration_is_fragile(P, &e, c_best))
            o->fragile_iteration = o->iterations;
        o->iterations += 1;
        if (st == ORA_NO_ELIGIBLE) {
            status = ORA_NO_ELIGIBLE;
            break;
        }
        if (e.goal_found) {
            c_best = e.goal_cost;
            if (o->n_solutions < o->hist_cap) {
                o->hist_cost[o->n_solutions] = c_best;
                o->hist_iter[o->n_solutions] = o->iterations - 1;
            }
            o->n_solutions += 1;
            o->best_cost = c_best;
            int64_t len = ora_extract_path(T, e.goal_idx, o->best_path, o->path_cap);
            o->best_path_len = len;
            for (int64_t t = 0; t < len; ++t) {
                int64_t v = o->best_path[t];
                memcpy(o->best_states + (size_t)t * d, T->states + (size_t)v * d, sizeof(double) * (size_t)d);
                memcpy(o->best_controls + (size_t)t * m, T->controls + (size_t)v * m, sizeof(double) * (size_t)m);
                o->best_steps[t] = T->steps[v];
            }
            if (o->stop_at_first) {
                status = ORA_GOAL_REACHED;
                break;
            }
            T->count = 1; /* fresh tree {(x_init, -, 0)}; the iteration counter continues */
        } else if (T->count >= T->cap) {
            T->count = 1;
            o->n_restarts += 1;
        }
    }
    if (status == ORA_BUDGET_EXPIRED && o->n_solutions > 0)
        status = ORA_GOAL_REACHED;
    o->status = status;

    free(e.samples);
    free(e.near);
    free(e.nn_d1);
    free(e.nn_d2);
    free(e.nn_fragile);
    free(e.u);
    free(e.S);
    free(e.outcome);
    free(e.x_end);
    free(e.cost_end);
    free(e.f_end);
    free(e.face_margin);
    free(e.goal_margin);
    free(e.in_goal);
    free(e.node);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Validation-only re-checks of an edge between the planner's substeps.        */
/* ------------------------------------------------------------------------- */

/* Re-integrate the edge at dt/sub and test validity at every fine step. */
int ora_recheck_edge_dense(const ora_problem *P, const double *x0, const double *u, int S, int sub)
{
    double x[ORA_MAX_D], xn[ORA_MAX_D];
    memcpy(x, x0, sizeof(double) * (size_t)P->d);
    double h = P->dt / (double)sub;
    for (int s = 0; s < S * sub; ++s) {
        ora_rk4_step(P, x, u, h, xn);
        memcpy(x, xn, sizeof(double) * (size_t)P->d);
        if (!ora_state_valid(P, x))
            return 1;
    }
    return 0;
}

/* Roots of a + b t + c t^2 = 0 in (0, T); returns how many were written. */
static int quad_roots(double a, double b, double c, double T, double *out)
{
    int n = 0;
    if (fabs(c) < 1e-300) {
        if (fabs(b) > 1e-300) {
            double t = -a / b;
            if (t > 0 && t < T)
                out[n++] = t;
        }
        return n;
    }
    double disc = b * b - 4 * a * c;
    if (disc < 0)
        return 0;
    double sq = sqrt(disc);
    double t1 = (-b - sq) / (2 * c), t2 = (-b + sq) / (2 * c);
    if (t1 > 0 && t1 < T)
        out[n++] = t1;
    if (t2 > 0 && t2 < T)
        out[n++] = t2;
    return n;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Double integrator only: p(t) = p0 + v0 t + u t^2 / 2 over the whole edge
 * t in [0, S dt].  Every time at which some coordinate crosses a face is a
 * root of a quadratic; between consecutive such times each inside/outside
 * status is constant, so testing those times and the midpoints between them
 * decides the continuous edge exactly (spheres fall back to a dense check). */
int ora_di_edge_hits_exact(const ora_problem *P, const double *x0, const double *u, int S)
{
    int pd = P->pdim;
    double T = S * P->dt;
    double times[4 + 4 * ORA_MAX_D + 64 * 4 * 3];
    int nt = 0;
    times[nt++] = 0.0;
    times[nt++] = T;
    /* state box faces */
    for (int a = 0; a < pd; ++a) {
        double lohi[2] = {P->x_lo[a], P->x_hi[a]};
        for (int e = 0; e < 2; ++e)
            nt += quad_roots(x0[a] - lohi[e], x0[pd + a], 0.5 * u[a], T, times + nt);
        double vlohi[2] = {P->x_lo[pd + a], P->x_hi[pd + a]};
        for (int e = 0; e < 2; ++e)
            nt += quad_roots(x0[pd + a] - vlohi[e], u[a], 0.0, T, times + nt);
    }
    int hit = 0;
    for (int b = 0; b < P->n_boxes && !hit; ++b) {
        const double *lo = P->boxes + (size_t)b * 2 * pd;
        const double *hi = lo + pd;
        double bt[2 + 4 * 3 + 8];
        int nb = 0;
        bt[nb++] = 0.0;
        bt[nb++] = T;
        for (int a = 0; a < pd; ++a) {
            nb += quad_roots(x0[a] - lo[a], x0[pd + a], 0.5 * u[a], T, bt + nb);
            nb += quad_roots(x0[a] - hi[a], x0[pd + a], 0.5 * u[a], T, bt + nb);
        }
        qsort(bt, (size_t)nb, sizeof(double), cmp_double);
        for (int t = 0; t < 2 * nb - 1 && !hit; ++t) {
            double tt = (t % 2 == 0) ? bt[t / 2] : 0.5 * (bt[t / 2] + bt[t / 2 + 1]);
            if (tt <= 0.0)
                continue; /* the parent state itself is not re-checked */
            int inside = 1;
            for (int a = 0; a < pd; ++a) {
                double p = x0[a] + x0[pd + a] * tt + 0.5 * u[a] * tt * tt;
                if (!(p >= lo[a] && p <= hi[a]))
                    inside = 0;
            }
            if (inside)
                hit = 1;
        }
    }
    if (hit)
        return 1;
    qsort(times, (size_t)nt, sizeof(double), cmp_double);
    for (int t = 0; t < 2 * nt - 1; ++t) {
        double tt = (t % 2 == 0) ? times[t / 2] : 0.5 * (times[t / 2] + times[t / 2 + 1]);
        if (tt <= 0.0)
            continue;
        for (int a = 0; a < pd; ++a) {
            double p = x0[a] + x0[pd + a] * tt + 0.5 * u[a] * tt * tt;
            double v = x0[pd + a] + u[a] * tt;
            if (!(p >= P->x_lo[a] && p <= P->x_hi[a]) || !(v >= P->x_lo[pd + a] && v <= P->x_hi[pd + a]))
                return 1;
        }
    }
    if (P->n_spheres > 0)
        return ora_recheck_edge_dense(P, x0, u, S, 64);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Smooth trajectory cost and its discrete adjoint (reverse mode through each  */
/* RK4 step).  Test infrastructure for the refinement kernels.                 */
/* ------------------------------------------------------------------------- */

/* a^T (df/dx), a^T (df/du) of the dynamics at (x, u). */
void ora_dynamics_vjp(const ora_problem *P, const double *x, const double *u, const double *a, double *gx,
                      double *gu)
{
    int d = P->d, m = P->m;
    for (int i = 0; i < d; ++i)
        gx[i] = 0.0;
    for (int j = 0; j < m; ++j)
        gu[j] = 0.0;
    switch (P->dyn) {
    case ORA_DI2:
    case ORA_DI3: {
        /* p' = v, v' = u */
        int pd = P->pdim;
        for (int i = 0; i < pd; ++i) {
            gx[pd + i] += a[i];
            gu[i] += a[pd + i];
        }
        break;
    }
    case ORA_QUAD12: {
        double mass = P->model[0], Ixx = P->model[1], Iyy = P->model[2], Izz = P->model[3], g = P->model[4];
        double phi = x[3], th = x[4], psi = x[5];
        double cf = cos(phi), sf = sin(phi), ct = cos(th), st = sin(th), cp = cos(psi), sp = sin(psi);
        double tt = st / ct;
        double v[3] = {x[6], x[7], x[8]}, w[3] = {x[9], x[10], x[11]};
        const double *ap = a, *ae = a + 3, *av = a + 6, *aw = a + 9;
        double R[3][3] = {{cp * ct, cp * st * sf - sp * cf, cp * st * cf + sp * sf},
                          {sp * ct, sp * st * sf + cp * cf, sp * st * cf - cp * sf},
                          {-st, ct * sf, ct * cf}};
        double dRf[3][3] = {{0, cp * st * cf + sp * sf, -cp * st * sf + sp * cf},
                            {0, sp * st * cf - cp * sf, -sp * st * sf - cp * cf},
                            {0, ct * cf, -ct * sf}};
        double dRt[3][3] = {{-cp * st, cp * ct * sf, cp * ct * cf},
                            {-sp * st, sp * ct * sf, sp * ct * cf},
                            {-ct, -st * sf, -st * cf}};
        double dRp[3][3] = {{-sp * ct, -sp * st * sf - cp * cf, -sp * st * cf + cp * sf},
                            {cp * ct, cp * st * sf - sp * cf, cp * st * cf + sp * sf},
                            {0, 0, 0}};
        /* p' = R v */
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                gx[6 + c] += R[r][c] * ap[r];
                gx[3] += ap[r] * dRf[r][c] * v[c];
                gx[4] += ap[r] * dRt[r][c] * v[c];
                gx[5] += ap[r] * dRp[r][c] * v[c];
            }
        /* eta' = W omega */
        double W[3][3] = {{1, sf * tt, cf * tt}, {0, cf, -sf}, {0, sf / ct, cf / ct}};
        double dWf[3][3] = {{0, cf * tt, -sf * tt}, {0, -sf, -cf}, {0, cf / ct, -sf / ct}};
        double c2 = ct * ct;
        double dWt[3][3] = {{0, sf / c2, cf / c2}, {0, 0, 0}, {0, sf * st / c2, cf * st / c2}};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                gx[9 + c] += W[r][c] * ae[r];
                gx[3] += ae[r] * dWf[r][c] * w[c];
                gx[4] += ae[r] * dWt[r][c] * w[c];
            }
        /* v' = v x w - g (third row of R) + T/m e3 */
        /* a . (v x w) = v . (w x a) = w . (a x v) */
        gx[6] += w[1] * av[2] - w[2] * av[1];
        gx[7] += w[2] * av[0] - w[0] * av[2];
        gx[8] += w[0] * av[1] - w[1] * av[0];
        gx[9] += av[1] * v[2] - av[2] * v[1];
        gx[10] += av[2] * v[0] - av[0] * v[2];
        gx[11] += av[0] * v[1] - av[1] * v[0];
        for (int c = 0; c < 3; ++c) {
            gx[3] += -g * av[c] * dRf[2][c];
            gx[4] += -g * av[c] * dRt[2][c];
        }
        gu[0] += av[2] / mass;
        /* w' = I^-1 (tau - w x I w) */
        double p_ = w[0], q_ = w[1], r_ = w[2];
        gu[1] += aw[0] / Ixx;
        gu[2] += aw[1] / Iyy;
        gu[3] += aw[2] / Izz;
        gx[9] += -(Ixx - Izz) * r_ * aw[1] / Iyy - (Iyy - Ixx) * q_ * aw[2] / Izz;
        gx[10] += -(Izz - Iyy) * r_ * aw[0] / Ixx - (Iyy - Ixx) * p_ * aw[2] / Izz;
        gx[11] += -(Izz - Iyy) * q_ * aw[0] / Ixx - (Ixx - Izz) * p_ * aw[1] / Iyy;
        break;
    }
    case ORA_DUBINS3D: {
        double yaw = x[3], pitch = x[4], vv = x[5];
        double cy = cos(yaw), sy = sin(yaw), cpi = cos(pitch), spi = sin(pitch);
        gx[3] += a[0] * (-vv * cpi * sy) + a[1] * (vv * cpi * cy);
        gx[4] += a[0] * (-vv * spi * cy) + a[1] * (-vv * spi * sy) + a[2] * (vv * cpi);
        gx[5] += a[0] * cpi * cy + a[1] * cpi * sy + a[2] * spi;
        gu[0] += a[3];
        gu[1] += a[4];
        gu[2] += a[5];
        break;
    }
    case ORA_UNICYCLE1: {
        double c = cos(x[2]), sn = sin(x[2]);
        gx[2] += a[0] * (-u[0] * sn) + a[1] * (u[0] * c);
        gu[0] += a[0] * c + a[1] * sn;
        gu[1] += a[2];
        break;
    }
    case ORA_UNICYCLE2: {
        double c = cos(x[2]), sn = sin(x[2]);
        gx[2] += a[0] * (-x[3] * sn) + a[1] * (x[3] * c);
        gx[3] += a[0] * c + a[1] * sn;
        gx[4] += a[2];
        gu[0] += a[3];
        gu[1] += a[4];
        break;
    }
    default:
        break;
    }
}

/* Exact signed distance from p to one box [lo, hi] (negative inside) and its
 * gradient in p. */
static double box_sdf(int pd, const double *lo, const double *hi, const double *p, double *grad)
{
    double q[3], out2 = 0.0, qmax = -INFINITY;
    int amax = 0;
    for (int a = 0; a < pd; ++a) {
        double ql = lo[a] - p[a], qh = p[a] - hi[a];
        q[a] = ql > qh ? ql : qh;
        if (q[a] > 0)
            out2 += q[a] * q[a];
        if (q[a] > qmax) {
            qmax = q[a];
            amax = a;
        }
    }
    for (int a = 0; a < pd; ++a)
        grad[a] = 0.0;
    if (out2 > 0) {
        double o = sqrt(out2);
        for (int a = 0; a < pd; ++a) {
            if (q[a] > 0) {
                double sgn = (lo[a] - p[a] > p[a] - hi[a]) ? -1.0 : 1.0;
                grad[a] = sgn * q[a] / o;
            }
        }
        return o;
    }
    grad[amax] = (lo[amax] - p[amax] > p[amax] - hi[amax]) ? -1.0 : 1.0;
    return qmax;
}

static double softplus_b(double z, double beta)
{
    double bz = beta * z;
    return (bz > 0 ? bz : 0.0) / beta + log1p(exp(-fabs(bz))) / beta;
}

static double sigmoid(double z)
{
    return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
}

/* Penalty sum_obstacles softplus_beta(margin - sdf(p)) and its gradient in p. */
static double obstacle_penalty(const ora_problem *P, const ora_traj_params *w, const double *p, double *grad)
{
    int pd = P->pdim;
    double total = 0.0, g[3];
    for (int a = 0; a < pd; ++a)
        grad[a] = 0.0;
    for (int b = 0; b < P->n_boxes; ++b) {
        const double *lo = P->boxes + (size_t)b * 2 * pd, *hi = lo + pd;
        double sdf = box_sdf(pd, lo, hi, p, g);
        double z = w->margin - sdf;
        total += softplus_b(z, w->beta);
        double s = sigmoid(w->beta * z);
        for (int a = 0; a < pd; ++a)
            grad[a] += -s * g[a];
    }
    for (int sidx = 0; sidx < P->n_spheres; ++sidx) {
        const double *c = P->spheres + (size_t)sidx * (pd + 1);
        double dd = 0.0;
        for (int a = 0; a < pd; ++a)
            dd += (p[a] - c[a]) * (p[a] - c[a]);
        double dist = sqrt(dd);
        double z = w->margin - (dist - c[pd]);
        total += softplus_b(z, w->beta);
        double s = sigmoid(w->beta * z);
        for (int a = 0; a < pd; ++a)
            grad[a] += dist > 0 ? -s * (p[a] - c[a]) / dist : 0.0;
    }
    return total;
}

double ora_traj_cost(const ora_problem *P, const double *x0, const double *U, int N, const ora_traj_params *w,
                     double *x_final)
{
    int d = P->d, m = P->m, pd = P->pdim;
    double x[ORA_MAX_D], xn[ORA_MAX_D], g[3];
    memcpy(x, x0, sizeof(double) * (size_t)d);
    double J = w->w_dur * N * P->dt;
    for (int n = 0; n < N; ++n) {
        const double *u = U + (size_t)n * m;
        for (int j = 0; j < m; ++j)
            J += w->w_u * u[j] * u[j] * P->dt;
        ora_rk4_step(P, x, u, P->dt, xn);
        double dd = 0.0;
        for (int a = 0; a < pd; ++a)
            dd += (xn[a] - x[a]) * (xn[a] - x[a]);
        J += w->w_len * sqrt(dd + w->len_eps * w->len_eps);
        memcpy(x, xn, sizeof(double) * (size_t)d);
        J += w->w_obs * obstacle_penalty(P, w, x, g) * P->dt;
    }
    double e2 = 0.0;
    for (int a = 0; a < pd; ++a)
        e2 += (x[a] - P->x_goal[a]) * (x[a] - P->x_goal[a]);
    J += w->w_goal * e2;
    if (x_final)
        memcpy(x_final, x, sizeof(double) * (size_t)d);
    return J;
}

/* Reverse mode: store every state, then pull the adjoint back through each
 * RK4 step's four stages.  Returns the cost; fills dJ/dU and dJ/dx0. */
double ora_traj_grad(const ora_problem *P, const double *x0, const double *U, int N, const ora_traj_params *w,
                     double *dU, double *dx0)
{
    int d = P->d, m = P->m, pd = P->pdim;
    double h = P->dt;
    double *X = (double *)malloc(sizeof(double) * (size_t)(N + 1) * d);
    memcpy(X, x0, sizeof(double) * (size_t)d);
    for (int n = 0; n < N; ++n)
        ora_rk4_step(P, X + (size_t)n * d, U + (size_t)n * m, h, X + (size_t)(n + 1) * d);
    double J = ora_traj_cost(P, x0, U, N, w, NULL);
    double lam[ORA_MAX_D], g3[3];
    /* adjoint of the final state: goal error + obstacle penalty at x_N */
    for (int i = 0; i < d; ++i)
        lam[i] = 0.0;
    const double *xN = X + (size_t)N * d;
    for (int a = 0; a < pd; ++a)
        lam[a] += 2.0 * w->w_goal * (xN[a] - P->x_goal[a]);
    obstacle_penalty(P, w, xN, g3);
    for (int a = 0; a < pd; ++a)
        lam[a] += w->w_obs * g3[a] * h;
    for (int n = N - 1; n >= 0; --n) {
        const double *xs = X + (size_t)n * d, *xe = X + (size_t)(n + 1) * d;
        const double *u = U + (size_t)n * m;
        /* path-length segment n -> n+1 */
        double dd = 0.0;
        for (int a = 0; a < pd; ++a)
            dd += (xe[a] - xs[a]) * (xe[a] - xs[a]);
        double L = sqrt(dd + w->len_eps * w->len_eps);
        for (int a = 0; a < pd; ++a)
            lam[a] += w->w_len * (xe[a] - xs[a]) / L;
        /* stages of the forward step */
        double k1[ORA_MAX_D], k2[ORA_MAX_D], k3[ORA_MAX_D], y2[ORA_MAX_D], y3[ORA_MAX_D], y4[ORA_MAX_D];
        ora_dynamics(P, xs, u, k1);
        for (int i = 0; i < d; ++i)
            y2[i] = xs[i] + 0.5 * h * k1[i];
        ora_dynamics(P, y2, u, k2);
        for (int i = 0; i < d; ++i)
            y3[i] = xs[i] + 0.5 * h * k2[i];
        ora_dynamics(P, y3, u, k3);
        for (int i = 0; i < d; ++i)
            y4[i] = xs[i] + h * k3[i];
        /* x' = x + h/6 (k1 + 2k2 + 2k3 + k4) */
        double a1[ORA_MAX_D], a2[ORA_MAX_D], a3[ORA_MAX_D], a4[ORA_MAX_D], gx[ORA_MAX_D], gu[ORA_MAX_M];
        double xb[ORA_MAX_D], ub[ORA_MAX_M];
        for (int i = 0; i < d; ++i) {
            xb[i] = lam[i];
            a1[i] = h / 6.0 * lam[i];
            a2[i] = h / 3.0 * lam[i];
            a3[i] = h / 3.0 * lam[i];
            a4[i] = h / 6.0 * lam[i];
        }
        for (int j = 0; j < m; ++j)
            ub[j] = 2.0 * w->w_u * u[j] * h;
        /* k4 = f(y4), y4 = x + h k3 */
        ora_dynamics_vjp(P, y4, u, a4, gx, gu);
        for (int i = 0; i < d; ++i) {
            xb[i] += gx[i];
            a3[i] += h * gx[i];
        }
        for (int j = 0; j < m; ++j)
            ub[j] += gu[j];
        /* k3 = f(y3), y3 = x + h/2 k2 */
        ora_dynamics_vjp(P, y3, u, a3, gx, gu);
        for (int i = 0; i < d; ++i) {
            xb[i] += gx[i];
            a2[i] += 0.5 * h * gx[i];
        }
        for (int j = 0; j < m; ++j)
            ub[j] += gu[j];
        /* k2 = f(y2), y2 = x + h/2 k1 */
        ora_dynamics_vjp(P, y2, u, a2, gx, gu);
        for (int i = 0; i < d; ++i) {
            xb[i] += gx[i];
            a1[i] += 0.5 * h * gx[i];
        }
        for (int j = 0; j < m; ++j)
            ub[j] += gu[j];
        /* k1 = f(x) */
        ora_dynamics_vjp(P, xs, u, a1, gx, gu);
        for (int i = 0; i < d; ++i)
            xb[i] += gx[i];
        for (int j = 0; j < m; ++j)
            ub[j] += gu[j];
        for (int j = 0; j < m; ++j)
            dU[(size_t)n * m + j] = ub[j];
        /* adjoint of x_n: the step's pull-back, the other end of the segment,
         * and the obstacle penalty at x_n (states 1..N carry it) */
        for (int i = 0; i < d; ++i)
            lam[i] = xb[i];
        for (int a = 0; a < pd; ++a)
            lam[a] -= w->w_len * (xe[a] - xs[a]) / L;
        if (n >= 1) {
            obstacle_penalty(P, w, xs, g3);
            for (int a = 0; a < pd; ++a)
                lam[a] += w->w_obs * g3[a] * h;
        }
    }
    if (dx0)
        memcpy(dx0, lam, sizeof(double) * (size_t)d);
    free(X);
    return J;
}
