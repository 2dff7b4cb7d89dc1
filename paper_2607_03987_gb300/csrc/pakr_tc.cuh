// Tensor-core nearest-neighbour support: inline PTX for tcgen05 / TMA / mbarrier,
// the packed node operand layout, and the error bound of the tensor-core filter.
//
// The filter computes, for every (query q, node x) pair,
//     a = |x - c|^2 - 2 (q - c) . (x - c)
// with c the centre of the weighted state box.  a + |q - c|^2 is the squared
// distance, so within one query a orders nodes like the distance.  Operands are
// FP16: centred coordinates are scaled by a power of two s that brings the box
// radius into [2^7, 2^8) (exact), and every FP32 value v is split as
// v = hi + lo + err with hi = fp16(v), lo = fp16(v - hi) (round to nearest,
// |err| <= 2^-22 |v| + 2^-25); the product is formed from hi.hi + hi.lo + lo.hi with
// FP32 accumulation, and |x - c|^2 (scaled by s^2 / 2^8) enters as hi + lo times
// 2^8.  One tcgen05.mma of kind::f16 with K = 16 covers sixteen of those columns.
// FP16 has TF32's 11-bit significand, so the split is as precise as a TF32 one, at
// twice the columns per MMA and half the operand bytes.
//
// Two layouts of the packed node row (TcShape<D>::SPLIT chooses):
//  - split (d = 5, 6, 12): the row is (x_hi, x_lo, |x|^2 hi, lo) in 2d + 2 columns rounded
//    up to 16, and the query has two operands: (-2q_hi against x_hi and x_lo, 2^8, 2^8)
//    over the whole row, and (-2q_lo) against the x_hi columns alone, issued as extra MMAs
//    into the same accumulator.  No column is stored twice;
//  - joint (d = 3, 4): the row is (x_hi, x_lo, x_hi, |x|^2 hi, lo) in 3d + 2 columns
//    rounded up to 16 against one query operand (-2q_hi, -2q_hi, -2q_lo, 2^8, 2^8): one MMA
//    per tile, where the split form would take two.
#pragma once
#include <cuda_fp16.h>

#include "pakr_internal.h"

namespace pakr {

// ---------------------------------------------------------------------------
// PTX wrappers (sm_100 family).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tc_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Potentially blocking test of the phase: the thread is suspended until the phase
// completes or a hardware time limit passes, so a waiting warp issues nothing.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity for at most limit_ns of device time (false on
// timeout) without spinning: polls would take issue slots and ALU cycles from the accumulator
// readers on the same scheduler, and a suspended thread wakes about as soon after the phase
// completes as a polling one sees it.
__device__ __forceinline__ bool mbar_wait_suspend(uint32_t bar, uint32_t parity, unsigned long long limit_ns)
{
    if (mbar_test_wait(bar, parity))
        return true;
    const unsigned long long t0 = tc_clock_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (tc_clock_ns() - t0 > limit_ns)
            return false;
    }
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (FP16 operands, FP32 accumulator), one CTA;
// the accumulate flag ACC is fixed at compile time (no predicate computed per MMA).
template <bool ACC>
__device__ __forceinline__ void mma_f16_ss_c(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc)
{
    if constexpr (ACC)
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "setp.eq.u32 p, 1, 1;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                     "l"(adesc), "l"(bdesc), "r"(idesc)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "setp.eq.u32 p, 1, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                     "l"(adesc), "l"(bdesc), "r"(idesc)
                     : "memory");
}
// Arrive on the mbarrier when every tcgen05 operation this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Order this thread's generic-proxy shared-memory writes before later async-proxy (TMA, MMA) accesses.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Bulk copy global -> shared (addresses 16-byte aligned, bytes a multiple of 16), completing on the
// mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst_smem, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst_smem),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Minimum of 16 consecutive FP32 accumulator columns of this thread's TMEM lane: tcgen05.ld
// with the min reduction (sm_103a) returns the per-lane minimum next to the loaded values, so
// no ALU work is spent on it; the values themselves are not needed and are dropped.  Waits for
// the load (its destination registers are written asynchronously until then).
__device__ __forceinline__ float tmem_ldred_min16(uint32_t taddr)
{
    uint32_t r[16];
    float m;
    asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, %16, [%17];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=f"(m)
                 : "r"(taddr)
                 : "memory");
    return m;
}
// The minima of two 16-column groups (at taddr and taddr + 16) from two reducing loads that
// are in flight together, with one wait for both.
__device__ __forceinline__ void tmem_ldred_min16x2(uint32_t taddr, float &m0, float &m1)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, %32, [%34];\n\t"
                 "tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 "
                 "{%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %33, [%35];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=f"(m0), "=f"(m1)
                 : "r"(taddr), "r"(taddr + 16u)
                 : "memory");
}
// Minima of NG consecutive 16-column groups, BATCH (1 or 2) loads in flight per wait.
template <int NG, int BATCH>
__device__ __forceinline__ void tmem_ldred_groups(uint32_t taddr, float (&m)[NG])
{
    static_assert(BATCH == 1 || (BATCH == 2 && NG % 2 == 0), "load batch");
    if constexpr (BATCH == 2) {
#pragma unroll
        for (int h = 0; h < NG; h += 2) {
            __syncwarp();
            tmem_ldred_min16x2(taddr + 16u * h, m[h], m[h + 1]);
        }
    } else {
#pragma unroll
        for (int h = 0; h < NG; ++h) {
            __syncwarp();
            m[h] = tmem_ldred_min16(taddr + 16u * h);
        }
    }
}
// Shared-memory matrix descriptor, no swizzle, K-major: LBO = byte distance of
// the two core matrices along K, SBO = byte distance of 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B f16 (type code 0), both
// K-major, N / 8 at bit 17, M / 16 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// Operand geometry.
// ---------------------------------------------------------------------------
constexpr int kTcElem = 2;        // bytes per operand element (FP16)
constexpr int kTcKStep = 16;      // K of one MMA (32 bytes of a row)
constexpr int kTcCoreK = 8;       // elements per 16-byte core-matrix row
constexpr int kTcM = 128;        // queries per CTA (MMA M)
constexpr int kTcN = 256;        // nodes per tile of the packed operand copy
constexpr int kTcBN = 128;       // nodes per pipeline stage and MMA (N): half a packed tile
constexpr int kTcAcc = 4 / kTcCtasPerSm;  // accumulators of kTcBN columns per CTA: an SM's 512 columns
constexpr int kTcCols = kTcAcc * kTcBN;  // TMEM columns per CTA
constexpr int kTcG = 16;         // nodes per filter group
constexpr int kTcRing = 8;       // candidate groups remembered per (query, reader)
// Scaled units (box radius X in [2^7, 2^8), queries within 2^9 of the centre): real filter
// values are below X^2 + 2 |2q| X < 2^19.  Ineligible and padding nodes get 2^15 in the
// |x - c|^2 hi column, 2^23 after the query's 2^8, and filter values at or above 2^22 are
// not eligible nodes.
constexpr float kTcSentinel = 32768.f;
constexpr float kTcEligible = 4194304.f;
constexpr float kTcNormA = 256.f;     // query operand's |x - c|^2 columns (the node's are scaled by 2^-8)
constexpr float kTcQueryMax2 = 262144.f;  // (2^9)^2: farther queries are rescanned exactly
// warp roles
constexpr int kTcLoadWarp = 0;   // lane 0: bulk copies of node half tiles and f-costs
constexpr int kTcMmaWarp = 1;    // lane 0: MMAs; the warp owns the TMEM allocation
constexpr int kTcPatch0 = 2;     // warps 2-3: mask ineligible rows, signal "stage masked"
constexpr int kTcReader0 = 4;    // warps 4 and up: accumulator readers (warp w reads lane quarter w % 4)

// Columns of the packed node row for state dimension d (see the two layouts above).
__host__ __device__ constexpr int tc_round_k(int c) { return (c + kTcKStep - 1) / kTcKStep * kTcKStep; }
__host__ __device__ constexpr int tc_cols_joint(int d) { return tc_round_k(3 * d + 2); }
__host__ __device__ constexpr int tc_cols_split(int d) { return tc_round_k(2 * d + 2); }
__host__ __device__ constexpr bool tc_split(int d)
{
    return tc_cols_split(d) < tc_cols_joint(d) &&
           tc_cols_split(d) / kTcKStep + tc_round_k(d) / kTcKStep <= tc_cols_joint(d) / kTcKStep;
}
__host__ __device__ constexpr int tc_node_cols(int d) { return tc_split(d) ? tc_cols_split(d) : tc_cols_joint(d); }

template <int D>
struct TcShape {
    static constexpr bool SPLIT = tc_split(D);
    static constexpr int KT = tc_node_cols(D);                 // columns of a packed node row
    static constexpr int KA2 = SPLIT ? tc_round_k(D) : 0;      // columns of the second query operand
    static constexpr int NORM = SPLIT ? 2 * D : 3 * D;         // column of |x|^2 hi (lo follows)
    static constexpr int MMAS = (KT + KA2) / kTcKStep;         // MMAs per stage
    static constexpr int LBO = 128, SBO = KT * kTcElem * 8;    // no-swizzle K-major core-matrix layout
    static constexpr int SBO2 = KA2 * kTcElem * 8;             // the same for the second query operand
    static constexpr int TILE_BYTES = kTcN * KT * kTcElem;     // one packed node tile, contiguous
    static constexpr int STAGE_BYTES = kTcBN * KT * kTcElem;   // half a packed tile: also contiguous
    static constexpr int A1_BYTES = kTcM * KT * kTcElem;
    static constexpr int A_BYTES = A1_BYTES + kTcM * KA2 * kTcElem;
    static constexpr int F_BYTES = kTcBN * 4;
    // reader warps per TMEM lane quarter: two (64 accumulator columns each) for d <= 8, one
    // (all 128) for larger d, whose resolve needs the registers (measured both ways: d = 6
    // gains 3 %, d = 12 loses 3-6 % with two)
    static constexpr int RH = D <= 8 ? 2 : 1;
    static constexpr int READERS = 128 * RH;
    static constexpr int THREADS = kTcReader0 * 32 + READERS;
    // TMEM loads a reader keeps in flight per wait: two where the launch leaves 128 registers
    // a thread (d > 8: quadrotor 333 -> 327 us at n = 1,000,000), one for d <= 8, where the
    // second load's destination registers spill at 80 (d = 6: 87.3 -> 90.3 us)
    static constexpr int LD_BATCH = D <= 8 ? 1 : 2;
    static constexpr int RING_BYTES = kTcRing * READERS * 8;
    // two CTAs per SM: each within half of the SM's 228 KB, static shared memory included
    static constexpr int NSTAGE_FIT = (100 * 1024 - A_BYTES - RING_BYTES) / (STAGE_BYTES + F_BYTES);
    static constexpr int NSTAGE = NSTAGE_FIT > 16 ? 16 : NSTAGE_FIT;  // half tiles staged in shared memory
    static constexpr int SMEM = A_BYTES + NSTAGE * (STAGE_BYTES + F_BYTES) + RING_BYTES;
    // and at least enough that no third CTA fits beside them (two CTAs take all 512 TMEM columns)
    static constexpr int SMEM_REQ = SMEM > 80 * 1024 ? SMEM : 80 * 1024;
    static_assert(NSTAGE >= 2 && NSTAGE >= kTcAcc, "shared memory stages");
    // after the tile loop the stages hold the resolve list: one (row, group) pair per ring entry
    static_assert(NSTAGE * STAGE_BYTES >= kTcRing * READERS * 8, "resolve list in the stages");
};

// Byte offset of (row r, column k) in a no-swizzle K-major tile with KT columns.
template <int D>
__host__ __device__ __forceinline__ uint32_t tc_off(int r, int k)
{
    return (uint32_t)((r >> 3) * TcShape<D>::SBO + (k / kTcCoreK) * TcShape<D>::LBO + (r & 7) * 16 +
                      (k % kTcCoreK) * kTcElem);
}
// The same in the second query operand (KA2 columns).
template <int D>
__host__ __device__ __forceinline__ uint32_t tc_off2(int r, int k)
{
    return (uint32_t)((r >> 3) * TcShape<D>::SBO2 + (k / kTcCoreK) * TcShape<D>::LBO + (r & 7) * 16 +
                      (k % kTcCoreK) * kTcElem);
}

__device__ __forceinline__ float f16_round(float v) { return __half2float(__float2half_rn(v)); }
// One 16-byte core-matrix row of kTcCoreK consecutive columns, from floats FP16 holds exactly.
__device__ __forceinline__ uint4 tc_chunk(const float *v)
{
    const __half2 h0 = __floats2half2_rn(v[0], v[1]), h1 = __floats2half2_rn(v[2], v[3]);
    const __half2 h2 = __floats2half2_rn(v[4], v[5]), h3 = __floats2half2_rn(v[6], v[7]);
    return make_uint4(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1),
                      *reinterpret_cast<const uint32_t *>(&h2), *reinterpret_cast<const uint32_t *>(&h3));
}
__device__ __forceinline__ void tc_store_elem(unsigned char *p, float v) { *reinterpret_cast<__half *>(p) = __float2half_rn(v); }
// v = hi + lo + err in FP16 (|v| well inside its range): round to nearest twice, |err| <=
// 2^-22 |v| + 2^-25 (the second term where lo is subnormal).  v - hi is exact in FP32.
__device__ __forceinline__ void tc_split_val(float v, float &hi, float &lo)
{
    hi = f16_round(v);
    lo = f16_round(v - hi);
}

// Bound on |a + |q - c|^2 - e| relative to R^2 = (|q - c| + X)^2, with e the exact FP32
// squared distance the result is defined by and X the bound on |x - c| over the state box,
// all in the scaled coordinates (X >= 2^7; scaling by a power of two commutes with FP32
// rounding).  Terms (u = 2^-24): the split leaves |v - hi - lo| <= 2^-22 |v| + 2^-25 per
// operand, so the three partial products miss -2 q.x by at most 3.01 2^-22 |2q||x| <=
// 1.505 2^-22 R^2 (|q||x| <= R^2 / 4), and |x|^2 by 2^-22 |x|^2 <= 2^-22 R^2; the subnormal
// floor adds 2^-25 (|2q|_1 + |x|_1) + 2^-25 2^8 (the norm's), below 0.05 u R^2 once X >= 2^7;
// FP32 |x - c|^2 adds gamma_d; the exact form e carries gamma_(d+2); rounding x - c and
// q - c moves the distance by at most 2.01 u R^2; the tensor-core accumulation is taken as
// 4 (MMAS + 1) u of the sum of |products|, which is at most R^2 (measured on this GPU: at most
// 6.1 u with 4 accumulating FP16 k-steps).  The total is doubled.
template <int D>
__host__ __device__ constexpr float tc_bound_coef()
{
    constexpr float u = 5.9604645e-8f;
    constexpr int MMAS = TcShape<D>::MMAS;
    return 2.f * (2.51f * 4.f * u + 0.05f * u + D * u / (1.f - D * u) + (D + 2) * u / (1.f - (D + 2) * u) +
                  1.01f * 4.f * (MMAS + 1) * u + 2.01f * u);
}

// Write node j's packed operand row (state x, unweighted) into the tree's tile copy: the
// centred coordinates scaled by P.tc_s and |x - c|^2 by P.tc_s^2 / 2^8 (powers of two,
// exact), each split into FP16 hi + lo.  Flag the tree when |x_w - c|^2 exceeds the box
// bound the error analysis assumes (its searches then rescan exactly).
template <int D>
__device__ __forceinline__ void tc_pack_node(const DevProblem &P, const DevTree &T, Ctl *ctl, int j, const float *x)
{
    if (!T.XT)
        return;
    using S = TcShape<D>;
    constexpr int KT = S::KT;
    float row[KT], v[D];
#pragma unroll
    for (int k = 0; k < KT; ++k)
        row[k] = 0.f;
    float xn = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        v[a] = x[a] * P.sw[a] - P.tc_c[a];
        xn = __fmaf_rn(v[a], v[a], xn);
    }
    // a node outside the box bound keeps a zero row: its scaled coordinates could overflow
    // FP16, and rows past the tree's end (of a later, smaller tree) still enter the products
    if (xn <= P.tc_xbox2) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float hi, lo;
            tc_split_val(v[a] * P.tc_s, hi, lo);
            row[a] = hi;
            row[D + a] = lo;
            if constexpr (!S::SPLIT)
                row[2 * D + a] = hi;
        }
        tc_split_val(xn * (P.tc_s * P.tc_s / kTcNormA), row[S::NORM], row[S::NORM + 1]);
    } else {
        atomicOr(&ctl->tc_flag, 1u);
    }
    unsigned char *tile = reinterpret_cast<unsigned char *>(T.XT) + (size_t)(j / kTcN) * TcShape<D>::TILE_BYTES;
    const int r = j % kTcN;
#pragma unroll
    for (int c = 0; c < KT / kTcCoreK; ++c)
        *reinterpret_cast<uint4 *>(tile + tc_off<D>(r, kTcCoreK * c)) = tc_chunk(row + kTcCoreK * c);
}

}  // namespace pakr
