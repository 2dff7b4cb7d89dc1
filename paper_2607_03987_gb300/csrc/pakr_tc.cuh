// Tensor-core nearest-neighbour support: inline PTX for tcgen05 / TMA / mbarrier,
// the packed node operand layout, and the error bound of the tensor-core filter.
//
// The filter computes, for every (query q, node x) pair,
//     a = |x - c|^2 - 2 (q - c) . (x - c)
// with c the centre of the weighted state box.  a + |q - c|^2 is the squared
// distance, so within one query a orders nodes like the distance.  Operands are
// FP32 values split into TF32 parts v = hi + lo (hi = v with the low 13
// mantissa bits cleared, lo = v - hi; the query operand truncates lo the same
// way, the packed node copy keeps it exact so that hi + lo gives v back, and
// the tensor core reads it as TF32); the product is formed from
// hi.hi + hi.lo + lo.hi, and |x - c|^2 enters as hi + lo times 1.
// One tcgen05.mma of kind::tf32 with K = 8 covers eight of those columns.
//
// Two layouts of the packed node row (TcShape<D>::SPLIT chooses):
//  - split (d = 3, 5, 6): the row is (x_hi, x_lo, |x|^2 hi, lo) in 2d + 2 columns rounded up
//    to 8, and the query has two operands: (-2q_hi against x_hi and x_lo, 1, 1) over the whole
//    row, and (-2q_lo) against the x_hi columns alone, issued as extra MMAs into the same
//    accumulator.  No column is stored twice;
//  - joint (other d): the row is (x_hi, x_lo, x_hi, |x|^2 hi, lo) in 3d + 2 columns rounded
//    up to 8 against one query operand (-2q_hi, -2q_hi, -2q_lo, 1, 1).  Used where the split
//    form would need more MMAs per tile (d = 12: 6 instead of 5) or save no bytes (d = 4).
#pragma once
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
// Wait for the phase with the given parity for at most limit_ns of device
// time; false on timeout.  Polls with the non-blocking test; after 64 failed
// polls the thread sleeps between polls (32 ns doubling to 256 ns).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned long long limit_ns)
{
    if (mbar_test_wait(bar, parity))
        return true;
    const unsigned long long t0 = tc_clock_ns();
    unsigned ns = 32;
    for (int it = 0;; ++it) {
        if (mbar_test_wait(bar, parity))
            return true;
        if (it >= 64) {
            __nanosleep(ns);
            ns = ns < 256 ? 2 * ns : 256;
        }
        if ((it & 15) == 15 && tc_clock_ns() - t0 > limit_ns)
            return false;
    }
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
// Wait for the phase for at most limit_ns of device time without spinning: for the warps
// that are not on the tensor pipe's critical path, whose polls would take issue slots and
// ALU cycles from the accumulator readers on the same scheduler.
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
// D[tmem] (+)= A[smem] * B[smem]^T, kind::tf32, one CTA; the accumulate flag ACC is fixed at
// compile time (no predicate computed per MMA).
template <bool ACC>
__device__ __forceinline__ void mma_tf32_ss_c(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc)
{
    if constexpr (ACC)
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "setp.eq.u32 p, 1, 1;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                     "l"(adesc), "l"(bdesc), "r"(idesc)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "setp.eq.u32 p, 1, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
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
// Shared-memory matrix descriptor, no swizzle, K-major: LBO = byte distance of
// the two core matrices along K, SBO = byte distance of 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// Operand geometry.
// ---------------------------------------------------------------------------
constexpr int kTcM = 128;        // queries per CTA (MMA M)
constexpr int kTcN = 256;        // nodes per tile of the packed operand copy
constexpr int kTcBN = 128;       // nodes per pipeline stage and MMA (N): half a packed tile
constexpr int kTcAcc = 4 / kTcCtasPerSm;  // accumulators of kTcBN columns per CTA: an SM's 512 columns
constexpr int kTcCols = kTcAcc * kTcBN;  // TMEM columns per CTA
constexpr int kTcG = 16;         // nodes per filter group
constexpr int kTcRing = 8;       // candidate groups remembered per (query, reader)
constexpr float kTcSentinel = 1.2676506e30f;  // 2^100: |x - c|^2 of ineligible and padding nodes
constexpr float kTcEligible = 6.338253e29f;   // 2^99: filter values at or above are not eligible nodes
// warp roles
constexpr int kTcLoadWarp = 0;   // lane 0: bulk copies of node half tiles and f-costs
constexpr int kTcMmaWarp = 1;    // lane 0: MMAs; the warp owns the TMEM allocation
constexpr int kTcPatch0 = 2;     // warps 2-3: mask ineligible rows, signal "stage masked"
constexpr int kTcReader0 = 4;    // warps 4 and up: accumulator readers (warp w reads lane quarter w % 4)

// Columns of the packed node row for state dimension d (see the two layouts above).
__host__ __device__ constexpr int tc_cols_joint(int d) { return ((3 * d + 2) + 7) / 8 * 8; }
__host__ __device__ constexpr int tc_cols_split(int d) { return ((2 * d + 2) + 7) / 8 * 8; }
__host__ __device__ constexpr bool tc_split(int d)
{
    return tc_cols_split(d) < tc_cols_joint(d) &&
           tc_cols_split(d) / 8 + (d + 7) / 8 <= tc_cols_joint(d) / 8;
}
__host__ __device__ constexpr int tc_node_cols(int d) { return tc_split(d) ? tc_cols_split(d) : tc_cols_joint(d); }

template <int D>
struct TcShape {
    static constexpr bool SPLIT = tc_split(D);
    static constexpr int KT = tc_node_cols(D);                 // columns of a packed node row
    static constexpr int KA2 = SPLIT ? (D + 7) / 8 * 8 : 0;    // columns of the second query operand
    static constexpr int NORM = SPLIT ? 2 * D : 3 * D;         // column of |x|^2 hi (lo follows)
    static constexpr int MMAS = KT / 8 + KA2 / 8;              // MMAs of K = 8 per stage
    static constexpr int LBO = 128, SBO = KT * 32;             // no-swizzle K-major core-matrix layout
    static constexpr int SBO2 = KA2 * 32;                      // the same for the second query operand
    static constexpr int TILE_BYTES = kTcN * KT * 4;           // one packed node tile, contiguous
    static constexpr int STAGE_BYTES = kTcBN * KT * 4;         // half a packed tile: also contiguous
    static constexpr int A1_BYTES = kTcM * KT * 4;
    static constexpr int A_BYTES = A1_BYTES + kTcM * KA2 * 4;
    static constexpr int F_BYTES = kTcBN * 4;
    // reader warps per TMEM lane quarter: two (64 accumulator columns each) for d <= 8, one
    // (all 128) for larger d, whose resolve needs the registers (measured both ways: d = 6
    // gains 3 %, d = 12 loses 3-6 % with two)
    static constexpr int RH = D <= 8 ? 2 : 1;
    static constexpr int READERS = 128 * RH;
    static constexpr int THREADS = kTcReader0 * 32 + READERS;
    static constexpr int RING_BYTES = kTcRing * READERS * 8;
    // two CTAs per SM: each within half of the SM's 228 KB, static shared memory included
    static constexpr int NSTAGE_FIT = (100 * 1024 - A_BYTES - RING_BYTES) / (STAGE_BYTES + F_BYTES);
    static constexpr int NSTAGE = NSTAGE_FIT > 8 ? 8 : NSTAGE_FIT;  // half tiles staged in shared memory
    static constexpr int SMEM = A_BYTES + NSTAGE * (STAGE_BYTES + F_BYTES) + RING_BYTES;
    // and at least enough that no third CTA fits beside them (two CTAs take all 512 TMEM columns)
    static constexpr int SMEM_REQ = SMEM > 80 * 1024 ? SMEM : 80 * 1024;
    static_assert(NSTAGE >= 2, "shared memory stages");
};

// Byte offset of (row r, column k) in a no-swizzle K-major tile with KT columns.
template <int D>
__host__ __device__ __forceinline__ uint32_t tc_off(int r, int k)
{
    return (uint32_t)((r >> 3) * TcShape<D>::SBO + (k >> 2) * TcShape<D>::LBO + (r & 7) * 16 + (k & 3) * 4);
}
// The same in the second query operand (KA2 columns).
template <int D>
__host__ __device__ __forceinline__ uint32_t tc_off2(int r, int k)
{
    return (uint32_t)((r >> 3) * TcShape<D>::SBO2 + (k >> 2) * TcShape<D>::LBO + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_trunc(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

// Bound on |a + |q - c|^2 - e| relative to R^2 = (|q - c| + X)^2, with e the exact FP32
// squared distance the result is defined by and X the bound on |x - c| over the state box.
// Terms (u = 2^-24): the hi/lo truncations leave |v - hi - lo| < 2^-20 |v| per operand, so
// the three partial products miss -2 q.x by at most 6 2^-20 |q||x| <= 1.5 2^-20 R^2, and
// |x|^2 by 2^-20 |x|^2; FP32 |x - c|^2 adds gamma_d; the exact form e carries gamma_(d+2);
// rounding x - c and q - c moves the distance by at most 2.01 u R^2; the tensor-core
// accumulation is taken as 4 (KT/8 + 1) u of the sum of |products| (measured on this GPU
// at most 5.2 u with 5 accumulating k-steps, 2.2 u with one; taken per MMA of the stage,
// whichever operand it reads).  The total is doubled.
template <int D>
__host__ __device__ constexpr float tc_bound_coef()
{
    constexpr float u = 5.9604645e-8f;
    constexpr int MMAS = TcShape<D>::MMAS;
    return 2.f * (2.5f * 16.f * u + D * u / (1.f - D * u) + (D + 2) * u / (1.f - (D + 2) * u) +
                  1.01f * 4.f * (MMAS + 1) * u + 2.01f * u);
}

// Write node j's packed operand row (state x, unweighted) into the tree's tile copy;
// flag the tree when |x_w - c|^2 exceeds the box bound the error analysis assumes.
template <int D>
__device__ __forceinline__ void tc_pack_node(const DevProblem &P, const DevTree &T, Ctl *ctl, int j, const float *x)
{
    if (!T.XT)
        return;
    using S = TcShape<D>;
    constexpr int KT = S::KT;
    float row[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k)
        row[k] = 0.f;
    float xn = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float v = x[a] * P.sw[a] - P.tc_c[a];
        xn = __fmaf_rn(v, v, xn);
        const float hi = tf32_trunc(v);
        row[a] = hi;
        row[D + a] = v - hi;  // exact; the tensor core reads it as TF32, the exact resolve adds it to hi
        if constexpr (!S::SPLIT)
            row[2 * D + a] = hi;
    }
    const float nh = tf32_trunc(xn);
    row[S::NORM] = nh;
    row[S::NORM + 1] = tf32_trunc(xn - nh);
    if (!(xn <= P.tc_xbox2))
        atomicOr(&ctl->tc_flag, 1u);
    unsigned char *tile = reinterpret_cast<unsigned char *>(T.XT) + (size_t)(j / kTcN) * TcShape<D>::TILE_BYTES;
    const int r = j % kTcN;
#pragma unroll
    for (int c = 0; c < KT / 4; ++c)
        *reinterpret_cast<float4 *>(tile + tc_off<D>(r, 4 * c)) =
            make_float4(row[4 * c], row[4 * c + 1], row[4 * c + 2], row[4 * c + 3]);
}

}  // namespace pakr
