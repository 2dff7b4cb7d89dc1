// k_nn_tc: cost-pruned nearest neighbour on the tensor cores (tcgen05, FP16 hi/lo split).
//
// Same result as k_nn (Algorithm 1 NearestNeighbor over the frozen snapshot,
// Sec. IV-A, IV-B): for each query the eligible node (f-cost below the bound)
// with the smallest exact FP32 squared distance, the lowest index on a tie.
//
// A CTA takes 128 queries (one query block) and a chunk of whole 128-node half tiles of the
// packed operand copy.  Per half tile the tensor cores compute the filter
// a = |x - c|^2 - 2 (q - c).(x - c) (in coordinates scaled by P.tc_s) for all 128 x 128
// pairs into TMEM; reader warps take each row's minimum over groups of 16 nodes and remember
// the groups whose minimum lies within `band` of the row's running minimum (band = 2 * B, B
// the bound of tc_bound_coef on |a + |q - c|^2 - e|).  After the chunk, every node whose
// exact distance could be the row's minimum lies in a remembered group (its filter value is
// at most m1 + band), so recomputing e from the tree's FP32 coordinates on those groups gives
// the exact argmin; the whole CTA does that last step, sixteen threads per (row, group) pair,
// so that the loads of all groups are in flight together.  A row whose candidate ring
// overflowed or whose query lies outside the
// filter's range, or a tree flagged as leaving the box bound, is rescanned exactly by the
// whole CTA.  Chunk results merge with a 64-bit atomicMin of (distance bits << 32 | index),
// as in k_nn.  Since a differs from the distance by a per-query constant, the chunks also
// share a per-query minimum of a (W.nn_amin) and prune their candidates against it.
//
// Two CTAs share an SM, each with two accumulators of 128 TMEM columns.  Within a CTA the
// work is one dependency chain (MMA, commit, readers, release, next MMA) whose mbarrier
// hand-offs cost on the order of a hundred cycles each; the second CTA's MMAs fill the
// tensor pipe while the first waits on that chain.  With P.tc_pair_share > 0 (one full wave)
// the CTAs launched first and second are paired on one node range and the first takes that
// share of it: the second CTA on an SM streams slower.
//
// Roles (TcShape<D>::THREADS: 12 warps per CTA for d <= 8, 8 for larger d):
//   warp 0 lane 0   bulk-copies packed half tiles (T.XT) and f-costs into a ring of stages;
//   warp 1 lane 0   waits "stage masked" and the release of the accumulator the tile will use
//                   (tile t - 2's), then issues MMAS MMAs (M 128, N 128, K 16);
//   warps 2-3       mask ineligible rows (|x|^2 hi column := 2^15), then signal "stage masked";
//   warps 4-        read the accumulators' 16-node group minima with TMEM loads that reduce
//                   (tcgen05.ld.red min, sm_103a) and keep candidate rings: for d <= 8 two
//                   warps per TMEM lane quarter, 64 columns each (two reader threads per query
//                   row); for larger d one per quarter, all 128 columns.
// Every role, the MMA thread included, waits with the suspending mbarrier.try_wait: a hop
// takes about as long as with a polling test_wait, and the waits take no issue slots from the
// readers on the same scheduler.  Every wait is bounded (1 s of device time);
// on timeout the CTA sets ERR_TC_TIMEOUT and stops issuing work.  Before the CTA frees its
// TMEM and leaves, the loader waits (bounded) until every bulk copy it issued has landed and
// the MMA thread waits (bounded) on a final commit that follows every MMA it issued, so no
// asynchronous copy or MMA still writes shared memory or TMEM after the CTA is gone.
#include <cmath>

#include "pakr_device.cuh"
#include "pakr_tc.cuh"

namespace pakr {

// Exact FP32 distance of node j to the centred query qv, from the tree's coordinates
// (the same form and rounding as k_nn's exact_dist2), +inf if ineligible.
template <int D>
__device__ __forceinline__ float tc_exact(const DevProblem &P, const DevTree &T, int j, float bound, const float *qv)
{
    const float f = T.fcost[j];
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float xc = __fsub_rn(__fmul_rn(T.X[(size_t)a * P.cap + j], P.sw[a]), P.tc_c[a]);
        const float diff = __fadd_rn(qv[a], -xc);
        acc = (a == 0) ? __fmul_rn(diff, diff) : __fmaf_rn(diff, diff, acc);
    }
    return (f < bound) ? acc : __int_as_float(0x7f800000);
}

// Order-preserving map of a float onto unsigned (smaller float, smaller key), so that the
// per-query filter minimum over node chunks can use the integer atomicMin.
__device__ __forceinline__ unsigned tc_ord(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float tc_unord(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// grid (chunks, ceil(K / 128)), TcShape<D>::THREADS threads, TcShape<D>::SMEM_REQ dynamic shared memory;
// two CTAs per SM.  T.fcost must be readable 4 floats past the node count (the f-cost copy
// rounds up to 16 bytes).
template <int D>
__global__ void __launch_bounds__(TcShape<D>::THREADS, kTcCtasPerSm)
    k_nn_tc(DevProblem P, Ctl *__restrict__ ctl, DevTree T, DevWork W)
{
    using S = TcShape<D>;
    constexpr int KT = S::KT;
    constexpr int NST = S::NSTAGE;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *sA = tc_smem;
    unsigned char *sB0 = tc_smem + S::A_BYTES;
    float *sF0 = reinterpret_cast<float *>(tc_smem + S::A_BYTES + NST * S::STAGE_BYTES);
    float *ring_val = reinterpret_cast<float *>(tc_smem + S::A_BYTES + NST * (S::STAGE_BYTES + S::F_BYTES));
    int *ring_grp = reinterpret_cast<int *>(ring_val + kTcRing * S::READERS);
    __shared__ __align__(8) unsigned long long s_loaded[NST], s_full[NST], s_free[NST];
    __shared__ __align__(8) unsigned long long s_done[kTcAcc], s_empty[kTcAcc], s_drain;
    __shared__ uint32_t s_tbase;
    __shared__ volatile int s_abort;
    __shared__ int s_nflag, s_nres, s_flag_qid[kTcM], s_ovf[kTcM];
    __shared__ float s_flag_q[kTcM][D];

    const int n = ctl->n_start;
    if (n < P.tc_min_n)
        return;  // small trees take k_nn
    // the chunk: whole half tiles of 128 nodes
    const int ntile_all = (n + kTcBN - 1) / kTcBN;
    int tile0, ntiles, qblock;
    if (P.tc_pair_share > 0.f) {
        // One full wave, two CTAs per SM: the CTAs launched second (the upper half of the linear
        // block order) stream about 8 % slower than the first.  Each query block takes half of
        // its CTAs from each half, in pairs over one node range, split in favour of the first.
        const int lin = blockIdx.y * gridDim.x + blockIdx.x;
        const int n_first = (gridDim.x * gridDim.y) / 2;
        const bool later = lin >= n_first;
        const int r = later ? lin - n_first : lin;
        const int pairs = gridDim.x / 2;  // pairs per query block
        qblock = r / pairs;
        const int per_pair = (ntile_all + pairs - 1) / pairs;
        const int p0 = min(ntile_all, (r % pairs) * per_pair), p1 = min(ntile_all, p0 + per_pair);
        const int a = min(p1 - p0, (int)((float)(p1 - p0) * P.tc_pair_share + 0.5f));
        tile0 = later ? p0 + a : p0;
        ntiles = later ? p1 - p0 - a : a;
    } else {
        const int tiles_per = (ntile_all + gridDim.x - 1) / gridDim.x;
        tile0 = blockIdx.x * tiles_per;
        ntiles = min(ntile_all, tile0 + tiles_per) - tile0;
        qblock = blockIdx.y;
    }
    if (ntiles <= 0)
        return;
    const int start = tile0 * kTcBN;
    const int end = min(n, start + ntiles * kTcBN);
    const float bound = ctl->bound;
    const bool flagged = ctl->tc_flag != 0;
    const int K = P.K;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int qbase = qblock * kTcM;
    const unsigned long long kWaitNs = 1000000000ull;

    // ---- setup: TMEM, barriers, the query operand ----
    if (warp == kTcMmaWarp) {
        tmem_alloc(smem_u32(&s_tbase), kTcCols);
        tmem_relinquish();
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) {
            mbar_init(smem_u32(&s_loaded[i]), 1);
            mbar_init(smem_u32(&s_full[i]), 2);
            mbar_init(smem_u32(&s_free[i]), 1);
        }
#pragma unroll
        for (int i = 0; i < kTcAcc; ++i) {
            mbar_init(smem_u32(&s_done[i]), 1);
            mbar_init(smem_u32(&s_empty[i]), S::READERS / 32);
        }
        mbar_init(smem_u32(&s_drain), 1);
        fence_mbar_init();
        s_abort = 0;
        s_nflag = 0;
        s_nres = 0;
    }
    if (tid < kTcM) {
        s_ovf[tid] = 0;
        // query operand: -2 (q - c) split as hi (against x_hi), hi (against x_lo) and lo (against
        // x_hi), and kTcNormA twice against |x|^2 hi, lo.  Split layout: (hi, hi, n, n) over the
        // node row and (lo) in the second operand; joint layout: (hi, hi, lo, n, n) in one row.
        const int q = qbase + tid;
        float row[KT], row2[S::KA2 > 0 ? S::KA2 : 1];
#pragma unroll
        for (int k = 0; k < KT; ++k)
            row[k] = 0.f;
#pragma unroll
        for (int k = 0; k < (S::KA2 > 0 ? S::KA2 : 1); ++k)
            row2[k] = 0.f;
        // coordinates scaled by P.tc_s; a query farther than 2^9 from the centre in those units
        // (twice the box radius and more) could leave the range the error bound and the
        // eligibility threshold assume: its row is rescanned exactly instead
        float qn = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const float v = q < K ? (W.xr[(size_t)a * K + q] * P.sw[a] - P.tc_c[a]) * P.tc_s : 0.f;
            qn = __fmaf_rn(v, v, qn);
        }
        if (q < K && !(qn <= kTcQueryMax2)) {
            s_ovf[tid] = 1;
        } else if (q < K) {
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float v = -2.f * (W.xr[(size_t)a * K + q] * P.sw[a] - P.tc_c[a]) * P.tc_s;
                float hi, lo;
                tc_split_val(v, hi, lo);
                row[a] = hi;
                row[D + a] = hi;
                if constexpr (S::SPLIT)
                    row2[a] = lo;
                else
                    row[2 * D + a] = lo;
            }
            row[S::NORM] = kTcNormA;
            row[S::NORM + 1] = kTcNormA;
        }
#pragma unroll
        for (int c = 0; c < KT / kTcCoreK; ++c)
            *reinterpret_cast<uint4 *>(sA + tc_off<D>(tid, kTcCoreK * c)) = tc_chunk(row + kTcCoreK * c);
        if constexpr (S::SPLIT) {
#pragma unroll
            for (int c = 0; c < S::KA2 / kTcCoreK; ++c)
                *reinterpret_cast<uint4 *>(sA + S::A1_BYTES + tc_off2<D>(tid, kTcCoreK * c)) =
                    tc_chunk(row2 + kTcCoreK * c);
        }
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = s_tbase;

    // reader state: two reader threads per query row, one per 64-column half of the accumulator
    const int quarter = warp & 3, half = (warp - kTcReader0) >> 2;
    const int qrow = 32 * quarter + lane;
    const int e = tid - kTcReader0 * 32;  // ring column
    const int qid = qbase + qrow;
    float m1 = kTcEligible;
    int pos = 0, ovf = 0;
    float band = 0.f;

    if (flagged) {
        // the tree has a node outside the box bound: no filter; the block rescans exactly below
    } else if (warp == kTcLoadWarp) {
        if (lane == 0) {
            const uint32_t sB = smem_u32(sB0), sF = smem_u32(sF0);
            int issued = 0;
            for (int t = 0; t < ntiles && !s_abort; ++t) {
                const int b = t % NST;
                if (t >= NST && !mbar_wait_suspend(smem_u32(&s_free[b]), ((t - NST) / NST) & 1, kWaitNs)) {
                    s_abort = 1;
                    atomicOr(&ctl->err, ERR_TC_TIMEOUT);
                    break;
                }
                const int h = tile0 + t;  // global half-tile index
                const int j0 = h * kTcBN;
                const uint32_t fbytes = (uint32_t)(((min(kTcBN, end - j0) + 3) & ~3) * 4);
                const uint32_t bar = smem_u32(&s_loaded[b]);
                mbar_arrive_expect_tx(bar, (uint32_t)S::STAGE_BYTES + fbytes);
                bulk_g2s(sB + b * S::STAGE_BYTES,
                         reinterpret_cast<const unsigned char *>(T.XT) + (size_t)(h >> 1) * S::TILE_BYTES +
                             (size_t)(h & 1) * S::STAGE_BYTES,
                         S::STAGE_BYTES, bar);
                bulk_g2s(sF + b * S::F_BYTES, T.fcost + j0, fbytes, bar);
                issued = t + 1;
            }
            // Drain: every copy this lane issued has landed before the CTA can leave (after an
            // abort nobody may have waited for the last stages).  A stage is re-armed only after
            // its previous phase was consumed, so the last phase armed per stage is the only one
            // that can still be open.
            for (int t = issued > NST ? issued - NST : 0; t < issued; ++t)
                if (!mbar_wait_suspend(smem_u32(&s_loaded[t % NST]), (t / NST) & 1, kWaitNs)) {
                    s_abort = 1;
                    atomicOr(&ctl->err, ERR_TC_TIMEOUT);
                }
        }
        __syncwarp();
    } else if (warp >= kTcPatch0 && warp < kTcReader0) {
        const int r0 = tid - kTcPatch0 * 32;  // rows r0 and r0 + 64 of every stage
        for (int t = 0; t < ntiles; ++t) {
            const int b = t % NST;
            const bool ok = !s_abort && mbar_wait_suspend(smem_u32(&s_loaded[b]), (t / NST) & 1, kWaitNs);
            if (!ok && !s_abort) {
                s_abort = 1;
                atomicOr(&ctl->err, ERR_TC_TIMEOUT);
            }
            if (ok) {
                bool wrote = false;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = r0 + 64 * h;
                    const int j = start + t * kTcBN + r;
                    if (!(j < end && sF0[b * kTcBN + r] < bound)) {
                        unsigned char *rowp = sB0 + b * S::STAGE_BYTES;
                        tc_store_elem(rowp + tc_off<D>(r, S::NORM), kTcSentinel);
                        tc_store_elem(rowp + tc_off<D>(r, S::NORM + 1), 0.f);
                        wrote = true;
                    }
                }
                if (wrote)
                    fence_async_smem();
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(smem_u32(&s_full[b]));
        }
    } else if (warp == kTcMmaWarp) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_f16(kTcM, kTcBN);
            // descriptors of stage 0 and k-step 0; the start-address field (address / 16, 14 bits)
            // takes the stage and k-step offsets directly (shared addresses stay below 256 KB)
            const uint64_t adesc = smem_desc(smem_u32(sA), S::LBO, S::SBO);
            const uint64_t adesc2 = S::SPLIT ? smem_desc(smem_u32(sA + S::A1_BYTES), S::LBO, S::SBO2) : 0ull;
            const uint64_t bdesc = smem_desc(smem_u32(sB0), S::LBO, S::SBO);
            // no per-tile poll of the abort flag (a shared-memory load that queues behind the
            // tile traffic): the masking warps signal every stage even after an abort, and a
            // wait that times out (also the release wait, once the readers have stopped) ends
            // the loop
            const uint32_t full0 = smem_u32(&s_full[0]), free0 = smem_u32(&s_free[0]);
            const uint32_t done0 = smem_u32(&s_done[0]), empty0 = smem_u32(&s_empty[0]);
            uint32_t st8 = 0, fpar = 0;  // stage * 8 (mbarrier byte offset), its phase parity
            uint64_t bd = bdesc;
            uint32_t epar = 0;  // phase parity of the accumulators' release barriers
            // two tiles per trip, one per accumulator, so that the accumulator is a constant
            for (int t = 0; t < ntiles; t += kTcAcc) {
                bool live = true;
#pragma unroll
                for (int ac = 0; ac < kTcAcc; ++ac) {
                    if (!live || t + ac >= ntiles)
                        break;
                    // the accumulator has been read (tile t + ac - 2's; usually the longer wait,
                    // so it comes first), and the stage is masked
                    if ((t > 0 && !mbar_wait_suspend(empty0 + 8 * ac, epar ^ 1u, kWaitNs)) ||
                        !mbar_wait_suspend(full0 + st8, fpar, kWaitNs)) {
                        s_abort = 1;
                        atomicOr(&ctl->err, ERR_TC_TIMEOUT);
                        live = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tbase + (uint32_t)(ac * kTcBN);
                    mma_f16_ss_c<false>(dt, adesc, bd, idesc);
#pragma unroll
                    for (int s = 1; s < KT / kTcKStep; ++s)
                        mma_f16_ss_c<true>(dt, adesc + (uint64_t)((2 * S::LBO * s) >> 4),
                                       bd + (uint64_t)((2 * S::LBO * s) >> 4), idesc);
                    // split layout: the lo part of the query against the x_hi columns
#pragma unroll
                    for (int s = 0; s < S::KA2 / kTcKStep; ++s)
                        mma_f16_ss_c<true>(dt, adesc2 + (uint64_t)((2 * S::LBO * s) >> 4),
                                       bd + (uint64_t)((2 * S::LBO * s) >> 4), idesc);
                    mma_commit(free0 + st8);
                    mma_commit(done0 + 8 * ac);
                    st8 += 8;
                    bd += (uint64_t)(S::STAGE_BYTES >> 4);
                    if (st8 == 8 * NST) {
                        st8 = 0;
                        fpar ^= 1u;
                        bd = bdesc;
                    }
                }
                if (!live)
                    break;
                epar ^= 1u;
            }
            // Drain: a final commit completes once every MMA issued above has finished, so no MMA
            // still writes the accumulators when TMEM is freed, also after an abort that left
            // accumulators unread.
            mma_commit(smem_u32(&s_drain));
            if (!mbar_wait_suspend(smem_u32(&s_drain), 0, kWaitNs)) {
                s_abort = 1;
                atomicOr(&ctl->err, ERR_TC_TIMEOUT);
            }
        }
        __syncwarp();
    } else if (warp >= kTcReader0) {
        // the query's coordinates are needed here for the band only, and again by the resolve:
        // they are recomputed there rather than kept in registers through the tile loop
        float qc2 = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const float v = (qid < K) ? __fsub_rn(__fmul_rn(W.xr[(size_t)a * K + qid], P.sw[a]), P.tc_c[a]) : 0.f;
            qc2 = __fmaf_rn(v, v, qc2);
        }
        const float Rq = (sqrtf(qc2) * 1.0001f + sqrtf(P.tc_xbox2)) * P.tc_s;
        band = 2.f * tc_bound_coef<D>() * Rq * Rq;
        float thr = kTcEligible;
        // The filter value a differs from the distance by a per-query constant, so minima from
        // other node chunks prune this chunk's candidates too: every 32 tiles the running
        // minimum is published (a fire-and-forget atomicMin) and the shared one is read back,
        // to be used one period later so that the load never stalls the loop.
        const bool pub = W.nn_amin != nullptr && qid < K && !s_ovf[qrow];  // (a row out of range publishes nothing)
        unsigned gkey = 0xFFFFFFFFu;
        constexpr int CW = kTcBN / S::RH;  // accumulator columns of this reader
        constexpr int NG = CW / kTcG;      // 16-node groups it reduces per tile
        const uint32_t tcol0 = tbase + (uint32_t)(CW * half) + ((uint32_t)(32 * quarter) << 16);
        uint32_t dpar = 0;  // phase parity of the accumulators' ready barriers
        // two tiles per trip, one per accumulator, so that the accumulator is a constant
        for (int t0 = 0; t0 < ntiles; t0 += kTcAcc) {
            bool stop = false;
#pragma unroll
            for (int b = 0; b < kTcAcc; ++b) {
                const int t = t0 + b;
                if (t >= ntiles)
                    break;
                const bool ok = __all_sync(0xFFFFFFFFu, mbar_wait_suspend(smem_u32(&s_done[b]), dpar, kWaitNs));
                if (!ok) {
                    if (lane == 0) {
                        s_abort = 1;
                        atomicOr(&ctl->err, ERR_TC_TIMEOUT);
                    }
                    stop = true;
                    break;
                }
                tc_fence_after();
                // minima of this reader's 16-node groups, then the accumulator is released; one
                // branch per tile (the candidate test rarely passes once the running minimum has
                // settled); the group minima come straight from the TMEM loads (min reduction,
                // sm_103a): one load per 16-node group, no ALU work on the values
                float m[NG];
                tmem_ldred_groups<NG, S::LD_BATCH>(tcol0 + (uint32_t)(b * kTcBN), m);
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(smem_u32(&s_empty[b]));
                if ((t & 31) == 31 && pub) {
                    const float g = tc_unord(gkey);  // the value read one period ago
                    if (g < m1)
                        thr = fminf(thr, g + band);
                    if (m1 < kTcEligible)
                        atomicMin(W.nn_amin + qid, tc_ord(m1));
                    gkey = __ldcg(W.nn_amin + qid);
                }
                float mm = m[0];
#pragma unroll
                for (int h = 1; h < NG; ++h)
                    mm = fminf(mm, m[h]);
                if (mm <= thr) {
#pragma unroll
                    for (int h8 = 0; h8 < NG; ++h8) {
                        if (m[h8] <= thr) {
                            if (m[h8] < m1) {
                                m1 = m[h8];
                                thr = fminf(thr, m1 + band);
                            }
                            const int slot = pos & (kTcRing - 1);
                            // an entry still within the band would be lost: the row falls back to a rescan
                            if (pos >= kTcRing && ring_val[slot * S::READERS + e] <= thr)
                                ovf = 1;
                            ring_val[slot * S::READERS + e] = m[h8];
                            ring_grp[slot * S::READERS + e] = start + t * kTcBN + CW * half + 16 * h8;
                            ++pos;
                        }
                    }
                }
            }
            if (stop)
                break;
            dpar ^= 1u;
        }
        if (pub && m1 < kTcEligible)
            atomicMin(W.nn_amin + qid, tc_ord(m1));
        if (ovf)
            s_ovf[qrow] = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kTcMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tbase, kTcCols);
    }
    if (s_abort)
        return;

    // ---- exact resolve of the candidate groups, by the whole CTA ----
    // Every CTA resolves at the same moment, so the resolve is latency: the surviving (row,
    // group) pairs go to one list, and sixteen threads take each pair, one node each, so that
    // all the groups' loads are in flight together.  The list lives in the stages, free now
    // (every copy has landed and every MMA has finished).
    int2 *rlist = reinterpret_cast<int2 *>(sB0);
    if (!flagged && warp >= kTcReader0 && qid < K && (m1 < kTcEligible || s_ovf[qrow])) {
        // against the smallest filter value any chunk has published by now (this chunk's
        // included): groups above it by more than the band cannot hold the nearest node
        const float thrf = (W.nn_amin ? fminf(m1, tc_unord(__ldcg(W.nn_amin + qid))) : m1) + band;
        // a row either of whose readers lost a candidate is rescanned instead (once)
        if (!s_ovf[qrow]) {
            const int np = min(pos, kTcRing);
#pragma unroll 1
            for (int s = 0; s < np; ++s)
                if (ring_val[s * S::READERS + e] <= thrf)
                    rlist[atomicAdd(&s_nres, 1)] = make_int2(qrow, ring_grp[s * S::READERS + e]);
        } else if (half == 0) {
            const int slot = atomicAdd(&s_nflag, 1);
            s_flag_qid[slot] = qid;
#pragma unroll
            for (int a = 0; a < D; ++a)
                s_flag_q[slot][a] = __fsub_rn(__fmul_rn(W.xr[(size_t)a * K + qid], P.sw[a]), P.tc_c[a]);
        }
    }
    if (flagged && tid < kTcM) {
        // every query of the block is rescanned exactly
        const int q = qbase + tid;
        if (q < K) {
            const int slot = atomicAdd(&s_nflag, 1);
            s_flag_qid[slot] = q;
#pragma unroll
            for (int a = 0; a < D; ++a)
                s_flag_q[slot][a] = __fsub_rn(__fmul_rn(W.xr[(size_t)a * K + q], P.sw[a]), P.tc_c[a]);
        }
    }
    __syncthreads();
    {
        // sixteen threads per (row, group), node g0 + k for thread k; the two halves of a warp take
        // neighbouring pairs and run the same trips, so that the shuffles stay warp-uniform
        const int nres = s_nres;
        const int sub = lane & (kTcG - 1);
        for (int base = 2 * warp; base < nres; base += S::THREADS / kTcG) {
            const int it = base + (lane >> 4);
            unsigned long long key = kNoKey;
            int q = 0;
            if (it < nres) {
                const int2 item = rlist[it];
                q = qbase + item.x;
                const int j = item.y + sub;
                if (j < end) {
                    float qv2[D];
#pragma unroll
                    for (int a = 0; a < D; ++a)
                        qv2[a] = __fsub_rn(__fmul_rn(W.xr[(size_t)a * K + q], P.sw[a]), P.tc_c[a]);
                    const float ed = tc_exact<D>(P, T, j, bound, qv2);
                    if (ed < __int_as_float(0x7f800000))
                        key = ((unsigned long long)__float_as_uint(ed) << 32) | (unsigned long long)(uint32_t)j;
                }
            }
#pragma unroll
            for (int o = kTcG / 2; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, key, o);
                key = other < key ? other : key;
            }
            if (sub == 0 && key != kNoKey)
                atomicMin(&W.nn_key[q], key);
        }
    }
    // exact rescans of the flagged queries by the whole block (coalesced nodes, warp minimum of packed keys)
    const int nflag = s_nflag;
    for (int f = 0; f < nflag; ++f) {
        float q2[D];
#pragma unroll
        for (int a = 0; a < D; ++a)
            q2[a] = s_flag_q[f][a];
        unsigned long long key = kNoKey;
        for (int j = start + tid; j < end; j += S::THREADS) {
            const float ed = tc_exact<D>(P, T, j, bound, q2);
            if (ed < __int_as_float(0x7f800000)) {
                const unsigned long long k2 =
                    ((unsigned long long)__float_as_uint(ed) << 32) | (unsigned long long)(uint32_t)j;
                key = k2 < key ? k2 : key;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, key, o);
            key = other < key ? other : key;
        }
        if (lane == 0 && key != kNoKey)
            atomicMin(&W.nn_key[s_flag_qid[f]], key);
    }
}

template <int D>
__global__ void k_tc_pack(DevProblem P, Ctl *ctl, DevTree T, int count)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count)
        return;
    float x[D];
#pragma unroll
    for (int a = 0; a < D; ++a)
        x[a] = T.X[(size_t)a * P.cap + j];
    tc_pack_node<D>(P, T, ctl, j, x);
}

template <int D>
static cudaError_t launch_nn_tc_d(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W,
                                  const LaunchCfg &L, cudaStream_t s)
{
    k_nn_tc<D><<<dim3(L.tc_chunks, L.tc_qblocks), TcShape<D>::THREADS, TcShape<D>::SMEM_REQ, s>>>(P, ctl, T, W);
    return cudaGetLastError();
}

template <int D>
static cudaError_t tc_configure_d()
{
    return cudaFuncSetAttribute(k_nn_tc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<D>::SMEM_REQ);
}

// Once per device before the first launch (outside any stream capture): the kernel
// takes more than 48 KB of dynamic shared memory.
cudaError_t tc_configure(const DevProblem &P)
{
    PAKR_DISPATCH_DYN(P.dyn, return tc_configure_d<Dims<DYN_>::D>());
    return cudaSuccess;
}

cudaError_t launch_nn_tc(const DevProblem &P, Ctl *ctl, const DevTree &T, const DevWork &W, const LaunchCfg &L,
                         cudaStream_t s)
{
    PAKR_DISPATCH_DYN(P.dyn, return launch_nn_tc_d<Dims<DYN_>::D>(P, ctl, T, W, L, s));
    return cudaSuccess;
}

cudaError_t launch_tc_pack(const DevProblem &P, Ctl *ctl, const DevTree &T, int count, cudaStream_t s)
{
    if (!T.XT || count <= 0)
        return cudaSuccess;
    PAKR_DISPATCH_DYN(P.dyn, (k_tc_pack<Dims<DYN_>::D><<<(count + 255) / 256, 256, 0, s>>>(P, ctl, T, count)));
    return cudaGetLastError();
}

int tc_operand_floats(int d)
{
    return tc_node_cols(d) * kTcElem / 4;
}

float tc_scale(float xbox2)
{
    int e = 0;
    std::frexp(std::sqrt((double)xbox2), &e);  // radius = m 2^e, m in [0.5, 1)
    return (float)std::ldexp(1.0, 8 - e);      // radius * scale = m 2^8 in [2^7, 2^8)
}

}  // namespace pakr
