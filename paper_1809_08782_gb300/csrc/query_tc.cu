// Query probing and re-rank on 5th-generation tensor cores (Section 3.3
// multi-probe with the exact re-rank of Eq. 1, batched over queries).
//
// Every (query, item) pair of a probed sub-dataset is handled as one entry of
// a dense product of a 128-query tile with 128-item tiles of S_j:
//
//   match counts  l(q, x) = (L + s_q . s_x) / 2, with s the +-1 sign vectors of
//                 the L code bits (bf16, zero past L).  The products and their
//                 sum (|s_q . s_x| <= 64) are exact in the FP32 accumulator, so
//                 l is exact: the same number as L - popcount(c_q xor c_x).
//   scores        q~ . x~ with q~ = q rounded to bf16 and x~ the bf16 items
//                 (fp32 items: rounded to bf16), FP32 accumulation; the interval
//                 [s - e, s + e], e = a_q ||x|| (a_q from the query's own bf16
//                 rounding error, query_bound_kernel), holds the FP64 score.
//
// Two epilogues share the kernel:
//   HIST     H[q][j][l] += 1 for every pair (private shared-memory counters per
//            query row, written out once per work item);
//   RERANK   a pair is a candidate when l >= lam_j(q), or it lies in the
//            boundary bucket (j*, l*) at a position <= pcut(q) (the r-th such
//            item); candidates are written with their score interval into the
//            query's list at offsets fixed beforehand from the histogram, so the
//            top-k pass sees exactly the probed items of Section 3.3.
//
// Persistent warp-specialised CTAs (320 threads, one per SM):
//   warp 0     one thread issues TMA loads: the query tile's operands once per
//              work item, then a ring of 16 KB stages (128 items x 64 K each);
//   warp 1     allocates 512 TMEM columns (two buffers of a 128-column score and a
//              128-column sign accumulator) and one thread issues tcgen05.mma
//              (M = 128 queries, N = 128 items, K = 16);
//   warps 2-9  read the accumulators (warp w: TMEM lanes 32 (w % 4).., columns
//              64 h.. with h = (w - 2) / 4) and run the epilogue.
// Every mbarrier wait is bounded; on a timeout the kernel records an error,
// stops issuing work, lets its own copies and MMAs land, frees TMEM and returns.
// The epilogue warps meet at named barriers a fixed number of times whatever
// happens, so an aborted run cannot leave one of them waiting.
#include "nrlsh_internal.cuh"
#include "tc_ops.cuh"

#include <algorithm>

namespace nrlsh {

using namespace tc;

namespace {

constexpr int kPM = 128;                  // queries per work item (MMA M)
constexpr int kPN = 128;                  // items per tile (MMA N)
constexpr uint32_t kChunk = 128 * 128;    // one 128-row x 64-element bf16 operand chunk
constexpr int kEpiWarps = 8;
constexpr int kPThreads = 32 * (2 + kEpiWarps);
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr uint32_t kTmemCols = 512;       // 2 buffers x (128 score + 128 sign columns)
constexpr int kMaxStages = 8;
constexpr int kWorkRing = 4;              // work items in flight between the roles

struct PairsArgs {
    const uint32_t* list;       // work items (j * nqt + query tile); null: all m * nqt
    const uint32_t* nlist;      // number of entries of list (device)
    int nwork_all;
    const int64_t* seg;         // m + 1 storage offsets
    int m, L, nqt, nkc, d, stages;
    int64_t nq;
    uint32_t* H;                // HIST: nq x m x (L + 1)
    const uint8_t* lam;         // RERANK: nq x m
    const uint32_t* off;        // nq x (m + 1) list offsets
    const TcBoundary* tb;       // nq
    const float* xnorm;         // n, storage order
    const float* qce;           // nq: a_q of the score interval
    uint32_t* cand;             // nq x cap
    float* lo;
    float* hi;
    int64_t cap;
    int* err;
    uint32_t* work_ctr;         // work items handed out so far (zeroed before the launch)
    uint32_t spin_first;        // polls of the MMA thread's first wait for a stage
};

// The histogram kernel's sign accumulators start at 1.5 2^23 instead of 0 (the
// epilogue writes that value back into each accumulator it has read), so the
// accumulated f = 1.5 2^23 + v, v = s_q . s_x an integer of L's parity in [-L, L],
// is exact and its bits are 0x4B400000 + v.  The counter of l = (L + v) / 2 in the
// [l][half][row] counters (1,024 bytes per l) is then at bits * 512 + k, k folding
// in the half, the row, the counters' base and L.  The unsigned min with the last
// counter keeps any value inside this CTA's shared memory.
constexpr uint32_t kSignBias = 0x4B400000u;   // 1.5 2^23 as an fp32 bit pattern

__device__ __forceinline__ uint32_t hist_addr(uint32_t fbits, uint32_t k, uint32_t last) {
    return min(fbits * 512u + k, last);
}

__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
}

template <bool kRerank>
__global__ void __launch_bounds__(kPThreads, 1)
    pairs_tc_kernel(const __grid_constant__ CUtensorMap map_qb,
                    const __grid_constant__ CUtensorMap map_qs,
                    const __grid_constant__ CUtensorMap map_xb,
                    const __grid_constant__ CUtensorMap map_xs, const __grid_constant__ PairsArgs a) {
    NRLSH_PDL_ENTRY();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int na = kRerank ? a.nkc + 1 : 1;     // operand chunks of the query tile
    const int nb = kRerank ? a.nkc + 1 : 1;     // operand chunks per item tile
    const int S = a.stages;
    uint8_t* a_tile = base;                     // na chunks; the sign chunk last
    uint8_t* ring = base + (size_t)na * kChunk;
    uint64_t* full = (uint64_t*)(ring + (size_t)S * kChunk);
    uint64_t* empty = full + S;
    uint64_t* acc_full = empty + S;             // 2
    uint64_t* acc_empty = acc_full + 2;         // 2
    uint64_t* a_full = acc_empty + 2;
    uint64_t* a_empty = a_full + 1;
    uint64_t* drain = a_empty + 1;
    uint64_t* wq_full = drain + 1;              // kWorkRing: a work item is published
    uint64_t* wq_empty = wq_full + kWorkRing;   // kWorkRing: the MMA thread and the
                                                // epilogue leader have read it
    volatile int* wq_item = (volatile int*)(wq_empty + kWorkRing);
    volatile int* epi_item = wq_item + kWorkRing;
    uint32_t* tmem_slot = (uint32_t*)(wq_item + kWorkRing + 4);
    volatile int* abort_s = (volatile int*)(tmem_slot + 1);
    uint32_t* extra = (uint32_t*)(tmem_slot + 4);
    // HIST: counters [l][half][row]; RERANK: staged xnorm [warp][64], counts
    // [2][128] and per-warp 32 x 33 transposition buffers
    uint32_t* hist = extra;
    float* xn_s = (float*)extra;
    uint32_t* cnt_x = extra + kEpiWarps * 64;
    float* tr_s = (float*)(cnt_x + 2 * kPM);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int nwork_s;

    if (threadIdx.x == 0) {
        // an earlier kernel of the call stopped early: its outputs are not to be used
        nwork_s = *a.err ? 0 : (a.list ? (int)*a.nlist : a.nwork_all);
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiThreads);
        }
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        mbar_init(drain, 1);
        for (int r = 0; r < kWorkRing; ++r) {
            mbar_init(&wq_full[r], 1);
            mbar_init(&wq_empty[r], 2);
        }
        *abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (!kRerank && warp >= 2)
        for (int i = threadIdx.x - 64; i < (a.L + 1) * 2 * kPM; i += kEpiThreads) hist[i] = 0;
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int nwork = nwork_s;            // one value for every role
    if (!kRerank) {
        // the sign accumulators of both buffers start at the bias (see hist_addr)
        if (warp >= 2) {
            const uint32_t la = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) +
                                128u + 64u * (uint32_t)((warp - 2) >> 2);
            for (int b = 0; b < 2; ++b) {
                tmem_fill32(la + 256u * b, kSignBias);
                tmem_fill32(la + 256u * b + 32u, kSignBias);
            }
            tmem_wait_st();
        }
        fence_before();
        __syncthreads();
        fence_after();
    }

    // Work items are handed out dynamically: the producer thread claims the next
    // index from the global counter and publishes it in the ring; the MMA thread
    // and the epilogue take the same sequence.  Indices run from the end of the
    // (sub-dataset major, ascending) order, so the highest-norm sub-datasets,
    // whose tiles hold the most candidates, start first.
    auto decode = [&](int i, int& j, int& qt, int64_t& p0, int& ntile) {
        const int ir = nwork - 1 - i;
        const uint32_t w = a.list ? a.list[ir] : (uint32_t)ir;
        j = (int)(w / (uint32_t)a.nqt);
        qt = (int)(w % (uint32_t)a.nqt);
        p0 = a.seg[j];
        ntile = (int)ceil_div(a.seg[j + 1] - p0, kPN);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer
            int stage = 0;
            uint32_t phase = 0, a_round = 0;
            int issued[kMaxStages];
            uint32_t issued_par[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) issued[s] = 0, issued_par[s] = 0;
            int a_issued = 0;
            for (int k = 0;; ++k) {
                const int rs = k % kWorkRing;
                int item = -1;
                if (!*abort_s) {
                    if (k >= kWorkRing && !mbar_wait(&wq_empty[rs], ((k / kWorkRing) - 1) & 1)) {
                        atomicCAS(a.err, 0, 16);
                        *abort_s = 1;
                    } else {
                        const uint32_t c = atomicAdd(a.work_ctr, 1u);
                        if (c < (uint32_t)nwork) item = (int)c;
                    }
                }
                wq_item[rs] = item;
                mbar_arrive(&wq_full[rs]);
                if (item < 0) break;
                int j, qt, ntile;
                int64_t p0;
                decode(item, j, qt, p0, ntile);
                if (ntile == 0) continue;
                if (!mbar_wait(a_empty, (a_round & 1) ^ 1)) {
                    atomicCAS(a.err, 0, 11);
                    *abort_s = 1;
                    break;
                }
                mbar_expect_tx(a_full, (uint32_t)na * kChunk);
                if (kRerank)
                    for (int c = 0; c < a.nkc; ++c)
                        tma_load_2d(a_tile + (size_t)c * kChunk, &map_qb, a_full, 64 * c, qt * kPM);
                tma_load_2d(a_tile + (size_t)(na - 1) * kChunk, &map_qs, a_full, 0, qt * kPM);
                a_issued = 1;
                ++a_round;
                for (int t = 0; t < ntile && !*abort_s; ++t) {
                    const int row = (int)(p0 + (int64_t)t * kPN);
                    for (int c = 0; c < nb; ++c) {
                        if (!mbar_wait(&empty[stage], phase ^ 1)) {
                            atomicCAS(a.err, 0, 12);
                            *abort_s = 1;
                            break;
                        }
                        mbar_expect_tx(&full[stage], kChunk);
                        uint8_t* dst = ring + (size_t)stage * kChunk;
                        if (c < nb - 1)
                            tma_load_2d(dst, &map_xb, &full[stage], 64 * c, row);
                        else
                            tma_load_2d(dst, &map_xs, &full[stage], 0, row);
                        issued[stage] = 1;
                        issued_par[stage] = phase;
                        if (++stage == S) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                }
            }
            if (*abort_s) {
                // let every copy in flight land before the CTA's memory goes away
                if (a_issued) mbar_wait(a_full, (a_round - 1) & 1);
                for (int s = 0; s < S; ++s)
                    if (issued[s]) mbar_wait(&full[s], issued_par[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t idesc = umma_idesc(kPM, kPN);
            const int ks_sign = (a.L + 15) / 16;
            int stage = 0, buf = 0;
            uint32_t phase = 0, acc_phase = 0, a_round = 0;
            bool ok = true, first = true;
            for (int k = 0; ok; ++k) {
                const int rs = k % kWorkRing;
                if (*abort_s || !mbar_wait(&wq_full[rs], (k / kWorkRing) & 1)) {
                    ok = false;
                    break;
                }
                const int item = wq_item[rs];
                mbar_arrive(&wq_empty[rs]);
                if (item < 0) break;
                int j, qt, ntile;
                int64_t p0;
                decode(item, j, qt, p0, ntile);
                if (ntile == 0) continue;
                if (!mbar_wait(a_full, a_round & 1)) {
                    ok = false;
                    break;
                }
                ++a_round;
                fence_after();
                for (int t = 0; ok && t < ntile; ++t) {
                    if (*abort_s || !mbar_wait(&acc_empty[buf], acc_phase ^ 1)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t d_score = tmem_base + (uint32_t)buf * 256;
                    const uint32_t d_sign = d_score + 128;
                    for (int c = 0; c < nb; ++c) {
                        const uint32_t lim = first ? a.spin_first : kSpinLimit;
                        first = false;
                        if (!mbar_wait(&full[stage], phase, lim)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint64_t bdesc = sw128_desc(ring + (size_t)stage * kChunk);
                        if (c < nb - 1) {
                            // score chunk c: K = 64 c .. 64 c + 63, only the steps below d
                            const uint64_t adesc = sw128_desc(a_tile + (size_t)c * kChunk);
                            const int ks = min(4, (a.d - 64 * c + 15) / 16);
                            for (int k = 0; k < ks; ++k)
                                umma_bf16(d_score, adesc + 2 * k, bdesc + 2 * k, idesc, (c | k) != 0);
                        } else {
                            // (histograms: accumulate onto the bias left by the epilogue)
                            const uint64_t adesc = sw128_desc(a_tile + (size_t)(na - 1) * kChunk);
                            for (int k = 0; k < ks_sign; ++k)
                                umma_bf16(d_sign, adesc + 2 * k, bdesc + 2 * k, idesc,
                                          !kRerank || k != 0);
                        }
                        umma_commit(&empty[stage]);
                        if (++stage == S) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                    if (!ok) break;
                    umma_commit(&acc_full[buf]);
                    if (++buf == 2) {
                        buf = 0;
                        acc_phase ^= 1;
                    }
                }
                umma_commit(a_empty);
            }
            if (!ok) {
                atomicCAS(a.err, 0, 13);
                *abort_s = 1;
            }
            // every MMA this thread issued has finished before TMEM is freed
            umma_commit(drain);
            mbar_wait(drain, 0);
        }
    } else {
        // ---- epilogue: warps 2..9
        const int quad = warp & 3, half = (warp - 2) >> 2;
        const int row = 32 * quad + lane;       // query row of the tile
        const int et = threadIdx.x - 64;        // epilogue thread index
        const int col_lo = 64 * half;
        const unsigned lt = (1u << lane) - 1u;
        float* xn_w = xn_s + (warp - 2) * 64;
        float* tr_w = tr_s + (warp - 2) * 32 * 33;
        const uint32_t lane_addr = (uint32_t)(32 * quad) << 16;
        int buf = 0;
        uint32_t acc_phase = 0;
        bool aborted = false;
        for (int k = 0;; ++k) {
            // one leader takes the next item (a bounded wait) and the 256 epilogue
            // threads meet once, so all of them follow the same sequence of items
            if (et == 0) {
                const int rs = k % kWorkRing;
                int item = -1;
                if (!*abort_s) {
                    if (mbar_wait(&wq_full[rs], (k / kWorkRing) & 1)) {
                        item = wq_item[rs];
                    } else {
                        atomicCAS(a.err, 0, 17);
                        *abort_s = 1;
                    }
                }
                *epi_item = item;
                mbar_arrive(&wq_empty[rs]);
            }
            epi_sync();
            const int item = *epi_item;     // read before the item's closing barriers
            if (item < 0) break;
            int j, qt, ntile;
            int64_t p0;
            decode(item, j, qt, p0, ntile);
            const int64_t q = (int64_t)qt * kPM + row;
            const bool qv = q < a.nq;
            const int64_t p1 = a.seg[j + 1];
            // per (query, sub-dataset) state of the candidate test; slots are
            // relative to the query's list (half 0 fills forward from the front of
            // the sub-dataset's range, half 1 backward from its end)
            float thrf = 3.0e38f, thrb = 3.0e38f, ce = 0.0f;
            int64_t pcut = -1;
            int32_t base_j = 0, cnt_j = 0, slot = -1;
            if (kRerank && qv) {
                thrf = (float)(2 * (int)a.lam[q * a.m + j] - a.L);
                const TcBoundary b = a.tb[q];
                if (b.j == j) {
                    thrb = (float)(2 * b.l - a.L);
                    pcut = b.pcut;
                }
                base_j = (int32_t)a.off[q * (a.m + 1) + j];
                cnt_j = (int32_t)(a.off[q * (a.m + 1) + j + 1] - (uint32_t)base_j);
                slot = half == 0 ? base_j : base_j + cnt_j - 1;
                ce = a.qce[q];
            }
            bool overflow = false;
            const uint32_t hist_k = smem_u32(hist) + 4u * (uint32_t)(half * kPM + row) +
                                    ((uint32_t)a.L - kSignBias) * 512u;
            const uint32_t hist_last = smem_u32(hist) + (uint32_t)(a.L + 1) * 2u * kPM * 4u - 4u;
            // the norms of the first tile's columns; each tile then fetches the next's
            float xn_next[2] = {0.0f, 0.0f};
            if (kRerank && ntile > 0) {
                for (int c2 = 0; c2 < 2; ++c2) {
                    const int c = col_lo + 32 * c2 + lane;
                    xn_next[c2] = p0 + c < p1 ? a.xnorm[p0 + c] : 0.0f;
                }
            }
            for (int t = 0; t < ntile; ++t) {
                const int64_t pos0 = p0 + (int64_t)t * kPN;
                const int ncols = (int)min((int64_t)kPN, p1 - pos0);
                if (kRerank) {
                    __syncwarp();
                    xn_w[lane] = xn_next[0];
                    xn_w[32 + lane] = xn_next[1];
                    __syncwarp();
                    const int64_t pn = pos0 + kPN;
                    for (int c2 = 0; c2 < 2; ++c2) {
                        const int c = col_lo + 32 * c2 + lane;
                        xn_next[c2] = t + 1 < ntile && pn + c < p1 ? a.xnorm[pn + c] : 0.0f;
                    }
                }
                if (!aborted && (*abort_s || !mbar_wait(&acc_full[buf], acc_phase))) {
                    aborted = true;
                    atomicCAS(a.err, 0, 14);
                    *abort_s = 1;
                }
                fence_after();
                const uint32_t t_score = tmem_base + lane_addr + (uint32_t)buf * 256;
                const uint32_t t_sign = t_score + 128;
                if (!kRerank) {
                    // both 32-column groups of this warp's half, then the counters
                    if (!aborted) {
                        uint32_t sg0[32], sg1[32];
                        tmem_ld32_nowait(t_sign + (uint32_t)col_lo, sg0);
                        tmem_ld32_nowait(t_sign + (uint32_t)(col_lo + 32), sg1);
                        tmem_wait_ld();
                        // the bias back in for the MMA that reuses this buffer
                        tmem_fill32(t_sign + (uint32_t)col_lo, kSignBias);
                        tmem_fill32(t_sign + (uint32_t)(col_lo + 32), kSignBias);
                        const int lim0 = min(32, ncols - col_lo), lim1 = min(32, ncols - col_lo - 32);
                        // (every index below is a constant after unrolling, so the
                        // values stay in registers; the ragged tail is predicated)
                        if (qv) {
                            if (lim0 == 32 && lim1 == 32) {
#pragma unroll
                                for (int ii = 0; ii < 32; ++ii) {
                                    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(
                                        hist_addr(sg0[ii], hist_k, hist_last)));
                                    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(
                                        hist_addr(sg1[ii], hist_k, hist_last)));
                                }
                            } else {
#pragma unroll
                                for (int ii = 0; ii < 32; ++ii) {
                                    if (ii < lim0)
                                        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(
                                            hist_addr(sg0[ii], hist_k, hist_last)));
                                    if (ii < lim1)
                                        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(
                                            hist_addr(sg1[ii], hist_k, hist_last)));
                                }
                            }
                        }
                        tmem_wait_st();
                    }
                } else {
                    for (int g = 0; g < 2 && !aborted; ++g) {
                        const int col = col_lo + 32 * g;
                        if (col >= ncols) break;                   // warp-uniform
                        const int lim = min(32, ncols - col);
                        uint32_t sg[32], sc[32];
                        tmem_ld32_nowait(t_sign + (uint32_t)col, sg);
                        tmem_ld32_nowait(t_score + (uint32_t)col, sc);
                        tmem_wait_ld();
                        // this lane's candidates among the group's columns, as a mask:
                        // the buckets probed whole, then (only in warps where some
                        // lane's boundary bucket reaches into the group) the cut of
                        // the boundary bucket
                        const int64_t pc64 = pcut - (pos0 + col);
                        const int pc = (int)max((int64_t)-1, min((int64_t)31, pc64));
                        // (four independent partial masks: no 32-long dependency chain)
                        uint32_t mp[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                        for (int ii = 0; ii < 32; ++ii)
                            mp[ii & 3] |= (uint32_t)(__uint_as_float(sg[ii]) >= thrf) << ii;
                        const bool bact = thrb < 1.0e30f && pc >= 0;
                        if (__any_sync(0xffffffffu, bact) && bact) {
#pragma unroll
                            for (int ii = 0; ii < 32; ++ii)
                                mp[ii & 3] |= (uint32_t)(__uint_as_float(sg[ii]) == thrb && ii <= pc)
                                              << ii;
                        }
                        uint32_t msk = (mp[0] | mp[1]) | (mp[2] | mp[3]);
                        if (lim < 32) msk &= (1u << lim) - 1u;
                        if (!qv) msk = 0;
                        const int cnt = __popc(msk);
                        // room in this half's share of the query's range
                        const bool room = half == 0 ? slot + cnt <= base_j + cnt_j
                                                    : slot - cnt + 1 >= base_j;
                        if (!room && cnt) {
                            overflow = true;
                            msk = 0;
                        }
                        const int tot = __reduce_add_sync(0xffffffffu, room ? cnt : 0);
                        if (tot == 0) continue;
                        // the scores through shared memory (row stride 33: no bank
                        // conflicts either way)
#pragma unroll
                        for (int ii = 0; ii < 32; ++ii) tr_w[lane * 33 + ii] = __uint_as_float(sc[ii]);
                        __syncwarp();
                        const int64_t row0 = (int64_t)qt * kPM + 32 * quad;
                        if (tot < 256) {
                            // sparse: every lane writes its own few candidates
                            uint32_t mm = msk;
                            int32_t sl = half == 0 ? slot : slot - cnt + 1;
                            while (mm) {
                                const int ii = __ffs(mm) - 1;
                                mm &= mm - 1;
                                const int64_t gi = (row0 + lane) * a.cap + sl++;
                                const float sv = tr_w[lane * 33 + ii];
                                const float e = __fmul_ru(ce, xn_w[col - col_lo + ii]);
                                a.cand[gi] = (uint32_t)(pos0 + col + ii);
                                a.lo[gi] = __fsub_rd(sv, e);
                                a.hi[gi] = __fadd_ru(sv, e);
                            }
                        } else {
                            // dense: one query's run at a time, written by consecutive
                            // lanes into consecutive slots, four queries per step
                            unsigned any = __ballot_sync(0xffffffffu, msk != 0);
                            const int64_t posl = pos0 + col + lane;
                            const float xl = xn_w[col - col_lo + lane];
                            for (int r0 = 0; r0 < 32; r0 += 4) {
                                if (!((any >> r0) & 0xFu)) continue;
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    const int r = r0 + u;
                                    const uint32_t mr = __shfl_sync(0xffffffffu, msk, r);
                                    const int32_t sr = __shfl_sync(0xffffffffu, slot, r);
                                    const float cer = __shfl_sync(0xffffffffu, ce, r);
                                    const int32_t first = half == 0 ? sr : sr - __popc(mr) + 1;
                                    if ((mr >> lane) & 1u) {
                                        const int64_t gi =
                                            (row0 + r) * a.cap + first + __popc(mr & lt);
                                        const float sv = tr_w[r * 33 + lane];
                                        const float e = __fmul_ru(cer, xl);
                                        a.cand[gi] = (uint32_t)posl;
                                        a.lo[gi] = __fsub_rd(sv, e);
                                        a.hi[gi] = __fadd_ru(sv, e);
                                    }
                                }
                            }
                        }
                        slot += half == 0 ? cnt : -cnt;
                        __syncwarp();
                    }
                }
                fence_before();
                mbar_arrive(&acc_empty[buf]);
                if (++buf == 2) {
                    buf = 0;
                    acc_phase ^= 1;
                }
            }
            // end of the work item: the same two barriers on every path
            if (kRerank) {
                const int32_t got = half == 0 ? slot - base_j : base_j + cnt_j - 1 - slot;
                cnt_x[half * kPM + row] = qv ? (overflow ? 0xFFFFFFFFu : (uint32_t)got) : 0u;
                epi_sync();
                if (half == 0 && qv && !aborted) {
                    const uint32_t other = cnt_x[kPM + row];
                    if (overflow || other == 0xFFFFFFFFu ||
                        (int64_t)cnt_x[row] + (int64_t)other != (int64_t)cnt_j)
                        atomicCAS(a.err, 0, 15);               // not the counted candidates
                }
                epi_sync();
            } else {
                epi_sync();
                // the two halves' counters of a query row add up to its histogram
                for (int idx = et; idx < kPM * (a.L + 1); idx += kEpiThreads) {
                    const int r = idx / (a.L + 1), l = idx - r * (a.L + 1);
                    const int64_t qq = (int64_t)qt * kPM + r;
                    uint32_t* h0 = &hist[l * 2 * kPM + r];
                    uint32_t* h1 = h0 + kPM;
                    if (qq < a.nq && !aborted)
                        a.H[(qq * a.m + j) * (a.L + 1) + l] = *h0 + *h1;
                    *h0 = 0;
                    *h1 = 0;
                }
                epi_sync();
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ------------------------------------------------------ operand preparation

// Qb[q][k] = bf16(q_k) (zero for d <= k < Kq); Qs[q][b] = +1 / -1 for code bit b
// set / clear (b < L), 0 beyond L.
template <typename C>
__global__ void prep_queries_kernel(const float* __restrict__ Q, int64_t nq, int d, int Kq,
                                    const C* __restrict__ qcodes, int L,
                                    __nv_bfloat16* __restrict__ Qb, __nv_bfloat16* __restrict__ Qs,
                                    int* __restrict__ err, uint32_t* __restrict__ hist_ctr) {
    NRLSH_PDL_ENTRY();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *err = 0;          // the call's error word starts clear
        *hist_ctr = 0;     // the histogram kernel's work counter
    }
    const int64_t total = nq * Kq;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / Kq;
        const int k = (int)(i - q * Kq);
        Qb[i] = __float2bfloat16_rn(k < d ? Q[q * d + k] : 0.0f);
        if (k < 64) {
            const uint64_t c = (uint64_t)qcodes[q];
            Qs[q * 64 + k] = __float2bfloat16_rn(k < L ? (((c >> k) & 1u) ? 1.0f : -1.0f) : 0.0f);
        }
    }
}

// Xs[p][b] as Qs, from the item codes (storage order); 8 bits per thread.
template <typename C>
__global__ void item_signs_kernel(const C* __restrict__ codes, int64_t n, int L,
                                  __nv_bfloat16* __restrict__ Xs) {
    NRLSH_PDL_ENTRY();
    const int64_t total = n * 8;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i >> 3;
        const int b0 = (int)(i & 7) * 8;
        const uint64_t c = (uint64_t)codes[p];
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t v = 0;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int b = b0 + 2 * h + e;
                // bf16 bit patterns: +1 = 0x3F80, -1 = 0xBF80, 0 = 0x0000
                const uint32_t bits = b < L ? (((c >> b) & 1u) ? 0x3F80u : 0xBF80u) : 0u;
                v |= bits << (16 * e);
            }
            w[h] = v;
        }
        ((uint4*)Xs)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ X, int64_t count,
                               __nv_bfloat16* __restrict__ Xb) {
    NRLSH_PDL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        Xb[i] = __float2bfloat16_rn(X[i]);
}

int grid_for(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), 152 * 16));
}

size_t pairs_smem_bytes(bool rerank, int nkc, int L, int stages) {
    const int na = rerank ? nkc + 1 : 1;
    const size_t extra = rerank ? (size_t)(kEpiWarps * 64 + 2 * kPM + kEpiWarps * 32 * 33) * 4
                                : (size_t)(L + 1) * 2 * kPM * 4;
    return 1024 + (size_t)(na + stages) * kChunk + (2 * (size_t)stages + 7 + 2 * kWorkRing) * 8 +
           (kWorkRing + 4) * 4 + 16 + extra;
}

int pairs_stages(bool rerank, int nkc, int L) {
    int s = kMaxStages;
    while (s > 2 && pairs_smem_bytes(rerank, nkc, L, s) > 225 * 1024) --s;
    return s;
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    return sms > 0 ? sms : 1;
}

}  // namespace

int tc_query_k_chunks(int d) { return (int)ceil_div(d, 64); }

bool tc_query_supported(int d, int L) {
    int dev = 0, major = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaGetLastError();
    if (major != 10 || L < 1 || L > 64 || tensor_map_encoder() == nullptr) return false;
    const int nkc = tc_query_k_chunks(d);
    return pairs_smem_bytes(true, nkc, L, 2) <= 225 * 1024;
}

// a_q of every query (a warp per query): with q~ = bf16(q), dq = q - q~ (exact in
// fp32 by Sterbenz's lemma) and x~ the bf16 items (x~ = x for bf16 items, else
// |x - x~| <= 2^-8 |x| elementwise: an 8-bit significand rounded to nearest),
//   |q.x - q~.x~| <= ||dq|| ||x|| + ||q~|| ||x - x~||,
//   the FP32 accumulation of the K (16-padded) products within (K + 8) 2^-20
//   ||q~|| ||x~|| (16x the first-order bound), and the canonical FP64 in-order
//   sum within (d + 2) 2^-53 ||q|| ||x||,
// with ||q~|| <= ||q|| + ||dq|| and ||x~|| <= (1 + rx) ||x||.  So e = a_q ||x||,
//   a_q = D + rx (Q + D) + (K + 8) 2^-20 (Q + D)(1 + rx) + (d + 2) 2^-53 Q,
// Q >= ||q|| the query norm bound, D >= ||dq|| (FP64 sum of the exact squares,
// enlarged by its own rounding), every step rounded up, times (1 + 2^-20).
__global__ void query_bound_kernel(const float* __restrict__ Q, int64_t nq, int d,
                                   const float* __restrict__ qnorm, int fp32_items,
                                   float* __restrict__ qce) {
    NRLSH_PDL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    double ss = 0.0;
    for (int k = lane; k < d; k += 32) {
        const float v = Q[q * d + k];
        const float r = v - __bfloat162float(__float2bfloat16_rn(v));
        ss = fma((double)r, (double)r, ss);
    }
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) {
        const double D = __dsqrt_ru(__dmul_ru(ss, 1.0 + (d + 40) * 0x1p-52));
        const double Qn = (double)qnorm[q];
        const double rx = fp32_items ? 0x1p-8 : 0.0;
        const double K = 16.0 * (double)ceil_div(d, 16);
        const double QD = __dadd_ru(Qn, D);
        double t = __dmul_ru(__dmul_ru((K + 8.0) * 0x1p-20, QD), 1.0 + rx);
        t = __dadd_ru(t, __dmul_ru(rx, QD));
        t = __dadd_ru(t, D);
        t = __dadd_ru(t, __dmul_ru((d + 2.0) * 0x1p-53, Qn));
        qce[q] = __double2float_ru(__dmul_ru(t, 1.0 + 0x1p-20));
    }
}

cudaError_t launch_query_bounds(const float* Q, int64_t nq, int d, const float* qnorm,
                                bool fp32_items, float* qce, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)ceil_div(nq * 32, (int64_t)256);
    return launch("query_bounds", query_bound_kernel, dim3(grid), dim3(256), 0, st, Q, nq, d, qnorm,
                  fp32_items ? 1 : 0, qce);
}

cudaError_t launch_prep_queries(const float* Q, int64_t nq, int d, int Kq, const void* qcodes,
                                int code_bytes, int L, __nv_bfloat16* Qb, __nv_bfloat16* Qs,
                                int* err, uint32_t* hist_ctr, cudaStream_t st) {
    const dim3 grid(grid_for(nq * Kq));
    if (code_bytes == 4)
        return launch("prep_queries", prep_queries_kernel<uint32_t>, grid, dim3(256), 0, st, Q, nq, d,
                      Kq, (const uint32_t*)qcodes, L, Qb, Qs, err, hist_ctr);
    return launch("prep_queries", prep_queries_kernel<uint64_t>, grid, dim3(256), 0, st, Q, nq, d, Kq,
                  (const uint64_t*)qcodes, L, Qb, Qs, err, hist_ctr);
}

__global__ void report_err_kernel(const int* __restrict__ err, int* __restrict__ report) {
    NRLSH_PDL_ENTRY();
    const int e = *err;
    if (e) atomicCAS(report, 0, e);
}

cudaError_t launch_report_err(const int* err, int* report, cudaStream_t st) {
    return launch("report_err", report_err_kernel, dim3(1), dim3(32), 0, st, err, report);
}

cudaError_t launch_item_signs(const void* codes, int code_bytes, int64_t n, int L,
                              __nv_bfloat16* Xs, cudaStream_t st) {
    const dim3 grid(grid_for(n * 8));
    if (code_bytes == 4)
        return launch("item_signs", item_signs_kernel<uint32_t>, grid, dim3(256), 0, st,
                      (const uint32_t*)codes, n, L, Xs);
    return launch("item_signs", item_signs_kernel<uint64_t>, grid, dim3(256), 0, st,
                  (const uint64_t*)codes, n, L, Xs);
}

cudaError_t launch_to_bf16(const float* X, int64_t count, __nv_bfloat16* Xb, cudaStream_t st) {
    return launch("to_bf16", to_bf16_kernel, dim3(grid_for(count)), dim3(256), 0, st, X, count, Xb);
}

cudaError_t launch_pairs_tc(bool rerank, const __nv_bfloat16* Qb, const __nv_bfloat16* Qs,
                            int64_t nq, const __nv_bfloat16* Xb, const __nv_bfloat16* Xs,
                            int64_t n, int d, int dp, int m, int L, const int64_t* seg,
                            const uint32_t* list, const uint32_t* nlist, uint32_t* H,
                            const uint8_t* lam, const uint32_t* off, const TcBoundary* tb,
                            const float* xnorm, const float* qce, uint32_t* cand,
                            float* lo, float* hi, int64_t cap, int* err, uint32_t* work_ctr,
                            cudaStream_t st, uint32_t spin_first) {
    if (nq <= 0) return cudaSuccess;
    const int nkc = tc_query_k_chunks(d);
    const int Kq = 64 * nkc;
    CUtensorMap map_qb, map_qs, map_xb, map_xs;
    if (!make_map_bf16(&map_qs, Qs, 64, (uint64_t)nq, 64, kPM) ||
        !make_map_bf16(&map_xs, Xs, 64, (uint64_t)n, 64, kPN))
        return cudaErrorNotSupported;
    if (rerank) {
        if (!make_map_bf16(&map_qb, Qb, (uint64_t)Kq, (uint64_t)nq, (uint64_t)Kq, kPM) ||
            !make_map_bf16(&map_xb, Xb, (uint64_t)d, (uint64_t)n, (uint64_t)dp, kPN))
            return cudaErrorNotSupported;
    } else {
        map_qb = map_qs;
        map_xb = map_xs;
    }
    PairsArgs a{};
    a.list = list;
    a.nlist = nlist;
    a.seg = seg;
    a.m = m;
    a.L = L;
    a.nqt = (int)ceil_div(nq, kPM);
    a.nwork_all = m * a.nqt;
    a.nkc = nkc;
    a.d = d;
    a.stages = pairs_stages(rerank, nkc, L);
    a.nq = nq;
    a.H = H;
    a.lam = lam;
    a.off = off;
    a.tb = tb;
    a.xnorm = xnorm;
    a.qce = qce;
    a.cand = cand;
    a.lo = lo;
    a.hi = hi;
    a.cap = cap;
    a.err = err;
    a.work_ctr = work_ctr;
    a.spin_first = spin_first;
    const size_t smem = pairs_smem_bytes(rerank, nkc, L, a.stages);
    // one CTA per SM (items are handed out dynamically; a work list's length is on
    // the device)
    const int grid = list ? sm_count() : (int)std::min<int64_t>(a.nwork_all, sm_count());
    if (rerank) {
        auto kern = pairs_tc_kernel<true>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return launch("rerank_tc", kern, dim3(grid), dim3(kPThreads), smem, st, map_qb, map_qs,
                      map_xb, map_xs, a);
    }
    auto kern = pairs_tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch("hist_tc", kern, dim3(grid), dim3(kPThreads), smem, st, map_qb, map_qs, map_xb,
                  map_xs, a);
}

}  // namespace nrlsh
