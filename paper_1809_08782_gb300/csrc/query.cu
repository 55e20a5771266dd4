// Query kernels (Section 3.3 multi-probe, Eq. 12 bucket order, exact re-rank, Eq. 1).
//
//   row_norm_bound   fp32 upper bound of ||q||, for the error bounds
//   hist             H[q][j][l] = #{x in S_j : l(q, x) = l}, XOR + popcount
//   threshold        walk the bucket order until the budget: lam_j, (j*, l*), r
//   select           ordered compaction of the probed items (storage positions)
//   rerank_fp32      gathered FP32 dot products with a proven error interval
//   topk             exact top-k: radix-select on the lower bounds, FP64 rescoring
//                    of the contenders, (score desc, id asc) selection
#include "nrlsh_internal.cuh"
#include "sign_tiers.cuh"

#include <unordered_map>
#include <utility>

#include <cfloat>

namespace nrlsh {

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive block scan of one uint32 per thread (blockDim.x == 256).
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total, uint32_t* warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < 8 ? warp_tot[lane] : 0;
        for (int o = 1; o < 8; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < 8) warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = warp ? warp_tot[warp - 1] : 0;
    *total = warp_tot[7];
    __syncthreads();
    return before + incl - v;
}

// ------------------------------------------------------------------ norms

__global__ void row_norm_bound_kernel(const float* __restrict__ Q, int64_t nq, int d,
                                      float* qnorm) {
    NRLSH_PDL_ENTRY();
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nq) return;
    double ss = 0.0;
    for (int c = lane; c < d; c += 32) {
        const double v = (double)Q[row * d + c];
        ss = fma(v, v, ss);
    }
    ss = warp_sum_d(ss);
    // the relative error of ss (< d 2^-53) is far inside the 4x margin of the bounds
    if (lane == 0) qnorm[row] = __fsqrt_ru(__double2float_ru(ss));
}

// --------------------------------------------------------------- histogram


// Block of 256 threads: one position tile (inside one sub-dataset, at most 4,096
// codes, staged in shared memory) x kHistQ queries, with kSplit = 256 / kHistQ
// threads per query each taking a contiguous share of the tile (a warp reads
// 16 bytes of codes at a time by broadcast).  Every thread keeps a private uint32
// histogram column indexed [l][thread], so increments never conflict on a bank;
// they are shared-memory reductions (no returned value), so consecutive
// increments of a thread do not wait on each other.  The columns of a query are summed at the end and added to
// H (stored, when every sub-dataset is one tile).
constexpr int kHistThreads = 256;

// The codes of one 16-byte vector counted into a thread's histogram column.
template <typename C>
__device__ __forceinline__ void hist_count_vec(const uint4& a, C cq, int L, uint32_t* hc);
template <>
__device__ __forceinline__ void hist_count_vec<uint32_t>(const uint4& a, uint32_t cq, int L,
                                                         uint32_t* hc) {
    atomicAdd(&hc[(L - __popc(cq ^ a.x)) * kHistThreads], 1u);
    atomicAdd(&hc[(L - __popc(cq ^ a.y)) * kHistThreads], 1u);
    atomicAdd(&hc[(L - __popc(cq ^ a.z)) * kHistThreads], 1u);
    atomicAdd(&hc[(L - __popc(cq ^ a.w)) * kHistThreads], 1u);
}
template <>
__device__ __forceinline__ void hist_count_vec<uint64_t>(const uint4& a, uint64_t cq, int L,
                                                         uint32_t* hc) {
    const uint64_t c0 = ((uint64_t)a.y << 32) | a.x, c1 = ((uint64_t)a.w << 32) | a.z;
    atomicAdd(&hc[(L - __popcll(cq ^ c0)) * kHistThreads], 1u);
    atomicAdd(&hc[(L - __popcll(cq ^ c1)) * kHistThreads], 1u);
}

template <typename C, int kHistQ>
__global__ void __launch_bounds__(kHistThreads)
    hist_kernel(const C* __restrict__ codes, const C* __restrict__ qcodes, int64_t nq, int m, int L,
                const PosTile* __restrict__ tiles, uint32_t* __restrict__ H, int exclusive) {
    NRLSH_PDL_ENTRY();
    constexpr int kSplit = kHistThreads / kHistQ;
    extern __shared__ unsigned char smem_raw[];
    C* cs = (C*)smem_raw;
    uint32_t* h = (uint32_t*)(smem_raw + 16384);        // [L+1][kHistThreads]
    const int tid = threadIdx.x;
    const int qi = tid % kHistQ, sp = tid / kHistQ;
    const PosTile t = tiles[blockIdx.x];
    const int64_t q0 = (int64_t)blockIdx.y * kHistQ;
    const int64_t q = q0 + qi;
#pragma unroll 4
    for (int i = tid; i < t.len; i += kHistThreads) cs[i] = codes[t.start + i];
    // (L+1) x 256 words: a multiple of 4, cleared 16 bytes at a time
    for (int i = tid; i < (L + 1) * kHistThreads / 4; i += kHistThreads)
        ((uint4*)h)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (q < nq) {
        // thread sp of a query takes a contiguous share of the tile's 16-byte code
        // vectors (a warp shares sp, so every vector load is a broadcast); the
        // codes past the last whole vector are taken strided
        const C cq = qcodes[q];
        uint32_t* hc = h + tid;
        constexpr int kPer = 16 / sizeof(C);
        const int nvec = t.len / kPer;
        const int v1 = (int)((int64_t)nvec * (sp + 1) / kSplit);
        const uint4* cs4 = (const uint4*)cs;
        int v = (int)((int64_t)nvec * sp / kSplit);
        for (; v + 3 < v1; v += 4) {
            const uint4 a = cs4[v], b = cs4[v + 1], c = cs4[v + 2], e = cs4[v + 3];
            hist_count_vec<C>(a, cq, L, hc);
            hist_count_vec<C>(b, cq, L, hc);
            hist_count_vec<C>(c, cq, L, hc);
            hist_count_vec<C>(e, cq, L, hc);
        }
        for (; v < v1; ++v) hist_count_vec<C>(cs4[v], cq, L, hc);
        for (int i = nvec * kPer + sp; i < t.len; i += kSplit)
            atomicAdd(&hc[(L - popc_word(cq ^ cs[i])) * kHistThreads], 1u);
    }
    __syncthreads();
    for (int e = tid; e < (L + 1) * kHistQ; e += kHistThreads) {
        const int l = e / kHistQ, qe = e % kHistQ;
        if (q0 + qe >= nq) continue;
        uint32_t v = 0;
#pragma unroll
        for (int s2 = 0; s2 < kSplit; ++s2) v += h[l * kHistThreads + s2 * kHistQ + qe];
        uint32_t* dst = &H[((q0 + qe) * m + t.seg) * (L + 1) + l];
        if (exclusive)
            *dst = v;                 // the only tile of its sub-dataset: H needs no clearing
        else if (v)
            atomicAdd(dst, v);
    }
}

// --------------------------------------------------------------- threshold

// Block phase (256 threads).  Walks the buckets in probing order with a block
// scan of their sizes until the running total reaches B' = min(B, n).  Buckets
// before the boundary bucket t* are taken whole; within sub-dataset j they are
// l = L, L-1, ..., so lam_j = L + 1 - (number of buckets of j before t*).
// cntj (m words) is scratch; lam_s receives lam_j; returns the boundary.
__device__ Boundary dev_threshold(const uint32_t* __restrict__ Hq, const uint32_t* __restrict__ order,
                                  int m, int L, int64_t n, int64_t B, uint32_t flags,
                                  uint32_t* cntj, uint8_t* lam_s) {
    __shared__ uint32_t warp_tot[8];
    __shared__ int tstar_s;
    __shared__ uint32_t before_s;
    __shared__ Boundary b_s;
    const int ncls = m * (L + 1);
    const uint32_t Bp = (uint32_t)(B < n ? B : n);
    for (int j = threadIdx.x; j < m; j += blockDim.x) cntj[j] = 0;
    if (threadIdx.x == 0) tstar_s = ncls;
    __syncthreads();
    uint32_t cum = 0;
    for (int base = 0; base < ncls; base += 256) {
        const int t = base + threadIdx.x;
        const uint32_t c = t < ncls ? Hq[order[t]] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(c, &total, warp_tot);
        if (t < ncls && cum + ex + c >= Bp && cum + ex < Bp) {  // exactly one thread
            tstar_s = t;
            before_s = cum + ex;
        }
        __syncthreads();
        if (tstar_s < ncls) break;
        cum += total;
    }
    const int tstar = tstar_s;
    for (int t = threadIdx.x; t < tstar; t += blockDim.x) atomicAdd(&cntj[order[t] / (L + 1)], 1u);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) lam_s[j] = (uint8_t)(L + 1 - cntj[j]);
    if (threadIdx.x == 0) {
        const uint32_t cid = order[tstar];
        Boundary b;
        b.j = (int32_t)(cid / (L + 1));
        b.l = (int32_t)(cid % (L + 1));
        b.full = (int32_t)before_s;
        b.r = (flags & NRLSH_WHOLE_BUCKETS) ? (int32_t)Hq[cid] : (int32_t)(Bp - before_s);
        b_s = b;
    }
    __syncthreads();
    return b_s;
}

__global__ void __launch_bounds__(256)
    threshold_kernel(const uint32_t* __restrict__ H, const uint32_t* __restrict__ order, int m,
                     int L, int64_t nq, int64_t n, int64_t budget,
                     const int64_t* __restrict__ budgets, uint32_t flags,
                     uint8_t* __restrict__ lam, Boundary* __restrict__ bnd) {
    NRLSH_PDL_ENTRY();
    extern __shared__ uint32_t cntj[];
    uint8_t* lam_s = (uint8_t*)(cntj + m);
    const int64_t q = blockIdx.x;
    const Boundary b = dev_threshold(H + q * m * (L + 1), order, m, L, n,
                                     budgets ? budgets[q] : budget, flags, cntj, lam_s);
    for (int j = threadIdx.x; j < m; j += 256) lam[q * m + j] = lam_s[j];
    if (threadIdx.x == 0) bnd[q] = b;
}

// ------------------------------------------------ walk for the tensor path

// Block per query (256 threads): the bucket walk of dev_threshold, then for every
// sub-dataset S_j the number of probed items, cnt_j = sum_{l >= lam_j} H[q][j][l]
// (+ r for the boundary sub-dataset), whose exclusive prefix over j is where the
// re-rank writes S_j's candidates (off[q][j], off[q][m] = min(B, n)).  The
// boundary bucket's first r items in storage (= id) order are the ones at
// positions <= pcut, found by one ordered sweep of S_j*.
template <typename C>
__global__ void __launch_bounds__(256)
    tc_walk_kernel(const uint32_t* __restrict__ H, const uint32_t* __restrict__ order, int m, int L,
                   int64_t n, const int64_t* __restrict__ seg, int64_t budget,
                   const int64_t* __restrict__ budgets, int64_t cap, uint32_t flags,
                   const C* __restrict__ codes, const C* __restrict__ qcodes,
                   uint8_t* __restrict__ lam, uint32_t* __restrict__ off, TcBoundary* __restrict__ tb,
                   Boundary* __restrict__ bnd, uint8_t* __restrict__ work_flag, int nqt,
                   const int* __restrict__ err) {
    NRLSH_PDL_ENTRY();
    extern __shared__ uint32_t cntj[];
    uint8_t* lam_s = (uint8_t*)(cntj + m);
    __shared__ uint32_t warp_tot[8];
    __shared__ int64_t pcut_s;
    const int64_t q = blockIdx.x;
    if (*err) {
        // the histograms are incomplete (a bounded wait ran out): nothing is probed,
        // so no later kernel of the call reads past what it owns
        for (int j = threadIdx.x; j <= m; j += blockDim.x) {
            off[q * (m + 1) + j] = 0;
            if (j < m) lam[q * m + j] = (uint8_t)(L + 1);
        }
        if (threadIdx.x == 0) {
            tb[q] = TcBoundary{0, 0, -1};
            bnd[q] = Boundary{0, 0, 0, 0};
        }
        return;
    }
    const int64_t Bq = min(max(budgets ? budgets[q] : budget, (int64_t)1), cap);
    const uint32_t* Hq = H + q * m * (L + 1);
    const Boundary b = dev_threshold(Hq, order, m, L, n, Bq, flags, cntj, lam_s);
    uint32_t run = 0;
    for (int base = 0; base < m; base += 256) {
        const int j = base + threadIdx.x;
        uint32_t c = 0;
        if (j < m) {
            const uint32_t* Hj = Hq + (int64_t)j * (L + 1);
            for (int l = lam_s[j]; l <= L; ++l) c += Hj[l];
            if (j == b.j) c += (uint32_t)b.r;
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(c, &tot, warp_tot);
        if (j < m) {
            off[q * (m + 1) + j] = run + ex;
            lam[q * m + j] = lam_s[j];
            if (c) work_flag[(int64_t)j * nqt + q / 128] = 1;
        }
        run += tot;
    }
    if (threadIdx.x == 0) {
        off[q * (m + 1) + m] = run;
        pcut_s = -1;
    }
    __syncthreads();
    const int64_t p_lo = seg[b.j], p_hi = seg[b.j + 1];
    const uint32_t in_bucket = Hq[(int64_t)b.j * (L + 1) + b.l];
    if ((uint32_t)b.r >= in_bucket) {
        if (threadIdx.x == 0) pcut_s = p_hi - 1;      // the whole bucket is probed
    } else {
        const C cq = qcodes[q];
        uint32_t cum = 0;
        for (int64_t p0 = p_lo; p0 < p_hi; p0 += 256) {
            const int64_t p = p0 + threadIdx.x;
            const uint32_t hit = p < p_hi && L - popc_word(cq ^ codes[p]) == b.l;
            uint32_t tot;
            const uint32_t ex = block_exclusive_scan(hit, &tot, warp_tot);
            if (hit && cum + ex + 1 == (uint32_t)b.r) pcut_s = p;
            cum += tot;
            if (cum >= (uint32_t)b.r) break;          // the same decision in every thread
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tb[q] = TcBoundary{b.j, b.l, pcut_s};
        bnd[q] = Boundary{b.j, b.l, 0, (int32_t)run};
    }
}

// One block of 1,024 threads: indices of the nonzero flags in ascending order.
__global__ void __launch_bounds__(1024)
    work_list_kernel(const uint8_t* __restrict__ flag, int nflag, uint32_t* __restrict__ list,
                     uint32_t* __restrict__ count) {
    NRLSH_PDL_ENTRY();
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nflag; base += 1024) {
        const int i = base + threadIdx.x;
        const bool f = i < nflag && flag[i] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = carry_s;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (f) list[before + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < 32; ++w) t += wsum[w];
            carry_s += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *count = carry_s;
        count[1] = 0;      // the consumer's work counter starts at zero
    }
}

// ------------------------------------------------------------------ select

// Block phase (256 threads): ordered compaction of the probed items of one
// query.  The positions from the first to the last sub-dataset the walk reached
// are swept once as one range (an unreached sub-dataset inside it has
// lam_j = L + 1 and contributes nothing); warp w owns a contiguous eighth and
// follows the sub-dataset of each lane's position as it advances.  A counting
// sweep, a scan over the 8 warps, and a writing sweep with ballot prefixes, each
// with kSelUnroll code loads in flight per lane.  Items of whole buckets go to
// out[0, full) in position order; boundary-bucket items go to
// out[full, full + r), the first r of them in position (= id) order.
constexpr int kSelUnroll = 4;

__device__ __forceinline__ int seg_find(const int64_t* __restrict__ seg, int jlo, int jhi, int64_t p) {
    // largest j in [jlo, jhi] with seg[j] <= p (then seg[j + 1] > p)
    int a = jlo, b = jhi;
    while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (seg[mid] <= p) a = mid; else b = mid - 1;
    }
    return a;
}

// msk: shared scratch of 2 x 8 x kMaskChunks words (shared with dev_topk's rows).
constexpr int kMaskChunks = 128;                // per warp: 32-position chunks whose masks are kept

template <typename C>
__device__ void dev_select(const C* __restrict__ codes, C cq, const int64_t* __restrict__ seg, int m, int L,
                           const uint8_t* lam_s, const Boundary& b, uint32_t* __restrict__ out,
                           uint32_t* msk) {
    __shared__ uint32_t wf[8], wb[8];
    uint32_t* mskf = msk;
    uint32_t* mskb = msk + 8 * kMaskChunks;
    __shared__ int jlo_s, jhi_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) {
        jlo_s = b.j;
        jhi_s = b.j;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        if (lam_s[j] <= L) {
            atomicMin(&jlo_s, j);
            atomicMax(&jhi_s, j);
        }
    }
    __syncthreads();
    const int jlo = jlo_s, jhi = jhi_s;
    const int64_t p_lo = seg[jlo], len = seg[jhi + 1] - p_lo;
    const int64_t w0 = p_lo + len * warp / 8, w1 = p_lo + len * (warp + 1) / 8;
    const int nchunk = (int)ceil_div(w1 - w0, 32);
    const bool keep = nchunk <= kMaskChunks;    // warp-uniform
    uint32_t* mf_w = mskf + warp * kMaskChunks;
    uint32_t* mb_w = mskb + warp * kMaskChunks;
    const int j_start = w0 + lane < w1 ? seg_find(seg, jlo, jhi, w0 + lane) : jlo;
    // the predicates at position p (lane's sub-dataset jl advances with p)
    auto test = [&](int64_t p, C cv, int& jl, int64_t& nxt, bool& f, bool& bb) {
        while (p >= nxt) nxt = seg[++jl + 1];
        const int l = L - popc_word(cq ^ cv);
        f = l >= lam_s[jl];
        bb = jl == b.j && l == b.l;
    };
    uint32_t cf = 0, cb = 0;
    {
        int jl = j_start;
        int64_t nxt = seg[jl + 1];
        for (int c0 = 0; c0 < nchunk; c0 += kSelUnroll) {
            C cv[kSelUnroll];
#pragma unroll
            for (int u = 0; u < kSelUnroll; ++u) {
                const int64_t p = w0 + 32 * (c0 + u) + lane;
                cv[u] = p < w1 ? codes[p] : (C)0;
            }
#pragma unroll
            for (int u = 0; u < kSelUnroll; ++u) {
                const int64_t p = w0 + 32 * (c0 + u) + lane;
                bool f = false, bb = false;
                if (p < w1) test(p, cv[u], jl, nxt, f, bb);
                const unsigned mf = __ballot_sync(0xffffffffu, f);
                const unsigned mb = __ballot_sync(0xffffffffu, bb);
                cf += __popc(mf);
                cb += __popc(mb);
                if (keep && lane == 0 && c0 + u < nchunk) {
                    mf_w[c0 + u] = mf;
                    mb_w[c0 + u] = mb;
                }
            }
        }
    }
    if (lane == 0) {
        wf[warp] = cf;
        wb[warp] = cb;
    }
    __syncthreads();
    uint32_t of = 0, ob = 0;
    for (int w = 0; w < warp; ++w) {
        of += wf[w];
        ob += wb[w];
    }
    auto emit = [&](int64_t p, unsigned mf, unsigned mb) {
        if ((mf >> lane) & 1u) out[of + __popc(mf & lt)] = (uint32_t)p;
        if ((mb >> lane) & 1u) {
            const uint32_t rank = ob + __popc(mb & lt);
            if (rank < (uint32_t)b.r) out[b.full + rank] = (uint32_t)p;
        }
        of += __popc(mf);
        ob += __popc(mb);
    };
    if (cf || (cb && ob < (uint32_t)b.r)) {
        if (keep) {
            for (int c = 0; c < nchunk; ++c) {
                const unsigned mf = mf_w[c], mb = mb_w[c];
                if (mf | mb) emit(w0 + 32 * c + lane, mf, mb);
            }
        } else {
            int jl = j_start;
            int64_t nxt = seg[jl + 1];
            for (int c0 = 0; c0 < nchunk; c0 += kSelUnroll) {
                C cv[kSelUnroll];
#pragma unroll
                for (int u = 0; u < kSelUnroll; ++u) {
                    const int64_t p = w0 + 32 * (c0 + u) + lane;
                    cv[u] = p < w1 ? codes[p] : (C)0;
                }
#pragma unroll
                for (int u = 0; u < kSelUnroll; ++u) {
                    const int64_t p = w0 + 32 * (c0 + u) + lane;
                    bool f = false, bb = false;
                    if (p < w1) test(p, cv[u], jl, nxt, f, bb);
                    emit(p, __ballot_sync(0xffffffffu, f), __ballot_sync(0xffffffffu, bb));
                }
            }
        }
    }
    __syncthreads();
}

template <typename C>
__global__ void __launch_bounds__(256)
    select_kernel(const C* __restrict__ codes, const C* __restrict__ qcodes,
                  const int64_t* __restrict__ seg, int m, int L,
                  const uint8_t* __restrict__ lam, const Boundary* __restrict__ bnd,
                  uint32_t* __restrict__ cand, int64_t cap) {
    NRLSH_PDL_ENTRY();
    extern __shared__ uint8_t lam_s[];
    const int64_t q = blockIdx.x;
    for (int j = threadIdx.x; j < m; j += 256) lam_s[j] = lam[q * m + j];
    __syncthreads();
    __shared__ __align__(16) uint32_t msk[16 * kMaskChunks];
    dev_select(codes, qcodes[q], seg, m, L, lam_s, bnd[q], cand + q * cap, msk);
}

// ------------------------------------------------------------------ rerank

constexpr int kRerankWarps = 8;
constexpr int kRerankUnroll = 4;  // candidate rows in flight per warp

template <typename T> struct RowDot;

template <> struct RowDot<float> {
    // dp is a multiple of 8, rows are 16-byte aligned
    template <int U>
    __device__ static void dot(const float* const* rows, const float* qs, int dp, int lane,
                               float (&acc)[U]) {
        const float4* q4 = (const float4*)qs;
        for (int c = lane; c < dp / 4; c += 32) {
            float4 x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) x[u] = ((const float4*)rows[u])[c];
            const float4 y = q4[c];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                acc[u] = fmaf(x[u].x, y.x, acc[u]);
                acc[u] = fmaf(x[u].y, y.y, acc[u]);
                acc[u] = fmaf(x[u].z, y.z, acc[u]);
                acc[u] = fmaf(x[u].w, y.w, acc[u]);
            }
        }
    }
};

template <> struct RowDot<__nv_bfloat16> {
    template <int U>
    __device__ static void dot(const __nv_bfloat16* const* rows, const float* qs, int dp, int lane,
                               float (&acc)[U]) {
        for (int c = lane; c < dp / 8; c += 32) {
            uint4 raw[U];
#pragma unroll
            for (int u = 0; u < U; ++u) raw[u] = ((const uint4*)rows[u])[c];
            const float* y = qs + c * 8;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const __nv_bfloat162* h = (const __nv_bfloat162*)&raw[u];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 x = __bfloat1622float2(h[i]);
                    acc[u] = fmaf(x.x, y[2 * i], acc[u]);
                    acc[u] = fmaf(x.y, y[2 * i + 1], acc[u]);
                }
            }
        }
    }
};

// Block phase: FP32 scores of candidates [i0, i1) of one query; a warp takes
// kRerankUnroll rows at a time.  The score interval [s - e, s + e] with
// e = kappa ||q|| ||x|| (FP32 summation bound, 4x margin) is stored rounded
// outward.  qs holds q zero-padded to dp.
template <typename T>
__device__ void dev_rerank(const T* __restrict__ Xp, int dp, const float* qs,
                           const uint32_t* __restrict__ candq, int64_t i0, int64_t i1,
                           const float* __restrict__ xnorm, float qn, float kappa,
                           float* __restrict__ loq, float* __restrict__ hiq) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t stride = (int64_t)(blockDim.x >> 5) * kRerankUnroll;
    int64_t i = i0 + (int64_t)warp * kRerankUnroll;
    // candidate positions one iteration ahead, so a row's address never waits
    uint32_t ps[kRerankUnroll];
#pragma unroll
    for (int u = 0; u < kRerankUnroll; ++u) ps[u] = i < i1 ? candq[min(i + u, i1 - 1)] : 0u;
    for (; i < i1; i += stride) {
        const T* rows[kRerankUnroll];
        float xn[kRerankUnroll];
#pragma unroll
        for (int u = 0; u < kRerankUnroll; ++u) {
            rows[u] = Xp + (int64_t)ps[u] * dp;
            xn[u] = xnorm[ps[u]];
        }
        const int64_t inext = i + stride;
        uint32_t nps[kRerankUnroll];
#pragma unroll
        for (int u = 0; u < kRerankUnroll; ++u)
            nps[u] = inext < i1 ? candq[min(inext + u, i1 - 1)] : 0u;
        float acc[kRerankUnroll];
#pragma unroll
        for (int u = 0; u < kRerankUnroll; ++u) acc[u] = 0.0f;
        RowDot<T>::template dot<kRerankUnroll>(rows, qs, dp, lane, acc);
        // transpose-reduction of the kRerankUnroll row sums: each level halves the
        // values a lane holds, then plain butterflies; afterwards lane
        // (32 / kRerankUnroll) r holds the sum of row r (any order meets the same
        // FP32 bound)
#pragma unroll
        for (int w = 16, cnt = kRerankUnroll; cnt > 1; w >>= 1, cnt >>= 1) {
            const bool up = (lane & w) != 0;
#pragma unroll
            for (int j = 0; j < cnt / 2; ++j) {
                const float send = up ? acc[j] : acc[j + cnt / 2];
                const float keep = up ? acc[j + cnt / 2] : acc[j];
                acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, w);
            }
        }
        for (int o = 16 / kRerankUnroll; o; o >>= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
        constexpr int kLanesPerRow = 32 / kRerankUnroll;
        const int r = lane / kLanesPerRow;
        if (lane % kLanesPerRow == 0 && i + r < i1) {
            const float sc = acc[0];
            float xr = xn[0];
#pragma unroll
            for (int u = 1; u < kRerankUnroll; ++u) xr = r == u ? xn[u] : xr;
            const float e = __fmul_ru(__fmul_ru(kappa, qn), xr);
            loq[i + r] = __fsub_rd(sc, e);
            hiq[i + r] = __fadd_ru(sc, e);
        }
#pragma unroll
        for (int u = 0; u < kRerankUnroll; ++u) ps[u] = nps[u];
    }
}

__device__ void load_query(const float* __restrict__ Q, int64_t q, int d, int dp, float* qs) {
    for (int c = threadIdx.x; c < dp; c += blockDim.x) qs[c] = c < d ? Q[q * d + c] : 0.0f;
}

// grid (nq, chunks): the re-rank alone, for very large budgets.
template <typename T>
__global__ void __launch_bounds__(kRerankWarps * 32)
    rerank_fp32_kernel(const T* __restrict__ Xp, int dp, int d, const float* __restrict__ Q,
                       const uint32_t* __restrict__ cand, int64_t cap, int per_block,
                       const Boundary* __restrict__ bnd, const float* __restrict__ xnorm,
                       const float* __restrict__ qnorm, float kappa, float* __restrict__ lo,
                       float* __restrict__ hi) {
    NRLSH_PDL_ENTRY();
    extern __shared__ __align__(16) float qs[];
    const int64_t q = blockIdx.x;
    load_query(Q, q, d, dp, qs);
    __syncthreads();
    const Boundary b = bnd[q];
    const int64_t count = (int64_t)b.full + b.r;
    const int64_t i0 = (int64_t)blockIdx.y * per_block;
    dev_rerank(Xp, dp, qs, cand + q * cap, i0, min(count, i0 + per_block), xnorm, qnorm[q], kappa,
               lo + q * cap, hi + q * cap);
}

// ------------------------------------------------------------------- top-k

__device__ __forceinline__ uint32_t float_order(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float order_float(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Order-preserving integer image of a double (larger value, larger key).
__device__ __forceinline__ unsigned long long double_key(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// The same for an interval end point, with -0 and +0 mapped alike (so that
// comparing keys is comparing the values), and its inverse.
__device__ __forceinline__ unsigned long long interval_key(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    if ((u << 1) == 0ull) u = 0ull;
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}

// (s, id) beats (s', id') when s > s', or s == s' and id < id'.
__device__ __forceinline__ bool better(double s, int64_t id, double s2, int64_t id2) {
    return s > s2 || (s == s2 && id < id2);
}

// Find the digit holding the rem-th largest key: bins are scanned from 255
// down; warp 0 sums 8 bins per lane, scans the lanes, and the crossing lane
// walks its 8 bins.  Writes the digit and the rank left inside it.
__device__ void select_digit(const uint32_t* hist, int rem, int* dg_out, int* rem_out) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    uint32_t part = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) part += hist[255 - (lane * 8 + i)];
    uint32_t incl = part;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t excl = incl - part;
    if (excl < (uint32_t)rem && incl >= (uint32_t)rem) {
        int r = rem - (int)excl;
        for (int i = 0; i < 8; ++i) {
            const int dg = 255 - (lane * 8 + i);
            const int c = (int)hist[dg];
            if (c >= r) {
                *dg_out = dg;
                *rem_out = r;
                break;
            }
            r -= c;
        }
    }
}

constexpr int kRescoreSmem = 16384;  // bytes of staged contender rows
constexpr int kDot2Max = 512;        // contenders scored by the compensated FP32 tier

// Compensated dot products of two rows with the query at once (their loads in
// flight together); row 1 may be null (then only row 0 is summed).
template <typename T> struct RowDot2;
template <> struct RowDot2<float> {
    __device__ static void dot(const float* xr0, const float* xr1, const float* qs, int dp,
                               int lane, float (&sh)[2], float (&sl)[2]) {
        const float4* a4 = (const float4*)xr0;
        const float4* b4 = (const float4*)(xr1 ? xr1 : xr0);
        const float4* q4 = (const float4*)qs;
#pragma unroll 2
        for (int c = lane; c < dp / 4; c += 32) {
            const float4 x = a4[c], z = b4[c], y = q4[c];
            dot2_step(x.x, y.x, sh[0], sl[0]);
            dot2_step(z.x, y.x, sh[1], sl[1]);
            dot2_step(x.y, y.y, sh[0], sl[0]);
            dot2_step(z.y, y.y, sh[1], sl[1]);
            dot2_step(x.z, y.z, sh[0], sl[0]);
            dot2_step(z.z, y.z, sh[1], sl[1]);
            dot2_step(x.w, y.w, sh[0], sl[0]);
            dot2_step(z.w, y.w, sh[1], sl[1]);
        }
    }
};
template <> struct RowDot2<__nv_bfloat16> {
    __device__ static void dot(const __nv_bfloat16* xr0, const __nv_bfloat16* xr1, const float* qs,
                               int dp, int lane, float (&sh)[2], float (&sl)[2]) {
        const uint4* a = (const uint4*)xr0;
        const uint4* b = (const uint4*)(xr1 ? xr1 : xr0);
        for (int c = lane; c < dp / 8; c += 32) {
            const uint4 ra = a[c], rb = b[c];
            const __nv_bfloat162* ha = (const __nv_bfloat162*)&ra;
            const __nv_bfloat162* hb = (const __nv_bfloat162*)&rb;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 x = __bfloat1622float2(ha[i]), z = __bfloat1622float2(hb[i]);
                const float y0 = qs[c * 8 + 2 * i], y1 = qs[c * 8 + 2 * i + 1];
                dot2_step(x.x, y0, sh[0], sl[0]);
                dot2_step(z.x, y0, sh[1], sl[1]);
                dot2_step(x.y, y1, sh[0], sl[0]);
                dot2_step(z.y, y1, sh[1], sl[1]);
            }
        }
    }
};

// FP64 dot product of one stored row with the query (both zero-padded to dp, a
// multiple of 8): lane-strided over float4 / 8 x bf16 groups, exact products,
// returns the lane's sum and its sum of magnitudes.
template <typename T> struct RowDot64;
template <> struct RowDot64<float> {
    __device__ static void dot(const float* xr, const float* qs, int dp, int lane, double& sd,
                               double& sa) {
        const float4* x4 = (const float4*)xr;
        const float4* q4 = (const float4*)qs;
        for (int c = lane; c < dp / 4; c += 32) {
            const float4 x = x4[c], y = q4[c];
            const double p0 = (double)x.x * y.x, p1 = (double)x.y * y.y;
            const double p2 = (double)x.z * y.z, p3 = (double)x.w * y.w;
            sd += p0; sd += p1; sd += p2; sd += p3;
            sa += fabs(p0) + fabs(p1) + fabs(p2) + fabs(p3);
        }
    }
};
template <> struct RowDot64<__nv_bfloat16> {
    __device__ static void dot(const __nv_bfloat16* xr, const float* qs, int dp, int lane,
                               double& sd, double& sa) {
        for (int c = lane; c < dp / 8; c += 32) {
            const uint4 raw = ((const uint4*)xr)[c];
            const __nv_bfloat162* h = (const __nv_bfloat162*)&raw;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 x = __bfloat1622float2(h[i]);
                const double p0 = (double)x.x * qs[c * 8 + 2 * i];
                const double p1 = (double)x.y * qs[c * 8 + 2 * i + 1];
                sd += p0; sd += p1;
                sa += fabs(p0) + fabs(p1);
            }
        }
    }
};

// Block phase (256 threads), one query.  tau = k-th largest lower bound (MSD
// radix select on the order-preserving integer image of the floats).  Every
// candidate whose upper bound reaches tau is a contender; any true top-k member
// is one, because k candidates have FP64 scores >= their lower bounds >= tau.
// Contenders are rescored in FP64 in the fixed order (rows staged in shared
// memory) and the top k by (score desc, id asc) are taken by k rounds of a block
// arg-max.  qs holds the query (fp32 values, exact in FP64).
template <typename T>
__device__ void dev_topk(const float* __restrict__ loq, const float* __restrict__ hiq,
                         const uint32_t* __restrict__ candq, int64_t count, int kq, int k_out,
                         const T* __restrict__ Xp, int dp, int d, const float* qs, float qn,
                         const float* __restrict__ xnorm, const uint32_t* __restrict__ perm,
                         uint32_t* __restrict__ contq, double* __restrict__ contsq,
                         int64_t* __restrict__ ids_out, float* __restrict__ sc_out,
                         float* rows_s) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t prefix_s, mask_s;
    __shared__ int rem_s, dg_s;
    __shared__ uint32_t nc_s;
    __shared__ double best_s[8];
    __shared__ int64_t bid_s[8];
    __shared__ int bc_s[8];
    // the contenders' score intervals as order-preserving integer keys (compared on
    // the integer pipes: GB300's FP64 rate is a small fraction of its FP32 rate)
    __shared__ unsigned long long rank_lo[kDot2Max], rank_hi[kDot2Max];
    __shared__ uint16_t flagged[kDot2Max], flagged2[kDot2Max];
    __shared__ uint32_t nflag_s, nflag2_s;
    __shared__ uint32_t idc_s[kDot2Max];      // original ids of the contenders (compensated tier)
    __shared__ uint32_t cpos_s[kDot2Max];     // their storage positions
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float tau = -FLT_MAX;
    if (count > kq) {
        if (threadIdx.x == 0) {
            prefix_s = 0;
            mask_s = 0;
            rem_s = kq;
        }
        for (int shift = 24; shift >= 0; shift -= 8) {
            hist[threadIdx.x] = 0;
            __syncthreads();
            const uint32_t prefix = prefix_s, mask = mask_s;
            const int rem = rem_s;
            for (int64_t i = threadIdx.x; i < count; i += 256) {
                const uint32_t key = float_order(loq[i]);
                if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 0xFFu], 1u);
            }
            __syncthreads();
            select_digit(hist, rem, &dg_s, &rem_s);
            __syncthreads();
            if (threadIdx.x == 0) {
                prefix_s = prefix | ((uint32_t)dg_s << shift);
                mask_s = mask | (0xFFu << shift);
            }
            __syncthreads();
        }
        tau = order_float(prefix_s);
    }
    if (threadIdx.x == 0) nc_s = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < count; i += 256) {
        if (hiq[i] >= tau) {
            const uint32_t slot = atomicAdd(&nc_s, 1u);
            contq[slot] = (uint32_t)i;
            if (slot < (uint32_t)kDot2Max) cpos_s[slot] = candq[i];
        }
    }
    __syncthreads();
    const uint32_t nc = nc_s;
    const int rb = max(1, min(256, kRescoreSmem / (int)(sizeof(float) * dp)));
    if (nc <= (uint32_t)kDot2Max) {
        // Compensated FP32 tier (Ogita, Rump, Oishi, "Accurate sum and dot product",
        // 2005): a warp per two contenders, TwoProduct by fma and TwoSum per lane,
        // the same transformations across lanes.  With m terms per lane (mlane) and 5
        // tree levels, |hi + lo - q^T x| <= u^2 (2m(m+1) + 10(dp+32)) sum|q x|,
        // u = 2^-24; the bound below takes 4x that, plus the FP64 rounding of the
        // canonical in-order sum ((d+2) 2^-53 sum|q x|) and of hi + lo.
        const int mlane = sizeof(T) == 4 ? 4 * ((dp / 4 + 31) / 32) : 8 * ((dp / 8 + 31) / 32);
        const double c2 = 4.0 * 0x1p-48 * (2.0 * mlane * (mlane + 1) + 10.0 * (dp + 32)) +
                          (double)(d + 2) * 0x1p-53;
        // two contenders per warp at a time (c and c + 8 of each 16)
        for (uint32_t c0 = warp; c0 < nc; c0 += 16) {
            const uint32_t c1 = c0 + 8;
            const bool two = c1 < nc;
            const uint32_t pos0 = cpos_s[c0];
            const uint32_t pos1 = two ? cpos_s[c1] : pos0;
            // the lane's row norm and id, loaded while the rows are
            const uint32_t posl = lane == 0 ? pos0 : pos1;
            const float xnl = lane < 2 ? xnorm[posl] : 0.0f;
            const uint32_t idl = lane < 2 ? perm[posl] : 0u;
            float sh[2] = {0.0f, 0.0f}, sl[2] = {0.0f, 0.0f};
            RowDot2<T>::dot(Xp + (int64_t)pos0 * dp, two ? Xp + (int64_t)pos1 * dp : nullptr, qs, dp,
                            lane, sh, sl);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                for (int o = 16; o; o >>= 1) {
                    const float oh = __shfl_xor_sync(0xffffffffu, sh[h], o);
                    const float ol = __shfl_xor_sync(0xffffffffu, sl[h], o);
                    const float s2 = __fadd_rn(sh[h], oh);
                    const float bb = __fsub_rn(s2, sh[h]);
                    const float t = __fadd_rn(__fsub_rn(sh[h], __fsub_rn(s2, bb)), __fsub_rn(oh, bb));
                    sh[h] = s2;
                    sl[h] = __fadd_rn(__fadd_rn(sl[h], ol), t);
                }
            }
            if (lane < 2 && (lane == 0 || two)) {
                const uint32_t c = lane == 0 ? c0 : c1;
                const float vh = lane == 0 ? sh[0] : sh[1], vl = lane == 0 ? sl[0] : sl[1];
                const double v = __dadd_rn((double)vh, (double)vl);
                const double e = c2 * (double)qn * (double)xnl * (1.0 + 0x1p-20) +
                                 0x1p-52 * fabs(v) + 0x1p-120;
                rank_lo[c] = interval_key(__dsub_rd(v, e));
                rank_hi[c] = interval_key(__dadd_ru(v, e));
                contsq[c] = v;
                idc_s[c] = idl;
            }
        }
        __syncthreads();
        // exact tier only where the interval could change the outcome: it straddles
        // an fp32 rounding boundary, or it overlaps another contender's interval
        if (threadIdx.x == 0) nflag_s = 0;
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < nc; c += 256) {
            const unsigned long long lo_c = rank_lo[c], hi_c = rank_hi[c];
            bool flag = __double2float_rn(key_value(lo_c)) != __double2float_rn(key_value(hi_c));
            for (uint32_t c1 = 0; c1 < nc && !flag; ++c1)
                flag = c1 != c && rank_lo[c1] <= hi_c && lo_c <= rank_hi[c1];
            if (flag) flagged[atomicAdd(&nflag_s, 1u)] = (uint16_t)c;
        }
        __syncthreads();
        uint32_t nf = nflag_s;
        if (nf) {
            // FP64 warp tier for the flagged: exact products summed lane-strided
            // (per_lane terms per lane) and by a 5-level tree, at most per_lane + 5
            // rounded additions deep; the canonical in-order sum is within (d - 1) u
            // sum|q x| of the exact value, u = 2^-53, so an interval of
            // (d + per_lane + 8) u sum|q x| (1 + 2^-30) each side holds it.  Each
            // interval is narrowed to its intersection with the FP32 one.
            const int per_lane = sizeof(T) == 4 ? 4 * ((dp / 4 + 31) / 32) : 8 * ((dp / 8 + 31) / 32);
            const double cw = (double)(d + per_lane + 8) * 0x1p-53 * (1.0 + 0x1p-30);
            for (uint32_t f = warp; f < nf; f += 8) {
                const uint32_t c = flagged[f];
                double sd = 0.0, sa = 0.0;
                RowDot64<T>::dot(Xp + (int64_t)candq[contq[c]] * dp, qs, dp, lane, sd, sa);
                for (int o = 16; o; o >>= 1) {
                    sd += __shfl_xor_sync(0xffffffffu, sd, o);
                    sa += __shfl_xor_sync(0xffffffffu, sa, o);
                }
                if (lane == 0) {
                    const double e = __dmul_ru(cw, sa);
                    rank_lo[c] = max(rank_lo[c], interval_key(__dsub_rd(sd, e)));
                    rank_hi[c] = min(rank_hi[c], interval_key(__dadd_ru(sd, e)));
                    contsq[c] = sd;
                }
            }
            __syncthreads();
            // still undecided: the interval straddles an fp32 rounding boundary or
            // overlaps another contender's (intervals only shrank, so contenders not
            // flagged before stay decided)
            if (threadIdx.x == 0) nflag2_s = 0;
            __syncthreads();
            for (uint32_t f = threadIdx.x; f < nf; f += 256) {
                const uint32_t c = flagged[f];
                const unsigned long long lo_c = rank_lo[c], hi_c = rank_hi[c];
                bool flag = __double2float_rn(key_value(lo_c)) != __double2float_rn(key_value(hi_c));
                for (uint32_t c1 = 0; c1 < nc && !flag; ++c1)
                    flag = c1 != c && rank_lo[c1] <= hi_c && lo_c <= rank_hi[c1];
                if (flag) flagged2[atomicAdd(&nflag2_s, 1u)] = (uint16_t)c;
            }
            __syncthreads();
            nf = nflag2_s;
            for (uint32_t f = threadIdx.x; f < nf; f += 256) flagged[f] = flagged2[f];
            __syncthreads();
        }
        for (uint32_t f0 = 0; f0 < nf; f0 += rb) {
            const int nr = (int)min((uint32_t)rb, nf - f0);
            for (int i = threadIdx.x; i < nr * dp; i += 256) {
                const int r = i / dp, col = i % dp;
                rows_s[r * dp + col] = to_f32(Xp[(int64_t)candq[contq[flagged[f0 + r]]] * dp + col]);
            }
            __syncthreads();
            if (threadIdx.x < nr) {
                const float* xr = rows_s + threadIdx.x * dp;
                double acc = 0.0;
                for (int kk = 0; kk < d; ++kk) acc = fma((double)xr[kk], (double)qs[kk], acc);
                contsq[flagged[f0 + threadIdx.x]] = acc;
            }
            __syncthreads();
        }
    } else {
        for (uint32_t c0 = 0; c0 < nc; c0 += rb) {
            const int nr = (int)min((uint32_t)rb, nc - c0);
            for (int i = threadIdx.x; i < nr * dp; i += 256) {
                const int r = i / dp, col = i % dp;
                rows_s[r * dp + col] = to_f32(Xp[(int64_t)candq[contq[c0 + r]] * dp + col]);
            }
            __syncthreads();
            if (threadIdx.x < nr) {
                const float* xr = rows_s + threadIdx.x * dp;
                double acc = 0.0;
                for (int kk = 0; kk < d; ++kk) acc = fma((double)xr[kk], (double)qs[kk], acc);
                contsq[c0 + threadIdx.x] = acc;
            }
            __syncthreads();
        }
    }
    const int kk_out = (int)min((int64_t)kq, (int64_t)nc);
    if (nc <= (uint32_t)(kRescoreSmem / 16)) {
        // rank every contender by (score desc, id asc) against all others; ranks are
        // unique (ids are), so rank < k places the item directly
        unsigned long long* key_s = (unsigned long long*)rows_s;
        int64_t* id_s = (int64_t*)(key_s + nc);
        const bool have_ids = nc <= (uint32_t)kDot2Max;   // fetched by the compensated tier
        for (uint32_t c = threadIdx.x; c < nc; c += 256) {
            key_s[c] = double_key(contsq[c]);
            id_s[c] = have_ids ? (int64_t)idc_s[c] : (int64_t)perm[candq[contq[c]]];
        }
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < nc; c += 256) {
            const unsigned long long k0 = key_s[c];
            const int64_t i0 = id_s[c];
            int rank = 0;
            for (uint32_t c1 = 0; c1 < nc; ++c1) {
                const unsigned long long k1 = key_s[c1];
                rank += (k1 > k0) || (k1 == k0 && id_s[c1] < i0);
            }
            if (rank < kq) {
                ids_out[rank] = i0;
                sc_out[rank] = __double2float_rn(contsq[c]);
            }
        }
        __syncthreads();
    } else {
    for (int r = 0; r < kk_out; ++r) {
        double bs = -DBL_MAX;
        int64_t bi = INT64_MAX;
        int bc = -1;
        for (uint32_t c = threadIdx.x; c < nc; c += 256) {
            const uint32_t ci = contq[c];
            if (ci & 0x80000000u) continue;  // taken
            const double sc = contsq[c];
            const int64_t id = perm[candq[ci]];
            if (bc < 0 || better(sc, id, bs, bi)) {
                bs = sc;
                bi = id;
                bc = (int)c;
            }
        }
        for (int o = 16; o; o >>= 1) {
            const double s2 = __shfl_xor_sync(0xffffffffu, bs, o);
            const int64_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            const int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
            if (c2 >= 0 && (bc < 0 || better(s2, i2, bs, bi))) {
                bs = s2;
                bi = i2;
                bc = c2;
            }
        }
        if (lane == 0) {
            best_s[warp] = bs;
            bid_s[warp] = bi;
            bc_s[warp] = bc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int w0 = -1;
            for (int w = 0; w < 8; ++w) {
                if (bc_s[w] < 0) continue;
                if (w0 < 0 || better(best_s[w], bid_s[w], best_s[w0], bid_s[w0])) w0 = w;
            }
            ids_out[r] = bid_s[w0];
            sc_out[r] = __double2float_rn(best_s[w0]);
            contq[bc_s[w0]] |= 0x80000000u;
        }
        __syncthreads();
    }
    }
    for (int r = kk_out + threadIdx.x; r < k_out; r += 256) {
        ids_out[r] = -1;
        sc_out[r] = -INFINITY;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
    topk_kernel(const float* __restrict__ lo, const float* __restrict__ hi,
                const uint32_t* __restrict__ cand, int64_t cap, const Boundary* __restrict__ bnd,
                int k, const int32_t* __restrict__ ks, const T* __restrict__ Xp, int dp, int d,
                const float* __restrict__ Q, const float* __restrict__ xnorm,
                const float* __restrict__ qnorm, const uint32_t* __restrict__ perm,
                uint32_t* __restrict__ cont, double* __restrict__ cont_s,
                int64_t* __restrict__ out_ids, float* __restrict__ out_scores, int out_ld,
                const int* __restrict__ skip, int* __restrict__ report) {
    NRLSH_PDL_ENTRY();
    extern __shared__ __align__(16) float qs[];
    const int64_t q = blockIdx.x;
    // skip != null: the candidate lists come from a call whose kernels may have
    // stopped early (a bounded wait ran out); the row is then padded and the
    // error passed on to *report
    const int e = skip ? *skip : 0;
    if (e) {
        for (int r = threadIdx.x; r < out_ld; r += blockDim.x) {
            out_ids[q * out_ld + r] = -1;
            out_scores[q * out_ld + r] = -INFINITY;
        }
        if (q == 0 && threadIdx.x == 0) atomicCAS(report, 0, e);
        return;
    }
    load_query(Q, q, d, dp, qs);
    __syncthreads();
    const Boundary b = bnd[q];
    __shared__ __align__(16) float rows_s[kRescoreSmem / sizeof(float)];
    dev_topk(lo + q * cap, hi + q * cap, cand + q * cap, (int64_t)b.full + b.r,
             ks ? min(max(ks[q], 1), k) : k,
             out_ld, Xp, dp, d, qs, qnorm[q], xnorm, perm, cont + q * cap, cont_s + q * cap,
             out_ids + q * out_ld, out_scores + q * out_ld, rows_s);
}

// ----------------------------------------------------- fused probe + rerank

// Block per query: the bucket walk, the ordered candidate selection, the FP32
// re-rank and the exact top-k back to back, with the query, lam and the walk's
// scratch in shared memory (dynamic: dp floats, m words, m bytes).
template <typename T, typename C>
__global__ void __launch_bounds__(256, 4)
    probe_rerank_kernel(const uint32_t* __restrict__ H, const uint32_t* __restrict__ order, int m,
                        int L, int64_t n, const int64_t* __restrict__ seg, int64_t budget, const int64_t* __restrict__ budgets,
                        uint32_t flags, const C* __restrict__ codes, const C* __restrict__ qcodes,
                        const T* __restrict__ Xp, int dp, int d, const float* __restrict__ Q,
                        const float* __restrict__ xnorm, const float* __restrict__ qnorm,
                        float kappa, const uint32_t* __restrict__ perm, int k,
                        const int32_t* __restrict__ ks, uint32_t* __restrict__ cand,
                        float* __restrict__ lo, float* __restrict__ hi, uint32_t* __restrict__ cont,
                        double* __restrict__ cont_s, int64_t cap, int64_t* __restrict__ out_ids,
                        float* __restrict__ out_scores, int out_ld) {
    NRLSH_PDL_ENTRY();
    extern __shared__ __align__(16) float qs[];
    uint32_t* cntj = (uint32_t*)(qs + dp);
    uint8_t* lam_s = (uint8_t*)(cntj + m);
    const int64_t q = blockIdx.x;
    load_query(Q, q, d, dp, qs);
    const Boundary b = dev_threshold(H + q * m * (L + 1), order, m, L, n,
                                     budgets ? budgets[q] : budget, flags, cntj, lam_s);
    uint32_t* candq = cand + q * cap;
    __shared__ __align__(16) float phase_s[kRescoreSmem / sizeof(float)];  // select masks, then top-k rows
    dev_select(codes, qcodes[q], seg, m, L, lam_s, b, candq, (uint32_t*)phase_s);
    __syncthreads();
    const int64_t count = (int64_t)b.full + b.r;
    dev_rerank(Xp, dp, qs, candq, 0, count, xnorm, qnorm[q], kappa, lo + q * cap, hi + q * cap);
    __syncthreads();
    dev_topk(lo + q * cap, hi + q * cap, candq, count, ks ? ks[q] : k, out_ld, Xp, dp, d, qs,
             qnorm[q], xnorm, perm, cont + q * cap, cont_s + q * cap, out_ids + q * out_ld,
             out_scores + q * out_ld, phase_s);
}

// Persistent form: CTAs take queries from a device work counter until it passes
// nq, each reusing its own scratch slab (cand, lo, hi, cont: cap words each;
// cont_s: cap doubles).  Per-query budgets and k; rows of the outputs are k_max
// wide, padded with (-1, -inf).
//
// R is the row type of the gathered re-rank: T itself, or (fp32 items) a bf16
// copy Xr of the rows, whose scores' intervals also cover the copy's rounding
// (kappa); the exact top-k tiers always rescore from the stored rows Xp.
template <typename T, typename C, typename R>
__global__ void __launch_bounds__(256, 4)
    probe_rerank_persistent_kernel(const uint32_t* __restrict__ H, const uint32_t* __restrict__ order,
                                   int m, int L, int64_t n, const int64_t* __restrict__ seg,
                                   int64_t budget, const int64_t* __restrict__ budgets,
                                   const C* __restrict__ codes, const C* __restrict__ qcodes,
                                   const T* __restrict__ Xp, const R* __restrict__ Xr, int dp, int d,
                                   const float* __restrict__ Q, const float* __restrict__ xnorm,
                                   const float* __restrict__ qnorm, float kappa,
                                   const uint32_t* __restrict__ perm, const int32_t* __restrict__ ks,
                                   int k_max, uint32_t* __restrict__ slabs, int64_t cap,
                                   unsigned* __restrict__ work, int64_t nq,
                                   int64_t* __restrict__ out_ids, float* __restrict__ out_scores) {
    NRLSH_PDL_ENTRY();
    extern __shared__ __align__(16) float qs[];
    uint32_t* cntj = (uint32_t*)(qs + dp);
    uint8_t* lam_s = (uint8_t*)(cntj + m);
    __shared__ int64_t q_s;
    __shared__ __align__(16) float phase_s[kRescoreSmem / sizeof(float)];  // select masks, then top-k rows
    uint32_t* slab = slabs + (size_t)blockIdx.x * 6 * cap;
    uint32_t* cand = slab;
    float* lo = (float*)(slab + cap);
    float* hi = (float*)(slab + 2 * cap);
    uint32_t* cont = slab + 3 * cap;
    double* cont_s = (double*)(slab + 4 * cap);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) q_s = (int64_t)atomicAdd(work, 1u);
        __syncthreads();
        const int64_t q = q_s;
        if (q >= nq) break;
        load_query(Q, q, d, dp, qs);
        const int64_t Bq = min(max(budgets ? budgets[q] : budget, (int64_t)1), cap);
        const Boundary b = dev_threshold(H + q * m * (L + 1), order, m, L, n, Bq, 0u, cntj, lam_s);
        dev_select(codes, qcodes[q], seg, m, L, lam_s, b, cand, (uint32_t*)phase_s);
        __syncthreads();
        const int64_t count = (int64_t)b.full + b.r;
        dev_rerank(Xr, dp, qs, cand, 0, count, xnorm, qnorm[q], kappa, lo, hi);
        __syncthreads();
        dev_topk(lo, hi, cand, count, ks ? min(max(ks[q], 1), k_max) : k_max, k_max, Xp, dp, d,
                 qs, qnorm[q],
                 xnorm, perm, cont, cont_s,
                 out_ids + q * k_max, out_scores + q * k_max, phase_s);
    }
}

// ------------------------------------------- multi-table single probe (Alg. 2)

// The index's L bits read as T tables of Lt = L / T bits.  Item x is probed when
// some table field of v = c_x xor c_q is zero, tested for all fields at once:
// (v - ONES) & ~v & HIGHS != 0, ONES holding the low bit and HIGHS the high bit
// of every field.  A borrow can only cross into a field above a zero field, so
// the test is exact.
template <typename C>
__device__ __forceinline__ bool table_hit(C v, C ones, C highs) {
    return ((C)(v - ones) & (C)~v & highs) != 0;
}

// Block phase (256 threads): ordered compaction of C(q) over all n positions
// (storage order: sub-dataset, then id).  Warps own contiguous position ranges;
// a counting sweep, a scan over the 8 warps, then a writing sweep with ballot
// prefixes.  The first min(|C(q)|, cap) positions go to out; returns |C(q)|.
template <typename C>
__device__ int64_t dev_select_tables(const C* __restrict__ codes, C cq, int64_t n, C ones, C highs,
                                     uint32_t* __restrict__ out, int64_t cap) {
    __shared__ uint32_t wc[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t w0 = n * warp / 8, w1 = n * (warp + 1) / 8;
    uint32_t c = 0;
    for (int64_t base = w0; base < w1; base += 32) {
        const int64_t p = base + lane;
        const bool hit = p < w1 && table_hit<C>(cq ^ codes[p], ones, highs);
        c += __popc(__ballot_sync(0xffffffffu, hit));
    }
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    int64_t off = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
        off += w < warp ? wc[w] : 0u;
        total += wc[w];
    }
    for (int64_t base = w0; base < w1 && off < cap; base += 32) {
        const int64_t p = base + lane;
        const bool hit = p < w1 && table_hit<C>(cq ^ codes[p], ones, highs);
        const unsigned b = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int64_t slot = off + __popc(b & lt);
            if (slot < cap) out[slot] = (uint32_t)p;
        }
        off += __popc(b);
    }
    __syncthreads();
    return total;
}

// Block per query: C(q) only.  bnd[q].full = min(|C(q)|, cap) (r = 0), so the
// re-rank and top-k kernels of the multi-probe path take the list as it is.
template <typename C>
__global__ void __launch_bounds__(256)
    multitable_select_kernel(const C* __restrict__ codes, const C* __restrict__ qcodes, int64_t n,
                             C ones, C highs, uint32_t* __restrict__ cand, int64_t cap,
                             Boundary* __restrict__ bnd, int64_t* __restrict__ probed) {
    NRLSH_PDL_ENTRY();
    const int64_t q = blockIdx.x;
    const int64_t total = dev_select_tables<C>(codes, qcodes[q], n, ones, highs, cand + q * cap, cap);
    if (threadIdx.x == 0) {
        if (probed) probed[q] = total;
        bnd[q] = Boundary{0, 0, 0, (int32_t)min(total, cap)};
    }
}

// Work list of the re-rank: query q owns items [work_off[q], work_off[q+1]) of
// ceil(count_q / kWorkChunk) chunks each (one block of 1,024 threads; exclusive
// scan in tiles with a running carry).
constexpr int kWorkChunk = 256;

__global__ void __launch_bounds__(1024)
    work_offsets_kernel(const Boundary* __restrict__ bnd, int64_t nq, int64_t* __restrict__ work_off) {
    NRLSH_PDL_ENTRY();
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < nq; base += 1024) {
        const int64_t q = base + threadIdx.x;
        const int64_t v = q < nq ? ceil_div((int64_t)bnd[q].full + bnd[q].r, kWorkChunk) : 0;
        int64_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int64_t carry = carry_s;
        if (q < nq) work_off[q] = carry + (warp ? wsum[warp - 1] : 0) + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) work_off[nq] = carry_s;
}

// Persistent FP32 re-rank over the work list: blocks take chunks from *work_ctr,
// find their query by binary search in work_off and score kWorkChunk candidates,
// so one query with a huge C(q) is spread over every SM.
template <typename T>
__global__ void __launch_bounds__(kRerankWarps * 32)
    rerank_work_kernel(const T* __restrict__ Xp, int dp, int d, const float* __restrict__ Q,
                       const uint32_t* __restrict__ cand, int64_t cap,
                       const Boundary* __restrict__ bnd, const int64_t* __restrict__ work_off,
                       int64_t nq, unsigned long long* __restrict__ work_ctr,
                       const float* __restrict__ xnorm, const float* __restrict__ qnorm,
                       float kappa, float* __restrict__ lo, float* __restrict__ hi) {
    NRLSH_PDL_ENTRY();
    extern __shared__ __align__(16) float qs[];
    __shared__ int64_t w_s;
    const int64_t total = work_off[nq];
    int64_t cur_q = -1;
    for (;;) {
        if (threadIdx.x == 0) w_s = (int64_t)atomicAdd(work_ctr, 1ull);
        __syncthreads();
        const int64_t w = w_s;
        if (w >= total) break;
        int64_t a = 0, b = nq;                 // work_off[a] <= w < work_off[b]
        while (b - a > 1) {
            const int64_t mid = (a + b) >> 1;
            if (work_off[mid] <= w) a = mid; else b = mid;
        }
        const int64_t q = a;
        if (q != cur_q) {
            load_query(Q, q, d, dp, qs);
            cur_q = q;
        }
        __syncthreads();
        const int64_t count = (int64_t)bnd[q].full + bnd[q].r;
        const int64_t i0 = (w - work_off[q]) * kWorkChunk;
        dev_rerank(Xp, dp, qs, cand + q * cap, i0, min(count, i0 + kWorkChunk), xnorm, qnorm[q],
                   kappa, lo + q * cap, hi + q * cap);
        __syncthreads();
    }
}

// Block per query: single-probe selection over the T tables, FP32 re-rank and the
// exact top-k of the first min(|C(q)|, cap) candidates; probed[q] = |C(q)|.  With
// cand_ids non-null only the candidates' ids are written (cand_ld per query).
template <typename T, typename C>
__global__ void __launch_bounds__(256)
    multitable_kernel(const C* __restrict__ codes, const C* __restrict__ qcodes, int64_t n, C ones,
                      C highs, const T* __restrict__ Xp, int dp, int d,
                      const float* __restrict__ Q, const float* __restrict__ xnorm,
                      const float* __restrict__ qnorm, float kappa,
                      const uint32_t* __restrict__ perm, int k, uint32_t* __restrict__ cand,
                      float* __restrict__ lo, float* __restrict__ hi, uint32_t* __restrict__ cont,
                      double* __restrict__ cont_s, int64_t cap, int64_t* __restrict__ out_ids,
                      float* __restrict__ out_scores, int out_ld, int64_t* __restrict__ probed,
                      int32_t* __restrict__ cand_ids, int64_t cand_ld) {
    NRLSH_PDL_ENTRY();
    extern __shared__ __align__(16) float qs[];
    const int64_t q = blockIdx.x;
    uint32_t* candq = cand + q * cap;
    const int64_t total = dev_select_tables<C>(codes, qcodes[q], n, ones, highs, candq, cap);
    const int64_t count = min(total, cap);
    if (threadIdx.x == 0 && probed) probed[q] = total;
    if (cand_ids) {
        for (int64_t i = threadIdx.x; i < count; i += blockDim.x)
            cand_ids[q * cand_ld + i] = (int32_t)perm[candq[i]];
        return;
    }
    load_query(Q, q, d, dp, qs);
    __syncthreads();
    dev_rerank(Xp, dp, qs, candq, 0, count, xnorm, qnorm[q], kappa, lo + q * cap, hi + q * cap);
    __syncthreads();
    __shared__ __align__(16) float rows_s[kRescoreSmem / sizeof(float)];
    dev_topk(lo + q * cap, hi + q * cap, candq, count, k, out_ld, Xp, dp, d, qs, qnorm[q], xnorm,
             perm, cont + q * cap, cont_s + q * cap, out_ids + q * out_ld, out_scores + q * out_ld,
             rows_s);
}

__global__ void cand_to_ids_kernel(const uint32_t* __restrict__ cand, int64_t cap,
                                   const Boundary* __restrict__ bnd,
                                   const uint32_t* __restrict__ perm, int32_t* out, int64_t out_cap,
                                   int64_t* count, const int* __restrict__ skip,
                                   int* __restrict__ report) {
    NRLSH_PDL_ENTRY();
    const int64_t q = blockIdx.x;
    const int e = skip ? *skip : 0;     // as in topk_kernel
    if (e) {
        if (threadIdx.x == 0) count[q] = 0;
        if (q == 0 && threadIdx.x == 0) atomicCAS(report, 0, e);
        return;
    }
    const Boundary b = bnd[q];
    const int64_t cnt = (int64_t)b.full + b.r;
    if (threadIdx.x == 0) count[q] = cnt;
    const int64_t lim = min(cnt, out_cap);
    for (int64_t i = threadIdx.x; i < lim; i += blockDim.x)
        out[q * out_cap + i] = (int32_t)perm[cand[q * cap + i]];
}

}  // namespace

// ---------------------------------------------------------------- launchers

// cudaFuncAttributeMaxDynamicSharedMemorySize raised as needed, per kernel,
// device and thread (the attribute only grows).
cudaError_t ensure_dyn_smem(const void* kern, size_t bytes) {
    static thread_local std::unordered_map<const void*, std::pair<int, size_t>> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    auto& s = set[kern];
    if (s.first == dev && s.second >= bytes) return cudaSuccess;
    if (s.first != dev) s = {dev, 0};
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) s.second = bytes;
    return e;
}

// CTAs of 256 threads that fit on the device at once (at most nq).
cudaError_t resident_ctas(const void* kern, size_t smem, int64_t nq, int* ctas) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    *ctas = (int)std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t)std::max(per_sm, 1) * sms));
    return cudaSuccess;
}

cudaError_t launch_row_norm_bound(const float* Q, int64_t nq, int d, float* qnorm,
                                  cudaStream_t st) {
    return launch("row_norm_bound", row_norm_bound_kernel, dim3((unsigned)ceil_div(nq * 32, 256)),
                  dim3(256), 0, st, Q, nq, d, qnorm);
}

cudaError_t launch_hist(const void* codes, const void* qcodes, int code_bytes, int64_t nq, int m,
                        int L, const PosTile* tiles, int ntiles, uint32_t* H, cudaStream_t st,
                        int queries_per_block, bool exclusive) {
    const int qb = queries_per_block;
    const dim3 grid((unsigned)ntiles, (unsigned)ceil_div(nq, qb));
    const size_t smem = 16384 + sizeof(uint32_t) * (size_t)(L + 1) * kHistThreads;
#define NRLSH_HIST_(C_, Q_)                                                                     \
    {                                                                                       \
        cudaError_t e = ensure_dyn_smem((const void*)hist_kernel<C_, Q_>, smem);            \
        if (e != cudaSuccess) return e;                                                     \
        return launch(sizeof(C_) == 4 ? "hist_u32" : "hist_u64", hist_kernel<C_, Q_>, grid,  \
                      dim3(kHistThreads), smem, st, (const C_*)codes, (const C_*)qcodes, nq, m, \
                      L, tiles, H, exclusive ? 1 : 0);                                      \
    }
    if (code_bytes == 4) {
        if (qb == 32) NRLSH_HIST_(uint32_t, 32)
        if (qb == 128) NRLSH_HIST_(uint32_t, 128)
        NRLSH_HIST_(uint32_t, 64)
    }
    if (qb == 32) NRLSH_HIST_(uint64_t, 32)
    if (qb == 128) NRLSH_HIST_(uint64_t, 128)
    NRLSH_HIST_(uint64_t, 64)
#undef NRLSH_HIST_
}

cudaError_t launch_threshold(const uint32_t* H, const uint32_t* order, int m, int L, int64_t nq,
                             int64_t n, int64_t budget, const int64_t* budgets, uint32_t flags,
                             uint8_t* lam, Boundary* bnd, cudaStream_t st) {
    return launch("threshold", threshold_kernel, dim3((unsigned)nq), dim3(256),
                  (sizeof(uint32_t) + 1) * (size_t)m, st, H, order, m, L, nq, n, budget, budgets,
                  flags, lam, bnd);
}

cudaError_t launch_tc_walk(const uint32_t* H, const uint32_t* order, int m, int L, int64_t n,
                           const int64_t* seg, int64_t nq, int64_t budget, const int64_t* budgets,
                           int64_t cap, uint32_t flags, const void* codes, const void* qcodes,
                           int code_bytes, uint8_t* lam, uint32_t* off, TcBoundary* tb,
                           Boundary* bnd, uint8_t* work_flag, int nqt, const int* err,
                           cudaStream_t st) {
    const size_t smem = (sizeof(uint32_t) + 1) * (size_t)m;
    if (code_bytes == 4)
        return launch("tc_walk", tc_walk_kernel<uint32_t>, dim3((unsigned)nq), dim3(256), smem, st, H,
                      order, m, L, n, seg, budget, budgets, cap, flags, (const uint32_t*)codes,
                      (const uint32_t*)qcodes, lam, off, tb, bnd, work_flag, nqt, err);
    return launch("tc_walk", tc_walk_kernel<uint64_t>, dim3((unsigned)nq), dim3(256), smem, st, H,
                  order, m, L, n, seg, budget, budgets, cap, flags, (const uint64_t*)codes,
                  (const uint64_t*)qcodes, lam, off, tb, bnd, work_flag, nqt, err);
}

cudaError_t launch_work_list(const uint8_t* flag, int nflag, uint32_t* list, uint32_t* count,
                             cudaStream_t st) {
    return launch("work_list", work_list_kernel, dim3(1), dim3(1024), 0, st, flag, nflag, list,
                  count);
}

cudaError_t launch_select(const void* codes, const void* qcodes, int code_bytes, const int64_t* seg, int m,
                          int L, int64_t nq, const uint8_t* lam, const Boundary* bnd,
                          uint32_t* cand, int64_t cap, cudaStream_t st) {
    if (code_bytes == 4)
        return launch("select_u32", select_kernel<uint32_t>, dim3((unsigned)nq), dim3(256),
                      (size_t)m, st, (const uint32_t*)codes, (const uint32_t*)qcodes, seg, m, L, lam,
                      bnd, cand, cap);
    return launch("select_u64", select_kernel<uint64_t>, dim3((unsigned)nq), dim3(256), (size_t)m,
                  st, (const uint64_t*)codes, (const uint64_t*)qcodes, seg, m, L, lam, bnd, cand,
                  cap);
}

cudaError_t launch_rerank_fp32(const void* Xp, nrlsh_dtype dt, int dp, int d, const float* Q,
                               int64_t nq, const uint32_t* cand, int64_t cap, const Boundary* bnd,
                               const float* xnorm, const float* qnorm, float* lo, float* hi,
                               cudaStream_t st) {
    int64_t per_block = 64;
    while (ceil_div(cap, per_block) > 65535) per_block *= 2;
    const dim3 grid((unsigned)nq, (unsigned)ceil_div(cap, per_block));
    const float kappa = (float)(d + 2) * 0x1p-22f;
    const size_t smem = sizeof(float) * (size_t)dp;
    if (dt == NRLSH_BF16)
        return launch("rerank_fp32_bf16", rerank_fp32_kernel<__nv_bfloat16>, grid,
                      dim3(kRerankWarps * 32), smem, st, (const __nv_bfloat16*)Xp, dp, d, Q, cand,
                      cap, (int)per_block, bnd, xnorm, qnorm, kappa, lo, hi);
    return launch("rerank_fp32", rerank_fp32_kernel<float>, grid, dim3(kRerankWarps * 32), smem, st,
                  (const float*)Xp, dp, d, Q, cand, cap, (int)per_block, bnd, xnorm, qnorm, kappa,
                  lo, hi);
}

cudaError_t launch_topk(const float* lo, const float* hi, const uint32_t* cand, int64_t cap,
                        const Boundary* bnd, int64_t nq, int k, const int32_t* ks,
                        const void* Xp, nrlsh_dtype dt, int dp, int d, const float* Q,
                        const float* xnorm, const float* qnorm, const uint32_t* perm,
                        uint32_t* cont, double* cont_s, int64_t* out_ids, float* out_scores,
                        int out_ld, cudaStream_t st, const int* skip, int* report) {
    const size_t smem = sizeof(float) * (size_t)dp;
    if (dt == NRLSH_BF16)
        return launch("topk_bf16", topk_kernel<__nv_bfloat16>, dim3((unsigned)nq), dim3(256), smem, st,
                      lo, hi, cand, cap, bnd, k, ks, (const __nv_bfloat16*)Xp, dp, d, Q, xnorm, qnorm,
                      perm, cont, cont_s, out_ids, out_scores, out_ld, skip, report);
    return launch("topk", topk_kernel<float>, dim3((unsigned)nq), dim3(256), smem, st, lo, hi, cand,
                  cap, bnd, k, ks, (const float*)Xp, dp, d, Q, xnorm, qnorm, perm, cont, cont_s,
                  out_ids, out_scores, out_ld, skip, report);
}

cudaError_t launch_probe_rerank(const uint32_t* H, const uint32_t* order, int m, int L, int64_t n,
                                const int64_t* seg, int64_t nq, int64_t budget,
                                const int64_t* budgets, uint32_t flags, const void* codes,
                                const void* qcodes, int code_bytes, const void* Xp, nrlsh_dtype dt,
                                int dp, int d, const float* Q, const float* xnorm,
                                const float* qnorm, const uint32_t* perm, int k, const int32_t* ks,
                                uint32_t* cand, float* lo, float* hi, uint32_t* cont,
                                double* cont_s, int64_t cap, int64_t* out_ids, float* out_scores,
                                int out_ld, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)dp + (sizeof(uint32_t) + 1) * (size_t)m;
    const float kappa = (float)(d + 2) * 0x1p-22f;
    const dim3 grid((unsigned)nq);
#define NRLSH_PR(T_, C_, NAME)                                                                  \
    {                                                                                           \
        auto kern = probe_rerank_kernel<T_, C_>;                                                \
        cudaError_t e = ensure_dyn_smem((const void*)kern, smem);                               \
        if (e != cudaSuccess) return e;                                                         \
        return launch(NAME, kern, grid, dim3(256), smem, st, H, order, m, L, n, seg, budget, budgets, \
                      flags, (const C_*)codes, (const C_*)qcodes, (const T_*)Xp, dp, d, Q, xnorm,\
                      qnorm, kappa, perm, k, ks, cand, lo, hi, cont, cont_s, cap, out_ids,       \
                      out_scores, out_ld);                                                      \
    }
    if (dt == NRLSH_BF16) {
        if (code_bytes == 4) NRLSH_PR(__nv_bfloat16, uint32_t, "probe_rerank_bf16")
        NRLSH_PR(__nv_bfloat16, uint64_t, "probe_rerank_bf16")
    }
    if (code_bytes == 4) NRLSH_PR(float, uint32_t, "probe_rerank")
    NRLSH_PR(float, uint64_t, "probe_rerank")
#undef NRLSH_PR
}

cudaError_t launch_probe_rerank_persistent(const uint32_t* H, const uint32_t* order, int m, int L,
                                           int64_t n, const int64_t* seg, int64_t budget,
                                           const int64_t* budgets,
                                           const void* codes, const void* qcodes, int code_bytes,
                                           const void* Xp, nrlsh_dtype dt, int dp, int d,
                                           const float* Q, const float* xnorm, const float* qnorm,
                                           const uint32_t* perm, const int32_t* ks, int k_max,
                                           uint32_t* slabs, int64_t cap, int ctas, unsigned* work,
                                           int64_t nq, int64_t* out_ids, float* out_scores,
                                           cudaStream_t st, const __nv_bfloat16* Xr16) {
    const size_t smem = sizeof(float) * (size_t)dp + (sizeof(uint32_t) + 1) * (size_t)m;
    const float kappa32 = (float)(d + 2) * 0x1p-22f;
    const float kappa = Xr16 && dt == NRLSH_F32 ? rerank_bf16_rows_bound(d) : kappa32;
#define NRLSH_PP(T_, C_, R_, XR_, NAME)                                                         \
    {                                                                                           \
        auto kern = probe_rerank_persistent_kernel<T_, C_, R_>;                                 \
        cudaError_t e = ensure_dyn_smem((const void*)kern, smem);                               \
        if (e != cudaSuccess) return e;                                                         \
        if (ctas <= 0) {                                                                        \
            e = resident_ctas((const void*)kern, smem, nq, &ctas);                              \
            if (e != cudaSuccess) return e;                                                     \
        }                                                                                       \
        return launch(NAME, kern, dim3((unsigned)ctas), dim3(256), smem, st, H, order, m, L, n,  \
                      seg, budget, budgets, (const C_*)codes, (const C_*)qcodes, (const T_*)Xp,  \
                      (const R_*)(XR_), dp, d, Q, xnorm, qnorm, kappa, perm, ks, k_max, slabs,   \
                      cap, work, nq, out_ids, out_scores);                                      \
    }
    if (dt == NRLSH_BF16) {
        if (code_bytes == 4)
            NRLSH_PP(__nv_bfloat16, uint32_t, __nv_bfloat16, Xp, "probe_rerank_persistent_bf16")
        NRLSH_PP(__nv_bfloat16, uint64_t, __nv_bfloat16, Xp, "probe_rerank_persistent_bf16")
    }
    if (Xr16) {
        if (code_bytes == 4)
            NRLSH_PP(float, uint32_t, __nv_bfloat16, Xr16, "probe_rerank_persistent_bf16rows")
        NRLSH_PP(float, uint64_t, __nv_bfloat16, Xr16, "probe_rerank_persistent_bf16rows")
    }
    if (code_bytes == 4) NRLSH_PP(float, uint32_t, float, Xp, "probe_rerank_persistent")
    NRLSH_PP(float, uint64_t, float, Xp, "probe_rerank_persistent")
#undef NRLSH_PP
}

float rerank_bf16_rows_bound(int d) {
    // x~ = bf16(x) = x (1 + delta), |delta| <= 2^-8 (an 8-bit significand, round to
    // nearest): |q.x~ - q.x| <= 2^-8 sum|q x|; the FP32 sum of the q_k x~_k within
    // (d + 2) 2^-22 sum|q x~| (4x the first-order bound), and the canonical FP64
    // in-order sum's own (d + 2) 2^-53, all relative to sum|q x| <= ||q|| ||x||
    const double c = (0x1p-8 + (d + 2.0) * 0x1p-22 * (1.0 + 0x1p-8) + (d + 2.0) * 0x1p-53) *
                     (1.0 + 0x1p-20);
    float f = (float)c;
    if ((double)f < c) f = nextafterf(f, 1.0f);
    return f;
}

cudaError_t launch_multitable(const void* codes, const void* qcodes, int code_bytes, int64_t n,
                              int L, int tables, const void* Xp, nrlsh_dtype dt, int dp, int d,
                              const float* Q, const float* xnorm, const float* qnorm,
                              const uint32_t* perm, int k, uint32_t* cand, float* lo, float* hi,
                              uint32_t* cont, double* cont_s, int64_t cap, int64_t nq,
                              int64_t* out_ids, float* out_scores, int out_ld, int64_t* probed,
                              int32_t* cand_ids, int64_t cand_ld, cudaStream_t st) {
    const int Lt = L / tables;
    uint64_t ones = 0;
    for (int t = 0; t < tables; ++t) ones |= 1ull << (t * Lt);
    const uint64_t highs = ones << (Lt - 1);
    const size_t smem = sizeof(float) * (size_t)dp;
    const float kappa = (float)(d + 2) * 0x1p-22f;
    const dim3 grid((unsigned)nq);
#define NRLSH_MT(T_, C_, NAME)                                                                 \
    {                                                                                          \
        auto kern = multitable_kernel<T_, C_>;                                                 \
        cudaError_t e = ensure_dyn_smem((const void*)kern, smem);                              \
        if (e != cudaSuccess) return e;                                                        \
        return launch(NAME, kern, grid, dim3(256), smem, st, (const C_*)codes,                 \
                      (const C_*)qcodes, n, (C_)ones, (C_)highs, (const T_*)Xp, dp, d, Q,      \
                      xnorm, qnorm, kappa, perm, k, cand, lo, hi, cont, cont_s, cap, out_ids,  \
                      out_scores, out_ld, probed, cand_ids, cand_ld);                          \
    }
    if (dt == NRLSH_BF16) {
        if (code_bytes == 4) NRLSH_MT(__nv_bfloat16, uint32_t, "multitable_bf16")
        NRLSH_MT(__nv_bfloat16, uint64_t, "multitable_bf16")
    }
    if (code_bytes == 4) NRLSH_MT(float, uint32_t, "multitable")
    NRLSH_MT(float, uint64_t, "multitable")
#undef NRLSH_MT
}

cudaError_t launch_multitable_select(const void* codes, const void* qcodes, int code_bytes,
                                     int64_t n, int L, int tables, uint32_t* cand, int64_t cap,
                                     int64_t nq, Boundary* bnd, int64_t* probed, cudaStream_t st) {
    const int Lt = L / tables;
    uint64_t ones = 0;
    for (int t = 0; t < tables; ++t) ones |= 1ull << (t * Lt);
    const uint64_t highs = ones << (Lt - 1);
    if (code_bytes == 4)
        return launch("multitable_select", multitable_select_kernel<uint32_t>, dim3((unsigned)nq),
                      dim3(256), 0, st, (const uint32_t*)codes, (const uint32_t*)qcodes, n,
                      (uint32_t)ones, (uint32_t)highs, cand, cap, bnd, probed);
    return launch("multitable_select", multitable_select_kernel<uint64_t>, dim3((unsigned)nq),
                  dim3(256), 0, st, (const uint64_t*)codes, (const uint64_t*)qcodes, n, ones, highs,
                  cand, cap, bnd, probed);
}

cudaError_t launch_rerank_work(const void* Xp, nrlsh_dtype dt, int dp, int d, const float* Q,
                               int64_t nq, const uint32_t* cand, int64_t cap, const Boundary* bnd,
                               int64_t* work_off, unsigned long long* work_ctr, const float* xnorm,
                               const float* qnorm, float* lo, float* hi, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(work_ctr, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = launch("work_offsets", work_offsets_kernel, dim3(1), dim3(1024), 0, st, bnd, nq, work_off);
    if (e != cudaSuccess) return e;
    const float kappa = (float)(d + 2) * 0x1p-22f;
    const size_t smem = sizeof(float) * (size_t)dp;
    const dim3 grid(4 * 152);
    if (dt == NRLSH_BF16)
        return launch("rerank_work_bf16", rerank_work_kernel<__nv_bfloat16>, grid,
                      dim3(kRerankWarps * 32), smem, st, (const __nv_bfloat16*)Xp, dp, d, Q, cand,
                      cap, bnd, (const int64_t*)work_off, nq, work_ctr, xnorm, qnorm, kappa, lo, hi);
    return launch("rerank_work", rerank_work_kernel<float>, grid, dim3(kRerankWarps * 32), smem, st,
                  (const float*)Xp, dp, d, Q, cand, cap, bnd, (const int64_t*)work_off, nq,
                  work_ctr, xnorm, qnorm, kappa, lo, hi);
}

int probe_rerank_ctas(nrlsh_dtype dt, int code_bytes, int dp, int m, int64_t nq) {
    const size_t smem = sizeof(float) * (size_t)dp + (sizeof(uint32_t) + 1) * (size_t)m;
    using BF = __nv_bfloat16;
    const void* kern =
        dt == NRLSH_BF16
            ? (code_bytes == 4 ? (const void*)probe_rerank_persistent_kernel<BF, uint32_t, BF>
                               : (const void*)probe_rerank_persistent_kernel<BF, uint64_t, BF>)
            : (code_bytes == 4 ? (const void*)probe_rerank_persistent_kernel<float, uint32_t, float>
                               : (const void*)probe_rerank_persistent_kernel<float, uint64_t, float>);
    int ctas = 1;
    if (ensure_dyn_smem(kern, smem) != cudaSuccess || resident_ctas(kern, smem, nq, &ctas) != cudaSuccess)
        return (int)std::max<int64_t>(1, std::min<int64_t>(nq, 152));
    return ctas;
}

cudaError_t launch_cand_to_ids(const uint32_t* cand, int64_t cap, const Boundary* bnd,
                               const uint32_t* perm, int64_t nq, int32_t* out, int64_t out_cap,
                               int64_t* count, cudaStream_t st, const int* skip, int* report) {
    return launch("cand_to_ids", cand_to_ids_kernel, dim3((unsigned)nq), dim3(256), 0, st, cand,
                  cap, bnd, perm, out, out_cap, count, skip, report);
}

}  // namespace nrlsh
