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

#include <cfloat>

namespace nrlsh {

namespace {

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

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

constexpr int kHistQ = 128;  // queries per block, one per thread

// Block: one position tile (inside one sub-dataset) x 128 queries.  The tile's
// codes sit in shared memory and are read by broadcast; each thread keeps a
// private histogram column (uint16, tile length <= 4096) indexed [l][thread],
// so increments never conflict on a bank.
template <typename C>
__global__ void __launch_bounds__(kHistQ)
    hist_kernel(const C* __restrict__ codes, const C* __restrict__ qcodes, int64_t nq, int m, int L,
                const PosTile* __restrict__ tiles, uint32_t* __restrict__ H) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int kTile = 16384 / sizeof(C);
    C* cs = (C*)smem_raw;
    uint16_t* hist = (uint16_t*)(smem_raw + 16384);
    const PosTile t = tiles[blockIdx.x];
    const int64_t q = (int64_t)blockIdx.y * kHistQ + threadIdx.x;
    for (int i = threadIdx.x; i < t.len; i += kHistQ) cs[i] = codes[t.start + i];
    for (int l = 0; l <= L; ++l) hist[l * kHistQ + threadIdx.x] = 0;
    __syncthreads();
    if (q >= nq) return;
    const C cq = qcodes[q];
    for (int i = 0; i < t.len; ++i) {
        const int l = L - popc_word(cq ^ cs[i]);
        hist[l * kHistQ + threadIdx.x] += 1;
    }
    uint32_t* Hq = H + ((int64_t)q * m + t.seg) * (L + 1);
    for (int l = 0; l <= L; ++l) {
        const uint32_t v = hist[l * kHistQ + threadIdx.x];
        if (v) atomicAdd(&Hq[l], v);
    }
    (void)kTile;
}

// --------------------------------------------------------------- threshold

// Block per query.  Walks the buckets in probing order with a block scan of
// their sizes until the running total reaches B' = min(B, n).  The boundary
// bucket t* and everything before it define the probe: buckets before t* are
// taken whole; within sub-dataset j they are l = L, L-1, ..., so
// lam_j = L + 1 - (number of buckets of j before t*).
__global__ void __launch_bounds__(256)
    threshold_kernel(const uint32_t* __restrict__ H, const uint32_t* __restrict__ order, int m,
                     int L, int64_t nq, int64_t n, int64_t budget,
                     const int64_t* __restrict__ budgets, uint32_t flags,
                     uint8_t* __restrict__ lam, Boundary* __restrict__ bnd) {
    extern __shared__ uint32_t cntj[];
    __shared__ uint32_t warp_tot[8];
    __shared__ int tstar_s;
    __shared__ uint32_t before_s;
    const int64_t q = blockIdx.x;
    const int ncls = m * (L + 1);
    const uint32_t* Hq = H + q * ncls;
    int64_t B = budgets ? budgets[q] : budget;
    const uint32_t Bp = (uint32_t)(B < n ? B : n);
    for (int j = threadIdx.x; j < m; j += 256) cntj[j] = 0;
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
    for (int t = threadIdx.x; t < tstar; t += 256) atomicAdd(&cntj[order[t] / (L + 1)], 1u);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += 256) lam[q * m + j] = (uint8_t)(L + 1 - cntj[j]);
    if (threadIdx.x == 0) {
        const uint32_t cid = order[tstar];
        Boundary b;
        b.j = (int32_t)(cid / (L + 1));
        b.l = (int32_t)(cid % (L + 1));
        b.full = (int32_t)before_s;
        b.r = (flags & NRLSH_WHOLE_BUCKETS) ? (int32_t)Hq[cid] : (int32_t)(Bp - before_s);
        bnd[q] = b;
    }
}

// ------------------------------------------------------------------ select

constexpr int kSelV = 4;  // consecutive positions per thread per step

// Block per query, ordered compaction over all storage positions.  Items of
// whole buckets go to cand[0, full) in position order; boundary-bucket items
// go to cand[full, full + r), the first r of them in position (= id) order.
template <typename C>
__global__ void __launch_bounds__(256)
    select_kernel(const C* __restrict__ codes, const C* __restrict__ qcodes, int64_t n, int m, int L,
                  const uint8_t* __restrict__ lam, const Boundary* __restrict__ bnd,
                  uint32_t* __restrict__ cand, int64_t cap) {
    extern __shared__ uint8_t lam_s[];
    __shared__ uint32_t warp_tot[8];
    const int64_t q = blockIdx.x;
    for (int j = threadIdx.x; j < m; j += 256) lam_s[j] = lam[q * m + j];
    const Boundary b = bnd[q];
    const C cq = qcodes[q];
    uint32_t* out = cand + q * cap;
    __syncthreads();
    uint32_t run_f = 0, run_b = 0;
    for (int64_t base = 0; base < n; base += 256 * kSelV) {
        const int64_t p0 = base + (int64_t)threadIdx.x * kSelV;
        bool f[kSelV], bb[kSelV];
        uint32_t tf = 0, tb = 0;
        if (p0 < n) {
            int32_t j = seg_of(p0, n, m);
            int64_t next = seg_start(j + 1, n, m);
#pragma unroll
            for (int i = 0; i < kSelV; ++i) {
                const int64_t p = p0 + i;
                f[i] = bb[i] = false;
                if (p < n) {
                    while (p >= next) next = seg_start(++j + 1, n, m);
                    const int l = L - popc_word(cq ^ codes[p]);
                    f[i] = l >= (int)lam_s[j];
                    bb[i] = (j == b.j) && (l == b.l);
                }
                tf += f[i];
                tb += bb[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < kSelV; ++i) f[i] = bb[i] = false;
        }
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(tf | (tb << 16), &total, warp_tot);
        uint32_t ef = run_f + (ex & 0xFFFFu), eb = run_b + (ex >> 16);
#pragma unroll
        for (int i = 0; i < kSelV; ++i) {
            const uint32_t p = (uint32_t)(p0 + i);
            if (f[i]) out[ef++] = p;
            if (bb[i]) {
                if (eb < (uint32_t)b.r) out[b.full + eb] = p;
                ++eb;
            }
        }
        run_f += total & 0xFFFFu;
        run_b += total >> 16;
        if (run_f >= (uint32_t)b.full && run_b >= (uint32_t)b.r) break;  // uniform
    }
}

// ------------------------------------------------------------------ rerank

constexpr int kRerankWarps = 8;

template <typename T> struct RowDot;

template <> struct RowDot<float> {
    // dp is a multiple of 8, rows are 16-byte aligned
    __device__ static float dot(const float* __restrict__ row, const float* qs, int dp, int lane) {
        const float4* r4 = (const float4*)row;
        const float4* q4 = (const float4*)qs;
        float acc = 0.0f;
        for (int c = lane; c < dp / 4; c += 32) {
            const float4 x = r4[c], y = q4[c];
            acc = fmaf(x.x, y.x, acc);
            acc = fmaf(x.y, y.y, acc);
            acc = fmaf(x.z, y.z, acc);
            acc = fmaf(x.w, y.w, acc);
        }
        return acc;
    }
};

template <> struct RowDot<__nv_bfloat16> {
    __device__ static float dot(const __nv_bfloat16* __restrict__ row, const float* qs, int dp,
                                int lane) {
        const uint4* r8 = (const uint4*)row;
        float acc = 0.0f;
        for (int c = lane; c < dp / 8; c += 32) {
            const uint4 raw = r8[c];
            const __nv_bfloat162* h = (const __nv_bfloat162*)&raw;
            const float* y = qs + c * 8;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 x = __bfloat1622float2(h[i]);
                acc = fmaf(x.x, y[2 * i], acc);
                acc = fmaf(x.y, y[2 * i + 1], acc);
            }
        }
        return acc;
    }
};

// grid (nq, chunks); a warp per candidate row; the score interval
// [s - e, s + e] with e = kappa ||q|| ||x|| (FP32 summation bound, 4x margin)
// is stored rounded outward.
template <typename T>
__global__ void __launch_bounds__(kRerankWarps * 32)
    rerank_fp32_kernel(const T* __restrict__ Xp, int dp, int d, const float* __restrict__ Q,
                       const uint32_t* __restrict__ cand, int64_t cap, int per_block,
                       const Boundary* __restrict__ bnd, const float* __restrict__ xnorm,
                       const float* __restrict__ qnorm, float kappa, float* __restrict__ lo,
                       float* __restrict__ hi) {
    extern __shared__ __align__(16) float qs[];
    const int64_t q = blockIdx.x;
    for (int c = threadIdx.x; c < dp; c += blockDim.x) qs[c] = c < d ? Q[q * d + c] : 0.0f;
    __syncthreads();
    const Boundary b = bnd[q];
    const int64_t count = (int64_t)b.full + b.r;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.y * per_block;
    const int64_t i1 = min(count, i0 + per_block);
    const float qn = qnorm[q];
    for (int64_t i = i0 + warp; i < i1; i += kRerankWarps) {
        const uint32_t p = cand[q * cap + i];
        const float s = warp_sum(RowDot<T>::dot(Xp + (int64_t)p * dp, qs, dp, lane));
        if (lane == 0) {
            const float e = __fmul_ru(__fmul_ru(kappa, qn), xnorm[p]);
            lo[q * cap + i] = __fsub_rd(s, e);
            hi[q * cap + i] = __fadd_ru(s, e);
        }
    }
}

// ------------------------------------------------------------------- top-k

__device__ __forceinline__ uint32_t float_order(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float order_float(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// (s, id) beats (s', id') when s > s', or s == s' and id < id'.
__device__ __forceinline__ bool better(double s, int64_t id, double s2, int64_t id2) {
    return s > s2 || (s == s2 && id < id2);
}

// Block per query.  tau = k-th largest lower bound (MSD radix select on the
// order-preserving integer image of the floats).  Every candidate whose upper
// bound reaches tau is a contender; any true top-k member is one, because k
// candidates have FP64 scores >= their lower bounds >= tau.  Contenders are
// rescored in FP64 in the fixed order and the top k by (score desc, id asc)
// are taken by k rounds of a block arg-max.
template <typename T>
__global__ void __launch_bounds__(256)
    topk_kernel(const float* __restrict__ lo, const float* __restrict__ hi,
                const uint32_t* __restrict__ cand, int64_t cap, const Boundary* __restrict__ bnd,
                int k, const int32_t* __restrict__ ks, const T* __restrict__ Xp, int dp, int d,
                const float* __restrict__ Q, const uint32_t* __restrict__ perm,
                uint32_t* __restrict__ cont, double* __restrict__ cont_s,
                int64_t* __restrict__ out_ids, float* __restrict__ out_scores, int out_ld) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t prefix_s, mask_s;
    __shared__ int rem_s;
    __shared__ uint32_t nc_s;
    __shared__ double best_s[8];
    __shared__ int64_t bid_s[8];
    __shared__ int bc_s[8];
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kq = ks ? ks[q] : k;
    const Boundary b = bnd[q];
    const int64_t count = (int64_t)b.full + b.r;
    const float* loq = lo + q * cap;
    const float* hiq = hi + q * cap;
    const uint32_t* candq = cand + q * cap;
    uint32_t* contq = cont + q * cap;
    double* contsq = cont_s + q * cap;

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
            for (int64_t i = threadIdx.x; i < count; i += 256) {
                const uint32_t key = float_order(loq[i]);
                if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 0xFFu], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int rem = rem_s;
                for (int dg = 255; dg >= 0; --dg) {
                    const int c = (int)hist[dg];
                    if (c >= rem) {
                        prefix_s = prefix | ((uint32_t)dg << shift);
                        mask_s = mask | (0xFFu << shift);
                        break;
                    }
                    rem -= c;
                }
                rem_s = rem;
            }
            __syncthreads();
        }
        tau = order_float(prefix_s);
    }
    if (threadIdx.x == 0) nc_s = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < count; i += 256) {
        if (hiq[i] >= tau) contq[atomicAdd(&nc_s, 1u)] = (uint32_t)i;
    }
    __syncthreads();
    const uint32_t nc = nc_s;
    const float* qrow = Q + q * d;
    for (uint32_t c = threadIdx.x; c < nc; c += 256) {
        const T* xrow = Xp + (int64_t)candq[contq[c]] * dp;
        double acc = 0.0;
        for (int kk = 0; kk < d; ++kk) acc = fma((double)to_f32(xrow[kk]), (double)qrow[kk], acc);
        contsq[c] = acc;
    }
    __syncthreads();
    const int kk_out = (int)min((int64_t)kq, (int64_t)nc);
    for (int r = 0; r < kk_out; ++r) {
        double bs = -DBL_MAX;
        int64_t bi = INT64_MAX;
        int bc = -1;
        for (uint32_t c = threadIdx.x; c < nc; c += 256) {
            const uint32_t ci = contq[c];
            if (ci & 0x80000000u) continue;  // taken
            const double s = contsq[c];
            const int64_t id = perm[candq[ci]];
            if (bc < 0 || better(s, id, bs, bi)) {
                bs = s;
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
            out_ids[q * out_ld + r] = bid_s[w0];
            out_scores[q * out_ld + r] = __double2float_rn(best_s[w0]);
            contq[bc_s[w0]] |= 0x80000000u;
        }
        __syncthreads();
    }
    for (int r = kk_out + threadIdx.x; r < kq; r += 256) {
        out_ids[q * out_ld + r] = -1;
        out_scores[q * out_ld + r] = -INFINITY;
    }
}

__global__ void cand_to_ids_kernel(const uint32_t* __restrict__ cand, int64_t cap,
                                   const Boundary* __restrict__ bnd,
                                   const uint32_t* __restrict__ perm, int32_t* out, int64_t out_cap,
                                   int64_t* count) {
    const int64_t q = blockIdx.x;
    const Boundary b = bnd[q];
    const int64_t cnt = (int64_t)b.full + b.r;
    if (threadIdx.x == 0) count[q] = cnt;
    const int64_t lim = min(cnt, out_cap);
    for (int64_t i = threadIdx.x; i < lim; i += blockDim.x)
        out[q * out_cap + i] = (int32_t)perm[cand[q * cap + i]];
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_row_norm_bound(const float* Q, int64_t nq, int d, float* qnorm,
                                  cudaStream_t st) {
    return launch("row_norm_bound", row_norm_bound_kernel, dim3((unsigned)ceil_div(nq * 32, 256)),
                  dim3(256), 0, st, Q, nq, d, qnorm);
}

cudaError_t launch_hist(const void* codes, const void* qcodes, int code_bytes, int64_t nq, int m,
                        int L, const PosTile* tiles, int ntiles, uint32_t* H, cudaStream_t st) {
    const dim3 grid((unsigned)ntiles, (unsigned)ceil_div(nq, kHistQ));
    const size_t smem = 16384 + sizeof(uint16_t) * (size_t)(L + 1) * kHistQ;
    if (code_bytes == 4)
        return launch("hist_u32", hist_kernel<uint32_t>, grid, dim3(kHistQ), smem, st,
                      (const uint32_t*)codes, (const uint32_t*)qcodes, nq, m, L, tiles, H);
    return launch("hist_u64", hist_kernel<uint64_t>, grid, dim3(kHistQ), smem, st,
                  (const uint64_t*)codes, (const uint64_t*)qcodes, nq, m, L, tiles, H);
}

cudaError_t launch_threshold(const uint32_t* H, const uint32_t* order, int m, int L, int64_t nq,
                             int64_t n, int64_t budget, const int64_t* budgets, uint32_t flags,
                             uint8_t* lam, Boundary* bnd, cudaStream_t st) {
    return launch("threshold", threshold_kernel, dim3((unsigned)nq), dim3(256),
                  sizeof(uint32_t) * (size_t)m, st, H, order, m, L, nq, n, budget, budgets, flags,
                  lam, bnd);
}

cudaError_t launch_select(const void* codes, const void* qcodes, int code_bytes, int64_t n, int m,
                          int L, int64_t nq, const uint8_t* lam, const Boundary* bnd,
                          uint32_t* cand, int64_t cap, cudaStream_t st) {
    if (code_bytes == 4)
        return launch("select_u32", select_kernel<uint32_t>, dim3((unsigned)nq), dim3(256),
                      (size_t)m, st, (const uint32_t*)codes, (const uint32_t*)qcodes, n, m, L, lam,
                      bnd, cand, cap);
    return launch("select_u64", select_kernel<uint64_t>, dim3((unsigned)nq), dim3(256), (size_t)m,
                  st, (const uint64_t*)codes, (const uint64_t*)qcodes, n, m, L, lam, bnd, cand,
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
                        const uint32_t* perm, uint32_t* cont, double* cont_s,
                        int64_t* out_ids, float* out_scores, int out_ld, cudaStream_t st) {
    if (dt == NRLSH_BF16)
        return launch("topk_bf16", topk_kernel<__nv_bfloat16>, dim3((unsigned)nq), dim3(256), 0, st,
                      lo, hi, cand, cap, bnd, k, ks, (const __nv_bfloat16*)Xp, dp, d, Q, perm, cont,
                      cont_s, out_ids, out_scores, out_ld);
    return launch("topk", topk_kernel<float>, dim3((unsigned)nq), dim3(256), 0, st, lo, hi, cand,
                  cap, bnd, k, ks, (const float*)Xp, dp, d, Q, perm, cont, cont_s, out_ids,
                  out_scores, out_ld);
}

cudaError_t launch_cand_to_ids(const uint32_t* cand, int64_t cap, const Boundary* bnd,
                               const uint32_t* perm, int64_t nq, int32_t* out, int64_t out_cap,
                               int64_t* count, cudaStream_t st) {
    return launch("cand_to_ids", cand_to_ids_kernel, dim3((unsigned)nq), dim3(256), 0, st, cand,
                  cap, bnd, perm, out, out_cap, count);
}

}  // namespace nrlsh
