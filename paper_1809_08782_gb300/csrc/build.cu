// Index building kernels (Algorithm 1, Eq. 8, Eq. 4, Eq. 12).
//
//   gen_projections   A ((d+1) x L) from Philox4x64-10 + Box-Muller, bf16-rounded
//   sqnorm            s_x = ||x||^2 in FP64, k = 0..d-1 in order
//   radix sort        stable LSD sort of (s_x bits, id) and of (sub-dataset, id)
//   segment_assign    percentile partition and U_j^2 = max s_x in S_j
//   gather_items      sub-dataset-major copy of the items, tau_x, norm bounds
//   project_fp32      sign(a^T [x; tau]) with an FP32 tier and an FP64 recompute
//   bucket_order      the sorted (U_j, l) structure of Section 3.3
#include "nrlsh_internal.cuh"

#include <cfloat>

namespace nrlsh {

// =====================================================================
// Projection matrix: Philox4x64-10 (Salmon et al., SC'11) and Box-Muller.
// =====================================================================

namespace {

constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

__device__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const uint64_t hi0 = __umul64hi(kPhiloxM0, c[0]), lo0 = kPhiloxM0 * c[0];
        const uint64_t hi1 = __umul64hi(kPhiloxM1, c[2]), lo1 = kPhiloxM1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// One rounding from double to the nearest bfloat16 value (8 significant bits),
// ties to even, returned as a double.
__device__ double round_to_bf16(double z) {
    if (z == 0.0) return 0.0;
    int ex;
    const double mant = frexp(z, &ex);  // z = mant * 2^ex, 0.5 <= |mant| < 1
    return ldexp(rint(mant * 256.0), ex - 8);
}

__global__ void gen_projections_kernel(float* A, int d, int L, uint64_t seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(d + 1) * L) return;
    uint64_t c[4] = {(uint64_t)(i / L), (uint64_t)(i % L), 0, 0};
    philox4x64_10(c, seed, 0);
    const double u1 = ((double)(c[0] >> 12) + 0.5) * 0x1p-52;
    const double u2 = ((double)(c[1] >> 12) + 0.5) * 0x1p-52;
    const double r = sqrt(-2.0 * log(u1));
    const double z = __dmul_rn(r, cos(__dmul_rn(6.283185307179586, u2)));
    A[i] = (float)round_to_bf16(z);
}

}  // namespace

cudaError_t launch_gen_projections(float* A, int d, int L, uint64_t seed, cudaStream_t s) {
    const int64_t total = (int64_t)(d + 1) * L;
    return launch("gen_projections", gen_projections_kernel, dim3((unsigned)ceil_div(total, 256)),
                  dim3(256), 0, s, A, d, L, seed);
}

// =====================================================================
// Squared norms: one thread per row, rows staged through shared memory so the
// global loads are coalesced; FP64 accumulation in column order.
// =====================================================================

namespace {

template <typename T>
__global__ void __launch_bounds__(128) sqnorm_kernel(const T* __restrict__ X, int64_t n, int d,
                                                     int64_t ld, double* __restrict__ s) {
    __shared__ float tile[128][33];
    const int64_t row0 = (int64_t)blockIdx.x * 128;
    double acc = 0.0;
    for (int c0 = 0; c0 < d; c0 += 32) {
        for (int i = threadIdx.x; i < 128 * 32; i += 128) {
            const int r = i >> 5, c = i & 31;
            const int64_t row = row0 + r;
            const int col = c0 + c;
            tile[r][c] = (row < n && col < d) ? to_f32(X[row * ld + col]) : 0.0f;
        }
        __syncthreads();
        const int cmax = min(32, d - c0);
        for (int c = 0; c < cmax; ++c) {
            const double v = (double)tile[threadIdx.x][c];
            acc = fma(v, v, acc);  // v*v is exact in FP64: same as add after multiply
        }
        __syncthreads();
    }
    const int64_t row = row0 + threadIdx.x;
    if (row < n) s[row] = acc;
}

}  // namespace

cudaError_t launch_sqnorm(const void* X, nrlsh_dtype dt, int64_t n, int d, int64_t ld, double* s,
                          cudaStream_t st) {
    const dim3 grid((unsigned)ceil_div(n, 128));
    if (dt == NRLSH_BF16)
        return launch("sqnorm_bf16", sqnorm_kernel<__nv_bfloat16>, grid, dim3(128), 0, st,
                      (const __nv_bfloat16*)X, n, d, ld, s);
    return launch("sqnorm_f32", sqnorm_kernel<float>, grid, dim3(128), 0, st, (const float*)X, n, d,
                  ld, s);
}

// =====================================================================
// Stable LSD radix sort, 8-bit digits.  Per pass: tile histograms, one
// exclusive scan over (digit, tile), and a stable scatter that ranks keys
// inside a tile with warp match + per-warp digit counts.  A pass whose digit
// is the same for every key (known from an OR-of-differences reduction) turns
// into a plain copy, so the buffers alternate the same way in every case.
// =====================================================================

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 4096 keys per tile
constexpr int kRadix = 256;

template <typename K>
__global__ void or_diff_kernel(const K* __restrict__ keys, int64_t n, unsigned long long* out) {
    const K k0 = keys[0];
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc |= (unsigned long long)(keys[i] ^ k0);
    for (int o = 16; o; o >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicOr(out, acc);
}

__device__ __forceinline__ bool digit_varies(const unsigned long long* varying, int shift) {
    return ((*varying >> shift) & 0xFFull) != 0;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
    radix_hist_kernel(const K* __restrict__ keys, int64_t n, int shift,
                      const unsigned long long* varying, uint32_t* __restrict__ counts,
                      int ntiles) {
    if (!digit_varies(varying, shift)) return;
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
        const int64_t p = base + i;
        if (p < n) atomicAdd(&h[(uint32_t)(keys[p] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan in place over total = 256 * ntiles counters, one block.
__global__ void __launch_bounds__(1024)
    radix_scan_kernel(uint32_t* counts, int64_t total, int shift,
                      const unsigned long long* varying) {
    if (!digit_varies(varying, shift)) return;
    __shared__ uint32_t part[1024];
    const int64_t per = ceil_div(total, 1024);
    const int64_t b = threadIdx.x * per, e = min(total, b + per);
    uint32_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += counts[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - sum;
    for (int64_t i = b; i < e; ++i) {
        const uint32_t c = counts[i];
        counts[i] = run;
        run += c;
    }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                         K* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                         const unsigned long long* varying, const uint32_t* __restrict__ offsets,
                         int ntiles) {
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    if (!digit_varies(varying, shift)) {
        for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
            const int64_t p = base + i;
            if (p < n) {
                kout[p] = kin[p];
                vout[p] = vin[p];
            }
        }
        return;
    }
    __shared__ uint32_t run_off[kRadix];
    __shared__ uint32_t warp_cnt[kSortThreads / 32][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int round = 0; round < kSortRounds; ++round) {
        uint32_t* wc = &warp_cnt[0][0];
        for (int i = threadIdx.x; i < (kSortThreads / 32) * kRadix; i += kSortThreads) wc[i] = 0;
        __syncthreads();
        const int64_t p = base + (int64_t)round * kSortThreads + threadIdx.x;
        const bool valid = p < n;
        const K key = valid ? kin[p] : (K)0;
        const uint32_t dg = (uint32_t)(key >> shift) & 0xFFu;
        // invalid lanes get a private value so they never match a real digit
        const unsigned peers = __match_any_sync(0xffffffffu, valid ? dg : 0x100u + lane);
        const int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) warp_cnt[warp][dg] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = run_off[threadIdx.x];
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const uint32_t c = warp_cnt[w][threadIdx.x];
                warp_cnt[w][threadIdx.x] = run;
                run += c;
            }
            run_off[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t dst = warp_cnt[warp][dg] + rank;
            kout[dst] = key;
            vout[dst] = vin[p];
        }
        __syncthreads();
    }
}

template <typename K>
cudaError_t radix_sort_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, int64_t n,
                            int key_bits, void* temp, bool* result_in_alt, cudaStream_t s,
                            const char* tag) {
    *result_in_alt = false;
    if (n <= 1) return cudaSuccess;
    const int ntiles = (int)ceil_div(n, kSortTile);
    unsigned long long* varying = (unsigned long long*)temp;
    uint32_t* counts = (uint32_t*)((char*)temp + 256);
    cudaError_t e = cudaMemsetAsync(varying, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int or_blocks = (int)std::min<int64_t>(ceil_div(n, 256), 1024);
    e = launch(tag, or_diff_kernel<K>, dim3(or_blocks), dim3(256), 0, s, (const K*)keys, n,
               varying);
    if (e != cudaSuccess) return e;
    K* src_k = keys;
    uint32_t* src_v = vals;
    K* dst_k = keys_alt;
    uint32_t* dst_v = vals_alt;
    for (int shift = 0; shift < key_bits; shift += 8) {
        e = launch("radix_hist", radix_hist_kernel<K>, dim3(ntiles), dim3(kSortThreads), 0, s,
                   (const K*)src_k, n, shift, (const unsigned long long*)varying, counts, ntiles);
        if (e != cudaSuccess) return e;
        e = launch("radix_scan", radix_scan_kernel, dim3(1), dim3(1024), 0, s, counts,
                   (int64_t)kRadix * ntiles, shift, (const unsigned long long*)varying);
        if (e != cudaSuccess) return e;
        e = launch("radix_scatter", radix_scatter_kernel<K>, dim3(ntiles), dim3(kSortThreads), 0,
                   s, (const K*)src_k, (const uint32_t*)src_v, dst_k, dst_v, n, shift,
                   (const unsigned long long*)varying, (const uint32_t*)counts, ntiles);
        if (e != cudaSuccess) return e;
        std::swap(src_k, dst_k);
        std::swap(src_v, dst_v);
        *result_in_alt = !*result_in_alt;
    }
    return cudaSuccess;
}

}  // namespace

size_t radix_sort_temp_bytes(int64_t n) {
    return 256 + sizeof(uint32_t) * (size_t)kRadix * (size_t)ceil_div(std::max<int64_t>(n, 1), kSortTile);
}

cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int key_bits, void* temp, bool* result_in_alt,
                           cudaStream_t s) {
    return radix_sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, key_bits, temp,
                                     result_in_alt, s, "radix_or_diff_u64");
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int key_bits, void* temp, bool* result_in_alt,
                           cudaStream_t s) {
    return radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, key_bits, temp,
                                     result_in_alt, s, "radix_or_diff_u32");
}

// =====================================================================
// Partition helpers.
// =====================================================================

namespace {

// s_x >= 0, so its IEEE bit pattern orders like the value (both zeros are +0).
__global__ void iota_keys_kernel(const double* __restrict__ s, uint64_t* keys, uint32_t* vals,
                                 int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = (uint64_t)__double_as_longlong(s[i] + 0.0);
    vals[i] = (uint32_t)i;
}

__global__ void iota_kernel(uint32_t* v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

__global__ void segment_assign_kernel(const uint64_t* __restrict__ sorted_keys,
                                      const uint32_t* __restrict__ sorted_ids, int64_t n, int m,
                                      uint32_t* sub_of_id, double* U2) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t j = seg_of(r, n, m);
    sub_of_id[sorted_ids[r]] = (uint32_t)j;
    if (r == seg_start(j + 1, n, m) - 1) U2[j] = __longlong_as_double((long long)sorted_keys[r]);
}

// One warp per storage position: copy the row (zero-padded to dp), the squared
// norm, tau = sqrt(U_j^2 - s) (1 when U_j = 0) and an fp32 upper bound of ||x||.
template <typename T>
__global__ void gather_items_kernel(const T* __restrict__ X, int64_t ld, int d, int dp,
                                    const uint32_t* __restrict__ perm, int64_t n, int m,
                                    const double* __restrict__ s_id, const double* __restrict__ U2,
                                    T* __restrict__ Xp, double* s_pos, double* tau64, float* tau32,
                                    float* xnorm) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n) return;
    const uint32_t id = perm[p];
    const T* src = X + (int64_t)id * ld;
    T* dst = Xp + p * dp;
    for (int c = lane; c < dp; c += 32) dst[c] = c < d ? src[c] : T(0.0f);
    if (lane == 0) {
        const double s = s_id[id];
        const double u2 = U2[seg_of(p, n, m)];
        const double t = (u2 == 0.0) ? 1.0 : sqrt(u2 - s);
        s_pos[p] = s;
        tau64[p] = t;
        tau32[p] = (float)t;
        xnorm[p] = __fsqrt_ru(__double2float_ru(s));
    }
}

}  // namespace

cudaError_t launch_iota_keys(const double* s, uint64_t* keys, uint32_t* vals, int64_t n,
                             cudaStream_t st) {
    return launch("iota_keys", iota_keys_kernel, dim3((unsigned)ceil_div(n, 256)), dim3(256), 0, st,
                  s, keys, vals, n);
}

cudaError_t launch_iota(uint32_t* v, int64_t n, cudaStream_t st) {
    return launch("iota", iota_kernel, dim3((unsigned)ceil_div(n, 256)), dim3(256), 0, st, v, n);
}

cudaError_t launch_segment_assign(const uint64_t* sorted_keys, const uint32_t* sorted_ids,
                                  int64_t n, int m, uint32_t* sub_of_id, double* U2,
                                  cudaStream_t st) {
    return launch("segment_assign", segment_assign_kernel, dim3((unsigned)ceil_div(n, 256)),
                  dim3(256), 0, st, sorted_keys, sorted_ids, n, m, sub_of_id, U2);
}

cudaError_t launch_gather_items(const void* X, nrlsh_dtype dt, int64_t ld, int d, int dp,
                                const uint32_t* perm, int64_t n, int m, const double* s_id,
                                const double* U2, void* Xp, double* s_pos, double* tau64,
                                float* tau32, float* xnorm, cudaStream_t st) {
    const dim3 grid((unsigned)ceil_div(n * 32, 256));
    if (dt == NRLSH_BF16)
        return launch("gather_items_bf16", gather_items_kernel<__nv_bfloat16>, grid, dim3(256), 0,
                      st, (const __nv_bfloat16*)X, ld, d, dp, perm, n, m, s_id, U2,
                      (__nv_bfloat16*)Xp, s_pos, tau64, tau32, xnorm);
    return launch("gather_items_f32", gather_items_kernel<float>, grid, dim3(256), 0, st,
                  (const float*)X, ld, d, dp, perm, n, m, s_id, U2, (float*)Xp, s_pos, tau64, tau32,
                  xnorm);
}

// =====================================================================
// Projection: the FP32 tier with a proven bound and the FP64 recompute.
// =====================================================================

namespace {

// A_pad: (d+1) x Lp, columns b >= L zero.  anorm[b]: fp32 upper bound of
// ||a_{0..d-1, b}||_2 (computed in FP64, rounded up).
__global__ void prepare_projections_kernel(const float* __restrict__ A, int d, int L, int Lp,
                                           float* A_pad, float* anorm) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Lp) return;
    double ss = 0.0;
    for (int k = 0; k <= d; ++k) {
        const float v = b < L ? A[(int64_t)k * L + b] : 0.0f;
        A_pad[(int64_t)k * Lp + b] = v;
        if (k < d) ss = fma((double)v, (double)v, ss);
    }
    anorm[b] = __fsqrt_ru(__double2float_ru(ss));
}

constexpr int kProjRows = 128;     // rows per block
constexpr int kProjThreads = 256;  // 8 warps: warp w owns bit group w, lane owns rows
constexpr int kProjKC = 32;        // columns of X staged per step

// Bit b of row x, FP64 in the fixed order: sum_k a_kb x_k (k = 0..d-1) then
// + fl(a_db * tau) for items.
template <typename T>
__device__ bool project_bit_fp64(const T* __restrict__ xrow, const float* __restrict__ A_pad,
                                 int Lp, int d, int b, bool has_tail, double tau) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k)
        acc = fma((double)to_f32(xrow[k]), (double)A_pad[(int64_t)k * Lp + b], acc);
    if (has_tail) acc = __dadd_rn(acc, __dmul_rn((double)A_pad[(int64_t)d * Lp + b], tau));
    return acc >= 0.0;
}

// Block: 128 rows x Lp bits.  Warp w owns bits [w BT, (w+1) BT), lane owns rows
// lane + 32 i.  X and A are staged kProjKC columns at a time; every (row, bit)
// accumulates in FP32 in column order.
template <typename T, typename C, int BT>
__global__ void __launch_bounds__(kProjThreads)
    project_fp32_kernel(const T* __restrict__ X, int64_t n, int d, int ldx, int L, int Lp,
                        const float* __restrict__ A_pad, const float* __restrict__ anorm,
                        const double* __restrict__ tau64, const float* __restrict__ tau32,
                        const float* __restrict__ xnorm, C* __restrict__ codes,
                        unsigned long long* ambiguous, float kappa) {
    __shared__ float As[kProjKC][8 * BT];
    __shared__ float Xs[kProjKC][kProjRows + 1];
    __shared__ unsigned long long code_s[kProjRows];
    __shared__ unsigned amb_s;

    const int lane = threadIdx.x & 31, bg = threadIdx.x >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * kProjRows;
    if (threadIdx.x < kProjRows) code_s[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) amb_s = 0;

    float acc[4][BT];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int b = 0; b < BT; ++b) acc[i][b] = 0.0f;

    for (int k0 = 0; k0 < d; k0 += kProjKC) {
        __syncthreads();
        for (int i = threadIdx.x; i < kProjRows * kProjKC; i += kProjThreads) {
            const int r = i / kProjKC, c = i % kProjKC;
            const int64_t row = row0 + r;
            const int col = k0 + c;
            Xs[c][r] = (row < n && col < d) ? to_f32(X[row * ldx + col]) : 0.0f;
        }
        for (int i = threadIdx.x; i < kProjKC * Lp; i += kProjThreads) {
            const int c = i / Lp, b = i % Lp;
            As[c][b] = (k0 + c < d) ? A_pad[(int64_t)(k0 + c) * Lp + b] : 0.0f;
        }
        __syncthreads();
        const int kc = min(kProjKC, d - k0);
        for (int c = 0; c < kc; ++c) {
            float xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = Xs[c][lane + 32 * i];
#pragma unroll
            for (int b = 0; b < BT; ++b) {
                const float a = As[c][bg * BT + b];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][b] = fmaf(xv[i], a, acc[i][b]);
            }
        }
    }

    const bool has_tail = tau64 != nullptr;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = lane + 32 * i;
        const int64_t row = row0 + r;
        if (row >= n) continue;
        const float xn = xnorm[row];
        const float t32 = has_tail ? tau32[row] : 0.0f;
        unsigned long long word = 0;
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const int bit = bg * BT + b;
            if (bit >= L) continue;
            const float ad = has_tail ? A_pad[(int64_t)d * Lp + bit] : 0.0f;
            const float v = has_tail ? fmaf(ad, t32, acc[i][b]) : acc[i][b];
            // |v - v64| <= bound: FP32 summation error with Cauchy-Schwarz for
            // sum |a_k x_k|, the tau rounding, and a 4x margin (kappa = (d+2) 2^-22).
            const float bound = kappa * anorm[bit] * xn + 0x1p-20f * fabsf(ad) * t32;
            bool set;
            if (fabsf(v) * (1.0f - 0x1p-21f) > bound) {
                set = v > 0.0f;
            } else {
                set = project_bit_fp64(X + row * ldx, A_pad, Lp, d, bit, has_tail,
                                       has_tail ? tau64[row] : 0.0);
                atomicAdd(&amb_s, 1u);
            }
            if (set) word |= 1ull << bit;
        }
        if (word) atomicOr(&code_s[r], word);
    }
    __syncthreads();
    if (threadIdx.x < kProjRows) {
        const int64_t row = row0 + threadIdx.x;
        if (row < n) codes[row] = (C)code_s[threadIdx.x];
    }
    if (threadIdx.x == 0 && amb_s) atomicAdd(ambiguous, (unsigned long long)amb_s);
}

template <typename T, typename C>
cudaError_t project_dispatch(const void* X, int64_t n, int d, int ldx, int L, int Lp,
                             const float* A_pad, const float* anorm, const double* tau64,
                             const float* tau32, const float* xnorm, void* codes,
                             unsigned long long* amb, cudaStream_t st, const char* name) {
    const float kappa = (float)(d + 2) * 0x1p-22f;
    const dim3 grid((unsigned)ceil_div(n, kProjRows));
    switch (Lp / 8) {
        case 1:
            return launch(name, project_fp32_kernel<T, C, 1>, grid, dim3(kProjThreads), 0, st,
                          (const T*)X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm,
                          (C*)codes, amb, kappa);
        case 2:
            return launch(name, project_fp32_kernel<T, C, 2>, grid, dim3(kProjThreads), 0, st,
                          (const T*)X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm,
                          (C*)codes, amb, kappa);
        case 4:
            return launch(name, project_fp32_kernel<T, C, 4>, grid, dim3(kProjThreads), 0, st,
                          (const T*)X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm,
                          (C*)codes, amb, kappa);
        case 8:
            return launch(name, project_fp32_kernel<T, C, 8>, grid, dim3(kProjThreads), 0, st,
                          (const T*)X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm,
                          (C*)codes, amb, kappa);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_prepare_projections(const float* A, int d, int L, int Lp, float* A_pad,
                                       float* anorm, cudaStream_t st) {
    return launch("prepare_projections", prepare_projections_kernel,
                  dim3((unsigned)ceil_div(Lp, 64)), dim3(64), 0, st, A, d, L, Lp, A_pad, anorm);
}

cudaError_t launch_project_fp32(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx,
                                int L, int Lp, const float* A_pad, const float* anorm,
                                const double* tau64, const float* tau32, const float* xnorm,
                                void* codes, int code_bytes, unsigned long long* ambiguous,
                                cudaStream_t st) {
    if (dt == NRLSH_BF16) {
        if (code_bytes == 4)
            return project_dispatch<__nv_bfloat16, uint32_t>(X, n, d, ldx, L, Lp, A_pad, anorm,
                                                             tau64, tau32, xnorm, codes, ambiguous,
                                                             st, "project_fp32_bf16");
        return project_dispatch<__nv_bfloat16, uint64_t>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64,
                                                         tau32, xnorm, codes, ambiguous, st,
                                                         "project_fp32_bf16");
    }
    if (code_bytes == 4)
        return project_dispatch<float, uint32_t>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32,
                                                 xnorm, codes, ambiguous, st, "project_fp32");
    return project_dispatch<float, uint64_t>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32,
                                             xnorm, codes, ambiguous, st, "project_fp32");
}

// =====================================================================
// Bucket order (Section 3.3): s_hat(j, l) = fl(U_j * c_l) with c_l the
// correctly rounded cos(pi (1 - eps)(L - l) / L), evaluated in double-double
// (Dekker/Knuth error-free transformations) and rounded once.
// =====================================================================

namespace {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double err = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, err};
}
__device__ __forceinline__ dd quick_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd two_prod(double a, double b) {
    const double p = __dmul_rn(a, b);
    return {p, fma(a, b, -p)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo = __dadd_rn(p.lo, __dadd_rn(__dmul_rn(a.hi, b.lo), __dmul_rn(a.lo, b.hi)));
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo = __dadd_rn(p.lo, __dmul_rn(a.lo, b));
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_div_d(dd a, double b) {
    const double q1 = __ddiv_rn(a.hi, b);
    dd p = two_prod(q1, b);
    dd r = two_sum(a.hi, -p.hi);
    r.lo = __dadd_rn(r.lo, __dsub_rn(a.lo, p.lo));
    const double q2 = __ddiv_rn(__dadd_rn(r.hi, r.lo), b);
    return quick_two_sum(q1, q2);
}

// Taylor series on |x| <= pi/4; 1/(2i)! terms fall below 2^-110 well before i = 14.
__device__ dd dd_cos_small(dd x) {
    const dd x2 = dd_mul(x, x);
    dd term = {1.0, 0.0}, sum = {1.0, 0.0};
    for (int i = 1; i < 16; ++i) {
        term = dd_div_d(dd_mul(term, dd_neg(x2)), (double)((2 * i - 1) * (2 * i)));
        sum = dd_add(sum, term);
    }
    return sum;
}
__device__ dd dd_sin_small(dd x) {
    const dd x2 = dd_mul(x, x);
    dd term = x, sum = x;
    for (int i = 1; i < 16; ++i) {
        term = dd_div_d(dd_mul(term, dd_neg(x2)), (double)((2 * i) * (2 * i + 1)));
        sum = dd_add(sum, term);
    }
    return sum;
}

// cos(pi (1 - eps) (L - l) / L) rounded to nearest.  The angle is exactly pi/2
// iff 2 (1 - eps)(L - l) = L, where cos is exactly 0; every other value this
// function can meet is irrational or +-1, +-1/2 (Niven), so rounding the
// double-double result once is correct.
__device__ double cos_class(int L, int l, double eps) {
    const double two_ml = 2.0 * (double)(L - l);
    if (eps * two_ml == two_ml - (double)L) return 0.0;  // both sides exact
    const dd pi = {3.141592653589793116, 1.2246467991473532e-16};
    dd t = two_sum(1.0, -eps);
    t = dd_div_d(dd_mul_d(t, (double)(L - l)), (double)L);
    const dd theta = dd_mul(pi, t);
    const dd half_pi = {pi.hi * 0.5, pi.lo * 0.5};
    const dd quarter_pi = {pi.hi * 0.25, pi.lo * 0.25};
    dd r;
    if (theta.hi <= quarter_pi.hi) {
        r = dd_cos_small(theta);
    } else if (theta.hi <= 3.0 * quarter_pi.hi) {
        r = dd_neg(dd_sin_small(dd_add(theta, dd_neg(half_pi))));
    } else {
        r = dd_neg(dd_cos_small(dd_add(pi, dd_neg(theta))));
    }
    return __dadd_rn(r.hi, r.lo);
}

// key = (s_hat, l, j), compared descending.
__global__ void bucket_keys_kernel(const double* __restrict__ U2, int m, int L, float eps,
                                   double* shat) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m * (L + 1)) return;
    const int j = c / (L + 1), l = c % (L + 1);
    const double cl = cos_class(L, l, (double)eps);
    const double U = sqrt(U2[j]);
    shat[c] = __dadd_rn(__dmul_rn(U, cl), 0.0);  // +0.0 turns -0 into +0
}

__device__ __forceinline__ bool key_greater(double s1, int l1, int j1, double s0, int l0, int j0) {
    if (s1 != s0) return s1 > s0;
    if (l1 != l0) return l1 > l0;
    return j1 > j0;
}

// rank(c) = number of buckets whose key is greater; order[rank] = c.
__global__ void bucket_rank_kernel(const double* __restrict__ shat, int m, int L,
                                   double* shat_sorted, uint32_t* order) {
    __shared__ double ks[256];
    const int ncls = m * (L + 1);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = c < ncls;
    const double s0 = valid ? shat[c] : 0.0;
    const int l0 = valid ? c % (L + 1) : 0, j0 = valid ? c / (L + 1) : 0;
    int rank = 0;
    for (int b = 0; b < ncls; b += 256) {
        __syncthreads();
        if (b + threadIdx.x < ncls) ks[threadIdx.x] = shat[b + threadIdx.x];
        __syncthreads();
        const int lim = min(256, ncls - b);
        for (int i = 0; i < lim; ++i) {
            const int c1 = b + i;
            rank += key_greater(ks[i], c1 % (L + 1), c1 / (L + 1), s0, l0, j0);
        }
    }
    if (valid) {
        order[rank] = (uint32_t)c;
        shat_sorted[rank] = s0;
    }
}

}  // namespace

cudaError_t launch_bucket_order(const double* U2, int m, int L, float eps, double* shat_sorted,
                                uint32_t* order, double* scratch_keys, cudaStream_t st) {
    const int ncls = m * (L + 1);
    const dim3 grid((unsigned)ceil_div(ncls, 256));
    cudaError_t e = launch("bucket_keys", bucket_keys_kernel, grid, dim3(256), 0, st, U2, m, L, eps,
                           scratch_keys);
    if (e != cudaSuccess) return e;
    return launch("bucket_rank", bucket_rank_kernel, grid, dim3(256), 0, st,
                  (const double*)scratch_keys, m, L, shat_sorted, order);
}

}  // namespace nrlsh
