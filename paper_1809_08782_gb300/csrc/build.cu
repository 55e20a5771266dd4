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
#include "sign_tiers.cuh"

#include <algorithm>
#include <cfloat>
#include <climits>

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

__device__ float projection_entry(int64_t r, int64_t b, uint64_t seed) {
    uint64_t c[4] = {(uint64_t)r, (uint64_t)b, 0, 0};
    philox4x64_10(c, seed, 0);
    const double u1 = ((double)(c[0] >> 12) + 0.5) * 0x1p-52;
    const double u2 = ((double)(c[1] >> 12) + 0.5) * 0x1p-52;
    const double rad = sqrt(-2.0 * log(u1));
    const double z = __dmul_rn(rad, cos(__dmul_rn(6.283185307179586, u2)));
    return (float)round_to_bf16(z);
}

// Block b fills column b of A ((d+1) x L) and of A_pad ((d+1) x Lp, zero for
// b >= L) and writes anorm[b], an fp32 upper bound of ||a_{0..d-1, b}||_2.
// Block b also writes row b of At (bf16, K-major: At[b][k] = a_{k,b}, zero for
// k >= d), the B operand of the tensor-core projection; At may be null.
__global__ void __launch_bounds__(256)
    projections_kernel(float* __restrict__ A, float* __restrict__ A_pad, float* __restrict__ anorm,
                       __nv_bfloat16* __restrict__ At, int dp, int d, int L, int Lp,
                       uint64_t seed) {
    NRLSH_PDL_ENTRY();
    __shared__ double part[8];
    const int b = blockIdx.x;
    double ss = 0.0;
    for (int r = threadIdx.x; r <= d; r += blockDim.x) {
        const float a = b < L ? projection_entry(r, b, seed) : 0.0f;
        if (b < L) A[(int64_t)r * L + b] = a;
        A_pad[(int64_t)r * Lp + b] = a;
        if (r < d) ss = fma((double)a, (double)a, ss);
        if (At && r < d) At[(int64_t)b * dp + r] = __float2bfloat16_rn(a);  // exact: a is bf16
    }
    if (At)
        for (int r = d + threadIdx.x; r < dp; r += blockDim.x) At[(int64_t)b * dp + r] = __float2bfloat16_rn(0.0f);
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        // the sum's relative error (< d 2^-53) is far inside the 4x bound margin
        anorm[b] = __fsqrt_ru(__double2float_ru(t));
    }
}

}  // namespace

cudaError_t launch_projections(float* A, float* A_pad, float* anorm, __nv_bfloat16* At, int dp,
                               int d, int L, int Lp, uint64_t seed, cudaStream_t s) {
    return launch("projections", projections_kernel, dim3((unsigned)Lp), dim3(256), 0, s, A, A_pad,
                  anorm, At, dp, d, L, Lp, seed);
}

// =====================================================================
// Zeroing of several small arrays in one launch.
// =====================================================================

namespace {

__global__ void zero_kernel(ZeroList z) {
    NRLSH_PDL_ENTRY();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int i = 0; i < z.k; ++i) {
        uint32_t* p = (uint32_t*)z.p[i];
        for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < (int64_t)z.words[i];
             w += stride)
            p[w] = 0u;
    }
}

}  // namespace

cudaError_t launch_zero(const ZeroList& z, cudaStream_t st) {
    size_t most = 1;
    for (int i = 0; i < z.k; ++i) most = std::max(most, z.words[i]);
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div((int64_t)most, 256), 2 * 152);
    return launch("zero", zero_kernel, dim3(grid), dim3(256), 0, st, z);
}

// =====================================================================
// Squared norms: s_x = sum_k x_k^2 exactly, rounded once to FP64.  16 lanes per
// row (rows of up to 512 values) or a warp per row; every x_k = M 2^E (M < 2^24)
// has x_k^2 = M^2 2^2E exactly.  The lanes
// add their terms into a 128-bit integer window [W0, W0 + 128) placed under the
// row's largest term with bitlen(d) + 1 bits of headroom, so 73 - bitlen(d) bits
// lie below the result's rounding bit inside the window; bits of terms below
// W0 are dropped and noted.  The dropped total is less than d units of 2^W0, so
// it can change the rounding only if the kept remainder lies within d units
// below the half-way point; such a row (none in practice; constructed tests
// have them) is summed again exactly in a 576-bit accumulator by one lane, and
// so is a row whose values are all subnormal.
// =====================================================================

namespace {

typedef unsigned __int128 u128;

__device__ __forceinline__ void f32_fields(float x, uint64_t& M2, int& E2) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xFFu, f = u & 0x7FFFFFu;
    const uint64_t M = e ? (f | 0x800000u) : f;
    M2 = M * M;                              // < 2^48
    E2 = 2 * (e ? (int)e - 150 : -149);      // x^2 = M2 2^E2
}

__device__ __forceinline__ int bitlen64(uint64_t v) { return v ? 64 - __clzll((long long)v) : 0; }

// 64-bit shifts whose amounts of 64 and more give 0 (the PTX shift semantics).
__device__ __forceinline__ uint64_t shl_clamped(uint64_t a, uint32_t s) {
    uint64_t r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(a), "r"(s));
    return r;
}
__device__ __forceinline__ uint64_t shr_clamped(uint64_t a, uint32_t s) {
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(a), "r"(s));
    return r;
}
// The exact sum of the row's squares in 9 words (bit i of the array has weight
// 2^(i - 298)), rounded to nearest even.  Slow; for ambiguous rows only.
template <typename T>
__device__ double sqnorm_exact_slow(const T* __restrict__ xr, int d) {
    uint64_t w[9];
    for (int i = 0; i < 9; ++i) w[i] = 0;
    for (int k = 0; k < d; ++k) {
        uint64_t M2;
        int E2;
        f32_fields(to_f32(xr[k]), M2, E2);
        if (!M2) continue;
        const int off = E2 + 298, wi = off >> 6, b = off & 63;
        uint64_t add_lo = M2 << b, add_hi = b ? (M2 >> (64 - b)) : 0;
        uint64_t old = w[wi];
        w[wi] += add_lo;
        uint64_t carry = w[wi] < old;
        for (int j = wi + 1; j < 9 && (add_hi | carry); ++j) {
            old = w[j];
            w[j] += add_hi + carry;
            carry = (w[j] < old) || (carry && add_hi == ~0ull);
            add_hi = 0;
        }
    }
    int top = -1;
    for (int j = 8; j >= 0 && top < 0; --j)
        if (w[j]) top = 64 * j + 63 - __clzll((long long)w[j]);
    if (top < 0) return 0.0;
    auto bit = [&](int i) -> uint64_t { return i < 0 ? 0 : (w[i >> 6] >> (i & 63)) & 1ull; };
    uint64_t mant = 0;
    for (int i = top; i > top - 53; --i) mant = (mant << 1) | bit(i);
    const uint64_t rb = bit(top - 53);
    bool sticky = false;
    for (int i = top - 54; i >= 0 && !sticky; --i)
        if ((i & 63) == 63 && !w[i >> 6]) i -= 63; else sticky = bit(i) != 0;
    int ex = top - 298;                      // value in [2^ex, 2^(ex+1))
    if (rb && (sticky || (mant & 1))) {
        if (++mant == (1ull << 53)) {
            mant >>= 1;
            ++ex;
        }
    }
    return __longlong_as_double((long long)(((uint64_t)(ex + 1023) << 52) | (mant & ((1ull << 52) - 1))));
}

// The row's elements as lane-strided groups of VEC consecutive values (one
// vector load each when VEC > 1).
template <typename T, int VEC>
struct RowGroups;
template <typename T>
struct RowGroups<T, 1> {
    __device__ static void load(const T* xr, int g, float (&v)[1]) { v[0] = to_f32(xr[g]); }
};
template <>
struct RowGroups<float, 4> {
    __device__ static void load(const float* xr, int g, float (&v)[4]) {
        const float4 f = ((const float4*)xr)[g];
        v[0] = f.x;
        v[1] = f.y;
        v[2] = f.z;
        v[3] = f.w;
    }
};
template <>
struct RowGroups<__nv_bfloat16, 4> {
    __device__ static void load(const __nv_bfloat16* xr, int g, float (&v)[4]) {
        const uint2 raw = ((const uint2*)xr)[g];
        const float2 a = __bfloat1622float2(*(const __nv_bfloat162*)&raw.x);
        const float2 b = __bfloat1622float2(*(const __nv_bfloat162*)&raw.y);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
    }
};

// The window for a row whose largest |x_k| is amax (normal): x^2 = T 2^(W0 + t)
// with T = M^2 2^16 and t = 2 max(e, 1) + tbase < 64.  Values whose t is at least
// 32 (all but values far below the row's largest) take the fast form; thr1 picks
// out the others: 0 < |x| with t < 32, and subnormal values.
struct SqWindow {
    int W0, tbase;
    uint32_t thr1;
};
__device__ __forceinline__ SqWindow sq_window(float amax, int d) {
    uint64_t M2m;
    int E2m;
    f32_fields(amax, M2m, E2m);
    const int top = E2m + bitlen64(M2m);          // the largest term ends below 2^top
    const int W0 = top + (32 - __clz(d)) + 1 - 128;
    const int tbase = -300 - W0 - 16;
    const int e32 = max((33 - tbase) >> 1, 1);    // the least exponent field with t >= 32
    return {W0, tbase, ((uint32_t)e32 << 23) - 1u};
}

// The 128-bit window as four 32-bit words, least significant first.
struct SqAcc {
    uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
    uint64_t dropped = 0;
};
__device__ __forceinline__ void add4(SqAcc& a, uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, %5;\n\taddc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, %7;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2), "+r"(a.w3)
        : "r"(x0), "r"(x1), "r"(x2), "r"(x3));
}

// x^2 (bits u) for any t < 64: the window part (h:l) and the bits below it.
struct SqTerm {
    uint64_t l, h, dropped;
};
__device__ __noinline__ SqTerm sq_term_any(uint32_t u, int tbase) {
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint32_t M8 = (u << 8) | (e ? 0x80000000u : 0u);   // M 2^8 < 2^32
    const uint64_t T = (uint64_t)M8 * M8;                    // M^2 2^16, exact
    const int t = 2 * (int)max(e, 1u) + tbase;
    const uint32_t tp = (uint32_t)max(t, 0), tn = (uint32_t)max(-t, 0);
    return {shr_clamped(shl_clamped(T, tp), tn), shr_clamped(T, 64u - tp),
            T & ~shl_clamped(~0ull, tn)};
}

// x^2 added into the window: for t in [32, 64) the term T 2^(t - 32) spans the
// words 1..3 (three funnel shifts and a three-word add); the rest go through sq_term_any.
__device__ __forceinline__ void sq_add(float x, const SqWindow& w, SqAcc& a) {
    const uint32_t u = __float_as_uint(x), mag = u & 0x7FFFFFFFu;
    if (mag - 1u < w.thr1) {
        const SqTerm r = sq_term_any(u, w.tbase);
        a.dropped |= r.dropped;
        add4(a, (uint32_t)r.l, (uint32_t)(r.l >> 32), (uint32_t)r.h, (uint32_t)(r.h >> 32));
        return;
    }
    const uint32_t e = mag >> 23;                            // 0 only for x = 0 here
    const uint32_t M8 = (u << 8) | (e ? 0x80000000u : 0u);
    const uint64_t T = (uint64_t)M8 * M8;
    const uint32_t T0 = (uint32_t)T, T1 = (uint32_t)(T >> 32);
    const uint32_t sh = 2 * e + (uint32_t)(w.tbase - 32);    // t - 32 (mod 32 in the shifts)
    const uint32_t x0 = __funnelshift_l(0u, T0, sh), x1 = __funnelshift_l(T0, T1, sh),
                   x2 = __funnelshift_l(T1, 0u, sh);
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
        : "+r"(a.w1), "+r"(a.w2), "+r"(a.w3)
        : "r"(x0), "r"(x1), "r"(x2));
}

// Sum of the windows of the lanes xor-paired up to `width` (a power of two).
__device__ __forceinline__ void sq_reduce(SqAcc& a, int width) {
    for (int o = width / 2; o; o >>= 1) {
        const uint32_t x0 = __shfl_xor_sync(0xffffffffu, a.w0, o);
        const uint32_t x1 = __shfl_xor_sync(0xffffffffu, a.w1, o);
        const uint32_t x2 = __shfl_xor_sync(0xffffffffu, a.w2, o);
        const uint32_t x3 = __shfl_xor_sync(0xffffffffu, a.w3, o);
        a.dropped |= __shfl_xor_sync(0xffffffffu, a.dropped, o);
        add4(a, x0, x1, x2, x3);
    }
}

// The row's s_x from its reduced window: round A 2^W0 (plus the dropped bits) to
// nearest even, or sum the row again exactly where the dropped bits could decide.
template <typename T>
__device__ double sq_finish(const SqAcc& acc, int W0, int d, const T* __restrict__ xr,
                            unsigned* fallbacks) {
    const uint64_t lo = ((uint64_t)acc.w1 << 32) | acc.w0, hi = ((uint64_t)acc.w3 << 32) | acc.w2;
    const bool dropped = acc.dropped != 0;
    const u128 A = ((u128)hi << 64) | lo;
    const int pos = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    const int cut = pos - 52;                 // >= 1: the bits below the mantissa
    uint64_t mant = (uint64_t)(A >> cut);
    const u128 rem = A & (((u128)1 << cut) - 1), half = (u128)1 << (cut - 1);
    int ex = W0 + pos;
    bool up;
    if (rem > half) {
        up = true;
    } else if (rem == half) {
        up = dropped || (mant & 1);
    } else {
        up = false;
        if (dropped && half - rem <= (u128)d) {
            atomicAdd(fallbacks, 1u);
            return sqnorm_exact_slow(xr, d);
        }
    }
    if (up && ++mant == (1ull << 53)) {
        mant >>= 1;
        ++ex;
    }
    return __longlong_as_double((long long)(((uint64_t)(ex + 1023) << 52) | (mant & ((1ull << 52) - 1))));
}

// Any row length: one warp per row, the row read twice (its maximum, then the
// window sums).
template <typename T, int VEC>
__global__ void __launch_bounds__(256)
    sqnorm_kernel(const T* __restrict__ X, int64_t n, int d, int64_t ld, double* __restrict__ s,
                  uint64_t* keys, uint32_t* vals, unsigned* fallbacks) {
    NRLSH_PDL_ENTRY();
    using G = RowGroups<T, VEC>;
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const T* xr = X + row * ld;
    const int ng = d / VEC;
    // the window: the row's largest term is the square of its largest |x_k|
    float amax = 0.0f;
#pragma unroll 4
    for (int g = lane; g < ng; g += 32) {
        float v[VEC];
        G::load(xr, g, v);
#pragma unroll
        for (int i = 0; i < VEC; ++i) amax = fmaxf(amax, fabsf(v[i]));
    }
    for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    double res = 0.0;
    if (amax > 0.0f && amax < 0x1p-126f) {   // every value subnormal: outside the window's range
        if (lane == 0) {
            atomicAdd(fallbacks, 1u);
            res = sqnorm_exact_slow(xr, d);
        }
    } else if (amax > 0.0f) {
        const SqWindow w = sq_window(amax, d);
        SqAcc acc;
#pragma unroll 4
        for (int g = lane; g < ng; g += 32) {
            float v[VEC];
            G::load(xr, g, v);
#pragma unroll
            for (int i = 0; i < VEC; ++i) sq_add(v[i], w, acc);
        }
        sq_reduce(acc, 32);
        if (lane == 0) res = sq_finish(acc, w.W0, d, xr, fallbacks);
    }
    if (lane == 0) {
        s[row] = res;
        if (keys) {
            keys[row] = (uint64_t)__double_as_longlong(res);
            vals[row] = (uint32_t)row;
        }
    }
}

// Rows of up to 16 NG VEC values: 16 lanes per row (two rows per warp), each lane
// holding its NG groups in registers, so the row is read once with all its loads
// in flight together.
template <typename T, int VEC, int NG>
__global__ void __launch_bounds__(256)
    sqnorm_half_kernel(const T* __restrict__ X, int64_t n, int d, int64_t ld,
                       double* __restrict__ s, uint64_t* keys, uint32_t* vals,
                       unsigned* fallbacks) {
    NRLSH_PDL_ENTRY();
    using G = RowGroups<T, VEC>;
    const int lane = threadIdx.x & 31, li = lane & 15;
    const int64_t row0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 2;
    if (row0 >= n) return;
    const int64_t row = row0 + (lane >> 4);
    const bool valid = row < n;
    const T* xr = X + (valid ? row : row0) * ld;
    const int ng = d / VEC;
    float v[NG][VEC];
#pragma unroll
    for (int j = 0; j < NG; ++j) {
        const int g = li + 16 * j;
        if (valid && g < ng) {
            G::load(xr, g, v[j]);
        } else {
#pragma unroll
            for (int i = 0; i < VEC; ++i) v[j][i] = 0.0f;
        }
    }
    float amax = 0.0f;
#pragma unroll
    for (int j = 0; j < NG; ++j)
#pragma unroll
        for (int i = 0; i < VEC; ++i) amax = fmaxf(amax, fabsf(v[j][i]));
    for (int o = 8; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    // both halves run the sums and reductions whatever their rows hold; a row with
    // no normal value takes no window below
    const SqWindow w = sq_window(fmaxf(amax, 0x1p-126f), d);
    SqAcc acc;
#pragma unroll
    for (int j = 0; j < NG; ++j)
        if (li + 16 * j < ng) {
#pragma unroll
            for (int i = 0; i < VEC; ++i) sq_add(v[j][i], w, acc);
        }
    sq_reduce(acc, 16);
    if (li == 0 && valid) {
        double res = 0.0;
        if (amax > 0.0f && amax < 0x1p-126f) {
            atomicAdd(fallbacks, 1u);
            res = sqnorm_exact_slow(xr, d);
        } else if (amax > 0.0f) {
            res = sq_finish(acc, w.W0, d, xr, fallbacks);
        }
        s[row] = res;
        if (keys) {
            keys[row] = (uint64_t)__double_as_longlong(res);
            vals[row] = (uint32_t)row;
        }
    }
}

}  // namespace

cudaError_t launch_sqnorm(const void* X, nrlsh_dtype dt, int64_t n, int d, int64_t ld, double* s,
                          uint64_t* keys, uint32_t* vals, unsigned* fallbacks, cudaStream_t st) {
    const dim3 grid((unsigned)ceil_div(n * 32, 256));
    // four values per load when every row starts on a 16-byte (fp32) or 8-byte
    // (bf16) boundary and d is a multiple of 4
    const size_t esz = dt == NRLSH_BF16 ? 2 : 4;
    const bool vec = d % 4 == 0 && (ld * esz) % (4 * esz) == 0 && ((uintptr_t)X % (4 * esz)) == 0;
    // rows of up to 512 values in four-value groups: 16 lanes per row
    const int ng = d / 4;
    const int NG = ng <= 32 ? 2 : ng <= 64 ? 4 : ng <= 128 ? 8 : 0;
    if (vec && NG) {
        const dim3 hgrid((unsigned)ceil_div(ceil_div(n, 2) * 32, 256));
#define NRLSH_SQH(T_, NG_)                                                                  \
    return launch("sqnorm_half", sqnorm_half_kernel<T_, 4, NG_>, hgrid, dim3(256), 0, st,    \
                  (const T_*)X, n, d, ld, s, keys, vals, fallbacks);
        if (dt == NRLSH_BF16) {
            if (NG == 2) NRLSH_SQH(__nv_bfloat16, 2)
            if (NG == 4) NRLSH_SQH(__nv_bfloat16, 4)
            NRLSH_SQH(__nv_bfloat16, 8)
        }
        if (NG == 2) NRLSH_SQH(float, 2)
        if (NG == 4) NRLSH_SQH(float, 4)
        NRLSH_SQH(float, 8)
#undef NRLSH_SQH
    }
    if (dt == NRLSH_BF16) {
        if (vec)
            return launch("sqnorm_bf16", sqnorm_kernel<__nv_bfloat16, 4>, grid, dim3(256), 0, st,
                          (const __nv_bfloat16*)X, n, d, ld, s, keys, vals, fallbacks);
        return launch("sqnorm_bf16", sqnorm_kernel<__nv_bfloat16, 1>, grid, dim3(256), 0, st,
                      (const __nv_bfloat16*)X, n, d, ld, s, keys, vals, fallbacks);
    }
    if (vec)
        return launch("sqnorm_f32", sqnorm_kernel<float, 4>, grid, dim3(256), 0, st, (const float*)X,
                      n, d, ld, s, keys, vals, fallbacks);
    return launch("sqnorm_f32", sqnorm_kernel<float, 1>, grid, dim3(256), 0, st, (const float*)X, n,
                  d, ld, s, keys, vals, fallbacks);
}

// =====================================================================
// Stable LSD radix sort, 8-bit digits.  One tile histogram pass up front;
// then per digit: one exclusive scan over (digit, tile) and one stable scatter
// that ranks keys inside a tile (warp match + per-warp digit counts) and, on
// the way, counts the next digit per destination tile for the next pass.  A pass
// whose digit is the same for every key (known from an OR-of-differences
// reduction) turns into a copy, so the buffers alternate the same way always.
// Tiles are 1,024 keys up to 1M keys (more blocks for small inputs) and 4,096
// beyond (a shorter scan).
// =====================================================================

namespace {

constexpr int kSortThreads = 256;
constexpr int kRadix = 256;
constexpr int kLocalOffsetTiles = 64;  // up to this many tiles, no separate scan launch

__device__ __forceinline__ bool digit_varies(const unsigned long long* varying, int shift) {
    return ((*varying >> shift) & 0xFFull) != 0;
}

// Tile histograms of digit 0 and, in the same sweep, the OR over all keys of
// (key xor key[0]): the bits that vary, which tell later passes to skip.
template <typename K, int ROUNDS>
__global__ void __launch_bounds__(kSortThreads)
    radix_first_hist_kernel(const K* __restrict__ keys, int64_t n, unsigned long long* varying,
                            uint32_t* __restrict__ counts, int ntiles) {
    NRLSH_PDL_ENTRY();
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const K k0 = keys[0];
    unsigned long long acc = 0;
    const int64_t base = (int64_t)blockIdx.x * kSortThreads * ROUNDS;
    for (int i = threadIdx.x; i < kSortThreads * ROUNDS; i += kSortThreads) {
        const int64_t p = base + i;
        if (p < n) {
            const K key = keys[p];
            acc |= (unsigned long long)(key ^ k0);
            atomicAdd(&h[(uint32_t)key & 0xFFu], 1u);
        }
    }
    for (int o = 16; o; o >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicOr(varying, acc);
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan in place over total = 256 * ntiles counters, one block of
// 1024 threads, each owning a contiguous run; warp shuffles, then one warp over
// the 32 warp totals.  Also clears the next pass's counters when the scatter
// will accumulate into them.
__global__ void __launch_bounds__(1024)
    radix_scan_kernel(uint32_t* counts, int64_t total, int shift, uint32_t* next_counts,
                      int next_shift, const unsigned long long* varying) {
    NRLSH_PDL_ENTRY();
    if (!digit_varies(varying, shift)) return;
    if (next_counts && digit_varies(varying, next_shift))
        for (int64_t i = threadIdx.x; i < total; i += 1024) next_counts[i] = 0;
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per = ceil_div(total, 1024);
    const int64_t b = threadIdx.x * per, e = min(total, b + per);
    uint32_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += counts[i];
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = (warp ? wsum[warp - 1] : 0) + incl - sum;
    for (int64_t i = b; i < e; ++i) {
        const uint32_t c = counts[i];
        counts[i] = run;
        run += c;
    }
}

// With local_offsets, `offsets` holds the raw tile counts of this digit and each
// block derives its own (digit, tile) offsets: the counts of earlier tiles plus
// an exclusive scan of the digit totals (for few tiles, instead of a scan
// launch); `zero` (same size) is cleared for the pass after next.
template <typename K, int ROUNDS>
__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                         K* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                         const unsigned long long* varying, const uint32_t* __restrict__ offsets,
                         int ntiles, uint32_t* __restrict__ next_counts, int next_shift,
                         int local_offsets, uint32_t* __restrict__ zero) {
    NRLSH_PDL_ENTRY();
    constexpr int kTile = kSortThreads * ROUNDS;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const bool count_next = next_counts != nullptr && digit_varies(varying, next_shift);
    __shared__ uint32_t run_off[kRadix];
    __shared__ uint32_t warp_cnt[kSortThreads / 32][kRadix];
    if (zero)
        for (int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; i < (int64_t)kRadix * ntiles;
             i += (int64_t)gridDim.x * kSortThreads)
            zero[i] = 0;
    if (!digit_varies(varying, shift)) {
        // keys keep their positions: this tile's next-digit histogram is local
        if (count_next) run_off[threadIdx.x] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < kTile; i += kSortThreads) {
            const int64_t p = base + i;
            if (p < n) {
                const K key = kin[p];
                kout[p] = key;
                vout[p] = vin[p];
                if (count_next) atomicAdd(&run_off[(uint32_t)(key >> next_shift) & 0xFFu], 1u);
            }
        }
        __syncthreads();
        if (count_next) next_counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = run_off[threadIdx.x];
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (local_offsets) {
        // thread = digit: count of this digit in earlier tiles, and in all tiles
        const uint32_t* row = offsets + (int64_t)threadIdx.x * ntiles;
        uint32_t before = 0, total = 0;
        for (int t = 0; t < ntiles; ++t) {
            const uint32_t c = row[t];
            before += t < (int)blockIdx.x ? c : 0u;
            total += c;
        }
        uint32_t incl = total;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_cnt[0][warp] = incl;
        __syncthreads();
        uint32_t wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += warp_cnt[0][w];
        run_off[threadIdx.x] = wbase + incl - total + before;
        __syncthreads();
    } else {
        run_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    }
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int round = 0; round < ROUNDS; ++round) {
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
            if (count_next)
                atomicAdd(&next_counts[(int64_t)((key >> next_shift) & 0xFFu) * ntiles + dst / kTile],
                          1u);
        }
        __syncthreads();
    }
}

template <typename K, int ROUNDS>
cudaError_t radix_sort_rounds(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, int64_t n,
                              int key_bits, void* temp, bool* result_in_alt, cudaStream_t s) {
    constexpr int kTile = kSortThreads * ROUNDS;
    const int ntiles = (int)ceil_div(n, kTile);
    const int64_t total = (int64_t)kRadix * ntiles;
    const bool local = ntiles <= kLocalOffsetTiles;
    unsigned long long* varying = (unsigned long long*)temp;
    uint32_t* counts[3] = {(uint32_t*)((char*)temp + 256), (uint32_t*)((char*)temp + 256) + total,
                           (uint32_t*)((char*)temp + 256) + 2 * total};
    cudaError_t e = cudaMemsetAsync(varying, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (local) {  // the write buffer of the first pass must start at zero
        e = cudaMemsetAsync(counts[1], 0, sizeof(uint32_t) * total, s);
        if (e != cudaSuccess) return e;
    }
    e = launch("radix_hist", radix_first_hist_kernel<K, ROUNDS>, dim3(ntiles), dim3(kSortThreads), 0,
               s, (const K*)keys, n, varying, counts[0], ntiles);
    if (e != cudaSuccess) return e;
    K* src_k = keys;
    uint32_t* src_v = vals;
    K* dst_k = keys_alt;
    uint32_t* dst_v = vals_alt;
    int r = 0, w = 1, z = 2;  // read, write (next digit), zero (the pass after next)
    for (int shift = 0; shift < key_bits; shift += 8) {
        const bool last = shift + 8 >= key_bits;
        uint32_t* nxt = last ? nullptr : counts[w];
        if (!local) {
            e = launch("radix_scan", radix_scan_kernel, dim3(1), dim3(1024), 0, s, counts[r], total,
                       shift, nxt, shift + 8, (const unsigned long long*)varying);
            if (e != cudaSuccess) return e;
        }
        e = launch("radix_scatter", radix_scatter_kernel<K, ROUNDS>, dim3(ntiles),
                   dim3(kSortThreads), 0, s, (const K*)src_k, (const uint32_t*)src_v, dst_k, dst_v,
                   n, shift, (const unsigned long long*)varying, (const uint32_t*)counts[r], ntiles,
                   nxt, shift + 8, local ? 1 : 0, local && !last ? counts[z] : nullptr);
        if (e != cudaSuccess) return e;
        std::swap(src_k, dst_k);
        std::swap(src_v, dst_v);
        *result_in_alt = !*result_in_alt;
        if (local) {
            const int r2 = w, w2 = z, z2 = r;
            r = r2;
            w = w2;
            z = z2;
        } else {
            std::swap(r, w);
        }
    }
    return cudaSuccess;
}

constexpr int64_t kSmallSort = 1 << 20;

template <typename K>
cudaError_t radix_sort_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, int64_t n,
                            int key_bits, void* temp, bool* result_in_alt, cudaStream_t s) {
    *result_in_alt = false;
    if (n <= 1 || key_bits <= 0) return cudaSuccess;
    if (n <= kSmallSort)
        return radix_sort_rounds<K, 4>(keys, vals, keys_alt, vals_alt, n, key_bits, temp,
                                       result_in_alt, s);
    return radix_sort_rounds<K, 16>(keys, vals, keys_alt, vals_alt, n, key_bits, temp,
                                    result_in_alt, s);
}

}  // namespace

size_t radix_sort_temp_bytes(int64_t n) {
    const int64_t tile = n <= kSmallSort ? 1024 : 4096;
    return 256 + 3 * sizeof(uint32_t) * (size_t)kRadix *
                     (size_t)ceil_div(std::max<int64_t>(n, 1), tile);
}

cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int key_bits, void* temp, bool* result_in_alt,
                           cudaStream_t s) {
    return radix_sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, key_bits, temp,
                                     result_in_alt, s);
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int key_bits, void* temp, bool* result_in_alt,
                           cudaStream_t s) {
    return radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, key_bits, temp,
                                     result_in_alt, s);
}

// =====================================================================
// Ranking for small inputs (n <= 64 tiles of 1,024): each tile of (s_x, id) keys
// is sorted in shared memory; a key's rank is the number of smaller keys,
// counted tile pair by tile pair by binary search; ranks give each item's
// percentile range, U_j^2 and a per-range bitmap of ids, and one block per range
// reads its bitmap in id order to lay out storage.  Four launches instead of a
// radix pass per 8-bit digit plus a second sort.
// =====================================================================

namespace {

constexpr int kRankTile = 1024;

__device__ __forceinline__ bool key_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Block per tile, one key per thread: bitonic sort of up to 1,024 (key, id) pairs
// in place (padded with the largest pair; exchanges less than 32 apart through
// warp shuffles, wider ones through shared memory).
__global__ void __launch_bounds__(kRankTile)
    tile_sort_kernel(uint64_t* __restrict__ keys, uint32_t* __restrict__ ids, int64_t n) {
    NRLSH_PDL_ENTRY();
    __shared__ uint64_t k_s[kRankTile];
    __shared__ uint32_t i_s[kRankTile];
    const int t = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kRankTile;
    const bool in = base + t < n;
    uint64_t k = in ? keys[base + t] : ~0ull;
    uint32_t id = in ? ids[base + t] : 0xFFFFFFFFu;
    for (int size = 2; size <= kRankTile; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            uint64_t k2;
            uint32_t i2;
            if (stride >= 32) {
                k_s[t] = k;
                i_s[t] = id;
                __syncthreads();
                k2 = k_s[t ^ stride];
                i2 = i_s[t ^ stride];
                __syncthreads();
            } else {
                k2 = __shfl_xor_sync(0xffffffffu, k, stride);
                i2 = __shfl_xor_sync(0xffffffffu, id, stride);
            }
            // the lower thread of a pair keeps the smaller pair in an ascending run
            const bool lower = (t & stride) == 0;
            const bool ascending = (t & size) == 0;
            if (key_less(k2, i2, k, id) == (lower == ascending)) {
                k = k2;
                id = i2;
            }
        }
    }
    if (in) {
        keys[base + t] = k;
        ids[base + t] = id;
    }
}

// Block (t, u) over sorted tiles: each key of tile t adds the number of smaller
// keys of tile u (binary search in shared memory; its own index when u = t) to
// its rank (rank: n words starting at 0).
__global__ void __launch_bounds__(512)
    tile_rank_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ids, int64_t n,
                     unsigned* __restrict__ rank) {
    NRLSH_PDL_ENTRY();
    __shared__ uint64_t k_s[kRankTile];
    __shared__ uint32_t i_s[kRankTile];
    const int64_t tb = (int64_t)blockIdx.x * kRankTile, ub = (int64_t)blockIdx.y * kRankTile;
    const int tlen = (int)min((int64_t)kRankTile, n - tb);
    const int ulen = (int)min((int64_t)kRankTile, n - ub);
    const bool self = blockIdx.x == blockIdx.y;
    if (!self) {
        for (int i = threadIdx.x; i < ulen; i += blockDim.x) {
            k_s[i] = keys[ub + i];
            i_s[i] = ids[ub + i];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < tlen; i += blockDim.x) {
        int lo = i;
        if (!self) {
            const uint64_t kq = keys[tb + i];
            const uint32_t iq = ids[tb + i];
            int hi = ulen;  // first index whose pair is not smaller
            lo = 0;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (key_less(k_s[mid], i_s[mid], kq, iq)) lo = mid + 1; else hi = mid;
            }
        }
        if (lo) atomicAdd(&rank[tb + i], (unsigned)lo);
    }
}

// Thread per key: its range j from its rank, sub_of_id, the bit of its id in
// range j's bitmap (W words per range, zeroed), and U_j^2 from the key at the
// range's last rank.
__global__ void __launch_bounds__(256)
    rank_place_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ids,
                      const unsigned* __restrict__ rank, int64_t n, int m, int64_t W,
                      uint32_t* __restrict__ bitmap, uint32_t* __restrict__ sub_of_id,
                      double* __restrict__ U2) {
    NRLSH_PDL_ENTRY();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int64_t r = rank[e];
    const int j = seg_of(r, n, m);
    const uint32_t id = ids[e];
    sub_of_id[id] = (uint32_t)j;
    atomicOr(&bitmap[(int64_t)j * W + id / 32], 1u << (id % 32));
    if (r == seg_start(j + 1, n, m) - 1) U2[j] = __longlong_as_double((long long)keys[e]);
}

// Block per range j: exclusive scan of the bitmap's popcounts, then every set bit
// in increasing id order goes to perm[seg_start(j) + its index].
__global__ void __launch_bounds__(256)
    range_order_kernel(const uint32_t* __restrict__ bitmap, int64_t n, int m, int64_t W,
                       uint32_t* __restrict__ perm) {
    NRLSH_PDL_ENTRY();
    __shared__ uint32_t wsum[8];
    __shared__ uint32_t carry_s;
    const int j = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t* bm = bitmap + (int64_t)j * W;
    uint32_t* out = perm + seg_start(j, n, m);
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t w0 = 0; w0 < W; w0 += blockDim.x) {
        const int64_t w = w0 + threadIdx.x;
        const uint32_t bits = w < W ? bm[w] : 0u;
        const uint32_t c = __popc(bits);
        uint32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t base = carry_s;
        for (int i = 0; i < warp; ++i) base += wsum[i];
        uint32_t pos = base + incl - c;
        for (uint32_t b = bits; b; b &= b - 1) out[pos++] = (uint32_t)(w * 32 + __ffs(b) - 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int i = 0; i < 8; ++i) tot += wsum[i];
            carry_s += tot;
        }
        __syncthreads();
    }
}

}  // namespace

bool small_rank_supported(int64_t n, int m) {
    return n >= 1 && n <= 64 * kRankTile && (int64_t)m * ceil_div(n, 32) <= ((int64_t)1 << 22);
}

size_t small_rank_temp_bytes(int64_t n, int m) {
    return sizeof(unsigned) * ((size_t)n + (size_t)m * ceil_div(n, 32));
}

cudaError_t launch_small_rank(uint64_t* keys, uint32_t* ids, int64_t n, int m,
                              void* temp, uint32_t* perm, uint32_t* sub_of_id, double* U2,
                              cudaStream_t st) {
    const int T = (int)ceil_div(n, kRankTile);
    const int64_t W = ceil_div(n, 32);
    unsigned* rank = (unsigned*)temp;
    uint32_t* bitmap = rank + n;
    cudaError_t e = launch("tile_sort", tile_sort_kernel, dim3(T), dim3(kRankTile), 0, st, keys, ids, n);
    if (e != cudaSuccess) return e;
    e = launch("tile_rank", tile_rank_kernel, dim3(T, T), dim3(512), 0, st, (const uint64_t*)keys,
               (const uint32_t*)ids, n, rank);
    if (e != cudaSuccess) return e;
    e = launch("rank_place", rank_place_kernel, dim3((unsigned)ceil_div(n, 256)), dim3(256), 0, st,
               keys, ids, (const unsigned*)rank, n, m, W, bitmap, sub_of_id, U2);
    if (e != cudaSuccess) return e;
    return launch("range_order", range_order_kernel, dim3(m), dim3(256), 0, st,
                  (const uint32_t*)bitmap, n, m, W, perm);
}

// =====================================================================
// Partition helpers.
// =====================================================================

namespace {

// Rank r -> sub-dataset j; U_j^2 from the last rank of each range.  Also writes
// the keys (j by id) and values (ids) of the stable sort into storage order.
__global__ void segment_assign_kernel(const uint64_t* __restrict__ sorted_keys,
                                      const uint32_t* __restrict__ sorted_ids, int64_t n, int m,
                                      uint32_t* sub_of_id, double* U2, uint32_t* jkeys,
                                      uint32_t* jvals) {
    NRLSH_PDL_ENTRY();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t j = seg_of(r, n, m);
    const uint32_t id = sorted_ids[r];
    sub_of_id[id] = (uint32_t)j;
    jkeys[id] = (uint32_t)j;
    jvals[r] = (uint32_t)r;
    if (r == seg_start(j + 1, n, m) - 1) U2[j] = __longlong_as_double((long long)sorted_keys[r]);
}

// Uniform norm ranges (the alternative partition of Section 5, Figure 3a):
// nu_x = sqrt(s_x), [nu_min, nu_max] cut into m equal ranges,
//   j(x) = min(m - 1, floor(fl(fl(fl(nu_x - nu_min) / w) * m))),  w = fl(nu_max - nu_min),
// every operation IEEE round-to-nearest (j = 0 for all items when w = 0).  Each
// step is monotone, so the ranges are contiguous in ||x||; some may be empty.
//
// First kernel: min and max of s (the bit patterns of non-negative doubles order
// like the values); the last block to finish stores nu_min, nu_max and w as the
// doubles range[2..4] (sqrt is monotone, so sqrt(min s) = min sqrt(s)).
__global__ void __launch_bounds__(256)
    norm_range_kernel(const double* __restrict__ s, int64_t n, unsigned long long* range,
                      unsigned* done) {
    NRLSH_PDL_ENTRY();
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(s[i] + 0.0);
        lo = u < lo ? u : lo;
        hi = u > hi ? u : hi;
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&range[0], lo);
        atomicMax(&range[1], hi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1u) == gridDim.x - 1) {
            __threadfence();
            const double nlo = sqrt(__longlong_as_double((long long)atomicAdd(&range[0], 0ull)));
            const double nhi = sqrt(__longlong_as_double((long long)atomicAdd(&range[1], 0ull)));
            range[2] = (unsigned long long)__double_as_longlong(nlo);
            range[3] = (unsigned long long)__double_as_longlong(nhi);
            range[4] = (unsigned long long)__double_as_longlong(__dsub_rn(nhi, nlo));
        }
    }
}

// Second kernel, one thread per id: j(x), the keys (j by id) and values (ids) of
// the stable sort into storage order, the sub-dataset sizes, and U_j^2 = max s
// over S_j (atomic max on the bit patterns; U2 starts at +0, so an empty S_j
// keeps U_j = 0).
__global__ void __launch_bounds__(256)
    uniform_assign_kernel(const double* __restrict__ s_id, int64_t n, int m,
                          const unsigned long long* __restrict__ range, uint32_t* sub_of_id,
                          unsigned long long* U2_bits, uint32_t* jkeys, uint32_t* jvals,
                          uint32_t* cnt) {
    NRLSH_PDL_ENTRY();
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const double s = s_id[id] + 0.0;
    const double lo = __longlong_as_double((long long)range[2]);
    const double w = __longlong_as_double((long long)range[4]);
    int j = 0;
    if (w > 0.0) {
        const double t = __dmul_rn(__ddiv_rn(__dsub_rn(sqrt(s), lo), w), (double)m);
        j = (int)fmin(floor(t), (double)(m - 1));
    }
    sub_of_id[id] = (uint32_t)j;
    jkeys[id] = (uint32_t)j;
    jvals[id] = (uint32_t)id;
    atomicAdd(&cnt[j], 1u);
    atomicMax(&U2_bits[j], (unsigned long long)__double_as_longlong(s));
}

// Exclusive scan over one block of 1024 threads (one value per thread).
__device__ int64_t block_scan_1024(int64_t v, int64_t* total, int64_t* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    const int64_t ex = (warp ? wsum[warp - 1] : 0) + incl - v;
    *total = wsum[31];
    __syncthreads();
    return ex;
}

// Segment offsets seg[0..m] (storage positions of each S_j: an exclusive scan of
// the sizes) and the histogram tiles (runs of at most `tile` positions inside one
// sub-dataset, in sub-dataset order); entries past the last tile, up to
// ntiles_max, get length 0.  One block; thread t owns sub-datasets
// [t per, (t + 1) per).
__global__ void __launch_bounds__(1024)
    segments_kernel(const uint32_t* __restrict__ cnt, int64_t n, int m, int64_t tile, int64_t* seg,
                    PosTile* tiles, int ntiles_max) {
    NRLSH_PDL_ENTRY();
    __shared__ int64_t wsum[32];
    const int per = (m + 1023) / 1024;
    const int b = min(m, (int)threadIdx.x * per), e = min(m, b + per);
    // sizes: counted (uniform ranges) or floor((j+1)n/m) - floor(jn/m) (percentiles)
    auto size_of = [&](int j) -> int64_t {
        return cnt ? (int64_t)cnt[j] : seg_start(j + 1, n, m) - seg_start(j, n, m);
    };
    int64_t items = 0, ntl = 0;
    for (int j = b; j < e; ++j) {
        items += size_of(j);
        ntl += ceil_div(size_of(j), tile);
    }
    int64_t items_total, tiles_total;
    int64_t pos = block_scan_1024(items, &items_total, wsum);
    int64_t t = block_scan_1024(ntl, &tiles_total, wsum);
    for (int j = b; j < e; ++j) {
        seg[j] = pos;
        const int64_t len = size_of(j);
        for (int64_t a = 0; a < len; a += tile) tiles[t++] = {pos + a, (int32_t)min(tile, len - a), j};
        pos += len;
    }
    if (threadIdx.x == 0) seg[m] = items_total;
    for (int64_t i = tiles_total + threadIdx.x; i < ntiles_max; i += 1024) tiles[i] = {0, 0, 0};
}

// Block of 256 threads per 32 storage positions.  Warp 0, lane i, first writes
// position i's squared norm, tau = sqrt(U_j^2 - s) (1 when U_j = 0) and an fp32
// upper bound of ||x||, so the FP64 square roots run on full warps; then warp w
// copies rows w, w + 8, ... (zero-padded to dp) and, when the FP32 sums of the
// item projection were computed beside the partition, decides the position's
// code bits (code_of_position).
struct GatherTail {
    double tau;
    float tau32, xn;
};
__device__ __forceinline__ GatherTail gather_tail(int64_t p, uint32_t id,
                                                  const uint32_t* __restrict__ sub_of_id,
                                                  const double* __restrict__ s_id,
                                                  const double* __restrict__ U2, double* s_pos,
                                                  double* tau64, float* tau32, float* xnorm) {
    const double s = s_id[id];
    const double u2 = U2[sub_of_id[id]];
    const double t = (u2 == 0.0) ? 1.0 : sqrt(u2 - s);
    const float xn = __fsqrt_ru(__double2float_ru(s));
    s_pos[p] = s;
    tau64[p] = t;
    tau32[p] = (float)t;
    xnorm[p] = xn;
    return {t, (float)t, xn};
}

constexpr int kGatherRows = 32;

// Per block: tau (FP64 and FP32) and the norm bound of each of its positions,
// written by warp 0 for the code decisions of all warps.
struct GatherShared {
    double tau64[kGatherRows];
    float tau32[kGatherRows], xn[kGatherRows];
};

// Warp 0 writes the tails of the block's positions (global arrays and sh); with
// code bits to take, every lane also loads a_db and ||a_b|| of bits lane and
// 32 + lane, and the block waits for the tails.
__device__ __forceinline__ void gather_prologue(const GatherCodes& gc, int64_t p0, int64_t n,
                                                const uint32_t* __restrict__ perm,
                                                const uint32_t* __restrict__ sub_of_id,
                                                const double* __restrict__ s_id,
                                                const double* __restrict__ U2, double* s_pos,
                                                double* tau64, float* tau32, float* xnorm,
                                                GatherShared& sh, float (&ad)[2], float (&an)[2]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0 && p0 + lane < n) {
        const GatherTail t =
            gather_tail(p0 + lane, perm[p0 + lane], sub_of_id, s_id, U2, s_pos, tau64, tau32, xnorm);
        sh.tau64[lane] = t.tau;
        sh.tau32[lane] = t.tau32;
        sh.xn[lane] = t.xn;
    }
    if (gc.vsum) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int b = 32 * h + lane;
            ad[h] = b < gc.L ? gc.A_pad[(int64_t)gc.d * gc.Lp + b] : 0.0f;
            an[h] = b < gc.L ? gc.anorm[b] : 0.0f;
        }
        __syncthreads();
    }
}

// Eq. 4 on the item of Eq. 8 at storage position p (item id, row src): bit b =
// [fl(a_db tau + sum_b) >= 0] with sum_b the FP32 sum a_b^T x computed beside the
// partition, decided where it lies outside (d + 2) 2^-22 ||a_b|| ||x|| + the tail's
// rounding; the other bits are settled by the warp (settle_bit_warp).
template <typename T>
__device__ void code_of_position(const GatherCodes& gc, int64_t p, uint32_t id,
                                 const T* __restrict__ src, const GatherShared& sh, int r,
                                 const float (&ad)[2], const float (&an)[2]) {
    const int lane = threadIdx.x & 31;
    const float* v = gc.vsum + (int64_t)id * gc.Lr;
    const float t32 = sh.tau32[r], xn = sh.xn[r];
    unsigned long long word = 0, undecided = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (32 * h >= gc.Lr) break;
        const int b = 32 * h + lane;
        bool set = false, open = false;
        if (b < gc.L) {
            const float s = fmaf(ad[h], t32, v[b]);
            const float bound = gc.kappa * an[h] * xn + 0x1p-20f * fabsf(ad[h]) * t32;
            if (fabsf(s) * (1.0f - 0x1p-21f) > bound)
                set = s > 0.0f;
            else
                open = true;
        }
        word |= (unsigned long long)__ballot_sync(0xffffffffu, set) << (32 * h);
        undecided |= (unsigned long long)__ballot_sync(0xffffffffu, open) << (32 * h);
    }
    if (undecided) {
        if (lane == 0) atomicAdd(gc.amb_count, (unsigned)__popcll(undecided));
        for (unsigned long long u = undecided; u; u &= u - 1) {
            const int b = __ffsll((long long)u) - 1;
            const float adb = __shfl_sync(0xffffffffu, b < 32 ? ad[0] : ad[1], b & 31);
            const float anb = __shfl_sync(0xffffffffu, b < 32 ? an[0] : an[1], b & 31);
            if (settle_bit_warp(src, gc.d, gc.At32 + (int64_t)b * gc.dpa, adb, sh.tau64[r], true, xn,
                                anb, gc.A_pad, gc.Lp, b))
                word |= 1ull << b;
        }
    }
    if (lane == 0) {
        if (gc.code_bytes == 4)
            static_cast<uint32_t*>(gc.codes)[p] = (uint32_t)word;
        else
            static_cast<uint64_t*>(gc.codes)[p] = word;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
    gather_items_kernel(const T* __restrict__ X, int64_t ld, int d, int dp,
                        const uint32_t* __restrict__ perm, int64_t n,
                        const uint32_t* __restrict__ sub_of_id, const double* __restrict__ s_id,
                        const double* __restrict__ U2, T* __restrict__ Xp,
                        __nv_bfloat16* __restrict__ Xb, __nv_bfloat16* __restrict__ Xb2,
                        double* s_pos, double* tau64, float* tau32, float* xnorm,
                        const GatherCodes gc) {
    NRLSH_PDL_ENTRY();
    __shared__ GatherShared sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * kGatherRows;
    float ad[2], an[2];
    gather_prologue(gc, p0, n, perm, sub_of_id, s_id, U2, s_pos, tau64, tau32, xnorm, sh, ad, an);
    for (int r = warp; r < kGatherRows; r += 8) {
        const int64_t p = p0 + r;
        if (p >= n) break;
        const uint32_t id = perm[p];
        const T* src = X + (int64_t)id * ld;
        T* dst = Xp + p * dp;
        for (int c = lane; c < dp; c += 32) {
            const T v = c < d ? src[c] : T(0.0f);
            dst[c] = v;
            if (Xb) {  // tensor-core copies: x = hi + lo + r, |r| <= 2^-16 |x|
                const float x = to_f32(v);
                const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                Xb[p * dp + c] = hi;
                if (Xb2) Xb2[p * dp + c] = __float2bfloat16_rn(x - __bfloat162float(hi));
            }
        }
        if (gc.vsum) code_of_position(gc, p, id, src, sh, r, ad, an);
    }
}

// Vectorised form of gather_items_kernel for rows whose length d is a multiple
// of the vector width (fp32: 4 per 16-byte load; bf16: 2 per 4-byte load) and
// whose source rows are aligned to it.  Same outputs.
template <typename T>
struct GatherVec;
template <>
struct GatherVec<float> {
    using V = float4;
    static constexpr int W = 4;
    __device__ static void to_f(const V& v, float (&f)[4]) {
        f[0] = v.x;
        f[1] = v.y;
        f[2] = v.z;
        f[3] = v.w;
    }
};
template <>
struct GatherVec<__nv_bfloat16> {
    using V = __nv_bfloat162;
    static constexpr int W = 2;
    __device__ static void to_f(const V& v, float (&f)[2]) {
        const float2 t = __bfloat1622float2(v);
        f[0] = t.x;
        f[1] = t.y;
    }
};

template <typename T>
__global__ void __launch_bounds__(256)
    gather_items_vec_kernel(const T* __restrict__ X, int64_t ld, int d, int dp,
                            const uint32_t* __restrict__ perm, int64_t n,
                            const uint32_t* __restrict__ sub_of_id,
                            const double* __restrict__ s_id, const double* __restrict__ U2,
                            T* __restrict__ Xp, __nv_bfloat16* __restrict__ Xb,
                            __nv_bfloat16* __restrict__ Xb2, double* s_pos, double* tau64,
                            float* tau32, float* xnorm, const GatherCodes gc) {
    NRLSH_PDL_ENTRY();
    using GV = GatherVec<T>;
    using V = typename GV::V;
    constexpr int W = GV::W;
    __shared__ GatherShared sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * kGatherRows;
    float ad[2], an[2];
    gather_prologue(gc, p0, n, perm, sub_of_id, s_id, U2, s_pos, tau64, tau32, xnorm, sh, ad, an);
    const int nv = d / W;
    for (int r = warp; r < kGatherRows; r += 8) {
        const int64_t p = p0 + r;
        if (p >= n) break;
        const uint32_t id = perm[p];
        const V* src = (const V*)(X + (int64_t)id * ld);
        V* dst = (V*)(Xp + p * dp);
        for (int c = lane; c < nv; c += 32) {
            const V v = src[c];
            dst[c] = v;
            if (Xb) {  // tensor-core copies: x = hi + lo + r, |r| <= 2^-16 |x|
                float f[W];
                GV::to_f(v, f);
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    const __nv_bfloat16 hi = __float2bfloat16_rn(f[i]);
                    Xb[p * dp + c * W + i] = hi;
                    if (Xb2)
                        Xb2[p * dp + c * W + i] = __float2bfloat16_rn(f[i] - __bfloat162float(hi));
                }
            }
        }
        for (int c = d + lane; c < dp; c += 32) {
            Xp[p * dp + c] = T(0.0f);
            if (Xb) Xb[p * dp + c] = __float2bfloat16_rn(0.0f);
            if (Xb2) Xb2[p * dp + c] = __float2bfloat16_rn(0.0f);
        }
        if (gc.vsum) code_of_position(gc, p, id, X + (int64_t)id * ld, sh, r, ad, an);
    }
}

}  // namespace

cudaError_t launch_segment_assign(const uint64_t* sorted_keys, const uint32_t* sorted_ids,
                                  int64_t n, int m, uint32_t* sub_of_id, double* U2,
                                  uint32_t* jkeys, uint32_t* jvals, cudaStream_t st) {
    return launch("segment_assign", segment_assign_kernel, dim3((unsigned)ceil_div(n, 256)),
                  dim3(256), 0, st, sorted_keys, sorted_ids, n, m, sub_of_id, U2, jkeys, jvals);
}

cudaError_t launch_uniform_assign(const double* s_id, int64_t n, int m, unsigned long long* range,
                                  uint32_t* sub_of_id, double* U2, uint32_t* jkeys,
                                  uint32_t* jvals, uint32_t* cnt, cudaStream_t st) {
    // range[0] = ~0 (min), range[1..4] = 0, done counter (range[5]) = 0
    cudaError_t e = cudaMemsetAsync(range, 0xFF, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(range + 1, 0, 5 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * m, st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n, 256), 2 * 152);
    e = launch("norm_range", norm_range_kernel, dim3(g), dim3(256), 0, st, s_id, n, range,
               (unsigned*)(range + 5));
    if (e != cudaSuccess) return e;
    return launch("uniform_assign", uniform_assign_kernel, dim3((unsigned)ceil_div(n, 256)),
                  dim3(256), 0, st, s_id, n, m, (const unsigned long long*)range, sub_of_id,
                  (unsigned long long*)U2, jkeys, jvals, cnt);
}

cudaError_t launch_segments(const uint32_t* cnt, int64_t n, int m, int64_t tile, int64_t* seg,
                            PosTile* tiles, int ntiles_max, cudaStream_t st) {
    return launch("segments", segments_kernel, dim3(1), dim3(1024), 0, st, cnt, n, m, tile, seg,
                  tiles, ntiles_max);
}

cudaError_t launch_gather_items(const void* X, nrlsh_dtype dt, int64_t ld, int d, int dp,
                                const uint32_t* perm, int64_t n, const uint32_t* sub_of_id,
                                const double* s_id, const double* U2, void* Xp,
                                __nv_bfloat16* Xb, __nv_bfloat16* Xb2, double* s_pos,
                                double* tau64, float* tau32, float* xnorm, const GatherCodes& gc,
                                cudaStream_t st) {
    const dim3 grid((unsigned)ceil_div(n, kGatherRows));
    if (gc.vsum && (gc.Lr > 64 || gc.d != d)) return cudaErrorInvalidValue;
    if (dt == NRLSH_BF16) {
        if (d % 2 == 0 && ld % 2 == 0 && ((uintptr_t)X & 3) == 0)
            return launch("gather_items_bf16", gather_items_vec_kernel<__nv_bfloat16>, grid,
                          dim3(256), 0, st, (const __nv_bfloat16*)X, ld, d, dp, perm, n, sub_of_id,
                          s_id, U2, (__nv_bfloat16*)Xp, (__nv_bfloat16*)nullptr,
                          (__nv_bfloat16*)nullptr, s_pos, tau64, tau32, xnorm, gc);
        return launch("gather_items_bf16", gather_items_kernel<__nv_bfloat16>, grid, dim3(256), 0,
                      st, (const __nv_bfloat16*)X, ld, d, dp, perm, n, sub_of_id, s_id, U2,
                      (__nv_bfloat16*)Xp, (__nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr, s_pos,
                      tau64, tau32, xnorm, gc);
    }
    if (d % 4 == 0 && ld % 4 == 0 && ((uintptr_t)X & 15) == 0)
        return launch("gather_items_f32", gather_items_vec_kernel<float>, grid, dim3(256), 0, st,
                      (const float*)X, ld, d, dp, perm, n, sub_of_id, s_id, U2, (float*)Xp, Xb, Xb2,
                      s_pos, tau64, tau32, xnorm, gc);
    return launch("gather_items_f32", gather_items_kernel<float>, grid, dim3(256), 0, st,
                  (const float*)X, ld, d, dp, perm, n, sub_of_id, s_id, U2, (float*)Xp, Xb, Xb2,
                  s_pos, tau64, tau32, xnorm, gc);
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

// 1/i! for i = 0..29 as double-double pairs (hi = 1/i! rounded to nearest,
// lo = the rounded remainder), written out from the exact rationals.
__constant__ dd kInvFact[30] = {
    {0x1.0000000000000p+0, 0x0.0p+0},  // 1/0!
    {0x1.0000000000000p+0, 0x0.0p+0},  // 1/1!
    {0x1.0000000000000p-1, 0x0.0p+0},  // 1/2!
    {0x1.5555555555555p-3, 0x1.5555555555555p-57},  // 1/3!
    {0x1.5555555555555p-5, 0x1.5555555555555p-59},  // 1/4!
    {0x1.1111111111111p-7, 0x1.1111111111111p-63},  // 1/5!
    {0x1.6c16c16c16c17p-10, -0x1.f49f49f49f49fp-65},  // 1/6!
    {0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-73},  // 1/7!
    {0x1.a01a01a01a01ap-16, 0x1.a01a01a01a01ap-76},  // 1/8!
    {0x1.71de3a556c734p-19, -0x1.c154f8ddc6c00p-73},  // 1/9!
    {0x1.27e4fb7789f5cp-22, 0x1.cbbc05b4fa99ap-76},  // 1/10!
    {0x1.ae64567f544e4p-26, -0x1.c062e06d1f209p-80},  // 1/11!
    {0x1.1eed8eff8d898p-29, -0x1.2aec959e14c06p-83},  // 1/12!
    {0x1.6124613a86d09p-33, 0x1.f28e0cc748ebep-87},  // 1/13!
    {0x1.93974a8c07c9dp-37, 0x1.05d6f8a2efd1fp-92},  // 1/14!
    {0x1.ae7f3e733b81fp-41, 0x1.1d8656b0ee8cbp-97},  // 1/15!
    {0x1.ae7f3e733b81fp-45, 0x1.1d8656b0ee8cbp-101},  // 1/16!
    {0x1.952c77030ad4ap-49, 0x1.ac981465ddc6cp-103},  // 1/17!
    {0x1.6827863b97d97p-53, 0x1.eec01221a8b0bp-107},  // 1/18!
    {0x1.2f49b46814157p-57, 0x1.2650f61dbdcb4p-112},  // 1/19!
    {0x1.e542ba4020225p-62, 0x1.ea72b4afe3c2fp-120},  // 1/20!
    {0x1.71b8ef6dcf572p-66, -0x1.d043ae40c4647p-120},  // 1/21!
    {0x1.0ce396db7f853p-70, -0x1.aebcdbd20331cp-124},  // 1/22!
    {0x1.761b41316381ap-75, -0x1.3423c7d91404fp-130},  // 1/23!
    {0x1.f2cf01972f578p-80, -0x1.9ada5fcc1ab14p-135},  // 1/24!
    {0x1.3f3ccdd165fa9p-84, -0x1.58ddadf344487p-139},  // 1/25!
    {0x1.88e85fc6a4e5ap-89, -0x1.71c37ebd16540p-143},  // 1/26!
    {0x1.d1ab1c2dccea3p-94, 0x1.054d0c78aea14p-149},  // 1/27!
    {0x1.0a18a2635085dp-98, 0x1.b9e2e28e1aa54p-153},  // 1/28!
    {0x1.259f98b4358adp-103, 0x1.eaf8c39dd9bc5p-157},  // 1/29!
};

// Taylor series on |x| <= pi/4 by Horner's rule in y = x^2; the first omitted
// term, x^30/30!, is below 2^-120.
__device__ dd dd_cos_small(dd x) {
    const dd my = dd_neg(dd_mul(x, x));
    dd p = kInvFact[28];
    for (int i = 13; i >= 0; --i) p = dd_add(kInvFact[2 * i], dd_mul(my, p));
    return p;
}
__device__ dd dd_sin_small(dd x) {
    const dd my = dd_neg(dd_mul(x, x));
    dd p = kInvFact[29];
    for (int i = 13; i >= 0; --i) p = dd_add(kInvFact[2 * i + 1], dd_mul(my, p));
    return dd_mul(x, p);
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

// Order-preserving image of a double as an unsigned integer.
__device__ __forceinline__ unsigned long long double_order(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double order_double(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}

constexpr int kBucketThreads = 256;

// c_l for l = 0..L (one thread each); independent of the data, so the build
// runs it on a side stream beside the norms and the sort.
__global__ void class_cos_kernel(int L, float eps, double* __restrict__ cl) {
    NRLSH_PDL_ENTRY();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l <= L) cl[l] = cos_class(L, l, (double)eps);
}

// The probing order in two launches.  First, one thread per bucket (j, l): the
// key s_hat = fl(U_j c_l), U_j = fl(sqrt(U_j^2)), as an order-preserving
// integer (-0 folded to +0), and the tie key l 2^16 + j.
__global__ void bucket_keys_kernel(const double* __restrict__ U2, const double* __restrict__ cl,
                                   int m, int L, unsigned long long* __restrict__ keys,
                                   uint32_t* __restrict__ tie) {
    NRLSH_PDL_ENTRY();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m * (L + 1)) return;
    const int j = c / (L + 1), l = c % (L + 1);
    keys[c] = double_order(__dadd_rn(__dmul_rn(sqrt(U2[j]), cl[l]), 0.0));
    tie[c] = ((uint32_t)l << 16) | (uint32_t)j;
}

// Then every block stages all keys in shared memory and each warp ranks buckets:
// rank(c) = number of buckets with a greater (s_hat, l, j), counted by the lanes
// over strided buckets and summed.  order[rank] = c, shat_sorted[rank] = s_hat.
// With keys_g null the block computes the keys itself from U2 and the cosines
// (staged in shared memory behind the keys), saving the first launch.
__global__ void __launch_bounds__(kBucketThreads)
    bucket_rank_kernel(const unsigned long long* __restrict__ keys_g,
                       const uint32_t* __restrict__ tie_g, int ncls,
                       double* __restrict__ shat_sorted, uint32_t* __restrict__ order,
                       const double* __restrict__ U2, const double* __restrict__ cl_g, int m,
                       int L) {
    NRLSH_PDL_ENTRY();
    extern __shared__ unsigned long long keys[];
    uint32_t* tie = (uint32_t*)(keys + ncls);
    if (keys_g) {
        for (int c = threadIdx.x; c < ncls; c += blockDim.x) {
            keys[c] = keys_g[c];
            tie[c] = tie_g[c];
        }
    } else {
        double* Uj = (double*)(tie + ((ncls + 1) & ~1));   // m norms, then L+1 cosines
        double* cl = Uj + m;
        for (int j = threadIdx.x; j < m; j += blockDim.x) Uj[j] = sqrt(U2[j]);
        for (int l = threadIdx.x; l <= L; l += blockDim.x) cl[l] = cl_g[l];
        __syncthreads();
        for (int c = threadIdx.x; c < ncls; c += blockDim.x) {
            const int j = c / (L + 1), l = c % (L + 1);
            keys[c] = double_order(__dadd_rn(__dmul_rn(Uj[j], cl[l]), 0.0));
            tie[c] = ((uint32_t)l << 16) | (uint32_t)j;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < ncls; c += gridDim.x * wpb) {
        const unsigned long long k0 = keys[c];
        const uint32_t t0 = tie[c];
        unsigned rank = 0;
        for (int c1 = lane; c1 < ncls; c1 += 32) {
            const unsigned long long k1 = keys[c1];
            rank += (k1 > k0) || (k1 == k0 && tie[c1] > t0);
        }
        rank = __reduce_add_sync(0xffffffffu, rank);
        if (lane == 0) {
            order[rank] = (uint32_t)c;
            shat_sorted[rank] = order_double(k0);
        }
    }
}

}  // namespace

cudaError_t launch_class_cos(int L, float eps, double* cl, cudaStream_t st) {
    return launch("class_cos", class_cos_kernel, dim3((unsigned)ceil_div(L + 1, 32)), dim3(32), 0, st,
                  L, eps, cl);
}

size_t bucket_order_temp_bytes(int m, int L) {
    return (size_t)m * (L + 1) * (sizeof(unsigned long long) + sizeof(uint32_t));
}

cudaError_t launch_bucket_order(const double* U2, const double* cl, int m, int L,
                                double* shat_sorted, uint32_t* order, void* temp,
                                cudaStream_t st) {
    const int ncls = m * (L + 1);
    const size_t key_bytes = (sizeof(unsigned long long) + sizeof(uint32_t)) * ncls + 8;
    const size_t fused_bytes = key_bytes + sizeof(double) * (m + L + 1);
    const bool fused = fused_bytes <= 200 * 1024;
    const size_t smem = fused ? fused_bytes : key_bytes;
    unsigned long long* keys = nullptr;
    uint32_t* tie = nullptr;
    cudaError_t e;
    if (!fused) {  // keys in global memory first (m (L+1) shared words would not fit)
        keys = (unsigned long long*)temp;
        tie = (uint32_t*)(keys + ncls);
        e = launch("bucket_keys", bucket_keys_kernel, dim3((unsigned)ceil_div(ncls, 256)), dim3(256),
                   0, st, U2, cl, m, L, keys, tie);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(bucket_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    const int wpb = kBucketThreads / 32;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(ncls, wpb), 2 * 152);
    return launch("bucket_order", bucket_rank_kernel, dim3(grid), dim3(kBucketThreads), smem, st,
                  (const unsigned long long*)keys, (const uint32_t*)tie, ncls, shat_sorted, order,
                  U2, cl, m, L);
}

}  // namespace nrlsh
