// Deciding one code bit exactly (Eq. 4 on the transformed item of Eq. 8): the
// canonical value is fl(A_seq + fl(a_d tau)) in FP64, A_seq the in-order FP64 sum
// of the exact products x_k a_k, and the bit is [value >= 0].  A bit that the FP32
// pass could not decide goes through two cheaper tiers before the canonical
// sequential form:
//   1. compensated FP32 (Ogita, Rump, Oishi, "Accurate sum and dot product",
//      2005): TwoProduct by fma and TwoSum per lane, lane-strided, then the same
//      transformations down a 5-level tree;
//   2. FP64: the exact products summed lane-strided and by a tree;
// each decides only when its estimate lies farther from zero than its error bound
// plus the canonical sum's own rounding error.
#pragma once

#include "nrlsh_internal.cuh"

namespace nrlsh {
namespace {

// The canonical bit, by one thread.
template <typename T>
__device__ bool project_bit_canonical(const T* __restrict__ xrow, const float* __restrict__ A_pad,
                                      int Lp, int d, int b, bool has_tail, double tau) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k)
        acc = fma((double)to_f32(xrow[k]), (double)A_pad[(int64_t)k * Lp + b], acc);
    if (has_tail) acc = __dadd_rn(acc, __dmul_rn((double)A_pad[(int64_t)d * Lp + b], tau));
    return acc >= 0.0;
}

// One lane's step of the compensated dot product: x y = pr + er exactly, and
// TwoSum(sh, pr) with its error added into sl together with er.
__device__ __forceinline__ void dot2_step(float x, float y, float& sh, float& sl) {
    const float pr = __fmul_rn(x, y);
    const float er = fmaf(x, y, -pr);            // pr + er = x y exactly
    const float s2 = __fadd_rn(sh, pr);          // TwoSum(sh, pr)
    const float bb = __fsub_rn(s2, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s2, bb)), __fsub_rn(pr, bb));
    sh = s2;
    sl = __fadd_rn(__fadd_rn(sl, t), er);
}

// The compensated pairs of all 32 lanes combined by a TwoSum tree (every lane
// ends with the warp's pair).
__device__ __forceinline__ void dot2_warp_reduce(float& sh, float& sl) {
    for (int o = 16; o; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
        const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
        const float s2 = __fadd_rn(sh, oh);
        const float bb = __fsub_rn(s2, sh);
        const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s2, bb)), __fsub_rn(oh, bb));
        sh = s2;
        sl = __fadd_rn(__fadd_rn(sl, ol), t);
    }
}

// Tier 1 bound.  Every transformation is error-free, so sh + (the exact sum of
// the error terms e_i) = x^T a; sl sums the e_i with at most K = 2m + 10
// roundings on any path (m terms per lane: 2 additions per term, 2 per tree
// level), so |sl - sum e_i| <= gamma_K sum|e_i|.  The product errors add up to at
// most u sum|x a|; a lane's TwoSum errors to u m (1 + gamma) times its share of
// sum|x a|, and each tree level's to u (1 + gamma) sum|x a|; so sum|e_i| <=
// u (m + 6) sum|x a| and |sh + sl - x^T a| <= u^2 (2m + 10)(m + 6) sum|x a|
// (u = 2^-24), doubled below.  The canonical in-order FP64 sum is within
// (d - 1) 2^-53 sum|x a| of x^T a, and the FP64 additions forming w are within
// 2^-52 (|w| + |tail|); FP32 underflow adds at most 2^-120.  Outside that total,
// sign(w) is the canonical sign.  xn >= ||x|| and an >= ||a_b|| bound sum|x a|
// (Cauchy-Schwarz).  Returns whether the pair (sh, sl), already reduced over the
// warp, decides the bit, and the bit in `set`.
__device__ __forceinline__ bool dot2_decides(float sh, float sl, double tail, int m, int d, float xn,
                                             float an, bool& set) {
    const double c = 2.0 * 0x1p-48 * (2.0 * m + 10.0) * (m + 6.0) + (d + 2.0) * 0x1p-53;
    const double w = __dadd_rn(__dadd_rn((double)sh, (double)sl), tail);
    const double bound = c * (double)xn * (double)an * (1.0 + 0x1p-20) +
                         0x1p-51 * (fabs(w) + fabs(tail)) + 0x1p-120;
    set = w > 0.0;
    return fabs(w) > bound;
}

// Bit b of the row xr (d values; column b of A is at[0..d) = A^T row b, the tail
// coefficient a_d = ad, tau), decided by the whole warp through the tiers.
template <typename T>
__device__ bool settle_bit_warp(const T* __restrict__ xr, int d, const float* __restrict__ at,
                                float ad, double tau, bool has_tail, float xn, float an,
                                const float* __restrict__ A_pad, int Lp, int b) {
    const int lane = threadIdx.x & 31;
    const double tail = has_tail ? __dmul_rn((double)ad, tau) : 0.0;
    {
        float sh = 0.0f, sl = 0.0f;
#pragma unroll 4
        for (int k = lane; k < d; k += 32) dot2_step(to_f32(xr[k]), at[k], sh, sl);
        dot2_warp_reduce(sh, sl);
        bool set;
        if (dot2_decides(sh, sl, tail, (d + 31) / 32, d, xn, an, set)) return set;
    }
    // Tier 2: FP64 lane-strided sum of the exact products and a tree, within
    // (2d + 8) 2^-53 (sum|a x| + |tail|) of the canonical in-order sum.
    double sd = 0.0, sa = 0.0;
#pragma unroll 4
    for (int k = lane; k < d; k += 32) {
        const double pr = (double)to_f32(xr[k]) * (double)at[k];
        sd += pr;
        sa += fabs(pr);
    }
    for (int o = 16; o; o >>= 1) {
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    const double v = __dadd_rn(sd, tail);
    const double bound = (2.0 * d + 8.0) * 0x1p-53 * (sa + fabs(tail)) + 0x1p-50 * fabs(v);
    if (fabs(v) > bound) return v > 0.0;
    int r = 0;
    if (lane == 0) r = project_bit_canonical(xr, A_pad, Lp, d, b, has_tail, tau);
    return __shfl_sync(0xffffffffu, r, 0) != 0;
}

}  // namespace
}  // namespace nrlsh
