// Projection of rows on CUDA cores (Eq. 4 on the Eq. 8 transform): the FP32
// tier with a proven bound, and the FP32 and FP64 tiers that decide the bits a
// first tier left open.
//
//   project_warp   warp per row, A^T in shared memory, transpose-reduction
//   project_fp32   register-tiled form for rows longer than 1,024
//   resolve_fp32   warp per undecided (row, bit): FP32, lane-strided
//   resolve_fp64   warp per undecided (row, bit): FP64, then the canonical order
#include "nrlsh_internal.cuh"
#include "sign_tiers.cuh"

#include <algorithm>
#include <unordered_map>

namespace nrlsh {

namespace {

constexpr int kProjThreads = 256;  // 8 warps: warp w owns bit group w, lane owns rows
constexpr int kProjKC = 32;        // columns of X staged per step

// Block: 32 RI rows x Lp bits.  Warp w owns bits [w BT, (w+1) BT), lane owns rows
// lane + 32 i (i < RI).  X and A are staged kProjKC columns at a time; every
// (row, bit) accumulates in FP32 in column order.  A bit whose FP32 value lies
// inside the error bound is left 0 and its (row, bit) pair is appended to
// `amb_list` for the resolve kernel (or, if the list is full, decided here by
// the canonical FP64 evaluation).
template <typename T, typename C, int BT, int RI>
__global__ void __launch_bounds__(kProjThreads)
    project_fp32_kernel(const T* __restrict__ X, int64_t n, int d, int ldx, int L, int Lp,
                        const float* __restrict__ A_pad, const float* __restrict__ anorm,
                        const double* __restrict__ tau64, const float* __restrict__ tau32,
                        const float* __restrict__ xnorm, C* __restrict__ codes,
                        unsigned long long* __restrict__ amb_list, unsigned* amb_count,
                        unsigned amb_cap, float kappa) {
    NRLSH_PDL_ENTRY();
    constexpr int kRows = 32 * RI;
    __shared__ float As[kProjKC][8 * BT];
    __shared__ float Xs[kProjKC][kRows + 1];
    __shared__ unsigned long long code_s[kRows];

    const int lane = threadIdx.x & 31, bg = threadIdx.x >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    if (threadIdx.x < kRows) code_s[threadIdx.x] = 0ull;

    float acc[RI][BT];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int b = 0; b < BT; ++b) acc[i][b] = 0.0f;

    for (int k0 = 0; k0 < d; k0 += kProjKC) {
        __syncthreads();
        for (int i = threadIdx.x; i < kRows * kProjKC; i += kProjThreads) {
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
            float xv[RI];
#pragma unroll
            for (int i = 0; i < RI; ++i) xv[i] = Xs[c][lane + 32 * i];
#pragma unroll
            for (int b = 0; b < BT; ++b) {
                const float a = As[c][bg * BT + b];
#pragma unroll
                for (int i = 0; i < RI; ++i) acc[i][b] = fmaf(xv[i], a, acc[i][b]);
            }
        }
    }

    const bool has_tail = tau64 != nullptr;
#pragma unroll
    for (int i = 0; i < RI; ++i) {
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
            if (fabsf(v) * (1.0f - 0x1p-21f) > bound) {
                if (v > 0.0f) word |= 1ull << bit;
            } else {
                const unsigned slot = atomicAdd(amb_count, 1u);
                if (slot < amb_cap) {
                    amb_list[slot] = ((unsigned long long)row << 6) | (unsigned)bit;
                } else if (project_bit_canonical(X + row * ldx, A_pad, Lp, d, bit, has_tail,
                                            has_tail ? tau64[row] : 0.0)) {
                    word |= 1ull << bit;
                }
            }
        }
        if (word) atomicOr(&code_s[r], word);
    }
    __syncthreads();
    if (threadIdx.x < kRows) {
        const int64_t row = row0 + threadIdx.x;
        if (row < n) codes[row] = (C)code_s[threadIdx.x];
    }
}

__device__ __forceinline__ void or_bit(uint32_t* w, int bit) { atomicOr(w, 1u << bit); }
__device__ __forceinline__ void or_bit(uint64_t* w, int bit) {
    atomicOr((unsigned long long*)w, 1ull << bit);
}

// Warp per undecided (row, bit): FP64 dot in lane-strided order, then a tree.
// Both that sum and the canonical in-order sum are within (d-1) 2^-53 sum|a_k x_k|
// of the exact value, so outside (2d + 8) 2^-53 (sum|a_k x_k| + |tail|) plus the
// final-add rounding the two have the same sign.  Otherwise lane 0 evaluates the
// canonical sequential form.
template <typename T, typename C>
__global__ void __launch_bounds__(256)
    resolve_kernel(const T* __restrict__ X, int d, int ldx, int Lp, const float* __restrict__ A_pad,
                   const double* __restrict__ tau64, const unsigned long long* __restrict__ list,
                   const unsigned* __restrict__ count, unsigned cap, C* __restrict__ codes) {
    NRLSH_PDL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned cnt = min(*count, cap);
    for (int64_t e = warp; e < cnt; e += nwarps) {
        const unsigned long long entry = list[e];
        const int64_t row = (int64_t)(entry >> 6);
        const int bit = (int)(entry & 63);
        const T* xr = X + row * ldx;
        double s = 0.0, sa = 0.0;
        for (int k = lane; k < d; k += 32) {
            const double p = (double)to_f32(xr[k]) * (double)A_pad[(int64_t)k * Lp + bit];
            s += p;
            sa += fabs(p);
        }
        for (int o = 16; o; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
        }
        const bool has_tail = tau64 != nullptr;
        const double tail = has_tail ? __dmul_rn((double)A_pad[(int64_t)d * Lp + bit], tau64[row]) : 0.0;
        const double v = __dadd_rn(s, tail);
        const double bound = (2.0 * d + 8.0) * 0x1p-53 * (sa + fabs(tail)) + 0x1p-50 * fabs(v);
        bool set;
        if (fabs(v) > bound) {
            set = v > 0.0;
        } else {
            int r = 0;
            if (lane == 0)
                r = project_bit_canonical(xr, A_pad, Lp, d, bit, has_tail, has_tail ? tau64[row] : 0.0);
            set = __shfl_sync(0xffffffffu, r, 0) != 0;
        }
        if (lane == 0 && set) or_bit(codes + row, bit);
    }
}

// The FP32 tier for pairs the bf16 tensor-core pass left undecided (fp32 items):
// warp per pair, FP32 dot of the exact fp32 row in lane-strided order and a
// tree, decided against (d+2) 2^-22 ||a|| ||x|| (any summation order) plus the
// tail rounding; still undecided pairs move on to the FP64 list.
template <typename T, typename C>
__global__ void __launch_bounds__(256)
    resolve_fp32_kernel(const T* __restrict__ X, int d, int ldx, int Lp,
                        const float* __restrict__ A_pad, const float* __restrict__ anorm,
                        const float* __restrict__ xnorm, const float* __restrict__ tau32,
                        const double* __restrict__ tau64, const unsigned long long* __restrict__ list,
                        const unsigned* __restrict__ count, unsigned cap, C* __restrict__ codes,
                        unsigned long long* __restrict__ list2, unsigned* count2, unsigned cap2,
                        float kappa) {
    NRLSH_PDL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned cnt = min(*count, cap);
    for (int64_t e = warp; e < cnt; e += nwarps) {
        const unsigned long long entry = list[e];
        const int64_t row = (int64_t)(entry >> 6);
        const int bit = (int)(entry & 63);
        const T* xr = X + row * ldx;
        float s = 0.0f;
        for (int k = lane; k < d; k += 32) s = fmaf(to_f32(xr[k]), A_pad[(int64_t)k * Lp + bit], s);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float ad = A_pad[(int64_t)d * Lp + bit];
        const float t32 = tau32[row];
        const float v = fmaf(ad, t32, s);
        const float bound = kappa * anorm[bit] * xnorm[row] + 0x1p-20f * fabsf(ad) * t32;
        if (lane == 0) {
            if (fabsf(v) * (1.0f - 0x1p-21f) > bound) {
                if (v > 0.0f) or_bit(codes + row, bit);
            } else {
                const unsigned slot = atomicAdd(count2, 1u);
                if (slot < cap2)
                    list2[slot] = entry;
                else if (project_bit_canonical(xr, A_pad, Lp, d, bit, true, tau64[row]))
                    or_bit(codes + row, bit);
            }
        }
    }
}

// Warp-per-row form of the FP32 tier.  A^T (bit-major, zero-padded) sits in
// shared memory; a warp keeps its row in registers (lane owns columns
// lane + 32 i), forms 32 bit-partials per pass, and reduces them with a
// transpose-reduction (31 shuffles) after which lane l holds the sum of bit
// 32 pass + l.  Any summation order satisfies the same FP32 bound.  The warp then
// settles its row's undecided bits in FP64 itself, so no list or second launch
// is needed (amb_count still counts them).
// One pass of the warp-per-row projection: FP32 sums a_b^T x of bits 32 pass
// .. 32 pass + 31 for ROWS rows held in registers (lane owns columns lane + 32 i),
// A^T read from shared memory (row stride dpa) once for all rows, and a
// transpose-reduction (31 shuffles) after which lane l holds bit 32 pass + l.
template <int NREG, int ROWS>
__device__ __forceinline__ void pass_sums(const float (&x)[ROWS][NREG], const float* At_s, int dpa,
                                          int pass, int lane, float (&out)[ROWS][1]) {
    float acc[ROWS][32];
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const float* ar = At_s + (pass * 32 + b) * dpa + lane;
        float a[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) a[r] = 0.0f;
#pragma unroll
        for (int i = 0; i < NREG; ++i) {
            const float av = ar[32 * i];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) a[r] = fmaf(x[r][i], av, a[r]);
        }
#pragma unroll
        for (int r = 0; r < ROWS; ++r) acc[r][b] = a[r];
    }
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int j = 0; j < w; ++j)
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const float send = up ? acc[r][j] : acc[r][j + w];
                const float keep = up ? acc[r][j + w] : acc[r][j];
                acc[r][j] = keep + __shfl_xor_sync(0xffffffffu, send, w);
            }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) out[r][0] = acc[r][0];
}

// The FP32 sums a_b^T x of every row and bit (no tail, no decision), in id order:
// vsum[row Lr + b].  Run beside the partition; the signs are taken once tau is
// known, by the gather that places each item.  A^T comes from the index's copy
// (At32).
template <typename T, int NREG, int ROWS>
__global__ void __launch_bounds__(256)
    project_dots_kernel(const T* __restrict__ X, int64_t n, int d, int ldx, int Lp, int dpa,
                        const float* __restrict__ At32, float* __restrict__ vsum) {
    NRLSH_PDL_ENTRY();
    extern __shared__ __align__(16) float At_s[];
    const int Lr = (Lp + 31) / 32 * 32;
    for (int i = threadIdx.x; i < Lr * dpa / 4; i += blockDim.x)
        ((float4*)At_s)[i] = ((const float4*)At32)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * ROWS; row0 < n;
         row0 += nwarps * ROWS) {
        float x[ROWS][NREG];
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
#pragma unroll
            for (int i = 0; i < NREG; ++i) {
                const int k = lane + 32 * i;
                x[r][i] = (row0 + r < n && k < d) ? to_f32(X[(row0 + r) * ldx + k]) : 0.0f;
            }
        for (int pass = 0; pass < Lr / 32; ++pass) {
            float acc[ROWS][1];
            pass_sums<NREG, ROWS>(x, At_s, dpa, pass, lane, acc);
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
                if (row0 + r < n) vsum[(row0 + r) * Lr + pass * 32 + lane] = acc[r][0];
        }
    }
}

template <typename T, int NREG, int ROWS>
__global__ void __launch_bounds__(256)
    project_warp_kernel(const T* __restrict__ X, int64_t n, int d, int ldx, int L, int Lp, int dpa,
                        const float* __restrict__ A_pad, const float* __restrict__ anorm,
                        const double* __restrict__ tau64, const float* __restrict__ tau32,
                        const float* __restrict__ xnorm, void* __restrict__ codes, int code_bytes,
                        unsigned* amb_count, float kappa, float* __restrict__ norm_out,
                        const float* __restrict__ At32) {
    NRLSH_PDL_ENTRY();
    extern __shared__ __align__(16) float At_s[];  // Lr x dpa, Lr = Lp rounded up to 32
    __shared__ float ad_s[64], an_s[64];
    const int Lr = (Lp + 31) / 32 * 32;
    if (At32) {  // the index keeps A^T in this layout: a straight vector copy
        for (int i = threadIdx.x; i < Lr * dpa / 4; i += blockDim.x)
            ((float4*)At_s)[i] = ((const float4*)At32)[i];
    } else {
        for (int i = threadIdx.x; i < Lr * dpa; i += blockDim.x) {
            const int b = i / dpa, k = i % dpa;
            At_s[i] = (b < L && k < d) ? A_pad[(int64_t)k * Lp + b] : 0.0f;
        }
    }
    if (threadIdx.x < 64) {
        const int b = threadIdx.x;
        ad_s[b] = (b < L && tau64) ? A_pad[(int64_t)d * Lp + b] : 0.0f;
        an_s[b] = b < L ? anorm[b] : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const bool has_tail = tau64 != nullptr;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // a warp takes ROWS consecutive rows at a time: every A^T element read from
    // shared memory serves all of them
    for (int64_t row0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * ROWS; row0 < n;
         row0 += nwarps * ROWS) {
        float x[ROWS][NREG];
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
#pragma unroll
            for (int i = 0; i < NREG; ++i) {
                const int k = lane + 32 * i;
                x[r][i] = (row0 + r < n && k < d) ? to_f32(X[(row0 + r) * ldx + k]) : 0.0f;
            }
        // fp32 upper bound of ||x||: given (items), or computed here from the row
        // in registers (queries; FP64 squares in lane-strided order and a tree)
        float xn[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            if (norm_out) {
                double ss = 0.0;
#pragma unroll
                for (int i = 0; i < NREG; ++i) ss = fma((double)x[r][i], (double)x[r][i], ss);
                for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
                xn[r] = __fsqrt_ru(__double2float_ru(ss));
                if (lane == 0 && row0 + r < n) norm_out[row0 + r] = xn[r];
            } else {
                xn[r] = row0 + r < n ? xnorm[row0 + r] : 0.0f;
            }
        }
        unsigned long long word[ROWS], undecided[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) word[r] = undecided[r] = 0;
        for (int pass = 0; pass < Lr / 32; ++pass) {
            float acc[ROWS][1];
            pass_sums<NREG, ROWS>(x, At_s, dpa, pass, lane, acc);
            const int bit = pass * 32 + lane;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                bool set = false, open = false;
                if (bit < L && row0 + r < n) {
                    const float t32 = has_tail ? tau32[row0 + r] : 0.0f;
                    const float ad = ad_s[bit];
                    const float v = has_tail ? fmaf(ad, t32, acc[r][0]) : acc[r][0];
                    const float bound = kappa * an_s[bit] * xn[r] + 0x1p-20f * fabsf(ad) * t32;
                    if (fabsf(v) * (1.0f - 0x1p-21f) > bound)
                        set = v > 0.0f;
                    else
                        open = true;
                }
                word[r] |= (unsigned long long)__ballot_sync(0xffffffffu, set) << (32 * pass);
                undecided[r] |= (unsigned long long)__ballot_sync(0xffffffffu, open) << (32 * pass);
            }
        }
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int64_t row = row0 + r;
            if (row >= n) break;
            // undecided bits, decided by this warp with the row still in registers:
            // the compensated FP32 tier (dot2_decides), then an FP64 lane-strided sum
            // and a tree (within (2d + 8) 2^-53 (sum|a x| + |tail|) of the canonical
            // in-order sum, as in resolve_kernel), and the canonical sequential form
            // by lane 0 only inside that bound
            if (undecided[r]) {
                if (lane == 0 && amb_count) atomicAdd(amb_count, (unsigned)__popcll(undecided[r]));
                const double tau = has_tail ? tau64[row] : 0.0;
                for (unsigned long long u = undecided[r]; u; u &= u - 1) {
                    const int b = __ffsll((long long)u) - 1;
                    const float* ar = At_s + b * dpa + lane;
                    {
                        float sh = 0.0f, sl = 0.0f;
#pragma unroll
                        for (int i = 0; i < NREG; ++i) dot2_step(x[r][i], ar[32 * i], sh, sl);
                        dot2_warp_reduce(sh, sl);
                        const double tail1 = has_tail ? __dmul_rn((double)ad_s[b], tau) : 0.0;
                        bool set1;
                        if (dot2_decides(sh, sl, tail1, NREG, d, xn[r], an_s[b], set1)) {
                            if (set1) word[r] |= 1ull << b;
                            continue;
                        }
                    }
                    double sd = 0.0, sa = 0.0;
#pragma unroll
                    for (int i = 0; i < NREG; ++i) {
                        const double pr = (double)x[r][i] * (double)ar[32 * i];
                        sd += pr;
                        sa += fabs(pr);
                    }
                    for (int o = 16; o; o >>= 1) {
                        sd += __shfl_xor_sync(0xffffffffu, sd, o);
                        sa += __shfl_xor_sync(0xffffffffu, sa, o);
                    }
                    const double tail = has_tail ? __dmul_rn((double)ad_s[b], tau) : 0.0;
                    const double v = __dadd_rn(sd, tail);
                    const double bound =
                        (2.0 * d + 8.0) * 0x1p-53 * (sa + fabs(tail)) + 0x1p-50 * fabs(v);
                    bool set;
                    if (fabs(v) > bound) {
                        set = v > 0.0;
                    } else {
                        int rr = 0;
                        if (lane == 0)
                            rr = project_bit_canonical(X + row * ldx, A_pad, Lp, d, b, has_tail, tau);
                        set = __shfl_sync(0xffffffffu, rr, 0) != 0;
                    }
                    if (set) word[r] |= 1ull << b;
                }
            }
            if (lane == 0) {
                if (code_bytes == 4)
                    static_cast<uint32_t*>(codes)[row] = (uint32_t)word[r];
                else
                    static_cast<uint64_t*>(codes)[row] = word[r];
            }
        }
    }
}

template <typename T, typename C, int BT>
cudaError_t project_rows(const void* X, int64_t n, int d, int ldx, int L, int Lp,
                         const float* A_pad, const float* anorm, const double* tau64,
                         const float* tau32, const float* xnorm, void* codes,
                         unsigned long long* amb_list, unsigned* amb_count, unsigned amb_cap,
                         float kappa, cudaStream_t st, const char* name) {
    return launch(name, project_fp32_kernel<T, C, BT, 2>, dim3((unsigned)ceil_div(n, 64)),
                  dim3(kProjThreads), 0, st, (const T*)X, n, d, ldx, L, Lp, A_pad, anorm, tau64,
                  tau32, xnorm, (C*)codes, amb_list, amb_count, amb_cap, kappa);
}

constexpr size_t kWarpProjMaxSmem = 227 * 1024;

// The bits the tensor-core pass left open, settled in one launch: a warp per
// listed (row, bit) runs the compensated FP32 tier, then (rarely) the FP64 tier and
// the canonical form (settle_bit_warp), with column b of A read contiguously from
// the fp32 A^T copy (row stride dpa).
template <typename T, typename C>
__global__ void __launch_bounds__(256)
    resolve_tiers_kernel(const T* __restrict__ X, int d, int ldx, int Lp, int dpa,
                         const float* __restrict__ At32, const float* __restrict__ A_pad,
                         const float* __restrict__ anorm, const float* __restrict__ xnorm,
                         const double* __restrict__ tau64, const unsigned long long* __restrict__ list,
                         const unsigned* __restrict__ count, unsigned cap, C* __restrict__ codes) {
    NRLSH_PDL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned cnt = min(*count, cap);
    for (int64_t e = warp; e < cnt; e += nwarps) {
        const unsigned long long entry = list[e];
        const int64_t row = (int64_t)(entry >> 6);
        const int bit = (int)(entry & 63);
        const bool set = settle_bit_warp(X + row * ldx, d, At32 + (int64_t)bit * dpa,
                                         A_pad[(int64_t)d * Lp + bit], tau64[row], true, xnorm[row],
                                         anorm[bit], A_pad, Lp, bit);
        if (lane == 0 && set) or_bit(codes + row, bit);
    }
}

}  // namespace

// Row stride (columns) of A^T for the warp-per-row projection, or 0 when it does
// not apply (rows longer than 1,024, or A^T beyond the shared memory of a block).
int warp_proj_stride(int d, int Lp) {
    const int nreg = (d + 31) / 32;
    if (nreg > 32) return 0;
    const int dpa = (nreg <= 4 ? 4 : nreg <= 10 ? 10 : 32) * 32;
    const size_t lr = (size_t)(Lp + 31) / 32 * 32;
    return sizeof(float) * lr * dpa <= kWarpProjMaxSmem ? dpa : 0;
}

size_t warp_proj_at_floats(int d, int Lp) {
    return (size_t)(Lp + 31) / 32 * 32 * warp_proj_stride(d, Lp);
}

namespace {

// A^T for the warp-per-row projection: row b holds a_{k,b}, k < d, zero-padded.
__global__ void transpose_a_kernel(const float* __restrict__ A_pad, int d, int L, int Lp, int dpa,
                                   float* __restrict__ At32) {
    NRLSH_PDL_ENTRY();
    const int b = blockIdx.x;
    for (int k = threadIdx.x; k < dpa; k += blockDim.x)
        At32[(int64_t)b * dpa + k] = (b < L && k < d) ? A_pad[(int64_t)k * Lp + b] : 0.0f;
}

// Per kernel (and thread): the dynamic shared memory the attribute allows so far
// (only ever raised, since launches with other code widths share the kernel)
// and the blocks per SM for the last size asked.
template <typename T, int NREG, int ROWS>
struct WarpKernelState {
    static thread_local int dev;
    static thread_local size_t attr, occ_smem;
    static thread_local int per_sm;
};
template <typename T, int NREG, int ROWS> thread_local int WarpKernelState<T, NREG, ROWS>::dev = -1;
template <typename T, int NREG, int ROWS> thread_local size_t WarpKernelState<T, NREG, ROWS>::attr = 0;
template <typename T, int NREG, int ROWS> thread_local size_t WarpKernelState<T, NREG, ROWS>::occ_smem = 0;
template <typename T, int NREG, int ROWS> thread_local int WarpKernelState<T, NREG, ROWS>::per_sm = 1;

template <typename T, typename C, int NREG, int ROWS>
cudaError_t project_warp_launch(const void* X, int64_t n, int d, int ldx, int L, int Lp,
                                const float* A_pad, const float* anorm, const double* tau64,
                                const float* tau32, const float* xnorm, void* codes,
                                unsigned* amb_count, float kappa, float* norm_out,
                                const float* At32, cudaStream_t st, const char* name) {
    using S = WarpKernelState<T, NREG, ROWS>;
    const int Lr = (Lp + 31) / 32 * 32, dpa = NREG * 32;
    const size_t smem = sizeof(float) * (size_t)Lr * dpa;
    auto kern = project_warp_kernel<T, NREG, ROWS>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != S::dev) {
        S::dev = dev;
        S::attr = 0;
        S::occ_smem = 0;
    }
    if (smem > S::attr) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        S::attr = smem;
    }
    if (smem != S::occ_smem) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&S::per_sm, kern, 256, smem);
        if (e != cudaSuccess) return e;
        S::per_sm = std::max(1, S::per_sm);
        S::occ_smem = smem;
    }
    const unsigned grid =
        (unsigned)std::min<int64_t>(ceil_div(n, 8 * ROWS), (int64_t)S::per_sm * 152);
    return launch(name, kern, dim3(grid), dim3(256), smem, st, (const T*)X, n, d, ldx, L, Lp, dpa,
                  A_pad, anorm, tau64, tau32, xnorm, codes, (int)sizeof(C), amb_count, kappa,
                  norm_out, At32);
}

template <typename T, typename C>
cudaError_t project_dispatch(const void* X, int64_t n, int d, int ldx, int L, int Lp,
                             const float* A_pad, const float* anorm, const double* tau64,
                             const float* tau32, const float* xnorm, void* codes,
                             unsigned long long* amb_list, unsigned* amb_count, unsigned amb_cap,
                             cudaStream_t st, const char* name, float* norm_out,
                             const float* At32) {
    const float kappa = (float)(d + 2) * 0x1p-22f;
    cudaError_t e;
    const int nreg_t = warp_proj_stride(d, Lp) / 32;
    if (nreg_t > 0) {
#define NRLSH_PW(R_, ROWS_)                                                                   \
    e = project_warp_launch<T, C, R_, ROWS_>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32,     \
                                             xnorm, codes, amb_count, kappa, norm_out, At32, st,  \
                                             name);                                               \
    break;
        switch (nreg_t) {
            case 4: NRLSH_PW(4, 2)
            case 10: NRLSH_PW(10, 2)
            default: NRLSH_PW(32, 1)
        }
#undef NRLSH_PW
        return e;
    }
    if (norm_out) {  // the register-tiled kernel reads the norm bounds
        e = launch_row_norm_bound((const float*)X, n, d, norm_out, st);
        if (e != cudaSuccess) return e;
        xnorm = norm_out;
    }
    switch (Lp / 8) {
        case 1:
            e = project_rows<T, C, 1>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm, codes,
                                      amb_list, amb_count, amb_cap, kappa, st, name);
            break;
        case 2:
            e = project_rows<T, C, 2>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm, codes,
                                      amb_list, amb_count, amb_cap, kappa, st, name);
            break;
        case 4:
            e = project_rows<T, C, 4>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm, codes,
                                      amb_list, amb_count, amb_cap, kappa, st, name);
            break;
        case 8:
            e = project_rows<T, C, 8>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm, codes,
                                      amb_list, amb_count, amb_cap, kappa, st, name);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(n * L / 256, 32), 8),
                                                      8 * 152);
    return launch("resolve_fp64", resolve_kernel<T, C>, dim3(grid), dim3(256), 0, st, (const T*)X, d,
                  ldx, Lp, A_pad, tau64, (const unsigned long long*)amb_list,
                  (const unsigned*)amb_count, amb_cap, (C*)codes);
}

}  // namespace

cudaError_t launch_transpose_a(const float* A_pad, int d, int L, int Lp, float* At32,
                               cudaStream_t st) {
    const int dpa = warp_proj_stride(d, Lp);
    if (dpa == 0) return cudaSuccess;
    return launch("transpose_a", transpose_a_kernel, dim3((unsigned)((Lp + 31) / 32 * 32)),
                  dim3(256), 0, st, A_pad, d, L, Lp, dpa, At32);
}

cudaError_t launch_project_fp32(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx,
                                int L, int Lp, const float* A_pad, const float* anorm,
                                const double* tau64, const float* tau32, const float* xnorm,
                                void* codes, int code_bytes, unsigned long long* amb_list,
                                unsigned* amb_count, unsigned amb_cap, const float* At32,
                                cudaStream_t st) {
    if (dt == NRLSH_BF16) {
        if (code_bytes == 4)
            return project_dispatch<__nv_bfloat16, uint32_t>(X, n, d, ldx, L, Lp, A_pad, anorm,
                                                             tau64, tau32, xnorm, codes, amb_list,
                                                             amb_count, amb_cap, st,
                                                             "project_fp32_bf16", nullptr, At32);
        return project_dispatch<__nv_bfloat16, uint64_t>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64,
                                                         tau32, xnorm, codes, amb_list, amb_count,
                                                         amb_cap, st, "project_fp32_bf16", nullptr,
                                                         At32);
    }
    if (code_bytes == 4)
        return project_dispatch<float, uint32_t>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32,
                                                 xnorm, codes, amb_list, amb_count, amb_cap, st,
                                                 "project_fp32", nullptr, At32);
    return project_dispatch<float, uint64_t>(X, n, d, ldx, L, Lp, A_pad, anorm, tau64, tau32, xnorm,
                                             codes, amb_list, amb_count, amb_cap, st,
                                             "project_fp32", nullptr, At32);
}

namespace {

// cudaFuncAttributeMaxDynamicSharedMemorySize raised as needed per kernel, device
// and thread, and the blocks per SM at the last size asked.
cudaError_t dyn_smem_blocks(const void* kern, size_t smem, int* per_sm) {
    struct St {
        int dev = -1;
        size_t attr = 0, occ = 0;
        int per_sm = 1;
    };
    static thread_local std::unordered_map<const void*, St> states;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    St& st = states[kern];
    if (st.dev != dev) st = St{dev, 0, 0, 1};
    if (smem > st.attr) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        st.attr = smem;
    }
    if (smem != st.occ) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&st.per_sm, kern, 256, smem);
        if (e != cudaSuccess) return e;
        st.per_sm = std::max(1, st.per_sm);
        st.occ = smem;
    }
    *per_sm = st.per_sm;
    return cudaSuccess;
}

template <typename T, int NREG, int ROWS>
cudaError_t dots_launch(const void* X, int64_t n, int d, int ldx, int Lp, const float* At32,
                        float* vsum, cudaStream_t st) {
    const int Lr = (Lp + 31) / 32 * 32, dpa = NREG * 32;
    const size_t smem = sizeof(float) * (size_t)Lr * dpa;
    auto kern = project_dots_kernel<T, NREG, ROWS>;
    int per_sm = 1;
    cudaError_t e = dyn_smem_blocks((const void*)kern, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 8 * ROWS), (int64_t)per_sm * 152);
    return launch("project_dots", kern, dim3(grid), dim3(256), smem, st, (const T*)X, n, d, ldx, Lp,
                  dpa, At32, vsum);
}

}  // namespace

bool split_projection_supported(int d, int Lp) { return warp_proj_stride(d, Lp) > 0; }

cudaError_t launch_project_dots(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx, int Lp,
                                const float* At32, float* vsum, cudaStream_t st) {
    const int nreg_t = warp_proj_stride(d, Lp) / 32;
    if (nreg_t == 0) return cudaErrorInvalidValue;
#define NRLSH_DOTS(T_)                                                                      \
    switch (nreg_t) {                                                                       \
        case 4: return dots_launch<T_, 4, 2>(X, n, d, ldx, Lp, At32, vsum, st);             \
        case 10: return dots_launch<T_, 10, 2>(X, n, d, ldx, Lp, At32, vsum, st);           \
        default: return dots_launch<T_, 32, 1>(X, n, d, ldx, Lp, At32, vsum, st);           \
    }
    if (dt == NRLSH_BF16) NRLSH_DOTS(__nv_bfloat16)
    NRLSH_DOTS(float)
#undef NRLSH_DOTS
}

cudaError_t launch_hash_queries(const float* Q, int64_t nq, int d, int L, int Lp,
                                const float* A_pad, const float* anorm, float* qnorm, void* codes,
                                int code_bytes, unsigned long long* amb_list, unsigned* amb_count,
                                unsigned amb_cap, const float* At32, cudaStream_t st) {
    if (warp_proj_stride(d, Lp) > 0) {
        amb_count = nullptr;  // the warp kernel settles its bits itself: nothing to count
    } else {
        cudaError_t e = cudaMemsetAsync(amb_count, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
    }
    if (code_bytes == 4)
        return project_dispatch<float, uint32_t>(Q, nq, d, d, L, Lp, A_pad, anorm, nullptr, nullptr,
                                                 nullptr, codes, amb_list, amb_count, amb_cap, st,
                                                 "hash_queries", qnorm, At32);
    return project_dispatch<float, uint64_t>(Q, nq, d, d, L, Lp, A_pad, anorm, nullptr, nullptr,
                                             nullptr, codes, amb_list, amb_count, amb_cap, st,
                                             "hash_queries", qnorm, At32);
}

cudaError_t launch_resolve_fp32(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx, int L,
                                int Lp, const float* A_pad, const float* anorm, const float* xnorm,
                                const float* tau32, const double* tau64,
                                const unsigned long long* list, const unsigned* count,
                                unsigned cap, void* codes, int code_bytes,
                                unsigned long long* list2, unsigned* count2, unsigned cap2,
                                cudaStream_t st) {
    const float kappa = (float)(d + 2) * 0x1p-22f;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(n * L / 32, 32), 8),
                                                      16 * 152);
#define NRLSH_R32(T_, C_)                                                                    \
    return launch("resolve_fp32", resolve_fp32_kernel<T_, C_>, dim3(grid), dim3(256), 0, st,  \
                  (const T_*)X, d, ldx, Lp, A_pad, anorm, xnorm, tau32, tau64, list, count,  \
                  cap, (C_*)codes, list2, count2, cap2, kappa);
    if (dt == NRLSH_BF16) {
        if (code_bytes == 4) NRLSH_R32(__nv_bfloat16, uint32_t)
        NRLSH_R32(__nv_bfloat16, uint64_t)
    }
    if (code_bytes == 4) NRLSH_R32(float, uint32_t)
    NRLSH_R32(float, uint64_t)
#undef NRLSH_R32
}

cudaError_t launch_resolve_tiers(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx, int L,
                                 int Lp, const float* At32, const float* A_pad, const float* anorm,
                                 const float* xnorm, const double* tau64,
                                 const unsigned long long* list, const unsigned* count,
                                 unsigned cap, void* codes, int code_bytes, cudaStream_t st) {
    const int dpa = warp_proj_stride(d, Lp);
    if (dpa == 0 || At32 == nullptr) return cudaErrorNotSupported;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(n * L / 32, 32), 8),
                                                      16 * 152);
#define NRLSH_RT(T_, C_)                                                                     \
    return launch("resolve_tiers", resolve_tiers_kernel<T_, C_>, dim3(grid), dim3(256), 0, st, \
                  (const T_*)X, d, ldx, Lp, dpa, At32, A_pad, anorm, xnorm, tau64, list, count, \
                  cap, (C_*)codes);
    if (dt == NRLSH_BF16) {
        if (code_bytes == 4) NRLSH_RT(__nv_bfloat16, uint32_t)
        NRLSH_RT(__nv_bfloat16, uint64_t)
    }
    if (code_bytes == 4) NRLSH_RT(float, uint32_t)
    NRLSH_RT(float, uint64_t)
#undef NRLSH_RT
}

cudaError_t launch_resolve_fp64(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx, int L,
                                int Lp, const float* A_pad, const double* tau64,
                                const unsigned long long* list, const unsigned* count,
                                unsigned cap, void* codes, int code_bytes, cudaStream_t st) {
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(n * L / 256, 32), 8),
                                                      8 * 152);
#define NRLSH_R64(T_, C_)                                                                    \
    return launch("resolve_fp64", resolve_kernel<T_, C_>, dim3(grid), dim3(256), 0, st,       \
                  (const T_*)X, d, ldx, Lp, A_pad, tau64, list, count, cap, (C_*)codes);
    if (dt == NRLSH_BF16) {
        if (code_bytes == 4) NRLSH_R64(__nv_bfloat16, uint32_t)
        NRLSH_R64(__nv_bfloat16, uint64_t)
    }
    if (code_bytes == 4) NRLSH_R64(float, uint32_t)
    NRLSH_R64(float, uint64_t)
#undef NRLSH_R64
}

size_t ambiguity_capacity(int64_t rows, int L) {
    return (size_t)std::max<int64_t>(4096, rows * L / 64);
}

}  // namespace nrlsh
