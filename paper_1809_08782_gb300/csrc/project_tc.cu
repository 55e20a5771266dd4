// Sign random projection of the items on 5th-generation tensor cores
// (Eq. 4 applied to the SIMPLE-LSH transform of Eq. 8): V = X~ A with X~ the
// bfloat16 items (n x d, row stride dp) and A the bfloat16-valued projections,
// accumulated in FP32 in tensor memory, then + a_d tau and the sign.
//
// Persistent warp-specialised CTAs (320 threads, two per SM when there are more
// tiles than SMs):
//   warp 0   one thread issues TMA loads: all of A^T once (K-major, 128-byte
//            swizzle), then a ring of stages, each a 128-item x 64-K tile of X~
//            (fp32 items: two tiles, the bf16 high and low parts of x);
//   warp 1   allocates 128 TMEM columns (two accumulators of up to 64 columns)
//            and one thread issues tcgen05.mma (M = 128, N = 16..64, K = 16);
//   warps 2-9 read the accumulator rows (warp w reads TMEM lanes 32 (w % 4)..;
//            warps 2-5 columns 0-31, warps 6-9 columns 32-63), add the tail
//            term, decide each bit against a proven bound and write their half
//            of the code word; undecided (item, bit) pairs go to a list that
//            the FP32 and FP64 tiers resolve.
// Every mbarrier wait is bounded; on a timeout the kernel records an error in
// *err, stops issuing work, waits (bounded) for its own copies, frees TMEM and
// returns.
#include "nrlsh_internal.cuh"
#include "tc_ops.cuh"

#include <mutex>

namespace nrlsh {

using namespace tc;

namespace {

constexpr int kTcM = 128;            // items per tile (MMA M)
constexpr int kTcKC = 64;            // K elements per stage: 128 bytes of bf16
constexpr int kTcMaxStages = 8;
constexpr int kAmbWarp = 64;         // undecided (item, bit) entries buffered per epilogue warp

__device__ __forceinline__ void set_code_bit(uint32_t* w, int bit) { atomicOr(w, 1u << bit); }
__device__ __forceinline__ void set_code_bit(uint64_t* w, int bit) {
    atomicOr((unsigned long long*)w, 1ull << bit);
}  // ring stages (each one or, for split fp32 items, two 16 KB tiles)
constexpr int kTcThreads = 320;
constexpr int kEpiWarps = 8;         // two per TMEM lane quadrant, one per 32-column half
constexpr uint32_t kTmemCols = 128;  // two accumulators of up to 64 fp32 columns
constexpr uint32_t kXStageBytes = kTcM * kTcKC * 2;


struct TcSmem {
    int nkc, N, split, stages;
    __device__ uint8_t* a_tile(uint8_t* base, int c) const { return base + (size_t)c * N * 128; }
    __device__ uint8_t* x_stage(uint8_t* base, int s, int part) const {
        return base + (size_t)nkc * N * 128 + ((size_t)s * split + part) * kXStageBytes;
    }
    __device__ uint64_t* bars(uint8_t* base) const {
        return (uint64_t*)(base + (size_t)nkc * N * 128 + (size_t)stages * split * kXStageBytes);
    }
};

template <typename C>
__global__ void __launch_bounds__(kTcThreads, 2)
    project_tc_kernel(const __grid_constant__ CUtensorMap map_x,
                      const __grid_constant__ CUtensorMap map_x2,
                      const __grid_constant__ CUtensorMap map_a, int split, int64_t n, int nkc, int L,
                      int N,
                      int Lp, int d, const float* __restrict__ A_pad,
                      const float* __restrict__ anorm, const float* __restrict__ tau32,
                      const float* __restrict__ xnorm, float kappa_tc, float round_x,
                      const void* __restrict__ X_exact, int fp32_items, int ldx,
                      const double* __restrict__ tau64, C* __restrict__ codes,
                      unsigned long long* __restrict__ amb_list, unsigned* amb_count,
                      unsigned amb_cap, int* err, uint32_t spin_first, int kTcStages) {
    NRLSH_PDL_ENTRY();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const TcSmem L_{nkc, N, split, kTcStages};
    const uint32_t stage_bytes = (uint32_t)split * kXStageBytes;
    uint64_t* bars = L_.bars(base);
    uint64_t* full = bars;                       // kTcStages
    uint64_t* empty = bars + kTcStages;          // kTcStages
    uint64_t* acc_full = bars + 2 * kTcStages;   // 2
    uint64_t* acc_empty = acc_full + 2;          // 2
    uint64_t* a_bar = acc_empty + 2;             // 1
    uint64_t* drain = a_bar + 1;                 // 1: all MMAs of this CTA done
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_s = (volatile int*)(tmem_slot + 1);
    float* s_c1 = (float*)(tmem_slot + 4);       // 64: (kappa_tc + round_x) ||a_b||
    float* s_c2 = s_c1 + 64;                     // 64: 2^-20 |a_{d,b}|
    float* s_ad = s_c2 + 64;                     // 64: a_{d,b}
    unsigned long long* amb_s = (unsigned long long*)(s_ad + 64);   // kEpiWarps x kAmbWarp entries

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = ceil_div(n, kTcM);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 32 * kEpiWarps);
        }
        mbar_init(a_bar, 1);
        mbar_init(drain, 1);
        *abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x < 64) {
        const int b = threadIdx.x;
        const float ad = b < L ? A_pad[(int64_t)d * Lp + b] : 0.0f;
        s_ad[b] = ad;
        s_c1[b] = b < L ? (kappa_tc + round_x) * anorm[b] : 0.0f;
        s_c2[b] = 0x1p-20f * fabsf(ad);
    }
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer
            mbar_expect_tx(a_bar, (uint32_t)(nkc * N * 128));
            for (int c = 0; c < nkc; ++c) tma_load_2d(L_.a_tile(base, c), &map_a, a_bar, c * kTcKC, 0);
            int stage = 0;
            uint32_t phase = 0;
            int issued[kTcMaxStages] = {0, 0, 0, 0, 0, 0, 0, 0};
            uint32_t issued_par[kTcMaxStages] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int64_t t = blockIdx.x; t < ntiles && !*abort_s; t += gridDim.x) {
                for (int c = 0; c < nkc; ++c) {
                    if (!mbar_wait(&empty[stage], phase ^ 1)) {
                        atomicExch(err, 1);
                        *abort_s = 1;
                        break;
                    }
                    mbar_expect_tx(&full[stage], stage_bytes);
                    tma_load_2d(L_.x_stage(base, stage, 0), &map_x, &full[stage], c * kTcKC,
                                (int)(t * kTcM));
                    if (split == 2)
                        tma_load_2d(L_.x_stage(base, stage, 1), &map_x2, &full[stage], c * kTcKC,
                                    (int)(t * kTcM));
                    issued[stage] = 1;
                    issued_par[stage] = phase;
                    if (++stage == kTcStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            if (*abort_s) {
                // let every copy in flight land before the CTA's memory goes away
                mbar_wait(a_bar, 0);
                for (int s = 0; s < kTcStages; ++s)
                    if (issued[s]) mbar_wait(&full[s], issued_par[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t idesc = umma_idesc(kTcM, N);
            bool ok = mbar_wait(a_bar, 0);
            int stage = 0;
            uint32_t phase = 0, acc_phase = 0;
            int buf = 0;
            bool first = true;  // the first wait for a stage takes spin_first polls at most
            for (int64_t t = blockIdx.x; ok && t < ntiles && !*abort_s; t += gridDim.x) {
                if (!mbar_wait(&acc_empty[buf], acc_phase ^ 1)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)buf * 64;
                for (int c = 0; c < nkc; ++c) {
                    const uint32_t lim = first ? spin_first : kSpinLimit;
                    first = false;
                    if (!mbar_wait(&full[stage], phase, lim)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint64_t bdesc = sw128_desc(L_.a_tile(base, c));
                    for (int part = 0; part < split; ++part) {
                        const uint64_t adesc = sw128_desc(L_.x_stage(base, stage, part));
#pragma unroll
                        for (int k = 0; k < kTcKC / 16; ++k)  // 32 bytes of K per MMA
                            umma_bf16(d_tmem, adesc + 2 * k, bdesc + 2 * k, idesc,
                                      (c | k | part) != 0);
                    }
                    umma_commit(&empty[stage]);
                    if (++stage == kTcStages) {
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
            if (!ok) {
                atomicExch(err, 2);
                *abort_s = 1;
            }
            // every MMA this thread issued has finished before TMEM is freed
            umma_commit(drain);
            mbar_wait(drain, 0);
        }
    } else {
        // ---- epilogue: warps 2..9, TMEM lanes 32 (warp % 4) + lane; warps 2..5 take
        // bits 0..31 of their rows, warps 6..9 bits 32..63
        const int sub = warp & 3;
        const int half = (warp - 2) >> 2;
        const bool has_bits = 32 * half < L;   // warp-uniform
        int buf = 0;
        uint32_t acc_phase = 0;
        // the row's norm bound and tau of the next tile are loaded while this
        // tile's accumulator is awaited
        auto row_of = [&](int64_t t) { return t * kTcM + 32 * sub + lane; };
        // the canonical FP64 form of one (row, bit), for entries the list has no room for
        auto canonical = [&](int64_t r, int bit) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k) {
                const double xk = fp32_items ? (double)((const float*)X_exact)[r * ldx + k]
                                             : (double)__bfloat162float(
                                                   ((const __nv_bfloat16*)X_exact)[r * ldx + k]);
                acc = fma(xk, (double)A_pad[(int64_t)k * Lp + bit], acc);
            }
            acc = __dadd_rn(acc, __dmul_rn((double)s_ad[bit], tau64[r]));
            return acc >= 0.0;
        };
        unsigned long long* wbuf = amb_s + (warp - 2) * kAmbWarp;
        uint32_t* codes32 = (uint32_t*)codes;
        unsigned wn = 0;   // entries in this warp's buffer (uniform in the warp)
        auto flush = [&]() {
            __syncwarp();
            if (wn == 0) return;
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(amb_count, wn);
            base = __shfl_sync(0xffffffffu, base, 0);
            for (unsigned i = lane; i < wn; i += 32) {
                const unsigned long long e = wbuf[i];
                if (base + i < amb_cap) {
                    amb_list[base + i] = e;
                } else {
                    const int64_t r = (int64_t)(e >> 6);
                    const int bit = (int)(e & 63);
                    if (canonical(r, bit)) set_code_bit(codes + r, bit);
                }
            }
            wn = 0;
            __syncwarp();
        };
        float xn_next = 0.0f, t32_next = 0.0f;
        if ((int64_t)blockIdx.x < ntiles && row_of(blockIdx.x) < n) {
            xn_next = xnorm[row_of(blockIdx.x)];
            t32_next = tau32[row_of(blockIdx.x)];
        }
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const float xn = xn_next, t32 = t32_next;
            const int64_t tn = t + gridDim.x;
            if (tn < ntiles && row_of(tn) < n) {
                xn_next = xnorm[row_of(tn)];
                t32_next = tau32[row_of(tn)];
            }
            if (*abort_s || !mbar_wait(&acc_full[buf], acc_phase)) {
                atomicExch(err, 3);
                *abort_s = 1;
                break;
            }
            fence_after();
            const int64_t row = row_of(t);
            const bool valid = row < n;
            uint32_t word = 0, undecided = 0;   // bits 32 half + i of the row's code
            uint32_t r[32];
            if (has_bits) {
                const uint32_t taddr = tmem_base + ((uint32_t)(32 * sub) << 16) +
                                       (uint32_t)(buf * 64 + 32 * half);
                tmem_ld32_nowait(taddr, r);
                tmem_wait_ld();
            }
            // the accumulator is in registers: the MMA may overwrite it now
            fence_before();
            mbar_arrive(&acc_empty[buf]);
            if (has_bits) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int bit = 32 * half + i;
                    if (!valid || bit >= L) continue;
                    const float v = fmaf(s_ad[bit], t32, __uint_as_float(r[i]));
                    // accumulation bound (kappa_tc) plus, for fp32 items, the bf16
                    // rounding of x (round_x); Cauchy-Schwarz for sum |a_k x_k|
                    const float bound = fmaf(s_c1[bit], xn, s_c2[bit] * t32);
                    if (fabsf(v) * (1.0f - 0x1p-21f) > bound) {
                        if (v > 0.0f) word |= 1u << i;
                    } else {
                        undecided |= 1u << i;
                    }
                }
            }
            // undecided pairs go to this warp's buffer in shared memory, flushed to
            // the global list (one reservation per flush) when it would overflow;
            // a flush only touches rows of earlier tiles, already stored
            const unsigned cnt = (unsigned)__popc(undecided);
            unsigned incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
            if (tot > 0 && wn + tot > (unsigned)kAmbWarp) flush();
            if (tot <= (unsigned)kAmbWarp) {
                unsigned pos = wn + incl - cnt;
                while (undecided) {
                    const int i = __ffs(undecided) - 1;
                    undecided &= undecided - 1;
                    wbuf[pos++] = ((unsigned long long)row << 6) | (unsigned)(32 * half + i);
                }
                wn += tot;
            } else {
                // more than a buffer in one tile: straight to the global list
                unsigned wbase = 0;
                if (lane == 31) wbase = atomicAdd(amb_count, tot);
                wbase = __shfl_sync(0xffffffffu, wbase, 31);
                unsigned slot = wbase + incl - cnt;
                while (undecided) {
                    const int i = __ffs(undecided) - 1;
                    undecided &= undecided - 1;
                    const int bit = 32 * half + i;
                    if (slot < amb_cap)
                        amb_list[slot] = ((unsigned long long)row << 6) | (unsigned)bit;
                    else if (canonical(row, bit))
                        word |= 1u << i;
                    ++slot;
                }
            }
            // each half stores its own 32 bits of the code (one word for L <= 32)
            if (valid && has_bits) {
                if (sizeof(C) == 4)
                    codes32[row] = word;
                else
                    codes32[2 * row + half] = word;
            }
            if (++buf == 2) {
                buf = 0;
                acc_phase ^= 1;
            }
        }
        flush();
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

bool make_map_bf16(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer,
                   uint64_t stride_elems, uint32_t box_rows) {
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {stride_elems * 2};
    const cuuint32_t box[2] = {64u, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t project_tc_smem_bytes(int d, int N, int split, int stages) {
    const int nkc = (int)ceil_div(d, kTcKC);
    return 1024 + (size_t)nkc * N * 128 + (size_t)stages * split * kXStageBytes + 256 + 3 * 64 * 4 +
           kEpiWarps * kAmbWarp * 8;
}

// With more tiles than SMs, the deepest ring (at most kTcMaxStages) that keeps two
// CTAs on an SM (two epilogues per SM); else, or if none does, the deepest that fits
// one.  0 if not even two stages fit.
int project_tc_stages(int d, int N, int split, bool two_per_sm, int* per_sm) {
    for (int s = kTcMaxStages; two_per_sm && s >= 2; --s)
        if (2 * project_tc_smem_bytes(d, N, split, s) <= 227 * 1024) {
            *per_sm = 2;
            return s;
        }
    for (int s = kTcMaxStages; s >= 2; --s)
        if (project_tc_smem_bytes(d, N, split, s) <= 220 * 1024) {
            *per_sm = 1;
            return s;
        }
    return 0;
}

bool project_tc_supported(int d, int L) {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaGetLastError();
    if (major != 10) return false;
    const int N = L <= 16 ? 16 : L <= 32 ? 32 : L <= 48 ? 48 : 64;
    int per_sm = 0;
    return project_tc_stages(d, N, 2, false, &per_sm) > 0 && tensor_map_encoder() != nullptr;
}

cudaError_t launch_project_tc(const __nv_bfloat16* Xb, const __nv_bfloat16* Xb2, const void* X_exact,
                              int64_t n, int d, int dp, int L, int Lp, const __nv_bfloat16* At,
                              const float* A_pad, const float* anorm, const float* tau32,
                              const double* tau64, const float* xnorm, bool fp32_items,
                              void* codes, int code_bytes, unsigned long long* amb_list,
                              unsigned* amb_count, unsigned amb_cap, int* err, cudaStream_t st,
                              uint32_t spin_first) {
    const int N = L <= 16 ? 16 : L <= 32 ? 32 : L <= 48 ? 48 : 64;
    const int nkc = (int)ceil_div(d, kTcKC);
    const int split = Xb2 ? 2 : 1;
    CUtensorMap map_x, map_x2, map_a;
    if (!make_map_bf16(&map_x, Xb, (uint64_t)d, (uint64_t)n, (uint64_t)dp, kTcM) ||
        !make_map_bf16(&map_x2, Xb2 ? Xb2 : Xb, (uint64_t)d, (uint64_t)n, (uint64_t)dp, kTcM) ||
        !make_map_bf16(&map_a, At, (uint64_t)d, (uint64_t)N, (uint64_t)dp, (uint32_t)N))
        return cudaErrorNotSupported;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = ceil_div(n, kTcM);
    int per_sm = 1;
    const int stages = project_tc_stages(d, N, split, ntiles > sms, &per_sm);
    if (stages == 0) return cudaErrorNotSupported;
    const size_t smem = project_tc_smem_bytes(d, N, split, stages);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)per_sm * sms);
    // accumulation bound: 16x the first-order FP32 bound (the adder's rounding mode
    // inside the tensor core is not assumed).  fp32 items enter as x = hi + lo + r
    // with hi, lo bf16 and |r| <= 2^-16 |x| (one bf16 part: |r| <= 2^-8 |x|).
    const float kappa_tc = (float)(nkc * kTcKC * split + 8) * 0x1p-20f;
    const float round_x = !fp32_items ? 0.0f : (split == 2 ? 0x1p-16f : 0x1p-8f) * (1.0f + 0x1p-7f);
#define NRLSH_TC(C_)                                                                         \
    {                                                                                        \
        auto kern = project_tc_kernel<C_>;                                                   \
        cudaError_t e =                                                                      \
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                      \
        return launch("project_tc", kern, dim3(grid), dim3(kTcThreads), smem, st, map_x, map_x2, \
                      map_a, split, n, nkc, L, N, Lp, d, A_pad, anorm, tau32, xnorm, kappa_tc, \
                      round_x, X_exact, fp32_items ? 1 : 0, dp, tau64, (C_*)codes, amb_list,  \
                      amb_count, amb_cap, err, spin_first, stages);                          \
    }
    if (code_bytes == 4) NRLSH_TC(uint32_t)
    NRLSH_TC(uint64_t)
#undef NRLSH_TC
}

}  // namespace nrlsh
