// Internal declarations shared by the translation units of libnrlsh.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <utility>

#include "../../include/nrlsh.h"

namespace nrlsh {

// ------------------------------------------------------------------ status

// Sets the thread-local message returned by nrlsh_last_error().
void set_error(const std::string& msg);
nrlsh_status cuda_status(cudaError_t e, const char* what);

#define NRLSH_CK(expr)                                                        \
    do {                                                                      \
        cudaError_t e_ = (expr);                                              \
        if (e_ != cudaSuccess) return ::nrlsh::cuda_status(e_, #expr);        \
    } while (0)

#define NRLSH_CKS(expr)                                                       \
    do {                                                                      \
        nrlsh_status s_ = (expr);                                             \
        if (s_ != NRLSH_OK) return s_;                                        \
    } while (0)

// ------------------------------------------------------- launch accounting

// Every kernel goes through launch(): it counts the launch and, when
// profiling is on, brackets it with CUDA events on its stream.  Kernels are
// launched as programmatic dependents of their predecessor on the stream: a
// kernel may be scheduled while the previous one drains, and waits at its
// entry (NRLSH_PDL_ENTRY) until that grid has completed and its writes are
// visible, so the launch latency between dependent kernels is hidden.
void prof_begin(const char* name, cudaStream_t s);
void prof_end(const char* name, cudaStream_t s);
void count_launch();
bool pdl_enabled();

// First statement of every kernel: wait for the predecessor grid (a no-op when
// launched without the attribute), then let the successor be scheduled.
#define NRLSH_PDL_ENTRY() \
    asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory")

template <typename... KArgs, typename... Args>
inline cudaError_t launch(const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                          size_t smem, cudaStream_t s, Args&&... args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
    count_launch();
    prof_begin(name, s);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e == cudaSuccess) e = cudaGetLastError();
    prof_end(name, s);
    return e;
}

// ------------------------------------------------------------ small helpers

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Sub-dataset j holds ranks (and storage positions) [seg_start(j), seg_start(j+1)),
// seg_start(j) = floor(j n / m)  (Algorithm 1, percentile ranges).
__host__ __device__ inline int64_t seg_start(int64_t j, int64_t n, int64_t m) {
    return (j * n) / m;
}
// The j with seg_start(j) <= r < seg_start(j+1): the largest j with j n < (r+1) m.
__host__ __device__ inline int32_t seg_of(int64_t r, int64_t n, int64_t m) {
    return (int32_t)(((r + 1) * m + n - 1) / n - 1);
}

template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// Code words: L <= 32 bits in uint32, otherwise uint64.
__device__ __forceinline__ int popc_word(uint32_t v) { return __popc(v); }
__device__ __forceinline__ int popc_word(uint64_t v) { return __popcll(v); }

// Histogram tile: a run of storage positions inside one sub-dataset.
struct PosTile {
    int64_t start;
    int32_t len;
    int32_t seg;
};

// ----------------------------------------------------------- build launchers

// Up to eight arrays of 4-byte words to clear with one launch.
struct ZeroList {
    void* p[8];
    size_t words[8];
    int k = 0;
    void add(void* ptr, size_t w) {
        p[k] = ptr;
        words[k] = w;
        ++k;
    }
};
cudaError_t launch_zero(const ZeroList& z, cudaStream_t st);
// All return cudaError_t of the last launch; pointers are device pointers.

// A ((d+1) x L), its zero-padded copy A_pad ((d+1) x Lp) and column-norm bounds anorm.
cudaError_t launch_projections(float* A, float* A_pad, float* anorm, __nv_bfloat16* At, int dp,
                               int d, int L, int Lp, uint64_t seed, cudaStream_t s);
// s_x = ||x||^2 rounded once to FP64; with keys/vals non-null also the partition's
// sort keys and ids.  *fallbacks counts rows summed by the exact slow path.
cudaError_t launch_sqnorm(const void* X, nrlsh_dtype dt, int64_t n, int d, int64_t ld, double* s,
                          uint64_t* keys, uint32_t* vals, unsigned* fallbacks, cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs by the low `key_bits` bits of the key.
// Buffers alternate; returns through *result_in_alt whether the result is in the alt pair.
size_t radix_sort_temp_bytes(int64_t n);
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int key_bits, void* temp, bool* result_in_alt,
                           cudaStream_t s);
cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int key_bits, void* temp, bool* result_in_alt,
                           cudaStream_t s);
// Percentile partition for small inputs (n <= 65,536 and m ceil(n/32) <= 4M):
// ranks the (keys, ids) pairs (sorting them by tiles in place), then writes perm
// (storage order), sub_of_id and U2.  temp: small_rank_temp_bytes(n, m), zeroed
// by the caller.
bool small_rank_supported(int64_t n, int m);
size_t small_rank_temp_bytes(int64_t n, int m);
cudaError_t launch_small_rank(uint64_t* keys, uint32_t* ids, int64_t n, int m,
                              void* temp, uint32_t* perm, uint32_t* sub_of_id, double* U2,
                              cudaStream_t st);
cudaError_t launch_segment_assign(const uint64_t* sorted_keys, const uint32_t* sorted_ids,
                                  int64_t n, int m, uint32_t* sub_of_id, double* U2,
                                  uint32_t* jkeys, uint32_t* jvals, cudaStream_t st);
// Uniform norm ranges (Section 5, Figure 3a): sub-dataset of every id, the
// sort keys/values into storage order, sizes cnt[j] and U_j^2 (U2 zeroed by the
// caller).  range: 6 words of scratch.
cudaError_t launch_uniform_assign(const double* s_id, int64_t n, int m, unsigned long long* range,
                                  uint32_t* sub_of_id, double* U2, uint32_t* jkeys,
                                  uint32_t* jvals, uint32_t* cnt, cudaStream_t st);
// Segment offsets seg[0..m] and histogram tiles from the sub-dataset sizes
// (cnt, or with cnt null the percentile sizes of n items in m ranges).
cudaError_t launch_segments(const uint32_t* cnt, int64_t n, int m, int64_t tile, int64_t* seg,
                            PosTile* tiles, int ntiles_max, cudaStream_t st);
// Code decisions fused into the gather (vsum null: none).  vsum holds the FP32
// sums a_b^T x of every item in id order (n x Lr floats, Lr = Lp rounded up to 32,
// at most 64); At32 is A^T (Lr x dpa); undecided bits are counted in amb_count.
struct GatherCodes {
    const float* vsum = nullptr;
    int Lr = 0, d = 0, L = 0, Lp = 0, dpa = 0, code_bytes = 4;
    const float* A_pad = nullptr;
    const float* At32 = nullptr;
    const float* anorm = nullptr;
    void* codes = nullptr;
    unsigned* amb_count = nullptr;
    float kappa = 0.0f;
};
cudaError_t launch_gather_items(const void* X, nrlsh_dtype dt, int64_t ld, int d, int dp,
                                const uint32_t* perm, int64_t n, const uint32_t* sub_of_id,
                                const double* s_id, const double* U2, void* Xp,
                                __nv_bfloat16* Xb, __nv_bfloat16* Xb2, double* s_pos,
                                double* tau64, float* tau32, float* xnorm, const GatherCodes& gc,
                                cudaStream_t st);
// Sign random projection of rows of X (row stride ldx, stored dtype) with the FP32
// fast tier; undecided (row, bit) pairs go through amb_list (capacity amb_cap,
// count in *amb_count, which must start at 0) to the FP64 resolve kernel.
// Items pass tau (tau64 != null); queries pass tau64 = tau32 = null.
// At32 (may be null): A^T as written by launch_transpose_a, copied straight into
// shared memory by the warp-per-row kernel.
cudaError_t launch_project_fp32(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx,
                                int L, int Lp, const float* A_pad, const float* anorm,
                                const double* tau64, const float* tau32, const float* xnorm,
                                void* codes, int code_bytes, unsigned long long* amb_list,
                                unsigned* amb_count, unsigned amb_cap, const float* At32,
                                cudaStream_t st);
// The item projection in two parts (where the warp-per-row projection applies):
// the FP32 sums a_b^T x of every item in id order (vsum: n x Lr floats, Lr = Lp
// rounded up to 32), which need no partition and run beside it; the signs are
// taken in the gather once tau is known (GatherCodes).
bool split_projection_supported(int d, int Lp);
cudaError_t launch_project_dots(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx, int Lp,
                                const float* At32, float* vsum, cudaStream_t st);
// A^T for the warp-per-row projection (warp_proj_at_floats(d, Lp) floats; no-op
// when that projection does not apply).
int warp_proj_stride(int d, int Lp);
size_t warp_proj_at_floats(int d, int Lp);
cudaError_t launch_transpose_a(const float* A_pad, int d, int L, int Lp, float* At32,
                               cudaStream_t st);
// Query codes (P(q) = [q; 0]) and the queries' fp32 norm bounds (qnorm, written
// here) in one pass where the warp-per-row projection applies.  amb_count need
// not be zeroed by the caller.
cudaError_t launch_hash_queries(const float* Q, int64_t nq, int d, int L, int Lp,
                                const float* A_pad, const float* anorm, float* qnorm, void* codes,
                                int code_bytes, unsigned long long* amb_list, unsigned* amb_count,
                                unsigned amb_cap, const float* At32, cudaStream_t st);
// Entries of the ambiguity list to reserve for `rows` rows of L bits.
size_t ambiguity_capacity(int64_t rows, int L);
// FP32 tier (fp32 items after the bf16 tensor-core pass) and FP64 tier on a list
// of undecided (row, bit) pairs; decided bits are OR-ed into the codes.
cudaError_t launch_resolve_fp32(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx, int L,
                                int Lp,
                                const float* A_pad, const float* anorm, const float* xnorm,
                                const float* tau32, const double* tau64,
                                const unsigned long long* list, const unsigned* count,
                                unsigned cap, void* codes, int code_bytes,
                                unsigned long long* list2, unsigned* count2, unsigned cap2,
                                cudaStream_t st);
// The tensor-core pass's open bits in one launch (compensated FP32, FP64, canonical
// tiers, a warp per listed pair); needs the fp32 A^T copy (At32, warp_proj_stride
// layout): cudaErrorNotSupported without it.
cudaError_t launch_resolve_tiers(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx, int L,
                                 int Lp, const float* At32, const float* A_pad, const float* anorm,
                                 const float* xnorm, const double* tau64,
                                 const unsigned long long* list, const unsigned* count,
                                 unsigned cap, void* codes, int code_bytes, cudaStream_t st);
cudaError_t launch_resolve_fp64(const void* X, nrlsh_dtype dt, int64_t n, int d, int ldx, int L,
                                int Lp, const float* A_pad, const double* tau64,
                                const unsigned long long* list, const unsigned* count,
                                unsigned cap, void* codes, int code_bytes, cudaStream_t st);
// tcgen05 projection of the items (bf16 copy Xb, n x dp; At = A^T bf16, 64 x dp).
bool project_tc_supported(int d, int L);
cudaError_t launch_project_tc(const __nv_bfloat16* Xb, const __nv_bfloat16* Xb2, const void* X_exact,
                              int64_t n, int d, int dp, int L, int Lp, const __nv_bfloat16* At,
                              const float* A_pad, const float* anorm, const float* tau32,
                              const double* tau64, const float* xnorm, bool fp32_items,
                              void* codes, int code_bytes, unsigned long long* amb_list,
                              unsigned* amb_count, unsigned amb_cap, int* err, cudaStream_t st,
                              uint32_t spin_first = 1u << 22);
// c_l = cos(pi (1 - eps)(L - l) / L), correctly rounded, l = 0..L.
cudaError_t launch_class_cos(int L, float eps, double* cl, cudaStream_t st);
// The sorted (U_j, l) structure: probing order of the m (L+1) buckets.
// temp: bucket_order_temp_bytes(m, L) bytes of scratch.
size_t bucket_order_temp_bytes(int m, int L);
cudaError_t launch_bucket_order(const double* U2, const double* cl, int m, int L,
                                double* shat_sorted, uint32_t* order, void* temp,
                                cudaStream_t st);

// ----------------------------------------------------------- query launchers

cudaError_t launch_row_norm_bound(const float* Q, int64_t nq, int d, float* qnorm,
                                  cudaStream_t st);
// queries_per_block: 32, 64 or 128 (the autotuned tile).  exclusive: every
// sub-dataset is exactly one tile, so H is stored whole and need not be cleared;
// otherwise H must start at zero.
cudaError_t launch_hist(const void* codes, const void* qcodes, int code_bytes, int64_t nq, int m,
                        int L, const PosTile* tiles, int ntiles, uint32_t* H, cudaStream_t st,
                        int queries_per_block = 64, bool exclusive = false);
struct Boundary {
    int32_t j;       // boundary bucket (j*, l*)
    int32_t l;
    int32_t r;       // items taken from the boundary bucket
    int32_t full;    // items in buckets probed whole
};
cudaError_t launch_threshold(const uint32_t* H, const uint32_t* order, int m, int L, int64_t nq,
                             int64_t n, int64_t budget, const int64_t* budgets, uint32_t flags,
                             uint8_t* lam, Boundary* bnd, cudaStream_t st);
cudaError_t launch_select(const void* codes, const void* qcodes, int code_bytes, const int64_t* seg, int m,
                          int L, int64_t nq, const uint8_t* lam, const Boundary* bnd,
                          uint32_t* cand, int64_t cap, cudaStream_t st);
cudaError_t launch_rerank_fp32(const void* Xp, nrlsh_dtype dt, int dp, int d, const float* Q,
                               int64_t nq, const uint32_t* cand, int64_t cap, const Boundary* bnd,
                               const float* xnorm, const float* qnorm, float* lo, float* hi,
                               cudaStream_t st);
cudaError_t launch_topk(const float* lo, const float* hi, const uint32_t* cand, int64_t cap,
                        const Boundary* bnd, int64_t nq, int k, const int32_t* ks,
                        const void* Xp, nrlsh_dtype dt, int dp, int d, const float* Q,
                        const float* xnorm, const float* qnorm, const uint32_t* perm,
                        uint32_t* cont, double* cont_s, int64_t* out_ids, float* out_scores,
                        int out_ld, cudaStream_t st, const int* skip = nullptr,
                        int* report = nullptr);
// Threshold walk, candidate selection, FP32 re-rank and exact top-k, one block
// per query (the main query path after the histograms).
cudaError_t launch_probe_rerank(const uint32_t* H, const uint32_t* order, int m, int L, int64_t n,
                                const int64_t* seg, int64_t nq, int64_t budget, const int64_t* budgets, uint32_t flags,
                                const void* codes, const void* qcodes, int code_bytes,
                                const void* Xp, nrlsh_dtype dt, int dp, int d, const float* Q,
                                const float* xnorm, const float* qnorm, const uint32_t* perm, int k,
                                const int32_t* ks, uint32_t* cand, float* lo, float* hi,
                                uint32_t* cont, double* cont_s, int64_t cap, int64_t* out_ids,
                                float* out_scores, int out_ld, cudaStream_t st);
// Persistent form: `ctas` CTAs pull queries from *work (zeroed by the caller).
// budgets/ks may be null: then every query uses budget / k_max.  ctas <= 0: as many
// CTAs as fit on the device at once.  slabs: ctas x 6 cap words.  Xr16 (fp32 items
// only, may be null): a bf16 copy of the stored rows for the gathered re-rank.
cudaError_t launch_probe_rerank_persistent(const uint32_t* H, const uint32_t* order, int m, int L,
                                           int64_t n, const int64_t* seg, int64_t budget,
                                           const int64_t* budgets, const void* codes,
                                           const void* qcodes, int code_bytes, const void* Xp,
                                           nrlsh_dtype dt, int dp, int d, const float* Q,
                                           const float* xnorm, const float* qnorm,
                                           const uint32_t* perm, const int32_t* ks, int k_max,
                                           uint32_t* slabs, int64_t cap, int ctas, unsigned* work,
                                           int64_t nq, int64_t* out_ids, float* out_scores,
                                           cudaStream_t st, const __nv_bfloat16* Xr16 = nullptr);
// Interval factor of the gathered re-rank over a bf16 copy of fp32 rows.
float rerank_bf16_rows_bound(int d);
// Multi-table single probe (Algorithm 2): L bits as `tables` tables of L / tables
// bits; block per query selects C(q), re-ranks and takes the exact top-k of its
// first min(|C(q)|, cap) items.  probed (may be null) receives |C(q)|; with
// cand_ids non-null only the candidate ids are written instead.
cudaError_t launch_multitable(const void* codes, const void* qcodes, int code_bytes, int64_t n,
                              int L, int tables, const void* Xp, nrlsh_dtype dt, int dp, int d,
                              const float* Q, const float* xnorm, const float* qnorm,
                              const uint32_t* perm, int k, uint32_t* cand, float* lo, float* hi,
                              uint32_t* cont, double* cont_s, int64_t cap, int64_t nq,
                              int64_t* out_ids, float* out_scores, int out_ld, int64_t* probed,
                              int32_t* cand_ids, int64_t cand_ld, cudaStream_t st);
// The same selection alone (bnd[q].full = min(|C(q)|, cap)), and a persistent
// FP32 re-rank whose blocks take 256-candidate chunks of any query from a work
// list (work_off: nq + 1 int64 scratch, work_ctr: one word), for lists too
// long or too uneven for a block per query.
cudaError_t launch_multitable_select(const void* codes, const void* qcodes, int code_bytes,
                                     int64_t n, int L, int tables, uint32_t* cand, int64_t cap,
                                     int64_t nq, Boundary* bnd, int64_t* probed, cudaStream_t st);
cudaError_t launch_rerank_work(const void* Xp, nrlsh_dtype dt, int dp, int d, const float* Q,
                               int64_t nq, const uint32_t* cand, int64_t cap, const Boundary* bnd,
                               int64_t* work_off, unsigned long long* work_ctr, const float* xnorm,
                               const float* qnorm, float* lo, float* hi, cudaStream_t st);
// CTAs of the persistent re-rank kernel resident at once (at most nq).
int probe_rerank_ctas(nrlsh_dtype dt, int code_bytes, int dp, int m, int64_t nq);
// ---------------------------------------------- tensor-core query path

// Boundary bucket of a query for the tensor-core re-rank: (j*, l*) and the
// storage position of the last item taken from it (-1: none).
struct TcBoundary {
    int32_t j;
    int32_t l;
    int64_t pcut;
};
// sm_100-family device, and the operands of rows of d values fit shared memory.
bool tc_query_supported(int d, int L);
// 64-element K chunks of a row of d values.
int tc_query_k_chunks(int d);
// qce[q] = a_q with |score_tc - score_fp64| <= a_q ||x|| for the bf16 tensor-core
// scores of query q (qnorm: the queries' norm bounds).
cudaError_t launch_query_bounds(const float* Q, int64_t nq, int d, const float* qnorm,
                                bool fp32_items, float* qce, cudaStream_t st);
// Qb (nq x 64 tc_query_k_chunks(d) bf16) and Qs (nq x 64 bf16 +-1 signs of the codes).
// Also clears the call's error word *err (the tensor-path kernels' timeouts) and
// the histogram kernel's work counter *hist_ctr.
cudaError_t launch_prep_queries(const float* Q, int64_t nq, int d, int Kq, const void* qcodes,
                                int code_bytes, int L, __nv_bfloat16* Qb, __nv_bfloat16* Qs,
                                int* err, uint32_t* hist_ctr, cudaStream_t st);
// *report = *err when *report is still 0 and *err is not.
cudaError_t launch_report_err(const int* err, int* report, cudaStream_t st);
// Xs (n x 64 bf16): the +-1 signs of the item codes, storage order.
cudaError_t launch_item_signs(const void* codes, int code_bytes, int64_t n, int L,
                              __nv_bfloat16* Xs, cudaStream_t st);
cudaError_t launch_to_bf16(const float* X, int64_t count, __nv_bfloat16* Xb, cudaStream_t st);
// The dense (query tile x item tile) tcgen05 kernel over the sub-datasets:
// rerank = false: the Hamming histograms H (every entry written; list may be null
// for all work items); rerank = true: the candidates of the work items in list
// (nlist entries, on the device) with their score intervals.
cudaError_t launch_pairs_tc(bool rerank, const __nv_bfloat16* Qb, const __nv_bfloat16* Qs,
                            int64_t nq, const __nv_bfloat16* Xb, const __nv_bfloat16* Xs,
                            int64_t n, int d, int dp, int m, int L, const int64_t* seg,
                            const uint32_t* list, const uint32_t* nlist, uint32_t* H,
                            const uint8_t* lam, const uint32_t* off, const TcBoundary* tb,
                            const float* xnorm, const float* qce, uint32_t* cand,
                            float* lo, float* hi, int64_t cap, int* err, uint32_t* work_ctr,
                            cudaStream_t st, uint32_t spin_first = 1u << 22);
// Bucket walk of every query (budgets per query or one budget, clamped to [1, cap]),
// then per sub-dataset the probed counts as list offsets off (nq x (m + 1)), the
// boundary cut (tb), bnd[q].full = min(B, n) (r = 0) for the top-k pass, and
// work_flag[j * nqt + q / 128] = 1 where query q probes S_j (flags zeroed first).
// With *err set (the histograms are incomplete) nothing is probed.
cudaError_t launch_tc_walk(const uint32_t* H, const uint32_t* order, int m, int L, int64_t n,
                           const int64_t* seg, int64_t nq, int64_t budget, const int64_t* budgets,
                           int64_t cap, uint32_t flags, const void* codes, const void* qcodes,
                           int code_bytes, uint8_t* lam, uint32_t* off, TcBoundary* tb,
                           Boundary* bnd, uint8_t* work_flag, int nqt, const int* err,
                           cudaStream_t st);
// Indices of the nonzero flags, ascending (list), their number (count[0]), and
// count[1] = 0 (the work counter of the kernel that consumes the list).
cudaError_t launch_work_list(const uint8_t* flag, int nflag, uint32_t* list, uint32_t* count,
                             cudaStream_t st);

// skip / report (may be null): as for launch_topk.
cudaError_t launch_cand_to_ids(const uint32_t* cand, int64_t cap, const Boundary* bnd,
                               const uint32_t* perm, int64_t nq, int32_t* out, int64_t out_cap,
                               int64_t* count, cudaStream_t st, const int* skip = nullptr,
                               int* report = nullptr);

}  // namespace nrlsh
