/*
 * nrlsh.h - C ABI of the GB300 norm-ranging LSH library (libnrlsh.so).
 *
 * Norm-ranging LSH for maximum inner product search (Yan, Li, Dai, Chen, Cheng,
 * NeurIPS 2018).  Given items x_1..x_n in R^d and a query q, MIPS returns the
 * item(s) with the largest q^T x (Eq. 1).  The index partitions the items into m
 * sub-datasets by 2-norm percentile, normalises each by its own largest norm U_j,
 * applies the SIMPLE-LSH transform P(x) = [x/U_j; sqrt(1 - ||x/U_j||^2)]
 * (Algorithm 1, Eq. 8) and stores L-bit sign-random-projection codes (Eq. 4).
 * A query probes buckets (sub-dataset j, number of identical bits l) in
 * descending order of s_hat = U_j cos[pi (1 - eps)(1 - l/L)] (Eq. 12 and the
 * sorted (U_j, l) structure of Section 3.3) until the probe budget B is reached,
 * re-ranks the probed items by exact inner product and returns the top k.
 *
 * Determinism.  Every floating-point value that decides an integer result is
 * fixed by a rule, so results are a deterministic function of the inputs:
 *   - squared norms s_x: the exact sum of the x_k^2 rounded once to FP64;
 *   - ranking for the partition: (s_x, id) ascending; sub-dataset j holds ranks
 *     [floor(j n / m), floor((j+1) n / m)); U_j^2 = max s_x in S_j;
 *   - code bit b of x in S_j: [fl(sum_k a_{k,b} x_k + fl(a_{d,b} tau_x)) >= 0] in
 *     FP64 with the sum taken in order k = 0..d-1, tau_x = fl(sqrt(fl(U_j^2 - s_x)))
 *     (tau_x = 1 if U_j = 0); query bit b: [sum_k a_{k,b} q_k >= 0] likewise.
 *     Fast tiers compute the projection in FP32 (or BF16 on tensor cores) with a
 *     proven error bound and recompute the undecided (item, bit) pairs in FP64;
 *   - A: (d+1) x L entries, Philox4x64-10 (Salmon et al., SC'11) with counter
 *     (row, col, 0, 0) and key (seed, 0), Box-Muller, rounded to bfloat16;
 *   - bucket order: s_hat = fl(U_j * c_l) with c_l = cos(pi (1-eps)(L-l)/L)
 *     correctly rounded, descending; ties by larger l, then larger j;
 *   - candidates: the first min(B, n) items in (bucket order, item id) order;
 *   - scores: FP64 sum of q_k x_k in order k = 0..d-1; top-k by (score desc,
 *     id asc); the reported score is that FP64 value rounded to fp32.
 *
 * Memory and streams.  Unless stated otherwise pointers may be device pointers
 * (any CUDA allocation of the current device, e.g. from PyTorch) or host
 * pointers.  Host inputs are copied into device memory before the call returns
 * (a build, nrlsh_query_ex and nrlsh_query_batched wait for those copies only,
 * queued ahead of the wait for the build, and leave their work queued); a call
 * with a host output synchronises its stream before returning.  With device pointers
 * only, calls are asynchronous on `stream` (NULL = the legacy default stream);
 * a query call on another stream than the index's build makes its stream wait
 * for the end of the build (an event recorded by the build).  The caller
 * keeps ownership of every buffer it passes; the index owns a copy of the items
 * and everything it derives from them.  Query calls allocate their scratch
 * with the stream-ordered allocator and free it on the same stream.
 *
 * Errors.  Every entry point validates its arguments before launching any work
 * and returns a status; a thread-local message is available from
 * nrlsh_last_error().  A CUDA error (including a sticky error left by earlier
 * work) is reported as NRLSH_ERR_CUDA.  No entry point aborts the process.
 * Every wait of the tensor-core kernels is bounded: one that runs out makes
 * the kernel stop, let its own copies and MMAs land and return, and records an
 * error word in the index, which nrlsh_get_info (and, for the build,
 * nrlsh_get_codes) report as NRLSH_ERR_TIMEOUT.  Test hook: the environment
 * variable NRLSH_TEST_SPIN_FIRST, read at each call, sets how many polls the
 * first such wait of the MMA thread takes (normally 4,194,304; 0 makes it run
 * out at once).
 */
#ifndef NRLSH_H
#define NRLSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define NRLSH_API __attribute__((visibility("default")))
#else
#define NRLSH_API
#endif

typedef struct nrlsh_index nrlsh_index;

typedef enum nrlsh_status {
    NRLSH_OK = 0,
    NRLSH_ERR_ARG = -1,          /* an argument is out of range or a pointer is NULL */
    NRLSH_ERR_OOM = -2,          /* a device or host allocation failed */
    NRLSH_ERR_CUDA = -3,         /* a CUDA call failed */
    NRLSH_ERR_TIMEOUT = -4,      /* a bounded device wait ran out */
    NRLSH_ERR_UNSUPPORTED = -5   /* valid request this library or device does not support */
} nrlsh_status;

typedef enum nrlsh_dtype {
    NRLSH_F32 = 0,               /* items are float32, row-major n x d */
    NRLSH_BF16 = 1               /* items are bfloat16, row-major n x d */
} nrlsh_dtype;

/* Query flags. */
#define NRLSH_WHOLE_BUCKETS 0x1u /* probe the boundary bucket whole (|C| may exceed B) */

/* Limits checked by the entry points. */
#define NRLSH_MAX_L 64
#define NRLSH_MAX_BUCKETS 16384  /* m * (L + 1) */
#define NRLSH_MAX_K 1024

/* How the item projections (Eq. 4 on the Eq. 8 transform) are computed. */
typedef enum nrlsh_projection {
    NRLSH_PROJECT_AUTO = 0,      /* tensor cores where the device has them, else CUDA cores */
    NRLSH_PROJECT_SIMT = 1,      /* FP32 on CUDA cores, undecided bits in FP64 */
    NRLSH_PROJECT_TENSOR = 2     /* bf16 tcgen05 MMA with FP32 accumulation, undecided bits
                                    in FP32 (fp32 items) and then FP64 */
} nrlsh_projection;

/* How the items are split into the m sub-datasets. */
typedef enum nrlsh_partition {
    NRLSH_PARTITION_PERCENTILE = 0, /* Algorithm 1: rank by (||x||^2, id); S_j holds ranks
                                       [floor(j n / m), floor((j + 1) n / m)) */
    NRLSH_PARTITION_UNIFORM = 1     /* Section 5 (Figure 3a): the norm domain [nu_min, nu_max]
                                       cut into m equal ranges, nu = sqrt(||x||^2),
                                       j = min(m - 1, floor(((nu - nu_min) / w) * m)),
                                       w = nu_max - nu_min, each operation rounded to
                                       nearest in FP64 (all j = 0 when w = 0); sub-datasets
                                       may be empty (U_j = 0) */
} nrlsh_partition;

typedef struct nrlsh_build_options {
    int32_t dtype;               /* nrlsh_dtype of the items */
    float eps;                   /* 0 < eps < 1 */
    int32_t projection;          /* nrlsh_projection */
    int32_t partition;           /* nrlsh_partition (0 = percentile) */
    void* stream;                /* cudaStream_t; NULL = legacy default stream */
    uint32_t flags;              /* NRLSH_BUILD_* (0 = none) */
} nrlsh_build_options;

/* Build flag: host items are read by the build's stream in order, and the call
 * returns without waiting for their copy.  The caller keeps the buffer unchanged
 * until the stream has passed the build (an event recorded after the call). */
#define NRLSH_BUILD_ASYNC_INPUT 0x1u

typedef struct nrlsh_info {
    int64_t n;
    int32_t d;
    int32_t m;
    int32_t L;
    int32_t dtype;               /* nrlsh_dtype */
    float eps;
    uint64_t seed;
    int32_t code_bytes;          /* 4 for L <= 32, 8 otherwise */
    int32_t row_stride;          /* elements per stored item row (d rounded up to 8) */
    int64_t device_bytes;        /* device memory owned by the index */
    int64_t ambiguous_bits;      /* (item, bit) pairs the first tier left undecided */
    int32_t projection;          /* nrlsh_projection used (SIMT or TENSOR) */
    int32_t device_error;        /* nonzero: a bounded device wait ran out during the build */
    int32_t partition;           /* nrlsh_partition used */
    int32_t norm_fallbacks;      /* rows whose squared norm needed the exact slow path */
    int32_t query_error;         /* nonzero: a tensor-core query kernel's bounded wait ran
                                    out, or it found other candidates than it counted */
} nrlsh_info;

/*
 * Index building (Algorithm 1).
 *   items   n x d row-major fp32 (nrlsh_build) or `dtype` (nrlsh_build_ex)
 *   n >= 1, d >= 1, 1 <= m <= n, 1 <= L <= 64, m * (L + 1) <= NRLSH_MAX_BUCKETS,
 *   0 < eps < 1 (nrlsh_build uses eps = 0.1), seed selects A.
 * On success *out receives a new index, released with nrlsh_free().  The items
 * are copied; the caller may free them once the call (and, for device items,
 * the work it queued on `stream`) has finished.
 */
NRLSH_API nrlsh_status nrlsh_build(const float* items, int64_t n, int32_t d, int32_t m,
                                   int32_t L, uint64_t seed, nrlsh_index** out);
NRLSH_API nrlsh_status nrlsh_build_ex(const void* items, int64_t n, int32_t d, int32_t m,
                                      int32_t L, uint64_t seed, nrlsh_dtype dtype, float eps,
                                      void* stream, nrlsh_index** out);
/* As nrlsh_build_ex, with the projection path chosen by opts->projection, the
 * partition by opts->partition and opts->flags (NRLSH_BUILD_ASYNC_INPUT).
 * NRLSH_PROJECT_TENSOR on a device without tcgen05 returns NRLSH_ERR_UNSUPPORTED;
 * an unknown partition or flag returns NRLSH_ERR_ARG.
 * Storage order is (sub-dataset, id) under either partition. */
NRLSH_API nrlsh_status nrlsh_build_opts(const void* items, int64_t n, int32_t d, int32_t m,
                                        int32_t L, uint64_t seed, const nrlsh_build_options* opts,
                                        nrlsh_index** out);

/*
 * Query processing (Section 3.3 multi-probe, exact re-rank, top-k; Eq. 1).
 *   queries       nq x d row-major fp32 (not normalised by the library)
 *   nq >= 0, 1 <= k <= NRLSH_MAX_K, probe_budget >= 1 (values above n act as n)
 *   ids           nq x k int64: original item ids, best first; -1 past the end
 *                 when fewer than k items were probed
 *   scores        nq x k fp32: the matching inner products; -inf past the end
 *   flags         NRLSH_WHOLE_BUCKETS: the boundary bucket is probed whole;
 *                 NRLSH_QUERY_TENSOR: the probing and the re-rank run on tensor
 *                 cores (below); results are the same;
 *                 NRLSH_QUERY_ASYNC_INPUT: host queries are read by `stream` in
 *                 order and the call does not wait for their copy (the caller
 *                 keeps the buffer unchanged until the stream has passed the call)
 * nrlsh_query runs on the legacy default stream with no flags.
 *
 * The tensor-core path handles every (query, item) pair of a probed sub-dataset
 * as one entry of a dense product of a 128-query tile with 128-item tiles:
 * match counts l(q, x) from the +-1 sign vectors of the codes (bf16 products,
 * exact in the FP32 accumulator) and scores from the bf16-rounded query and
 * items with FP32 accumulation, kept as intervals [s - e, s + e] that provably
 * hold the FP64 score; the exact top-k then rescores the contenders.  It needs
 * an sm_100-family GPU (else NRLSH_ERR_UNSUPPORTED).  Its first call on an index
 * makes the index's sign matrix (n x 128 bytes, kept until nrlsh_free) on that
 * call's stream; make it before any stream capture.
 */
#define NRLSH_QUERY_TENSOR 0x8u
#define NRLSH_QUERY_ASYNC_INPUT 0x40u   /* also taken by nrlsh_query_batched (ks, budgets too) */
NRLSH_API nrlsh_status nrlsh_query(const nrlsh_index* index, const float* queries, int64_t nq,
                                   int32_t k, int64_t probe_budget, int64_t* ids,
                                   float* scores);
NRLSH_API nrlsh_status nrlsh_query_ex(const nrlsh_index* index, const float* queries,
                                      int64_t nq, int32_t k, int64_t probe_budget,
                                      uint32_t flags, int64_t* ids, float* scores,
                                      void* stream);

/*
 * Batched query processing with per-query budgets and k (the batching form of the
 * Section 3.3 multi-probe query): the queries are hashed, their Hamming histograms
 * computed, and a persistent fused kernel takes queries from a device work
 * counter, each CTA running the bucket walk, selection, FP32 re-rank and exact
 * top-k in its own scratch slab.  Results equal nrlsh_query_ex per query.
 *   ks            nq int32: k of each query, clamped into [1, k_max]
 *   budgets       nq int64: probe budget of each query, clamped into [1, min(budget_max, n)]
 *   k_max         1 <= k_max <= NRLSH_MAX_K; ids/scores rows are k_max wide, padded
 *                 with (-1, -inf) past each query's k
 *   budget_max    >= 1: the largest budget honoured (sizes the scratch slabs)
 *   flags         NRLSH_QUERY_GRAPH: capture the launches in a CUDA graph on the first
 *                 call with these pointers and sizes, and replay it on later identical
 *                 calls (needs a non-NULL stream; the graph and its workspace live
 *                 until nrlsh_free); NRLSH_QUERY_ASYNC_INPUT: host queries, ks and
 *                 budgets are read by `stream` in order and the call does not wait
 *                 for their copies; the path flags below.
 * The tensor-core path runs the queries in chunks whose workspace is at most an
 * eighth of the device's memory (at most 32 GiB).
 * The first call for a given shape (device, the index's n, d, m, L, dtype and eps,
 * and the call's nq, k_max, budget_max and path flags) times the candidate
 * configurations on a prefix of the batch (the autotuner) and keeps the fastest
 * for every later call of that shape, on any index of the process:
 *   - the FP32 re-rank: popcount histograms with 32, 64 or 128 queries per block,
 *     the persistent re-rank at 1, 2 or 4 CTAs per SM, gathering the stored rows
 *     or (fp32 items) a bf16 copy of them: the scores' intervals then also cover
 *     that copy's rounding, and the exact top-k still rescores from the stored rows;
 *   - the tensor-core path of nrlsh_query_ex's NRLSH_QUERY_TENSOR (histograms on
 *     tensor cores or by popcount).
 * NRLSH_QUERY_TENSOR, NRLSH_QUERY_FP32 and NRLSH_QUERY_BF16 (at most one) restrict
 * it.  Every path returns the same ids and scores.  Make that first call before
 * any stream capture of your own.  ks and budgets may be device or host pointers
 * like the other arrays.
 */
#define NRLSH_QUERY_GRAPH 0x2u
#define NRLSH_QUERY_NO_TUNE 0x4u   /* skip the autotuner: last tuned (or default) tiles */
#define NRLSH_QUERY_FP32 0x10u     /* the FP32 re-rank over the stored rows only */
#define NRLSH_QUERY_BF16 0x20u     /* bf16 operands only: tensor cores, or the FP32 re-rank
                                      over bf16 rows (NRLSH_QUERY_TENSOR: tensor cores only;
                                      none of the three: the autotuner picks among all) */
NRLSH_API nrlsh_status nrlsh_query_batched(const nrlsh_index* index, const float* queries,
                                           int64_t nq, const int32_t* ks, const int64_t* budgets,
                                           int32_t k_max, int64_t budget_max, uint32_t flags,
                                           int64_t* ids, float* scores, void* stream);
/* Device scratch (bytes) one nrlsh_query_batched call with these sizes and flags
 * allocates from the stream-ordered pool (device-pointer arguments, no graph), for
 * callers that admit work by memory.  It follows the configuration that call would
 * use: the tuned one for these sizes, else the last one used. */
NRLSH_API nrlsh_status nrlsh_batched_scratch_bytes(const nrlsh_index* index, int64_t nq,
                                                   int32_t k_max, int64_t budget_max,
                                                   uint32_t flags, int64_t* bytes);
/* The autotuned configuration last used for this index: histogram queries per
 * block and persistent CTAs per SM (0, 0 before any batched call), and in
 * *tensor bit 0 = histograms on tensor cores, bit 1 = re-rank on tensor cores,
 * bit 2 = the FP32 re-rank gathers a bf16 copy of fp32 rows.
 * Any output may be NULL. */
NRLSH_API nrlsh_status nrlsh_get_tuning(const nrlsh_index* index, int32_t* hist_queries_per_block,
                                        int32_t* ctas_per_sm, int32_t* tensor);

/*
 * Query processing without any device allocation.  The paper has no counterpart:
 * this exists for callers that must not allocate device memory while they query,
 * for example a serving process whose memory is owned by another allocator, or
 * code whose latency budget cannot absorb an allocator call.  It computes exactly
 * what nrlsh_query_ex computes (no flags), using as scratch one fixed array of
 * NRLSH_NOALLOC_SCRATCH_BYTES (32 MiB) compiled into the library; every GPU on
 * which the library is used keeps that array until the process exits.
 *   queries, ids, scores   DEVICE pointers only (host pointers: NRLSH_ERR_ARG)
 *   the other arguments    as for nrlsh_query_ex
 * Queries are processed in chunks that fit the array.  A probe budget whose single
 * query needs more scratch than the array holds (about 1.4M candidates for the
 * largest bucket tables) is rejected with NRLSH_ERR_ARG before any work is queued.
 * The first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * share the one array and leave their contents in it, so calls whose GPU work
 * overlaps (on different streams, or from different threads) race and must be
 * serialised by the caller.  No allocation or free of any kind is made.
 */
#define NRLSH_NOALLOC_SCRATCH_BYTES (32u << 20)
NRLSH_API nrlsh_status nrlsh_query_noalloc(const nrlsh_index* index, const float* queries,
                                           int64_t nq, int32_t k, int64_t probe_budget,
                                           int64_t* ids, float* scores, void* stream);

/*
 * Multi-table single-probe query (Algorithm 2 with several hash tables).  The L
 * code bits of the index are read as `tables` hash tables of L / tables bits:
 * table t holds bits [t L / tables, (t + 1) L / tables).  For every sub-dataset
 * S_j, a single probe of each table visits the bucket equal to the query's code
 * in that table, so the probed items are
 *     C(q) = { x : code_t(x) = code_t(q) for some table t }  (all sub-datasets),
 * and the result is the exact top-k of C(q) by q^T x (scores and tie rule as in
 * nrlsh_query_ex): Algorithm 2's best item over the sub-datasets, extended to k.
 *   tables          1 <= tables <= L, L % tables == 0
 *   max_candidates  0: C(q) is re-ranked whole; > 0: only the first
 *                   max_candidates items of C(q) in storage order (sub-dataset,
 *                   then id) are re-ranked
 *   ids, scores     nq x k, best first, padded with (-1, -inf) past |C(q)|
 *   probed          nq int64 or NULL: |C(q)| before the cap
 * Scratch of about 24 bytes per (query, candidate slot) is taken in chunks of
 * queries of at most 1 GiB.
 */
NRLSH_API nrlsh_status nrlsh_query_multitable(const nrlsh_index* index, const float* queries,
                                              int64_t nq, int32_t tables, int32_t k,
                                              int64_t max_candidates, int64_t* ids,
                                              float* scores, int64_t* probed, void* stream);
/* The first min(|C(q)|, cap) items of C(q) of nrlsh_query_multitable, as original
 * ids in storage order (cand: nq x cap int32), and |C(q)| (count: nq int64). */
NRLSH_API nrlsh_status nrlsh_multitable_candidates(const nrlsh_index* index,
                                                   const float* queries, int64_t nq,
                                                   int32_t tables, int64_t cap, int32_t* cand,
                                                   int64_t* count, void* stream);

/*
 * Introspection of the query path, for testing against a reference.  Device or
 * host pointers as above.
 * nrlsh_hash_queries: codes (nq uint64; bit b of the code is hash bit b).
 * nrlsh_query_histograms: H (nq x m x (L+1) uint32), H[q][j][l] = number of
 *   items of sub-dataset j sharing exactly l hash bits with query q; flags
 *   NRLSH_QUERY_TENSOR counts them on tensor cores (the same numbers).
 * nrlsh_query_candidates: the probed items of each query (Section 3.3):
 *   cand (nq x cap int32 original ids) and count (nq int64).  For each query the
 *   ids of the buckets probed whole come first, in storage order (sub-dataset,
 *   then id), followed by the items taken from the boundary bucket, by id.  Fails
 *   with NRLSH_ERR_ARG if a query has more than `cap` candidates (count is still
 *   written).  Without NRLSH_WHOLE_BUCKETS, count = min(B, n).  With
 *   NRLSH_QUERY_TENSOR the candidates come from the tensor-core path: the same
 *   set, grouped by ascending sub-dataset but in no set order inside one.
 */
NRLSH_API nrlsh_status nrlsh_hash_queries(const nrlsh_index* index, const float* queries,
                                          int64_t nq, uint64_t* codes, void* stream);
NRLSH_API nrlsh_status nrlsh_query_histograms(const nrlsh_index* index, const float* queries,
                                              int64_t nq, uint32_t* H, uint32_t flags,
                                              void* stream);
NRLSH_API nrlsh_status nrlsh_query_candidates(const nrlsh_index* index, const float* queries,
                                              int64_t nq, int64_t probe_budget, uint32_t flags,
                                              int64_t cap, int32_t* cand, int64_t* count,
                                              void* stream);

/*
 * Index introspection.  These copy into caller-owned HOST buffers and
 * synchronise the index's build stream.
 * nrlsh_get_codes:       n uint64 codes in original id order.
 * nrlsh_get_partition:   sub_of_id (n int32), U2 (m doubles, U_j^2), sqnorm (n doubles,
 *                        s_x in id order); any of the three may be NULL.
 * nrlsh_get_segments:    seg (m+1 int64): S_j occupies storage positions
 *                        [seg[j], seg[j+1]); seg[0] = 0, seg[m] = n.
 * nrlsh_get_projections: A ((d+1) x L floats, row-major; every value is bf16).
 * nrlsh_get_buckets:     the probing order: bucket_j, bucket_l (m(L+1) int32 each)
 *                        and s_hat (m(L+1) doubles) in probing order; any may be NULL.
 * nrlsh_get_info:        sizes and build statistics; NRLSH_ERR_TIMEOUT (info still
 *                        filled) when device_error or query_error is set.
 */
NRLSH_API nrlsh_status nrlsh_get_codes(const nrlsh_index* index, uint64_t* codes);
NRLSH_API nrlsh_status nrlsh_get_partition(const nrlsh_index* index, int32_t* sub_of_id,
                                           double* U2, double* sqnorm);
NRLSH_API nrlsh_status nrlsh_get_segments(const nrlsh_index* index, int64_t* seg);
NRLSH_API nrlsh_status nrlsh_get_projections(const nrlsh_index* index, float* A);
NRLSH_API nrlsh_status nrlsh_get_buckets(const nrlsh_index* index, int32_t* bucket_j,
                                         int32_t* bucket_l, double* s_hat);
NRLSH_API nrlsh_status nrlsh_get_info(const nrlsh_index* index, nrlsh_info* info);

/* Releases the index and its device memory (after synchronising its stream). */
NRLSH_API void nrlsh_free(nrlsh_index* index);

/* Message for the last failed call on this thread ("" if none). */
NRLSH_API const char* nrlsh_last_error(void);

/*
 * Instrumentation.  nrlsh_launch_count: kernels this library has launched in
 * this process.  With profiling on, every kernel launch is bracketed by CUDA
 * events on its stream; nrlsh_profile_read synchronises those events, adds up
 * the time per kernel name and clears the record.  names receives a
 * '\n'-separated list (up to names_cap bytes), ms and launches one entry per
 * name (up to cap).  Returns the number of distinct names through *count.
 */
NRLSH_API uint64_t nrlsh_launch_count(void);
/* Read bandwidth of device memory for the rooflines of the bandwidth-bound kernels:
 * every SM reads the `bytes` (a multiple of 16; buf 16-byte aligned) of buf with
 * 16-byte loads that bypass L1, `reps` times, after one untimed pass; *gbps =
 * bytes x reps / the event-timed duration on `stream`.  A buffer well inside L2
 * gives the L2 read rate, one much larger than L2 the HBM read rate. */
NRLSH_API nrlsh_status nrlsh_read_bandwidth(const void* buf, int64_t bytes, int32_t reps,
                                            void* stream, double* gbps);
NRLSH_API nrlsh_status nrlsh_set_profiling(int32_t enable);
NRLSH_API nrlsh_status nrlsh_profile_read(char* names, int64_t names_cap, double* ms,
                                          int64_t* launches, int32_t cap, int32_t* count);

#ifdef __cplusplus
}
#endif

#endif /* NRLSH_H */
