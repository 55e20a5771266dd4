// C ABI of libnrlsh.so: argument checks, device memory ownership, the order of
// kernel launches for index building (Algorithm 1) and query processing
// (Section 3.3), host<->device staging, introspection and instrumentation.
#include "nrlsh_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

// Autotuned configuration of the batched query path.
struct nrlsh_batch_cfg {
    int hist_qb = 64;       // queries per histogram block (popcount histogram)
    int ctas_per_sm = 2;    // persistent probe/re-rank CTAs per SM (FP32 re-rank)
    int hist_tc = 0;        // 1: histograms on tensor cores (sign products)
    int rerank_tc = 0;      // 1: candidates and score intervals on tensor cores
    int rows_bf16 = 0;      // 1: the FP32 re-rank gathers a bf16 copy of fp32 rows
    bool operator==(const nrlsh_batch_cfg& o) const {
        return hist_qb == o.hist_qb && ctas_per_sm == o.ctas_per_sm && hist_tc == o.hist_tc &&
               rerank_tc == o.rerank_tc && rows_bf16 == o.rows_bf16;
    }
};

// A captured batched-query launch sequence with its fixed workspace.
struct nrlsh_graph_entry {
    std::tuple<const void*, int64_t, const void*, const void*, int, int64_t, const void*,
               const void*, void*> key;
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> workspace;
    nrlsh_batch_cfg cfg{0, 0, 0, 0};   // the captured configuration
};

struct nrlsh_index {
    int64_t n = 0;
    int32_t d = 0, m = 0, L = 0, Lp = 0, dp = 0, code_bytes = 0, ncls = 0;
    nrlsh_dtype dtype = NRLSH_F32;
    float eps = 0.1f;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t built = nullptr;   // recorded on `stream` at the end of the build
    int device = 0;
    int64_t device_bytes = 0;
    std::vector<void*> owned;
    // device arrays (storage order = sub-dataset major, id ascending inside)
    void* Xp = nullptr;            // n x dp items, stored dtype, zero padded
    uint32_t* perm = nullptr;      // position -> original id
    uint32_t* sub_of_id = nullptr; // id -> sub-dataset
    double* s_id = nullptr;        // id -> ||x||^2
    double* s_pos = nullptr;       // position -> ||x||^2
    double* tau64 = nullptr;       // position -> sqrt(U_j^2 - ||x||^2)
    float* tau32 = nullptr;
    float* xnorm = nullptr;        // position -> fp32 upper bound of ||x||
    double* U2 = nullptr;          // m
    float* A = nullptr;            // (d+1) x L
    float* A_pad = nullptr;        // (d+1) x Lp
    float* anorm = nullptr;        // Lp
    void* codes = nullptr;         // n code words, position order
    uint32_t* order = nullptr;     // ncls bucket ids j*(L+1)+l in probing order
    double* shat_sorted = nullptr; // ncls
    const double* ccos = nullptr;  // L+1 bucket cosines c_l (the library's cache, not owned)
    int32_t partition = NRLSH_PARTITION_PERCENTILE;
    int64_t* seg = nullptr;        // m+1 storage offsets of the sub-datasets
    nrlsh::PosTile* tiles = nullptr;
    int32_t ntiles = 0;
    bool tiles_exclusive = false;  // every sub-dataset is exactly one histogram tile
    unsigned* ambiguous = nullptr;  // (item, bit) pairs the first tier left undecided
    unsigned* norm_fb = nullptr;    // rows whose squared norm took the exact slow path
    int projection = NRLSH_PROJECT_SIMT;
    __nv_bfloat16* At = nullptr;     // A^T in bf16, 64 x dp (tensor-core B operand)
    float* At32 = nullptr;           // A^T in fp32, the warp-per-row projection's layout
    __nv_bfloat16* Xb = nullptr;     // fp32 items: bf16 high part, n x dp (tensor-core A operand)
    __nv_bfloat16* Xb2 = nullptr;    // fp32 items: bf16 low part (x - hi rounded), n x dp
    int* dev_err = nullptr;          // set by bounded device waits that ran out
    int* query_err = nullptr;        // the same for the tensor-core query kernels
    // tensor-core query operands, made on first use: the +-1 signs of the codes
    // (n x 64 bf16) and, for fp32 items, their bf16 rounding (n x dp)
    mutable std::mutex tc_mu;
    mutable __nv_bfloat16* tc_xs = nullptr;
    mutable __nv_bfloat16* tc_xb = nullptr;
    mutable cudaEvent_t tc_ready = nullptr;
    mutable std::vector<void*> tc_owned;
    // batched queries: the configuration last used and the graph cache
    mutable std::mutex batch_mu;
    mutable nrlsh_batch_cfg last_cfg{0, 0, 0, 0};
    mutable std::vector<nrlsh_graph_entry> graphs;
};

namespace nrlsh {

// ------------------------------------------------------------ error state

namespace state {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

struct ProfRecord {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRecord> g_prof;
std::vector<cudaEvent_t> g_event_pool;
thread_local cudaEvent_t t_pending = nullptr;

cudaEvent_t take_event() {
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace state

using namespace state;

void set_error(const std::string& msg) { g_last_error = msg; }

nrlsh_status cuda_status(cudaError_t e, const char* what) {
    set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return NRLSH_ERR_OOM;
    return NRLSH_ERR_CUDA;
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Programmatic dependent launches are on unless NRLSH_NO_PDL is set (to 1) in the
// environment when the library first launches a kernel.
bool pdl_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("NRLSH_NO_PDL");
        return !(v && v[0] == '1');
    }();
    return on;
}

// Polls of the tensor-core kernels' first wait for an operand stage: the
// NRLSH_TEST_SPIN_FIRST environment variable when set (a test hook that makes a
// bounded wait run out on purpose), else the kernels' normal limit.
uint32_t test_spin_first() {
    const char* v = std::getenv("NRLSH_TEST_SPIN_FIRST");
    if (!v || !*v) return 1u << 22;
    return (uint32_t)std::strtoul(v, nullptr, 10);
}

void prof_begin(const char*, cudaStream_t s) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    t_pending = take_event();
    cudaEventRecord(t_pending, s);
}

void prof_end(const char* name, cudaStream_t s) {
    if (!t_pending) return;
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.push_back({name, t_pending, b});
    t_pending = nullptr;
}

}  // namespace nrlsh

using namespace nrlsh;

namespace {

nrlsh_status arg_error(const std::string& msg) {
    set_error(msg);
    return NRLSH_ERR_ARG;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The stream-ordered pool keeps freed blocks for reuse instead of returning
// them to the driver at every synchronisation.
void keep_pool_memory(int device) {
    static std::once_flag once[64];
    if (device < 0 || device >= 64) return;
    std::call_once(once[device], [device] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    });
}

// Scratch memory of one call: bump-allocated (256-byte aligned) from blocks of the
// stream-ordered pool, released on its stream at scope exit.
struct Scratch {
    static constexpr size_t kBlock = (size_t)8 << 20;
    cudaStream_t s;
    std::vector<void*> blocks;
    char* cur = nullptr;
    size_t left = 0;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void* p : blocks) cudaFreeAsync(p, s);
    }
    template <typename T>
    nrlsh_status get(T** out, size_t count) {
        *out = nullptr;
        const size_t bytes = (std::max<size_t>(count * sizeof(T), 16) + 255) & ~(size_t)255;
        if (bytes > left) {
            void* p = nullptr;
            const size_t bb = std::max(bytes, kBlock);
            cudaError_t e = cudaMallocAsync(&p, bb, s);
            if (e != cudaSuccess) return cuda_status(e, "cudaMallocAsync");
            blocks.push_back(p);
            cur = (char*)p;
            left = bb;
        }
        *out = (T*)cur;
        cur += bytes;
        left -= bytes;
        return NRLSH_OK;
    }
};

// Carves the index's arrays out of one allocation: a first pass with base null
// only adds up the (256-byte aligned) sizes, a second assigns the pointers.
struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    void take(T** out, size_t count) {
        off = (off + 255) & ~(size_t)255;
        if (base) *out = (T*)(base + off);
        off += std::max<size_t>(count * sizeof(T), 16);
    }
};

void destroy(nrlsh_index* ix) {
    if (!ix) return;
    cudaStreamSynchronize(ix->stream);
    for (auto& g : ix->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        for (void* p : g.workspace) cudaFree(p);
    }
    cudaDeviceSynchronize();
    for (void* p : ix->owned) cudaFreeAsync(p, ix->stream);
    cudaStreamSynchronize(ix->stream);
    for (void* p : ix->tc_owned) cudaFreeAsync(p, ix->stream);
    cudaStreamSynchronize(ix->stream);
    if (ix->built) cudaEventDestroy(ix->built);
    if (ix->tc_ready) cudaEventDestroy(ix->tc_ready);
    delete ix;
}

// Per-thread side streams for the data-independent parts of the build.  A fork
// makes a side stream wait for everything queued on the main stream so far; its
// join event (recorded after the side work) is what the main stream waits for at
// the point where the side work's first consumer is queued.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ~SideStream() {
        if (s) cudaStreamDestroy(s);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
    }
};
thread_local SideStream t_side[2];

cudaStream_t side_stream(int i) { return t_side[i].s; }

cudaError_t side_stream_fork(cudaStream_t main, int i) {
    SideStream& t = t_side[i];
    if (!t.s) {
        cudaError_t e = cudaStreamCreateWithFlags(&t.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t.join, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaEventRecord(t.fork, main);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(t.s, t.fork, 0);
}

// Marks the end of the copy of a host input, which is all a call must wait for
// before its caller may reuse that buffer.
thread_local cudaEvent_t t_staged = nullptr;
cudaError_t record_staged(cudaStream_t st) {
    if (!t_staged) {
        cudaError_t e = cudaEventCreateWithFlags(&t_staged, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    return cudaEventRecord(t_staged, st);
}

// The bucket cosines c_l = cos(pi (1 - eps)(L - l) / L) depend on (L, eps) alone:
// each (device, L, eps) is computed once, into an array the library keeps until
// the process exits, and later builds wait for its event instead of recomputing it.
struct CosEntry {
    double* cl = nullptr;
    cudaEvent_t ready = nullptr;
};
std::mutex g_cos_mu;
std::map<std::tuple<int, int, uint32_t>, CosEntry> g_cos;

// *cl receives the cached array; the cosines are queued on `side` the first time
// and `wait_on` waits for them.
nrlsh_status class_cos_cached(int device, int L, float eps, cudaStream_t side,
                              cudaStream_t wait_on, const double** cl) {
    uint32_t eb;
    std::memcpy(&eb, &eps, 4);
    std::lock_guard<std::mutex> g(g_cos_mu);
    CosEntry& e = g_cos[std::make_tuple(device, L, eb)];
    if (!e.cl) {
        void* p = nullptr;
        NRLSH_CK(cudaMalloc(&p, sizeof(double) * (L + 1)));
        cudaEvent_t ev = nullptr;
        cudaError_t er = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (er == cudaSuccess) er = launch_class_cos(L, eps, (double*)p, side);
        if (er == cudaSuccess) er = cudaEventRecord(ev, side);
        if (er != cudaSuccess) {
            cudaFree(p);
            if (ev) cudaEventDestroy(ev);
            return cuda_status(er, "bucket cosines");
        }
        e.cl = (double*)p;
        e.ready = ev;
    }
    NRLSH_CK(cudaStreamWaitEvent(wait_on, e.ready, 0));
    *cl = e.cl;
    return NRLSH_OK;
}

// Records the end of the side work queued so far.
cudaError_t side_stream_join(int i) { return cudaEventRecord(t_side[i].join, t_side[i].s); }

// The main stream's later work waits for the side work (its earlier work is
// unaffected, and the side kernels run meanwhile).
cudaError_t side_stream_wait(cudaStream_t main, int i) {
    return cudaStreamWaitEvent(main, t_side[i].join, 0);
}

// Work queued on another stream than the index's build stream waits for the
// build to finish (on the same stream, stream order suffices).
cudaError_t wait_for_build(const nrlsh_index* ix, cudaStream_t st) {
    if (st == ix->stream || !ix->built) return cudaSuccess;
    return cudaStreamWaitEvent(st, ix->built, 0);
}

int bits_for(int64_t v) {  // smallest b with 2^b >= v
    int b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return b;
}

// Copy `bytes` from a host or device pointer into fresh device scratch when the
// pointer is not device memory; otherwise return it unchanged.
nrlsh_status stage_in(Scratch& sc, const void* src, size_t bytes, const void** dev) {
    if (is_device_ptr(src)) {
        *dev = src;
        return NRLSH_OK;
    }
    char* d = nullptr;
    NRLSH_CKS(sc.get(&d, bytes));
    NRLSH_CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, sc.s));
    *dev = d;
    return NRLSH_OK;
}

nrlsh_status build_impl(const void* items, int64_t n, int32_t d, int32_t m, int32_t L,
                        uint64_t seed, nrlsh_dtype dtype, float eps, void* stream, int projection,
                        int partition, nrlsh_index** out, uint32_t build_flags = 0) {
    if (!out) return arg_error("out is NULL");
    *out = nullptr;
    if (!items) return arg_error("items is NULL");
    if (n < 1 || n > (int64_t)INT32_MAX) return arg_error("need 1 <= n <= 2^31 - 1");
    if (d < 1) return arg_error("need d >= 1");
    if (m < 1 || m > n) return arg_error("need 1 <= m <= n");
    if (L < 1 || L > NRLSH_MAX_L) return arg_error("need 1 <= L <= 64");
    if ((int64_t)m * (L + 1) > NRLSH_MAX_BUCKETS) return arg_error("need m * (L + 1) <= 16384");
    if (!(eps > 0.0f && eps < 1.0f)) return arg_error("need 0 < eps < 1");
    if (dtype != NRLSH_F32 && dtype != NRLSH_BF16) return arg_error("unknown dtype");
    if (projection < NRLSH_PROJECT_AUTO || projection > NRLSH_PROJECT_TENSOR)
        return arg_error("unknown projection path");
    if (partition != NRLSH_PARTITION_PERCENTILE && partition != NRLSH_PARTITION_UNIFORM)
        return arg_error("unknown partition");
    const size_t esz = dtype == NRLSH_BF16 ? 2 : 4;
    if ((int64_t)d * (int64_t)esz * n / n != (int64_t)d * (int64_t)esz) return arg_error("n*d overflows");

    cudaStream_t st = (cudaStream_t)stream;
    const bool host_items = !is_device_ptr(items);
    nrlsh_index* ix = new nrlsh_index();
    ix->n = n;
    ix->d = d;
    ix->m = m;
    ix->L = L;
    ix->Lp = L <= 8 ? 8 : L <= 16 ? 16 : L <= 32 ? 32 : 64;
    ix->dp = (d + 7) / 8 * 8;
    ix->code_bytes = L <= 32 ? 4 : 8;
    ix->ncls = m * (L + 1);
    ix->dtype = dtype;
    ix->eps = eps;
    ix->seed = seed;
    ix->partition = partition;
    ix->stream = st;
    cudaGetDevice(&ix->device);
    keep_pool_memory(ix->device);
    const bool tc_ok = project_tc_supported(d, L);
    if (projection == NRLSH_PROJECT_TENSOR && !tc_ok) {
        delete ix;
        set_error("the tensor-core projection needs an sm_100-family GPU and d <= ~1000");
        return NRLSH_ERR_UNSUPPORTED;
    }
    ix->projection = projection == NRLSH_PROJECT_AUTO ? NRLSH_PROJECT_SIMT : projection;

    auto fail = [&](nrlsh_status s) {
        destroy(ix);
        return s;
    };
#define B_CK(expr)                                            \
    do {                                                      \
        nrlsh_status s_ = (expr);                             \
        if (s_ != NRLSH_OK) return fail(s_);                  \
    } while (0)
#define B_CU(expr)                                            \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return fail(cuda_status(e_, #expr)); \
    } while (0)

    // sticky errors from earlier work surface here rather than mid-build
    B_CU(cudaGetLastError());
    // histogram tiles: runs of positions inside one sub-dataset.  Percentile
    // ranges have known sizes: offsets and tiles are made here; uniform ranges
    // get them from the device after the assignment (at most this many tiles).
    const int64_t tile = 16384 / ix->code_bytes;
    const bool uniform = partition == NRLSH_PARTITION_UNIFORM;
    if (!uniform) {
        int64_t nt = 0;
        for (int32_t j = 0; j < m; ++j) nt += ceil_div(seg_start(j + 1, n, m) - seg_start(j, n, m), tile);
        ix->ntiles = (int32_t)nt;
        ix->tiles_exclusive = nt == m;
    } else {
        ix->ntiles = (int32_t)(ceil_div(n, tile) + m);
    }

    // the index's device arrays: one allocation, carved in 256-byte aligned pieces
    const bool tc = ix->projection == NRLSH_PROJECT_TENSOR;
    auto carve = [&](Carver& c) {
        c.take((char**)&ix->Xp, (size_t)n * ix->dp * esz);
        c.take(&ix->perm, n);
        c.take(&ix->sub_of_id, n);
        c.take(&ix->s_id, n);
        c.take(&ix->s_pos, n);
        c.take(&ix->tau64, n);
        c.take(&ix->tau32, n);
        c.take(&ix->xnorm, n);
        c.take(&ix->U2, m);
        c.take(&ix->seg, (size_t)m + 1);
        c.take(&ix->A, (size_t)(d + 1) * L);
        c.take(&ix->A_pad, (size_t)(d + 1) * ix->Lp);
        c.take(&ix->anorm, ix->Lp);
        c.take((char**)&ix->codes, (size_t)n * ix->code_bytes);
        c.take(&ix->order, ix->ncls);
        c.take(&ix->shat_sorted, ix->ncls);
        c.take(&ix->ambiguous, 1);
        c.take(&ix->norm_fb, 1);
        c.take(&ix->dev_err, 1);
        c.take(&ix->query_err, 1);
        c.take(&ix->tiles, (size_t)ix->ntiles);
        if (warp_proj_stride(d, ix->Lp) > 0) c.take(&ix->At32, warp_proj_at_floats(d, ix->Lp));
        if (tc) {
            c.take(&ix->At, (size_t)64 * ix->dp);
            if (dtype == NRLSH_F32) {
                c.take(&ix->Xb, (size_t)n * ix->dp);
                c.take(&ix->Xb2, (size_t)n * ix->dp);
            }
        }
    };
    {
        Carver sizing;
        carve(sizing);
        void* base = nullptr;
        cudaError_t e = cudaMallocAsync(&base, sizing.off, st);
        if (e != cudaSuccess) return fail(cuda_status(e, "cudaMallocAsync (index)"));
        ix->owned.push_back(base);
        ix->device_bytes = (int64_t)sizing.off;
        Carver real{(char*)base, 0};
        carve(real);
    }

    {
        Scratch sc(st);
        // host items: the copy is queued after the side streams fork, so that
        // their item-independent work runs while it is in flight
        const void* X = items;
        char* X_stage = nullptr;
        if (host_items) B_CK(sc.get(&X_stage, (size_t)n * d * esz));
        uint64_t *keys, *keys_alt;
        uint32_t *vals, *vals_alt, *jkeys, *jkeys_alt;
        char* sort_tmp;
        unsigned long long *amb_list, *amb_list2 = nullptr;
        unsigned* amb_count2 = nullptr;
        // the bf16 pass on fp32 items leaves a few percent of the bits to the FP32 tier
        const size_t amb_cap = tc ? std::max<size_t>(4096, (size_t)n * L / 16)
                                  : ambiguity_capacity(n, L);
        const size_t amb_cap2 = ambiguity_capacity(n, L);
        B_CK(sc.get(&keys, std::max<int64_t>(n, 8)));      // uniform ranges: sizes (m words)
        B_CK(sc.get(&keys_alt, std::max<int64_t>(n, 8)));  // uniform ranges: 6 range words
        B_CK(sc.get(&vals, n));
        B_CK(sc.get(&vals_alt, n));
        B_CK(sc.get(&jkeys, n));
        B_CK(sc.get(&jkeys_alt, n));
        B_CK(sc.get(&sort_tmp, std::max(radix_sort_temp_bytes(n),
                                        small_rank_supported(n, m) ? small_rank_temp_bytes(n, m) : 0)));
        char* bo_tmp;
        B_CK(sc.get(&bo_tmp, bucket_order_temp_bytes(m, L)));
        B_CK(sc.get(&amb_list, amb_cap));
        if (tc) {
            B_CK(sc.get(&amb_list2, amb_cap2));
            B_CK(sc.get(&amb_count2, 1));
        }
        // FP32 sums of the item projection, computed in id order beside the partition
        const bool split = !tc && split_projection_supported(d, ix->Lp);
        float* vsum = nullptr;
        if (split) B_CK(sc.get(&vsum, (size_t)n * ((ix->Lp + 31) / 32 * 32)));
        // everything that starts at zero, in one launch
        const bool small = !uniform && small_rank_supported(n, m);
        {
            ZeroList z;
            z.add(ix->dev_err, 1);
            z.add(ix->query_err, 1);
            z.add(ix->ambiguous, 1);
            z.add(ix->norm_fb, 1);
            z.add(ix->U2, 2 * (size_t)m);
            if (tc) z.add(amb_count2, 1);
            if (small) z.add(sort_tmp, small_rank_temp_bytes(n, m) / 4);
            B_CU(launch_zero(z, st));
        }
        // Side stream 0: A and A^T, needed by the projection.  Side stream 1: the
        // bucket cosines and the percentile offsets, needed by the bucket order
        // and the queries.  Both run while the main stream ranks the items.
        B_CU(side_stream_fork(st, 0));
        B_CU(side_stream_fork(st, 1));
        cudaStream_t side0 = side_stream(0), side1 = side_stream(1);
        if (host_items) {
            B_CU(cudaMemcpyAsync(X_stage, items, (size_t)n * d * esz, cudaMemcpyHostToDevice, st));
            B_CU(record_staged(st));
            X = X_stage;
        }
        B_CU(launch_projections(ix->A, ix->A_pad, ix->anorm, ix->At, ix->dp, d, L, ix->Lp, seed,
                                side0));
        if (ix->At32) B_CU(launch_transpose_a(ix->A_pad, d, L, ix->Lp, ix->At32, side0));
        // the FP32 part of the item projection needs no partition: it runs here too
        // (after the items' copy, when they come from the host)
        if (split) {
            if (host_items) B_CU(cudaStreamWaitEvent(side0, t_staged, 0));
            B_CU(launch_project_dots(X, dtype, n, d, d, ix->Lp, ix->At32, vsum, side0));
        }
        B_CU(side_stream_join(0));
        B_CK(class_cos_cached(ix->device, L, eps, side1, side1, &ix->ccos));
        if (!uniform)  // percentile ranges: offsets and tiles follow from n and m
            B_CU(launch_segments(nullptr, n, m, tile, ix->seg, ix->tiles, ix->ntiles, side1));
        B_CU(side_stream_join(1));
        const int jbits = (bits_for(m) + 7) / 8 * 8;
        bool alt = false;
        uint32_t *jv = nullptr, *jv_alt = nullptr;
        if (small) {
            // Algorithm 1 for small inputs: tile sort, rank, per-range id sort
            B_CU(launch_sqnorm(X, dtype, n, d, d, ix->s_id, keys, vals, ix->norm_fb, st));
            B_CU(launch_small_rank(keys, vals, n, m, sort_tmp, ix->perm, ix->sub_of_id, ix->U2,
                                   st));
        } else if (!uniform) {
            // Algorithm 1: rank by norm, percentile partition, U_j
            B_CU(launch_sqnorm(X, dtype, n, d, d, ix->s_id, keys, vals, ix->norm_fb, st));
            B_CU(radix_sort_u64(keys, vals, keys_alt, vals_alt, n, 64, sort_tmp, &alt, st));
            // storage order: stable sort of ids by sub-dataset
            jv = alt ? vals : vals_alt;       // the pair the sort did not end in
            jv_alt = alt ? vals_alt : vals;
            B_CU(launch_segment_assign(alt ? keys_alt : keys, alt ? vals_alt : vals, n, m,
                                       ix->sub_of_id, ix->U2, jkeys, jv, st));
        } else {
            // Section 5: uniform norm ranges, then the same stable sort by sub-dataset
            B_CU(launch_sqnorm(X, dtype, n, d, d, ix->s_id, nullptr, nullptr, ix->norm_fb, st));
            jv = vals;
            jv_alt = vals_alt;
            B_CU(launch_uniform_assign(ix->s_id, n, m, (unsigned long long*)keys_alt, ix->sub_of_id,
                                       ix->U2, jkeys, jv, (uint32_t*)keys, st));
            B_CU(launch_segments((const uint32_t*)keys, n, m, tile, ix->seg, ix->tiles,
                                 ix->ntiles, st));
        }
        if (!small) {
            B_CU(radix_sort_u32(jkeys, jv, jkeys_alt, jv_alt, n, jbits, sort_tmp, &alt, st));
            B_CU(cudaMemcpyAsync(ix->perm, alt ? jv_alt : jv, sizeof(uint32_t) * n,
                                 cudaMemcpyDeviceToDevice, st));
        }
        // Eq. 8 per sub-dataset: sub-dataset-major copy and tau = sqrt(U_j^2 - s)
        // with the projection split, the gather takes the signs: it waits for the
        // FP32 sums (side stream 0)
        GatherCodes gc;
        if (split) {
            B_CU(side_stream_wait(st, 0));
            gc.vsum = vsum;
            gc.Lr = (ix->Lp + 31) / 32 * 32;
            gc.d = d;
            gc.L = L;
            gc.Lp = ix->Lp;
            gc.dpa = warp_proj_stride(d, ix->Lp);
            gc.code_bytes = ix->code_bytes;
            gc.A_pad = ix->A_pad;
            gc.At32 = ix->At32;
            gc.anorm = ix->anorm;
            gc.codes = ix->codes;
            gc.amb_count = ix->ambiguous;
            gc.kappa = (float)(d + 2) * 0x1p-22f;
        }
        B_CU(launch_gather_items(X, dtype, d, d, ix->dp, ix->perm, n, ix->sub_of_id, ix->s_id,
                                 ix->U2, ix->Xp, ix->Xb, ix->Xb2, ix->s_pos, ix->tau64, ix->tau32,
                                 ix->xnorm, gc, st));
        B_CU(side_stream_wait(st, 0));  // A and A^T are ready
        // Eq. 4: sign random projection codes
        if (split) {
            // the codes were taken in the gather
        } else if (!tc) {
            B_CU(launch_project_fp32(ix->Xp, dtype, n, d, ix->dp, L, ix->Lp, ix->A_pad, ix->anorm,
                                     ix->tau64, ix->tau32, ix->xnorm, ix->codes, ix->code_bytes,
                                     amb_list, ix->ambiguous, (unsigned)amb_cap, ix->At32, st));
        } else {
            const __nv_bfloat16* xb = dtype == NRLSH_F32 ? ix->Xb : (const __nv_bfloat16*)ix->Xp;
            B_CU(launch_project_tc(xb, ix->Xb2, ix->Xp, n, d, ix->dp, L, ix->Lp, ix->At, ix->A_pad,
                                   ix->anorm, ix->tau32, ix->tau64, ix->xnorm, dtype == NRLSH_F32,
                                   ix->codes, ix->code_bytes, amb_list, ix->ambiguous,
                                   (unsigned)amb_cap, ix->dev_err, st, test_spin_first()));
            // bits the tensor-core bound left open: compensated FP32, FP64 and canonical
            // tiers in one launch (with the fp32 A^T copy), else FP32 then FP64 lists
            if (ix->At32) {
                B_CU(launch_resolve_tiers(ix->Xp, dtype, n, d, ix->dp, L, ix->Lp, ix->At32,
                                          ix->A_pad, ix->anorm, ix->xnorm, ix->tau64, amb_list,
                                          ix->ambiguous, (unsigned)amb_cap, ix->codes,
                                          ix->code_bytes, st));
            } else {
                B_CU(launch_resolve_fp32(ix->Xp, dtype, n, d, ix->dp, L, ix->Lp, ix->A_pad,
                                         ix->anorm, ix->xnorm, ix->tau32, ix->tau64, amb_list,
                                         ix->ambiguous, (unsigned)amb_cap, ix->codes,
                                         ix->code_bytes, amb_list2, amb_count2,
                                         (unsigned)amb_cap2, st));
                B_CU(launch_resolve_fp64(ix->Xp, dtype, n, d, ix->dp, L, ix->Lp, ix->A_pad,
                                         ix->tau64, amb_list2, amb_count2, (unsigned)amb_cap2,
                                         ix->codes, ix->code_bytes, st));
            }
        }
        // Eq. 12 and the sorted (U_j, l) structure (the cosines, and for the
        // queries the offsets, come from side stream 1)
        B_CU(side_stream_wait(st, 1));
        B_CU(launch_bucket_order(ix->U2, ix->ccos, m, L, ix->shat_sorted, ix->order, bo_tmp, st));
    }
    B_CU(cudaEventCreateWithFlags(&ix->built, cudaEventDisableTiming));
    B_CU(cudaEventRecord(ix->built, st));
    // the caller may reuse a host item buffer once its copy is done; the build
    // itself stays queued
    if (host_items && !(build_flags & NRLSH_BUILD_ASYNC_INPUT)) B_CU(cudaEventSynchronize(t_staged));
#undef B_CK
#undef B_CU
    *out = ix;
    return NRLSH_OK;
}

// ------------------------------------------------------------------ queries

struct QueryOut {
    int64_t* ids = nullptr;      // nq x k_ld
    float* scores = nullptr;
    int32_t k_ld = 0;
    // candidates mode
    int32_t* cand = nullptr;     // nq x cand_cap
    int64_t cand_cap = 0;
    int64_t* count = nullptr;
    // histogram mode
    uint32_t* H = nullptr;
    // hash mode
    uint64_t* codes = nullptr;
};

enum class Stage { Hash, Hist, Cand, TopK };

__global__ void widen_codes_kernel(const uint32_t* in, uint64_t* out, int64_t nq) {
    NRLSH_PDL_ENTRY();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nq) out[i] = in[i];
}

// Runs the query path up to `stage` for queries [0, nq) (device pointers).
nrlsh_status run_queries(const nrlsh_index* ix, const float* Q, int64_t nq, int32_t k,
                         int64_t budget, uint32_t flags, Stage stage, const QueryOut& o,
                         cudaStream_t st) {
    const int64_t n = ix->n;
    const int64_t Bp = std::min(budget, n);
    const bool whole = (flags & NRLSH_WHOLE_BUCKETS) != 0;
    // per-query scratch beyond the candidate arrays
    const int64_t fixed = (int64_t)ix->ncls * 4 + ix->m + 64 + 8 + 4;
    int64_t cap = Bp;
    const int64_t per_cand = 4 + 4 + 4 + 4 + 8;
    const int64_t budget_bytes = (int64_t)1 << 30;
    int64_t chunk = std::max<int64_t>(1, budget_bytes / (fixed + (stage >= Stage::Cand ? cap * per_cand : 0)));
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(nq, 1));
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t qc = std::min(chunk, nq - q0);
        const float* Qc = Q + q0 * ix->d;
        Scratch sc(st);
        float* qnorm;
        char* qcodes;
        unsigned* qamb;
        unsigned long long* qamb_list;
        const size_t qamb_cap = ambiguity_capacity(qc, ix->L);
        NRLSH_CKS(sc.get(&qnorm, qc));
        NRLSH_CKS(sc.get(&qamb, 1));
        NRLSH_CKS(sc.get(&qamb_list, qamb_cap));
        NRLSH_CKS(sc.get(&qcodes, qc * ix->code_bytes));
        // P(q) = [q; 0] (Eq. 8), hashed by Eq. 4
        NRLSH_CK(launch_hash_queries(Qc, qc, ix->d, ix->L, ix->Lp, ix->A_pad, ix->anorm, qnorm,
                                     qcodes, ix->code_bytes, qamb_list, qamb, (unsigned)qamb_cap, ix->At32, st));
        if (stage == Stage::Hash) {
            if (ix->code_bytes == 8) {
                NRLSH_CK(cudaMemcpyAsync(o.codes + q0, qcodes, 8 * qc, cudaMemcpyDeviceToDevice, st));
            } else {
                NRLSH_CK(launch("widen_codes", widen_codes_kernel, dim3((unsigned)ceil_div(qc, 256)),
                                dim3(256), 0, st, (const uint32_t*)qcodes, o.codes + q0, qc));
            }
            continue;
        }
        uint32_t* H;
        if (stage == Stage::Hist) {
            H = o.H + q0 * ix->ncls;
        } else {
            NRLSH_CKS(sc.get(&H, qc * ix->ncls));
        }
        if (!ix->tiles_exclusive)
            NRLSH_CK(cudaMemsetAsync(H, 0, sizeof(uint32_t) * qc * ix->ncls, st));
        NRLSH_CK(launch_hist(ix->codes, qcodes, ix->code_bytes, qc, ix->m, ix->L, ix->tiles,
                             ix->ntiles, H, st, 64, ix->tiles_exclusive));
        if (stage == Stage::Hist) continue;
        if (stage == Stage::TopK && !whole) {
            // one fused launch: walk, selection, re-rank, exact top-k, by CTAs that
            // stay resident and take queries from a counter
            const int ctas = probe_rerank_ctas(ix->dtype, ix->code_bytes, ix->dp, ix->m, qc);
            uint32_t* slabs;
            unsigned* work;
            NRLSH_CKS(sc.get(&slabs, (size_t)ctas * 6 * cap));
            NRLSH_CKS(sc.get(&work, 1));
            NRLSH_CK(cudaMemsetAsync(work, 0, sizeof(unsigned), st));
            NRLSH_CK(launch_probe_rerank_persistent(
                H, ix->order, ix->m, ix->L, n, ix->seg, budget, nullptr, ix->codes, qcodes,
                ix->code_bytes, ix->Xp, ix->dtype, ix->dp, ix->d, Qc, ix->xnorm, qnorm, ix->perm,
                nullptr, k, slabs, cap, ctas, work, qc, o.ids + q0 * o.k_ld,
                o.scores + q0 * o.k_ld, st));
            continue;
        }
        uint8_t* lam;
        Boundary* bnd;
        NRLSH_CKS(sc.get(&lam, qc * ix->m));
        NRLSH_CKS(sc.get(&bnd, qc));
        NRLSH_CK(launch_threshold(H, ix->order, ix->m, ix->L, qc, n, budget, nullptr, flags, lam,
                                  bnd, st));
        int64_t ccap = cap;
        if (whole) {  // the boundary bucket may overshoot B: size the lists first
            std::vector<Boundary> hb(qc);
            NRLSH_CK(cudaMemcpyAsync(hb.data(), bnd, sizeof(Boundary) * qc, cudaMemcpyDeviceToHost, st));
            NRLSH_CK(cudaStreamSynchronize(st));
            ccap = 1;
            for (auto& b : hb) ccap = std::max<int64_t>(ccap, (int64_t)b.full + b.r);
        }
        uint32_t* cand;
        NRLSH_CKS(sc.get(&cand, qc * ccap));
        NRLSH_CK(launch_select(ix->codes, qcodes, ix->code_bytes, ix->seg, ix->m, ix->L, qc, lam, bnd,
                               cand, ccap, st));
        if (stage == Stage::Cand) {
            NRLSH_CK(launch_cand_to_ids(cand, ccap, bnd, ix->perm, qc, o.cand + q0 * o.cand_cap,
                                        o.cand_cap, o.count + q0, st));
            continue;
        }
        float *lo, *hi;
        uint32_t* cont;
        double* cont_s;
        NRLSH_CKS(sc.get(&lo, qc * ccap));
        NRLSH_CKS(sc.get(&hi, qc * ccap));
        NRLSH_CKS(sc.get(&cont, qc * ccap));
        NRLSH_CKS(sc.get(&cont_s, qc * ccap));
        NRLSH_CK(launch_rerank_fp32(ix->Xp, ix->dtype, ix->dp, ix->d, Qc, qc, cand, ccap, bnd,
                                    ix->xnorm, qnorm, lo, hi, st));
        NRLSH_CK(launch_topk(lo, hi, cand, ccap, bnd, qc, k, nullptr, ix->Xp, ix->dtype, ix->dp,
                             ix->d, Qc, ix->xnorm, qnorm, ix->perm, cont, cont_s,
                             o.ids + q0 * o.k_ld, o.scores + q0 * o.k_ld, o.k_ld, st));
    }
    return NRLSH_OK;
}

// ------------------------------------------------- tensor-core query path

// Workspace of one chunk of qc queries on the tensor-core path.
struct TcWs {
    float* qnorm = nullptr;
    unsigned* qamb = nullptr;
    unsigned long long* qamb_list = nullptr;
    size_t qamb_cap = 0;
    char* qcodes = nullptr;
    __nv_bfloat16* Qb = nullptr;
    __nv_bfloat16* Qs = nullptr;
    uint32_t* H = nullptr;
    uint8_t* lam = nullptr;
    uint32_t* off = nullptr;
    TcBoundary* tb = nullptr;
    Boundary* bnd = nullptr;
    uint8_t* flag = nullptr;
    uint32_t* list = nullptr;
    uint32_t* nlist = nullptr;
    uint32_t* cand = nullptr;
    float* lo = nullptr;
    float* hi = nullptr;
    uint32_t* cont = nullptr;
    double* cont_s = nullptr;
    int* err = nullptr;           // the call's error word (copied into the index's at the end)
    float* qce = nullptr;         // per-query score interval factors
    int64_t qc = 0;
    int64_t cap = 0;
};

int tc_nqt(int64_t qc) { return (int)ceil_div(qc, 128); }

// Buffer sizes (bytes) of a TcWs for qc queries and list capacity cap, in TcWs order.
std::vector<size_t> tc_ws_sizes(const nrlsh_index* ix, int64_t qc, int64_t cap) {
    const size_t q = (size_t)qc, c = (size_t)cap;
    const size_t Kq = 64 * (size_t)tc_query_k_chunks(ix->d);
    const size_t nw = (size_t)ix->m * tc_nqt(qc);
    return {q * 4, 16, ambiguity_capacity(qc, ix->L) * 8, q * ix->code_bytes, q * Kq * 2, q * 128,
            q * ix->ncls * 4, q * ix->m, q * (ix->m + 1) * 4, q * sizeof(TcBoundary),
            q * sizeof(Boundary), nw, nw * 4, 16, q * c * 4, q * c * 4, q * c * 4, q * c * 4,
            q * c * 8, 16, q * 4};
}

size_t tc_ws_bytes(const nrlsh_index* ix, int64_t qc, int64_t cap) {
    size_t t = 0;
    for (size_t b : tc_ws_sizes(ix, qc, cap)) t += (std::max<size_t>(b, 16) + 255) / 256 * 256;
    return t;
}

void tc_ws_assign(TcWs& w, const std::vector<void*>& p, const nrlsh_index* ix, int64_t qc,
                  int64_t cap) {
    w.qnorm = (float*)p[0];
    w.qamb = (unsigned*)p[1];
    w.qamb_list = (unsigned long long*)p[2];
    w.qamb_cap = ambiguity_capacity(qc, ix->L);
    w.qcodes = (char*)p[3];
    w.Qb = (__nv_bfloat16*)p[4];
    w.Qs = (__nv_bfloat16*)p[5];
    w.H = (uint32_t*)p[6];
    w.lam = (uint8_t*)p[7];
    w.off = (uint32_t*)p[8];
    w.tb = (TcBoundary*)p[9];
    w.bnd = (Boundary*)p[10];
    w.flag = (uint8_t*)p[11];
    w.list = (uint32_t*)p[12];
    w.nlist = (uint32_t*)p[13];
    w.cand = (uint32_t*)p[14];
    w.lo = (float*)p[15];
    w.hi = (float*)p[16];
    w.cont = (uint32_t*)p[17];
    w.cont_s = (double*)p[18];
    w.err = (int*)p[19];
    w.qce = (float*)p[20];
    w.qc = qc;
    w.cap = cap;
}

nrlsh_status tc_ws_scratch(Scratch& sc, TcWs& w, const nrlsh_index* ix, int64_t qc, int64_t cap) {
    std::vector<void*> p;
    for (size_t b : tc_ws_sizes(ix, qc, cap)) {
        char* q = nullptr;
        NRLSH_CKS(sc.get(&q, b));
        p.push_back(q);
    }
    tc_ws_assign(w, p, ix, qc, cap);
    return NRLSH_OK;
}

// Queries per chunk of the tensor-core path: the chunk's workspace within an eighth
// of the device's memory, at most 32 GiB (a fixed function of the device, so that
// the workspace a call sizes and the chunks it runs always agree).  Fewer, larger
// chunks leave less of each kernel's last wave idle.
int64_t tc_chunk(const nrlsh_index* ix, int64_t nq, int64_t cap) {
    static const int64_t budget = [] {
        size_t fr = 0, total = 0;
        if (cudaMemGetInfo(&fr, &total) != cudaSuccess) {
            cudaGetLastError();
            total = (size_t)64 << 30;
        }
        return std::max<int64_t>((int64_t)1 << 30, std::min<int64_t>((int64_t)32 << 30, (int64_t)(total / 8)));
    }();
    const int64_t per = (int64_t)tc_ws_bytes(ix, 128, cap) / 128 + 1;
    int64_t c = std::max<int64_t>(128, budget / per);
    return std::min<int64_t>(c, std::max<int64_t>(nq, 1));
}

bool tc_path_supported(const nrlsh_index* ix) { return tc_query_supported(ix->d, ix->L); }

// The index's tensor-path operands (the sign matrix of the codes, the bf16 copy
// of fp32 items), made on the first call on stream st: later calls on other
// streams wait for them (not during a stream capture, which must come after
// the first call).
nrlsh_status ensure_tc_items(const nrlsh_index* ix, cudaStream_t st, bool capturing) {
    std::lock_guard<std::mutex> g(ix->tc_mu);
    if (ix->tc_xs) {
        if (!capturing) NRLSH_CK(cudaStreamWaitEvent(st, ix->tc_ready, 0));
        return NRLSH_OK;
    }
    if (capturing) {
        set_error("the first tensor-core query on an index must come before any stream capture");
        return NRLSH_ERR_UNSUPPORTED;
    }
    void* xs = nullptr;
    void* xb = nullptr;
    NRLSH_CK(cudaMallocAsync(&xs, (size_t)ix->n * 64 * 2, st));
    ix->tc_owned.push_back(xs);
    if (ix->dtype == NRLSH_F32 && !ix->Xb) {
        NRLSH_CK(cudaMallocAsync(&xb, (size_t)ix->n * ix->dp * 2, st));
        ix->tc_owned.push_back(xb);
    }
    NRLSH_CK(launch_item_signs(ix->codes, ix->code_bytes, ix->n, ix->L, (__nv_bfloat16*)xs, st));
    if (xb) NRLSH_CK(launch_to_bf16((const float*)ix->Xp, ix->n * ix->dp, (__nv_bfloat16*)xb, st));
    if (!ix->tc_ready) NRLSH_CK(cudaEventCreateWithFlags(&ix->tc_ready, cudaEventDisableTiming));
    NRLSH_CK(cudaEventRecord(ix->tc_ready, st));
    ix->tc_xs = (__nv_bfloat16*)xs;
    ix->tc_xb = ix->dtype == NRLSH_BF16 ? (__nv_bfloat16*)ix->Xp
                                         : (ix->Xb ? ix->Xb : (__nv_bfloat16*)xb);
    return NRLSH_OK;
}

nrlsh_status cuda_status_ok(cudaError_t e) {
    return e == cudaSuccess ? NRLSH_OK : cuda_status(e, "kernel launch");
}

nrlsh_status tensor_query_prologue(const nrlsh_index* ix, cudaStream_t st) {
    if (!tc_path_supported(ix)) {
        set_error("the tensor-core query path needs an sm_100-family GPU and rows that fit its tiles");
        return NRLSH_ERR_UNSUPPORTED;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st) NRLSH_CK(cudaStreamIsCapturing(st, &cs));
    return ensure_tc_items(ix, st, cs != cudaStreamCaptureStatusNone);
}

// One chunk of queries [0, qc) on the tensor-core path (device pointers): hash,
// histograms (tensor cores when hist_tc, else the popcount kernel with hist_qb
// queries per block), walk with the list offsets, the dense candidate re-rank on
// tensor cores, and the exact top-k.  ks / budgets may be null (one k / budget).
// With H_out the histograms are written there and the chunk stops; with cand_out
// the candidates' ids (grouped by ascending sub-dataset, unordered inside one)
// and their number are written instead of the top-k.
nrlsh_status run_tc_chunk(const nrlsh_index* ix, const float* Q, int64_t qc, const int32_t* ks,
                          int k, const int64_t* budgets, int64_t budget, uint32_t flags,
                          bool hist_tc, int hist_qb, const TcWs& w, int64_t* ids, float* scores,
                          int out_ld, cudaStream_t st, uint32_t* H_out = nullptr,
                          int32_t* cand_out = nullptr, int64_t cand_cap = 0,
                          int64_t* count_out = nullptr) {
    uint32_t* H = H_out ? H_out : w.H;
    const int Kq = 64 * tc_query_k_chunks(ix->d);
    const int nqt = tc_nqt(qc);
    NRLSH_CK(launch_hash_queries(Q, qc, ix->d, ix->L, ix->Lp, ix->A_pad, ix->anorm, w.qnorm,
                                 w.qcodes, ix->code_bytes, w.qamb_list, w.qamb, (unsigned)w.qamb_cap,
                                 ix->At32, st));
    NRLSH_CK(launch_prep_queries(Q, qc, ix->d, Kq, w.qcodes, ix->code_bytes, ix->L, w.Qb, w.Qs,
                                 w.err, w.nlist + 2, st));
    if (hist_tc) {
        NRLSH_CK(launch_pairs_tc(false, w.Qb, w.Qs, qc, ix->tc_xb, ix->tc_xs, ix->n, ix->d, ix->dp,
                                 ix->m, ix->L, ix->seg, nullptr, nullptr, H, nullptr, nullptr,
                                 nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                                 w.err, w.nlist + 2, st, test_spin_first()));
    } else {
        if (!ix->tiles_exclusive)
            NRLSH_CK(cudaMemsetAsync(H, 0, sizeof(uint32_t) * qc * ix->ncls, st));
        NRLSH_CK(launch_hist(ix->codes, w.qcodes, ix->code_bytes, qc, ix->m, ix->L, ix->tiles,
                             ix->ntiles, H, st, hist_qb, ix->tiles_exclusive));
    }
    if (H_out) return cuda_status_ok(launch_report_err(w.err, ix->query_err, st));
    NRLSH_CK(cudaMemsetAsync(w.flag, 0, (size_t)ix->m * nqt, st));
    NRLSH_CK(launch_tc_walk(H, ix->order, ix->m, ix->L, ix->n, ix->seg, qc, budget, budgets, w.cap,
                            flags, ix->codes, w.qcodes, ix->code_bytes, w.lam, w.off, w.tb, w.bnd,
                            w.flag, nqt, w.err, st));
    NRLSH_CK(launch_work_list(w.flag, ix->m * nqt, w.list, w.nlist, st));
    NRLSH_CK(launch_query_bounds(Q, qc, ix->d, w.qnorm, ix->dtype == NRLSH_F32, w.qce, st));
    NRLSH_CK(launch_pairs_tc(true, w.Qb, w.Qs, qc, ix->tc_xb, ix->tc_xs, ix->n, ix->d, ix->dp,
                             ix->m, ix->L, ix->seg, w.list, w.nlist, nullptr, w.lam, w.off, w.tb,
                             ix->xnorm, w.qce, w.cand, w.lo, w.hi, w.cap, w.err,
                             w.nlist + 1, st, test_spin_first()));
    // the last kernel skips its work when the call's error word is set and
    // copies that word into the index's
    if (cand_out)
        return cuda_status_ok(launch_cand_to_ids(w.cand, w.cap, w.bnd, ix->perm, qc, cand_out,
                                                 cand_cap, count_out, st, w.err, ix->query_err));
    NRLSH_CK(launch_topk(w.lo, w.hi, w.cand, w.cap, w.bnd, qc, k, ks, ix->Xp, ix->dtype, ix->dp,
                         ix->d, Q, ix->xnorm, w.qnorm, ix->perm, w.cont, w.cont_s, ids, scores,
                         out_ld, st, w.err, ix->query_err));
    return NRLSH_OK;
}

// The query path on tensor cores up to `stage` (TopK, Cand or Hist; outputs as
// for run_queries): chunks of queries, scratch from the pool.
nrlsh_status run_queries_tc(const nrlsh_index* ix, const float* Q, int64_t nq, int32_t k,
                            int64_t budget, uint32_t flags, Stage stage, const QueryOut& o,
                            cudaStream_t st) {
    const bool whole = (flags & NRLSH_WHOLE_BUCKETS) != 0;
    // with whole buckets a query's list can exceed B: room for all n items
    const int64_t cap = stage == Stage::Hist ? 1 : whole ? ix->n : std::min(budget, ix->n);
    const int64_t chunk = tc_chunk(ix, nq, cap);
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t qc = std::min(chunk, nq - q0);
        Scratch sc(st);
        TcWs w;
        NRLSH_CKS(tc_ws_scratch(sc, w, ix, qc, cap));
        const float* Qc = Q + q0 * ix->d;
        const uint32_t fl = flags & NRLSH_WHOLE_BUCKETS;
        if (stage == Stage::Hist) {
            NRLSH_CKS(run_tc_chunk(ix, Qc, qc, nullptr, 1, nullptr, 1, fl, true, 64, w, nullptr,
                                   nullptr, 1, st, o.H + q0 * ix->ncls));
        } else if (stage == Stage::Cand) {
            NRLSH_CKS(run_tc_chunk(ix, Qc, qc, nullptr, 1, nullptr, budget, fl, true, 64, w,
                                   nullptr, nullptr, 1, st, nullptr, o.cand + q0 * o.cand_cap,
                                   o.cand_cap, o.count + q0));
        } else {
            NRLSH_CKS(run_tc_chunk(ix, Qc, qc, nullptr, k, nullptr, budget, fl, true, 64, w,
                                   o.ids + q0 * o.k_ld, o.scores + q0 * o.k_ld, o.k_ld, st));
        }
    }
    return NRLSH_OK;
}

// Multi-table single probe (Algorithm 2) for queries [0, nq): hash, then select
// C(q) and take the exact top-k of its first `cap` items (or, with cand_ids,
// report their ids).  Queries go in chunks whose scratch stays within 1 GiB.
constexpr int64_t kMultitableFusedCap = 4096;

nrlsh_status run_multitable(const nrlsh_index* ix, const float* Q, int64_t nq, int32_t tables,
                            int32_t k, int64_t cap, int64_t* ids, float* scores, int64_t* probed,
                            int32_t* cand_ids, cudaStream_t st) {
    const int64_t per_query = cap * (4 + 4 + 4 + 4 + 8) + ix->code_bytes + 64;
    int64_t chunk = std::max<int64_t>(1, ((int64_t)1 << 30) / per_query);
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(nq, 1));
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t qc = std::min(chunk, nq - q0);
        const float* Qc = Q + q0 * ix->d;
        Scratch sc(st);
        float* qnorm;
        char* qcodes;
        unsigned* qamb;
        unsigned long long* qamb_list;
        const size_t qamb_cap = ambiguity_capacity(qc, ix->L);
        NRLSH_CKS(sc.get(&qnorm, qc));
        NRLSH_CKS(sc.get(&qamb, 1));
        NRLSH_CKS(sc.get(&qamb_list, qamb_cap));
        NRLSH_CKS(sc.get(&qcodes, qc * ix->code_bytes));
        // P(q) = [q; 0] (Eq. 8), hashed by Eq. 4
        NRLSH_CK(launch_hash_queries(Qc, qc, ix->d, ix->L, ix->Lp, ix->A_pad, ix->anorm, qnorm,
                                     qcodes, ix->code_bytes, qamb_list, qamb, (unsigned)qamb_cap, ix->At32, st));
        uint32_t *cand, *cont = nullptr;
        float *lo = nullptr, *hi = nullptr;
        double* cont_s = nullptr;
        NRLSH_CKS(sc.get(&cand, qc * cap));
        if (!cand_ids) {
            NRLSH_CKS(sc.get(&lo, qc * cap));
            NRLSH_CKS(sc.get(&hi, qc * cap));
            NRLSH_CKS(sc.get(&cont, qc * cap));
            NRLSH_CKS(sc.get(&cont_s, qc * cap));
        }
        if (cand_ids || cap <= kMultitableFusedCap) {
            // short lists: selection, re-rank and top-k in one block per query
            NRLSH_CK(launch_multitable(ix->codes, qcodes, ix->code_bytes, ix->n, ix->L, tables,
                                       ix->Xp, ix->dtype, ix->dp, ix->d, Qc, ix->xnorm, qnorm,
                                       ix->perm, k, cand, lo, hi, cont, cont_s, cap, qc,
                                       ids ? ids + q0 * k : nullptr,
                                       scores ? scores + q0 * k : nullptr, k,
                                       probed ? probed + q0 : nullptr,
                                       cand_ids ? cand_ids + q0 * cap : nullptr, cap, st));
            continue;
        }
        // long or uneven lists: the re-rank is spread over all SMs by a work list
        Boundary* bnd;
        int64_t* work_off;
        unsigned long long* work_ctr;
        NRLSH_CKS(sc.get(&bnd, qc));
        NRLSH_CKS(sc.get(&work_off, qc + 1));
        NRLSH_CKS(sc.get(&work_ctr, 1));
        NRLSH_CK(launch_multitable_select(ix->codes, qcodes, ix->code_bytes, ix->n, ix->L, tables,
                                          cand, cap, qc, bnd, probed ? probed + q0 : nullptr, st));
        NRLSH_CK(launch_rerank_work(ix->Xp, ix->dtype, ix->dp, ix->d, Qc, qc, cand, cap, bnd,
                                    work_off, work_ctr, ix->xnorm, qnorm, lo, hi, st));
        NRLSH_CK(launch_topk(lo, hi, cand, cap, bnd, qc, k, nullptr, ix->Xp, ix->dtype, ix->dp,
                             ix->d, Qc, ix->xnorm, qnorm, ix->perm, cont, cont_s, ids + q0 * k,
                             scores + q0 * k, k, st));
    }
    return NRLSH_OK;
}

nrlsh_status check_query_args(const nrlsh_index* ix, const float* Q, int64_t nq) {
    if (!ix) return arg_error("index is NULL");
    if (nq < 0) return arg_error("need nq >= 0");
    if (nq > 0 && !Q) return arg_error("queries is NULL");
    return NRLSH_OK;
}

// Stage host output buffers: returns a device pointer to write into and
// remembers the host destination for the copy back.
struct OutStage {
    void* host = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
};

template <typename T>
nrlsh_status stage_out(Scratch& sc, T* p, size_t count, OutStage& os, T** dev) {
    if (is_device_ptr(p)) {
        *dev = p;
        return NRLSH_OK;
    }
    T* d = nullptr;
    NRLSH_CKS(sc.get(&d, count));
    os.host = p;
    os.dev = d;
    os.bytes = count * sizeof(T);
    *dev = d;
    return NRLSH_OK;
}

nrlsh_status finish_out(cudaStream_t st, std::initializer_list<OutStage*> outs, bool any_host) {
    for (OutStage* o : outs)
        if (o->host) NRLSH_CK(cudaMemcpyAsync(o->host, o->dev, o->bytes, cudaMemcpyDeviceToHost, st));
    if (any_host) NRLSH_CK(cudaStreamSynchronize(st));
    return NRLSH_OK;
}

// The copies of a call's host inputs, queued before the call waits for the build
// (so they do not queue behind it): with device outputs the call returns once they
// have landed, without waiting for its kernels.
struct InputCopies {
    cudaEvent_t ev = nullptr;
    ~InputCopies() {
        if (ev) cudaEventDestroy(ev);
    }
    nrlsh_status mark(cudaStream_t st, bool any_host, uint32_t flags) {
        if (!any_host || (flags & NRLSH_QUERY_ASYNC_INPUT)) return NRLSH_OK;
        NRLSH_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        NRLSH_CK(cudaEventRecord(ev, st));
        return NRLSH_OK;
    }
};

nrlsh_status finish_out(cudaStream_t st, std::initializer_list<OutStage*> outs,
                        const InputCopies& in) {
    bool host_out = false;
    for (OutStage* o : outs) host_out = host_out || o->host;
    if (host_out) return finish_out(st, outs, true);
    if (in.ev) NRLSH_CK(cudaEventSynchronize(in.ev));
    return NRLSH_OK;
}

}  // namespace

// ===================================================================== C ABI

extern "C" {

NRLSH_API nrlsh_status nrlsh_build(const float* items, int64_t n, int32_t d, int32_t m, int32_t L,
                                   uint64_t seed, nrlsh_index** out) {
    return build_impl(items, n, d, m, L, seed, NRLSH_F32, 0.1f, nullptr, NRLSH_PROJECT_AUTO,
                      NRLSH_PARTITION_PERCENTILE, out);
}

NRLSH_API nrlsh_status nrlsh_build_ex(const void* items, int64_t n, int32_t d, int32_t m,
                                      int32_t L, uint64_t seed, nrlsh_dtype dtype, float eps,
                                      void* stream, nrlsh_index** out) {
    return build_impl(items, n, d, m, L, seed, dtype, eps, stream, NRLSH_PROJECT_AUTO,
                      NRLSH_PARTITION_PERCENTILE, out);
}

NRLSH_API nrlsh_status nrlsh_build_opts(const void* items, int64_t n, int32_t d, int32_t m,
                                        int32_t L, uint64_t seed, const nrlsh_build_options* opts,
                                        nrlsh_index** out) {
    if (!opts) return arg_error("opts is NULL");
    if (opts->flags & ~NRLSH_BUILD_ASYNC_INPUT) return arg_error("unknown build flags");
    return build_impl(items, n, d, m, L, seed, (nrlsh_dtype)opts->dtype, opts->eps, opts->stream,
                      opts->projection, opts->partition, out, opts->flags);
}

NRLSH_API nrlsh_status nrlsh_query_ex(const nrlsh_index* ix, const float* queries, int64_t nq,
                                      int32_t k, int64_t probe_budget, uint32_t flags,
                                      int64_t* ids, float* scores, void* stream) {
    NRLSH_CKS(check_query_args(ix, queries, nq));
    if (k < 1 || k > NRLSH_MAX_K) return arg_error("need 1 <= k <= 1024");
    if (probe_budget < 1) return arg_error("need probe_budget >= 1");
    if (flags & ~(NRLSH_WHOLE_BUCKETS | NRLSH_QUERY_TENSOR | NRLSH_QUERY_ASYNC_INPUT))
        return arg_error("unknown flags");
    if (nq > 0 && (!ids || !scores)) return arg_error("ids/scores is NULL");
    const bool tensor = (flags & NRLSH_QUERY_TENSOR) != 0;
    if (tensor && !tc_path_supported(ix)) {
        set_error("the tensor-core query path needs an sm_100-family GPU and rows that fit its tiles");
        return NRLSH_ERR_UNSUPPORTED;
    }
    if (nq == 0) return NRLSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    Scratch sc(st);
    const void* Qd;
    NRLSH_CKS(stage_in(sc, queries, sizeof(float) * nq * ix->d, &Qd));
    InputCopies in;
    NRLSH_CKS(in.mark(st, Qd != queries, flags));
    NRLSH_CK(wait_for_build(ix, st));
    if (tensor) NRLSH_CKS(tensor_query_prologue(ix, st));
    OutStage oi, os;
    QueryOut o;
    NRLSH_CKS(stage_out(sc, ids, (size_t)nq * k, oi, &o.ids));
    NRLSH_CKS(stage_out(sc, scores, (size_t)nq * k, os, &o.scores));
    o.k_ld = k;
    if (tensor)
        NRLSH_CKS(run_queries_tc(ix, (const float*)Qd, nq, k, probe_budget, flags, Stage::TopK, o, st));
    else
        NRLSH_CKS(run_queries(ix, (const float*)Qd, nq, k, probe_budget, flags, Stage::TopK, o, st));
    return finish_out(st, {&oi, &os}, in);
}

NRLSH_API nrlsh_status nrlsh_query(const nrlsh_index* ix, const float* queries, int64_t nq,
                                   int32_t k, int64_t probe_budget, int64_t* ids, float* scores) {
    return nrlsh_query_ex(ix, queries, nq, k, probe_budget, 0u, ids, scores, nullptr);
}

NRLSH_API nrlsh_status nrlsh_hash_queries(const nrlsh_index* ix, const float* queries, int64_t nq,
                                          uint64_t* codes, void* stream) {
    NRLSH_CKS(check_query_args(ix, queries, nq));
    if (nq > 0 && !codes) return arg_error("codes is NULL");
    if (nq == 0) return NRLSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    NRLSH_CK(wait_for_build(ix, st));
    Scratch sc(st);
    const void* Qd;
    NRLSH_CKS(stage_in(sc, queries, sizeof(float) * nq * ix->d, &Qd));
    OutStage oc;
    QueryOut o;
    NRLSH_CKS(stage_out(sc, codes, (size_t)nq, oc, &o.codes));
    NRLSH_CKS(run_queries(ix, (const float*)Qd, nq, 1, 1, 0u, Stage::Hash, o, st));
    return finish_out(st, {&oc}, oc.host || Qd != queries);
}

NRLSH_API nrlsh_status nrlsh_query_histograms(const nrlsh_index* ix, const float* queries,
                                              int64_t nq, uint32_t* H, uint32_t flags,
                                              void* stream) {
    NRLSH_CKS(check_query_args(ix, queries, nq));
    if (nq > 0 && !H) return arg_error("H is NULL");
    if (flags & ~NRLSH_QUERY_TENSOR) return arg_error("unknown flags");
    if (nq == 0) return NRLSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    NRLSH_CK(wait_for_build(ix, st));
    const bool tensor = (flags & NRLSH_QUERY_TENSOR) != 0;
    if (tensor) NRLSH_CKS(tensor_query_prologue(ix, st));
    Scratch sc(st);
    const void* Qd;
    NRLSH_CKS(stage_in(sc, queries, sizeof(float) * nq * ix->d, &Qd));
    OutStage oh;
    QueryOut o;
    NRLSH_CKS(stage_out(sc, H, (size_t)nq * ix->ncls, oh, &o.H));
    if (tensor)
        NRLSH_CKS(run_queries_tc(ix, (const float*)Qd, nq, 1, 1, 0u, Stage::Hist, o, st));
    else
        NRLSH_CKS(run_queries(ix, (const float*)Qd, nq, 1, 1, 0u, Stage::Hist, o, st));
    return finish_out(st, {&oh}, oh.host || Qd != queries);
}

NRLSH_API nrlsh_status nrlsh_query_multitable(const nrlsh_index* ix, const float* queries,
                                              int64_t nq, int32_t tables, int32_t k,
                                              int64_t max_candidates, int64_t* ids,
                                              float* scores, int64_t* probed, void* stream) {
    NRLSH_CKS(check_query_args(ix, queries, nq));
    if (tables < 1 || tables > ix->L || ix->L % tables != 0)
        return arg_error("need 1 <= tables <= L with L % tables == 0");
    if (k < 1 || k > NRLSH_MAX_K) return arg_error("need 1 <= k <= 1024");
    if (max_candidates < 0) return arg_error("need max_candidates >= 0");
    if (nq > 0 && (!ids || !scores)) return arg_error("ids/scores is NULL");
    if (nq == 0) return NRLSH_OK;
    const int64_t cap = max_candidates == 0 ? ix->n : std::min(max_candidates, ix->n);
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    NRLSH_CK(wait_for_build(ix, st));
    Scratch sc(st);
    const void* Qd;
    NRLSH_CKS(stage_in(sc, queries, sizeof(float) * nq * ix->d, &Qd));
    OutStage oi, os, op;
    int64_t* di;
    float* ds;
    int64_t* dp = nullptr;
    NRLSH_CKS(stage_out(sc, ids, (size_t)(nq * k), oi, &di));
    NRLSH_CKS(stage_out(sc, scores, (size_t)(nq * k), os, &ds));
    if (probed) NRLSH_CKS(stage_out(sc, probed, (size_t)nq, op, &dp));
    NRLSH_CKS(run_multitable(ix, (const float*)Qd, nq, tables, k, cap, di, ds, dp, nullptr, st));
    return finish_out(st, {&oi, &os, &op}, oi.host || os.host || op.host);
}

NRLSH_API nrlsh_status nrlsh_multitable_candidates(const nrlsh_index* ix, const float* queries,
                                                   int64_t nq, int32_t tables, int64_t cap,
                                                   int32_t* cand, int64_t* count, void* stream) {
    NRLSH_CKS(check_query_args(ix, queries, nq));
    if (tables < 1 || tables > ix->L || ix->L % tables != 0)
        return arg_error("need 1 <= tables <= L with L % tables == 0");
    if (cap < 1) return arg_error("need cap >= 1");
    if (nq > 0 && (!cand || !count)) return arg_error("cand/count is NULL");
    if (nq == 0) return NRLSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    NRLSH_CK(wait_for_build(ix, st));
    Scratch sc(st);
    const void* Qd;
    NRLSH_CKS(stage_in(sc, queries, sizeof(float) * nq * ix->d, &Qd));
    OutStage oc, on;
    int32_t* dc;
    int64_t* dn;
    NRLSH_CKS(stage_out(sc, cand, (size_t)(nq * cap), oc, &dc));
    NRLSH_CKS(stage_out(sc, count, (size_t)nq, on, &dn));
    NRLSH_CKS(run_multitable(ix, (const float*)Qd, nq, tables, 1, cap, nullptr, nullptr, dn, dc,
                             st));
    return finish_out(st, {&oc, &on}, oc.host || on.host);
}

NRLSH_API nrlsh_status nrlsh_query_candidates(const nrlsh_index* ix, const float* queries,
                                              int64_t nq, int64_t probe_budget, uint32_t flags,
                                              int64_t cap, int32_t* cand, int64_t* count,
                                              void* stream) {
    NRLSH_CKS(check_query_args(ix, queries, nq));
    if (probe_budget < 1) return arg_error("need probe_budget >= 1");
    if (cap < 1) return arg_error("need cap >= 1");
    if (flags & ~(NRLSH_WHOLE_BUCKETS | NRLSH_QUERY_TENSOR)) return arg_error("unknown flags");
    if (nq > 0 && (!cand || !count)) return arg_error("cand/count is NULL");
    if (nq == 0) return NRLSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    NRLSH_CK(wait_for_build(ix, st));
    const bool tensor = (flags & NRLSH_QUERY_TENSOR) != 0;
    if (tensor) NRLSH_CKS(tensor_query_prologue(ix, st));
    Scratch sc(st);
    const void* Qd;
    NRLSH_CKS(stage_in(sc, queries, sizeof(float) * nq * ix->d, &Qd));
    OutStage oc, on;
    QueryOut o;
    NRLSH_CKS(stage_out(sc, cand, (size_t)(nq * cap), oc, &o.cand));
    NRLSH_CKS(stage_out(sc, count, (size_t)nq, on, &o.count));
    o.cand_cap = cap;
    if (tensor)
        NRLSH_CKS(run_queries_tc(ix, (const float*)Qd, nq, 1, probe_budget, flags, Stage::Cand, o, st));
    else
        NRLSH_CKS(run_queries(ix, (const float*)Qd, nq, 1, probe_budget, flags, Stage::Cand, o, st));
    NRLSH_CKS(finish_out(st, {&oc, &on}, true));
    // counts are needed on the host to report an overflow of `cap`
    std::vector<int64_t> hc(nq);
    const int64_t* cnt = on.host ? (const int64_t*)on.host : nullptr;
    if (!cnt) {
        NRLSH_CK(cudaMemcpy(hc.data(), count, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost));
        cnt = hc.data();
    }
    for (int64_t i = 0; i < nq; ++i)
        if (cnt[i] > cap) return arg_error("a query has more candidates than cap");
    return NRLSH_OK;
}

NRLSH_API nrlsh_status nrlsh_get_codes(const nrlsh_index* ix, uint64_t* codes) {
    if (!ix || !codes) return arg_error("NULL argument");
    NRLSH_CK(cudaStreamSynchronize(ix->stream));
    int derr = 0;
    NRLSH_CK(cudaMemcpy(&derr, ix->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (derr) {
        set_error("a bounded device wait of the index build ran out: its codes are incomplete");
        return NRLSH_ERR_TIMEOUT;
    }
    const int64_t n = ix->n;
    std::vector<uint32_t> perm(n);
    std::vector<unsigned char> raw((size_t)n * ix->code_bytes);
    NRLSH_CK(cudaMemcpy(perm.data(), ix->perm, 4 * n, cudaMemcpyDeviceToHost));
    NRLSH_CK(cudaMemcpy(raw.data(), ix->codes, raw.size(), cudaMemcpyDeviceToHost));
    for (int64_t p = 0; p < n; ++p) {
        uint64_t c = 0;
        if (ix->code_bytes == 4) {
            uint32_t v;
            std::memcpy(&v, raw.data() + 4 * p, 4);
            c = v;
        } else {
            std::memcpy(&c, raw.data() + 8 * p, 8);
        }
        codes[perm[p]] = c;
    }
    return NRLSH_OK;
}

NRLSH_API nrlsh_status nrlsh_get_partition(const nrlsh_index* ix, int32_t* sub_of_id, double* U2,
                                           double* sqnorm) {
    if (!ix) return arg_error("index is NULL");
    NRLSH_CK(cudaStreamSynchronize(ix->stream));
    if (sub_of_id)
        NRLSH_CK(cudaMemcpy(sub_of_id, ix->sub_of_id, 4 * ix->n, cudaMemcpyDeviceToHost));
    if (U2) NRLSH_CK(cudaMemcpy(U2, ix->U2, 8 * ix->m, cudaMemcpyDeviceToHost));
    if (sqnorm) NRLSH_CK(cudaMemcpy(sqnorm, ix->s_id, 8 * ix->n, cudaMemcpyDeviceToHost));
    return NRLSH_OK;
}

NRLSH_API nrlsh_status nrlsh_get_segments(const nrlsh_index* ix, int64_t* seg) {
    if (!ix || !seg) return arg_error("NULL argument");
    NRLSH_CK(cudaStreamSynchronize(ix->stream));
    NRLSH_CK(cudaMemcpy(seg, ix->seg, sizeof(int64_t) * (ix->m + 1), cudaMemcpyDeviceToHost));
    return NRLSH_OK;
}

NRLSH_API nrlsh_status nrlsh_get_projections(const nrlsh_index* ix, float* A) {
    if (!ix || !A) return arg_error("NULL argument");
    NRLSH_CK(cudaStreamSynchronize(ix->stream));
    NRLSH_CK(cudaMemcpy(A, ix->A, sizeof(float) * (ix->d + 1) * ix->L, cudaMemcpyDeviceToHost));
    return NRLSH_OK;
}

NRLSH_API nrlsh_status nrlsh_get_buckets(const nrlsh_index* ix, int32_t* bucket_j,
                                         int32_t* bucket_l, double* s_hat) {
    if (!ix) return arg_error("index is NULL");
    NRLSH_CK(cudaStreamSynchronize(ix->stream));
    std::vector<uint32_t> ord(ix->ncls);
    NRLSH_CK(cudaMemcpy(ord.data(), ix->order, 4 * ix->ncls, cudaMemcpyDeviceToHost));
    for (int i = 0; i < ix->ncls; ++i) {
        if (bucket_j) bucket_j[i] = (int32_t)(ord[i] / (ix->L + 1));
        if (bucket_l) bucket_l[i] = (int32_t)(ord[i] % (ix->L + 1));
    }
    if (s_hat)
        NRLSH_CK(cudaMemcpy(s_hat, ix->shat_sorted, 8 * ix->ncls, cudaMemcpyDeviceToHost));
    return NRLSH_OK;
}

NRLSH_API nrlsh_status nrlsh_get_info(const nrlsh_index* ix, nrlsh_info* info) {
    if (!ix || !info) return arg_error("NULL argument");
    NRLSH_CK(cudaStreamSynchronize(ix->stream));
    unsigned amb = 0;
    NRLSH_CK(cudaMemcpy(&amb, ix->ambiguous, sizeof(amb), cudaMemcpyDeviceToHost));
    info->n = ix->n;
    info->d = ix->d;
    info->m = ix->m;
    info->L = ix->L;
    info->dtype = ix->dtype;
    info->eps = ix->eps;
    info->seed = ix->seed;
    info->code_bytes = ix->code_bytes;
    info->row_stride = ix->dp;
    info->device_bytes = ix->device_bytes;
    info->ambiguous_bits = (int64_t)amb;
    int derr = 0;
    NRLSH_CK(cudaMemcpy(&derr, ix->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    info->projection = ix->projection;
    info->device_error = derr;
    info->partition = ix->partition;
    unsigned nfb = 0;
    NRLSH_CK(cudaMemcpy(&nfb, ix->norm_fb, sizeof(nfb), cudaMemcpyDeviceToHost));
    info->norm_fallbacks = (int32_t)nfb;
    int qerr = 0;
    NRLSH_CK(cudaMemcpy(&qerr, ix->query_err, sizeof(int), cudaMemcpyDeviceToHost));
    info->query_error = qerr;
    // the statistics are filled either way; the status reports what went wrong
    if (derr) {
        set_error("a bounded device wait of the index build ran out (code " +
                  std::to_string(derr) + "): its codes are incomplete");
        return NRLSH_ERR_TIMEOUT;
    }
    if (qerr == 15) {
        set_error("a tensor-core query kernel found other candidates than it counted");
        return NRLSH_ERR_CUDA;
    }
    if (qerr) {
        set_error("a bounded device wait of a tensor-core query kernel ran out (code " +
                  std::to_string(qerr) + "): that call's results are invalid");
        return NRLSH_ERR_TIMEOUT;
    }
    return NRLSH_OK;
}

NRLSH_API void nrlsh_free(nrlsh_index* ix) { destroy(ix); }

NRLSH_API const char* nrlsh_last_error(void) { return g_last_error.c_str(); }

NRLSH_API uint64_t nrlsh_launch_count(void) { return g_launches.load(); }

}  // extern "C"

namespace {

// Every thread reads 16-byte words of the buffer, grid-strided, `reps` times, from
// L2 (ld.global.cg); the folded words are written only if they match an
// impossible value, which keeps the loads.
__global__ void __launch_bounds__(256) read_probe_kernel(const uint4* __restrict__ buf, int64_t words,
                                                         int reps, uint32_t* __restrict__ sink) {
    NRLSH_PDL_ENTRY();
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = i + u * stride;
                v[u] = k < words ? __ldcg(buf + k) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
        acc = acc * 2654435761u + (uint32_t)r;
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;
}

}  // namespace

extern "C" {

NRLSH_API nrlsh_status nrlsh_read_bandwidth(const void* buf, int64_t bytes, int32_t reps,
                                            void* stream, double* gbps) {
    if (!buf || !gbps) return arg_error("NULL argument");
    if (bytes < 16 || bytes % 16 != 0) return arg_error("need bytes >= 16, a multiple of 16");
    if (((uintptr_t)buf & 15) != 0) return arg_error("buf must be 16-byte aligned");
    if (reps < 1) return arg_error("need reps >= 1");
    if (!is_device_ptr(buf)) return arg_error("buf must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    int dev = 0, sms = 0;
    NRLSH_CK(cudaGetDevice(&dev));
    NRLSH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    Scratch sc(st);
    uint32_t* sink;
    NRLSH_CKS(sc.get(&sink, 1));
    const dim3 grid((unsigned)(sms * 8));
    // one untimed pass brings an L2-sized buffer into L2
    NRLSH_CK(launch("read_probe", read_probe_kernel, grid, dim3(256), 0, st, (const uint4*)buf,
                    bytes / 16, 1, sink));
    cudaEvent_t e0, e1;
    NRLSH_CK(cudaEventCreate(&e0));
    NRLSH_CK(cudaEventCreate(&e1));
    NRLSH_CK(cudaEventRecord(e0, st));
    const cudaError_t le = launch("read_probe", read_probe_kernel, grid, dim3(256), 0, st,
                                  (const uint4*)buf, bytes / 16, (int)reps, sink);
    NRLSH_CK(cudaEventRecord(e1, st));
    NRLSH_CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    NRLSH_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    NRLSH_CK(le);
    *gbps = (double)bytes * reps / (ms * 1e-3) / 1e9;
    return NRLSH_OK;
}

NRLSH_API nrlsh_status nrlsh_set_profiling(int32_t enable) {
    g_prof_on.store(enable != 0);
    return NRLSH_OK;
}

NRLSH_API nrlsh_status nrlsh_profile_read(char* names, int64_t names_cap, double* ms,
                                          int64_t* launches, int32_t cap, int32_t* count) {
    std::vector<ProfRecord> recs;
    {
        std::lock_guard<std::mutex> g(g_prof_mu);
        recs.swap(g_prof);
    }
    std::map<std::string, std::pair<double, int64_t>> agg;
    std::vector<std::string> order;
    for (auto& r : recs) {
        NRLSH_CK(cudaEventSynchronize(r.b));
        float t = 0.f;
        NRLSH_CK(cudaEventElapsedTime(&t, r.a, r.b));
        auto it = agg.find(r.name);
        if (it == agg.end()) {
            order.push_back(r.name);
            agg[r.name] = {t, 1};
        } else {
            it->second.first += t;
            it->second.second += 1;
        }
    }
    {
        std::lock_guard<std::mutex> g(g_prof_mu);
        for (auto& r : recs) {
            g_event_pool.push_back(r.a);
            g_event_pool.push_back(r.b);
        }
    }
    std::string all;
    int32_t i = 0;
    for (auto& nm : order) {
        if (i < cap) {
            if (ms) ms[i] = agg[nm].first;
            if (launches) launches[i] = agg[nm].second;
        }
        all += nm;
        all += '\n';
        ++i;
    }
    if (count) *count = (int32_t)order.size();
    if (names && names_cap > 0) {
        const size_t nb = std::min<size_t>(all.size(), (size_t)names_cap - 1);
        std::memcpy(names, all.data(), nb);
        names[nb] = 0;
    }
    return NRLSH_OK;
}

}  // extern "C"


// ------------------------------------------------------------- batched queries

namespace {

struct BatchWs {
    float* qnorm = nullptr;
    unsigned* qamb = nullptr;
    unsigned long long* qamb_list = nullptr;
    size_t qamb_cap = 0;
    char* qcodes = nullptr;
    uint32_t* H = nullptr;
    int64_t hq = 0;           // queries per histogram chunk
    unsigned* work = nullptr;
    uint32_t* slabs = nullptr;
    int ctas = 0;
};

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Persistent CTAs for a configuration, limited so the slabs stay under 4 GB.
int batch_ctas(const nrlsh_batch_cfg& cfg, int64_t cap) {
    const int64_t by_mem = std::max<int64_t>(1, ((int64_t)4 << 30) / (24 * cap));
    return (int)std::min<int64_t>((int64_t)cfg.ctas_per_sm * device_sms(), by_mem);
}

// Sizes of the workspace buffers (bytes), in BatchWs order.
std::vector<size_t> batch_ws_sizes(const nrlsh_index* ix, int64_t nq, int64_t cap, int ctas) {
    const int64_t hq = std::min<int64_t>(nq, std::max<int64_t>(1, ((int64_t)1 << 30) / (ix->ncls * 4)));
    return {sizeof(float) * (size_t)nq, 16, sizeof(unsigned long long) * ambiguity_capacity(nq, ix->L),
            (size_t)ix->code_bytes * nq, sizeof(uint32_t) * (size_t)hq * ix->ncls, 16,
            (size_t)ctas * 24 * (size_t)cap};
}

void batch_ws_assign(BatchWs& w, const std::vector<void*>& p, const nrlsh_index* ix, int64_t nq,
                     int ctas) {
    w.qnorm = (float*)p[0];
    w.qamb = (unsigned*)p[1];
    w.qamb_list = (unsigned long long*)p[2];
    w.qamb_cap = ambiguity_capacity(nq, ix->L);
    w.qcodes = (char*)p[3];
    w.H = (uint32_t*)p[4];
    w.hq = std::min<int64_t>(nq, std::max<int64_t>(1, ((int64_t)1 << 30) / (ix->ncls * 4)));
    w.work = (unsigned*)p[5];
    w.slabs = (uint32_t*)p[6];
    w.ctas = ctas;
}

// Workspace buffers of a configuration: the persistent FP32 path's, or one chunk
// of the tensor-core path's.
std::vector<size_t> cfg_ws_sizes(const nrlsh_index* ix, const nrlsh_batch_cfg& cfg, int64_t nq,
                                 int64_t cap) {
    if (cfg.rerank_tc) return tc_ws_sizes(ix, tc_chunk(ix, nq, cap), cap);
    return batch_ws_sizes(ix, nq, cap, batch_ctas(cfg, cap));
}

// The launch sequence of a batch (device pointers only) in workspace p.
nrlsh_status run_batched(const nrlsh_index* ix, const float* Q, int64_t nq, const int32_t* ks,
                         const int64_t* budgets, int k_max, int64_t cap, const nrlsh_batch_cfg& cfg,
                         const std::vector<void*>& p, int64_t* ids, float* scores, cudaStream_t st) {
    if (cfg.rerank_tc) {
        const int64_t chunk = tc_chunk(ix, nq, cap);
        TcWs w;
        tc_ws_assign(w, p, ix, chunk, cap);
        for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
            const int64_t qc = std::min(chunk, nq - q0);
            NRLSH_CKS(run_tc_chunk(ix, Q + q0 * ix->d, qc, ks + q0, k_max, budgets + q0, 0, 0u,
                                   cfg.hist_tc != 0, cfg.hist_qb, w, ids + q0 * k_max,
                                   scores + q0 * k_max, k_max, st));
        }
        return NRLSH_OK;
    }
    BatchWs w;
    batch_ws_assign(w, p, ix, nq, batch_ctas(cfg, cap));
    const __nv_bfloat16* xr16 = cfg.rows_bf16 && ix->dtype == NRLSH_F32 ? ix->tc_xb : nullptr;
    NRLSH_CK(launch_hash_queries(Q, nq, ix->d, ix->L, ix->Lp, ix->A_pad, ix->anorm, w.qnorm,
                                 w.qcodes, ix->code_bytes, w.qamb_list, w.qamb,
                                 (unsigned)w.qamb_cap, ix->At32, st));
    for (int64_t q0 = 0; q0 < nq; q0 += w.hq) {
        const int64_t qc = std::min(w.hq, nq - q0);
        const char* qcodes = w.qcodes + q0 * ix->code_bytes;
        if (!ix->tiles_exclusive)
            NRLSH_CK(cudaMemsetAsync(w.H, 0, sizeof(uint32_t) * qc * ix->ncls, st));
        NRLSH_CK(launch_hist(ix->codes, qcodes, ix->code_bytes, qc, ix->m, ix->L, ix->tiles,
                             ix->ntiles, w.H, st, cfg.hist_qb, ix->tiles_exclusive));
        NRLSH_CK(cudaMemsetAsync(w.work, 0, sizeof(unsigned), st));
        NRLSH_CK(launch_probe_rerank_persistent(
            w.H, ix->order, ix->m, ix->L, ix->n, ix->seg, 0, budgets + q0, ix->codes, qcodes,
            ix->code_bytes,
            ix->Xp, ix->dtype, ix->dp, ix->d, Q + q0 * ix->d, ix->xnorm, w.qnorm + q0, ix->perm,
            ks + q0, k_max, w.slabs, cap, w.ctas, w.work, qc, ids + q0 * k_max,
            scores + q0 * k_max, st, xr16));
    }
    return NRLSH_OK;
}

nrlsh_status check_batch_flags(uint32_t flags) {
    const uint32_t path = NRLSH_QUERY_TENSOR | NRLSH_QUERY_FP32 | NRLSH_QUERY_BF16;
    if (flags & ~(NRLSH_QUERY_GRAPH | NRLSH_QUERY_NO_TUNE | NRLSH_QUERY_ASYNC_INPUT | path))
        return arg_error("unknown flags");
    const uint32_t p = flags & path;
    if (p & (p - 1))
        return arg_error("NRLSH_QUERY_TENSOR, NRLSH_QUERY_FP32 and NRLSH_QUERY_BF16 exclude each other");
    return NRLSH_OK;
}

// Which paths a batched call may use: 0 any (autotuned), 1 tensor cores only,
// 2 the FP32 re-rank over the stored rows only, 3 bf16 operands only (tensor
// cores, or the FP32 re-rank over bf16 rows).
int batch_mode(uint32_t flags) {
    return (flags & NRLSH_QUERY_TENSOR) ? 1
           : (flags & NRLSH_QUERY_FP32) ? 2
           : (flags & NRLSH_QUERY_BF16) ? 3
                                        : 0;
}

// bf16 copies of the rows exist (or can be made) for this index.
bool bf16_rows_ok(const nrlsh_index* ix) {
    return ix->dtype == NRLSH_BF16 || tc_path_supported(ix);
}

// Whether a configuration belongs to the paths `mode` allows.
bool cfg_allowed(const nrlsh_index* ix, int mode, const nrlsh_batch_cfg& c) {
    switch (mode) {
        case 1: return c.rerank_tc != 0;
        case 2: return !c.rerank_tc && !c.rows_bf16;
        case 3: return c.rerank_tc || c.rows_bf16 || ix->dtype == NRLSH_BF16;
        default: return true;
    }
}

// A path's configuration when nothing was tuned for it.
nrlsh_batch_cfg default_cfg(const nrlsh_index* ix, int mode) {
    nrlsh_batch_cfg c;
    if (mode == 1) c.rerank_tc = c.hist_tc = 1;
    if (mode == 3 && ix->dtype == NRLSH_F32) c.rows_bf16 = 1;
    return c;
}

// The autotuner's results, shared by every index of the process: a configuration
// depends on the device, the index's shape and the batch's sizes, not on the
// values, so a rebuilt index of the same shape reuses it.
using TuneKey = std::tuple<int, int64_t, int, int, int, int, int, uint32_t, int64_t, int, int64_t, int>;
std::mutex g_tune_mu;
std::map<TuneKey, nrlsh_batch_cfg> g_tuned;

TuneKey tune_key(const nrlsh_index* ix, int64_t nq, int k_max, int64_t cap, int mode) {
    int dev = 0;
    cudaGetDevice(&dev);
    uint32_t eb;
    std::memcpy(&eb, &ix->eps, 4);
    return TuneKey(dev, ix->n, ix->d, ix->m, ix->L, (int)ix->dtype, ix->code_bytes, eb, nq, k_max,
                   cap, mode);
}

// Time the candidate configurations on a prefix of the batch; keep the fastest.
// FP32 re-rank: the popcount histogram's query tile (32, 64, 128) and the
// persistent re-rank's CTAs per SM (1, 2, 4), over the stored rows or (fp32
// items) their bf16 copy.  Tensor-core path: histograms on tensor cores or by
// popcount (best tile), candidates and scores on tensor cores.
nrlsh_status autotune(const nrlsh_index* ix, const float* Q, int64_t nq, const int32_t* ks,
                      const int64_t* budgets, int k_max, int64_t cap, int mode, int64_t* ids,
                      float* scores, cudaStream_t st, nrlsh_batch_cfg* best) {
    const int64_t nt = std::min<int64_t>(nq, 2048);
    cudaEvent_t e0, e1;
    NRLSH_CK(cudaEventCreate(&e0));
    NRLSH_CK(cudaEventCreate(&e1));
    auto time_cfg = [&](const nrlsh_batch_cfg& c, float* ms) -> nrlsh_status {
        Scratch sc(st);
        std::vector<void*> p;
        for (size_t b : cfg_ws_sizes(ix, c, nt, cap)) {
            char* q = nullptr;
            NRLSH_CKS(sc.get(&q, b));
            p.push_back(q);
        }
        NRLSH_CKS(run_batched(ix, Q, nt, ks, budgets, k_max, cap, c, p, ids, scores, st));  // warm
        NRLSH_CK(cudaEventRecord(e0, st));
        NRLSH_CKS(run_batched(ix, Q, nt, ks, budgets, k_max, cap, c, p, ids, scores, st));
        NRLSH_CK(cudaEventRecord(e1, st));
        NRLSH_CK(cudaEventSynchronize(e1));
        NRLSH_CK(cudaEventElapsedTime(ms, e0, e1));
        return NRLSH_OK;
    };
    float best_ms = 1e30f;
    auto consider = [&](const nrlsh_batch_cfg& c) -> nrlsh_status {
        float ms;
        NRLSH_CKS(time_cfg(c, &ms));
        if (ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
        return NRLSH_OK;
    };
    nrlsh_batch_cfg c;
    int best_qb = 64;
    // the re-rank's row copy the tile sweep runs with
    const int rb = mode == 3 && ix->dtype == NRLSH_F32 ? 1 : 0;
    {
        // the popcount histogram's tile (FP32 re-rank at 2 CTAs per SM)
        float qb_ms = 1e30f;
        for (int qb : {32, 64, 128}) {
            c = nrlsh_batch_cfg{};
            c.hist_qb = qb;
            c.ctas_per_sm = 2;
            c.rows_bf16 = rb;
            float ms;
            NRLSH_CKS(time_cfg(c, &ms));
            if (ms < qb_ms) {
                qb_ms = ms;
                best_qb = qb;
            }
            if (mode != 1 && ms < best_ms) {
                best_ms = ms;
                *best = c;
            }
        }
    }
    if (mode != 1) {
        for (int cps : {1, 4}) {
            c = nrlsh_batch_cfg{};
            c.hist_qb = best_qb;
            c.ctas_per_sm = cps;
            c.rows_bf16 = rb;
            NRLSH_CKS(consider(c));
        }
    }
    if (mode == 0 && ix->dtype == NRLSH_F32 && bf16_rows_ok(ix)) {
        for (int cps : {2, 4}) {
            c = nrlsh_batch_cfg{};
            c.hist_qb = best_qb;
            c.ctas_per_sm = cps;
            c.rows_bf16 = 1;
            NRLSH_CKS(consider(c));
        }
    }
    if ((mode == 0 || mode == 1 || mode == 3) && tc_path_supported(ix)) {
        for (int htc : {1, 0}) {
            c = nrlsh_batch_cfg{};
            c.hist_qb = best_qb;
            c.rerank_tc = 1;
            c.hist_tc = htc;
            NRLSH_CKS(consider(c));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return NRLSH_OK;
}

}  // namespace

extern "C" NRLSH_API nrlsh_status nrlsh_query_batched(const nrlsh_index* ix, const float* queries,
                                                      int64_t nq, const int32_t* ks,
                                                      const int64_t* budgets, int32_t k_max,
                                                      int64_t budget_max, uint32_t flags,
                                                      int64_t* ids, float* scores, void* stream) {
    NRLSH_CKS(check_query_args(ix, queries, nq));
    if (k_max < 1 || k_max > NRLSH_MAX_K) return arg_error("need 1 <= k_max <= 1024");
    if (budget_max < 1) return arg_error("need budget_max >= 1");
    NRLSH_CKS(check_batch_flags(flags));
    if (nq > 0 && (!ids || !scores || !ks || !budgets)) return arg_error("NULL array");
    const int mode = batch_mode(flags);
    if (mode == 1 && !tc_path_supported(ix)) {
        set_error("the tensor-core query path needs an sm_100-family GPU and rows that fit its tiles");
        return NRLSH_ERR_UNSUPPORTED;
    }
    if (mode == 3 && !bf16_rows_ok(ix)) {
        set_error("the bf16 query paths need an sm_100-family GPU and rows that fit its tiles");
        return NRLSH_ERR_UNSUPPORTED;
    }
    if (nq == 0) return NRLSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    const int64_t cap = std::min<int64_t>(budget_max, ix->n);
    const bool graph = (flags & NRLSH_QUERY_GRAPH) && st != nullptr;
    if (graph && !(is_device_ptr(queries) && is_device_ptr(ks) && is_device_ptr(budgets) &&
                   is_device_ptr(ids) && is_device_ptr(scores)))
        return arg_error("NRLSH_QUERY_GRAPH needs device pointers");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st) NRLSH_CK(cudaStreamIsCapturing(st, &cs));
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    Scratch sc(st);
    const void *Qd, *ksd, *bd;
    NRLSH_CKS(stage_in(sc, queries, sizeof(float) * nq * ix->d, &Qd));
    NRLSH_CKS(stage_in(sc, ks, sizeof(int32_t) * nq, &ksd));
    NRLSH_CKS(stage_in(sc, budgets, sizeof(int64_t) * nq, &bd));
    InputCopies in;
    NRLSH_CKS(in.mark(st, Qd != queries || ksd != ks || bd != budgets, flags));
    NRLSH_CK(wait_for_build(ix, st));
    // the bf16 paths' index operands exist before any tuning or capture
    if (mode != 2 && tc_path_supported(ix)) NRLSH_CKS(ensure_tc_items(ix, st, capturing));
    OutStage oi, os;
    int64_t* idsd;
    float* scd;
    NRLSH_CKS(stage_out(sc, ids, (size_t)nq * k_max, oi, &idsd));
    NRLSH_CKS(stage_out(sc, scores, (size_t)nq * k_max, os, &scd));

    nrlsh_batch_cfg cfg = default_cfg(ix, mode);
    {
        std::lock_guard<std::mutex> g(ix->batch_mu);
        const TuneKey key = tune_key(ix, nq, k_max, cap, mode);
        bool found = false;
        {
            std::lock_guard<std::mutex> gt(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                cfg = it->second;
                found = true;
            }
        }
        if (!found && (flags & NRLSH_QUERY_NO_TUNE)) {
            const nrlsh_batch_cfg& l = ix->last_cfg;
            if (l.hist_qb && cfg_allowed(ix, mode, l)) cfg = l;
        } else if (!found && !capturing) {
            NRLSH_CKS(autotune(ix, (const float*)Qd, nq, (const int32_t*)ksd, (const int64_t*)bd,
                               k_max, cap, mode, idsd, scd, st, &cfg));
            std::lock_guard<std::mutex> gt(g_tune_mu);
            g_tuned[key] = cfg;
        }
        ix->last_cfg = cfg;
    }
    if (!graph) {
        std::vector<void*> p;
        for (size_t b : cfg_ws_sizes(ix, cfg, nq, cap)) {
            char* q = nullptr;
            NRLSH_CKS(sc.get(&q, b));
            p.push_back(q);
        }
        NRLSH_CKS(run_batched(ix, (const float*)Qd, nq, (const int32_t*)ksd, (const int64_t*)bd,
                              k_max, cap, cfg, p, idsd, scd, st));
        return finish_out(st, {&oi, &os}, in);
    }
    // graph mode: replay a captured sequence for identical calls
    std::lock_guard<std::mutex> g(ix->batch_mu);
    const auto key = std::make_tuple((const void*)queries, nq, (const void*)ks, (const void*)budgets,
                                     (int)k_max, cap, (const void*)ids, (const void*)scores, stream);
    for (auto& e : ix->graphs)
        if (e.key == key && e.cfg == cfg) {
            NRLSH_CK(cudaGraphLaunch(e.exec, st));
            return NRLSH_OK;
        }
    nrlsh_graph_entry e;
    e.key = key;
    e.cfg = cfg;
    for (size_t b : cfg_ws_sizes(ix, cfg, nq, cap)) {
        void* q = nullptr;
        cudaError_t err = cudaMalloc(&q, std::max<size_t>(b, 16));
        if (err != cudaSuccess) {
            for (void* x : e.workspace) cudaFree(x);
            return cuda_status(err, "cudaMalloc (graph workspace)");
        }
        e.workspace.push_back(q);
    }
    cudaGraph_t gr = nullptr;
    NRLSH_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const nrlsh_status rs = run_batched(ix, queries, nq, ks, budgets, k_max, cap, cfg, e.workspace,
                                        ids, scores, st);
    const cudaError_t ce = cudaStreamEndCapture(st, &gr);
    if (rs != NRLSH_OK || ce != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        for (void* x : e.workspace) cudaFree(x);
        return rs != NRLSH_OK ? rs : cuda_status(ce, "cudaStreamEndCapture");
    }
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, gr, 0);
    cudaGraphDestroy(gr);
    if (ie != cudaSuccess) {
        for (void* x : e.workspace) cudaFree(x);
        return cuda_status(ie, "cudaGraphInstantiate");
    }
    NRLSH_CK(cudaGraphLaunch(e.exec, st));
    ix->graphs.push_back(std::move(e));
    return NRLSH_OK;
}

extern "C" NRLSH_API nrlsh_status nrlsh_batched_scratch_bytes(const nrlsh_index* ix, int64_t nq,
                                                              int32_t k_max, int64_t budget_max,
                                                              uint32_t flags, int64_t* bytes) {
    if (!ix || !bytes) return arg_error("NULL argument");
    if (nq < 0 || k_max < 1 || budget_max < 1) return arg_error("bad sizes");
    NRLSH_CKS(check_batch_flags(flags));
    const int mode = batch_mode(flags);
    const int64_t cap = std::min<int64_t>(budget_max, ix->n);
    const int64_t qn = std::max<int64_t>(nq, 1);
    // the configuration nrlsh_query_batched would use for these sizes and flags: the
    // tuned one when it exists, else the last one used when the flags allow it,
    // else the path's default
    std::vector<nrlsh_batch_cfg> cfgs;
    {
        std::lock_guard<std::mutex> g(ix->batch_mu);
        {
            std::lock_guard<std::mutex> gt(g_tune_mu);
            auto it = g_tuned.find(tune_key(ix, nq, k_max, cap, mode));
            if (it != g_tuned.end()) cfgs.push_back(it->second);
        }
        if (cfgs.empty()) {
            const nrlsh_batch_cfg& l = ix->last_cfg;
            nrlsh_batch_cfg c = default_cfg(ix, mode);
            if (l.hist_qb && cfg_allowed(ix, mode, l)) c = l;
            cfgs.push_back(c);
        }
    }
    int64_t total = 0;
    for (const auto& cfg : cfgs) {
        int64_t t = 0;
        for (size_t b : cfg_ws_sizes(ix, cfg, qn, cap))
            t += (int64_t)((std::max<size_t>(b, 16) + 255) / 256 * 256);
        total = std::max(total, t);
    }
    *bytes = total;
    return NRLSH_OK;
}

extern "C" NRLSH_API nrlsh_status nrlsh_get_tuning(const nrlsh_index* ix, int32_t* hist_qb,
                                                   int32_t* ctas_per_sm, int32_t* tensor) {
    if (!ix) return arg_error("index is NULL");
    std::lock_guard<std::mutex> g(ix->batch_mu);
    if (hist_qb) *hist_qb = ix->last_cfg.hist_qb;
    if (ctas_per_sm) *ctas_per_sm = ix->last_cfg.ctas_per_sm;
    if (tensor)
        *tensor = (ix->last_cfg.hist_tc ? 1 : 0) | (ix->last_cfg.rerank_tc ? 2 : 0) |
                  (ix->last_cfg.rows_bf16 ? 4 : 0);
    return NRLSH_OK;
}

// ============================================================ no-allocation
// nrlsh_query_noalloc: the query path of nrlsh_query_ex for callers that must
// not allocate device memory while they query.  Its scratch is one fixed array
// in this translation unit; host code must not use the array's name as a device
// address, so the address is looked up once per device with that device current.

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[NRLSH_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_base[kNoallocMaxDevices] = {};

nrlsh_status noalloc_base(void** out) {
    int dev = 0;
    NRLSH_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return arg_error("device ordinal out of range");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return NRLSH_OK;
}

constexpr size_t kArenaAlign = 256;

size_t arena_round(size_t b) { return (b + kArenaAlign - 1) / kArenaAlign * kArenaAlign; }

// Bytes of scratch one chunk of qc queries takes (every buffer 256-byte aligned).
size_t noalloc_chunk_bytes(const nrlsh_index* ix, int64_t qc, int64_t cap) {
    const size_t q = (size_t)qc, c = (size_t)cap;
    return arena_round(q * sizeof(float))                      // qnorm
         + arena_round(sizeof(unsigned))                       // ambiguity counter
         + arena_round(ambiguity_capacity(qc, ix->L) * sizeof(unsigned long long))
         + arena_round(q * ix->code_bytes)                     // query codes
         + arena_round(q * ix->ncls * sizeof(uint32_t))        // histograms
         + arena_round(q * c * sizeof(uint32_t))               // candidates
         + 2 * arena_round(q * c * sizeof(float))              // lo, hi
         + arena_round(q * c * sizeof(uint32_t))               // contenders
         + arena_round(q * c * sizeof(double));                // contender scores
}

struct Arena {
    char* base;
    size_t off;
    template <typename T>
    T* take(size_t count) {
        T* p = (T*)(base + off);
        off += arena_round(count * sizeof(T));
        return p;
    }
};

}  // namespace

extern "C" NRLSH_API nrlsh_status nrlsh_query_noalloc(const nrlsh_index* ix, const float* queries,
                                                      int64_t nq, int32_t k, int64_t probe_budget,
                                                      int64_t* ids, float* scores, void* stream) {
    NRLSH_CKS(check_query_args(ix, queries, nq));
    if (k < 1 || k > NRLSH_MAX_K) return arg_error("need 1 <= k <= 1024");
    if (probe_budget < 1) return arg_error("need probe_budget >= 1");
    if (nq > 0 && (!ids || !scores)) return arg_error("ids/scores is NULL");
    if (nq == 0) return NRLSH_OK;
    if (!is_device_ptr(queries) || !is_device_ptr(ids) || !is_device_ptr(scores))
        return arg_error("nrlsh_query_noalloc takes device pointers only");
    const int64_t cap = std::min<int64_t>(probe_budget, ix->n);
    if (noalloc_chunk_bytes(ix, 1, cap) > (size_t)NRLSH_NOALLOC_SCRATCH_BYTES)
        return arg_error("probe budget too large for the 32 MiB no-allocation scratch");
    void* base = nullptr;
    NRLSH_CKS(noalloc_base(&base));
    cudaStream_t st = (cudaStream_t)stream;
    NRLSH_CK(cudaGetLastError());
    NRLSH_CK(wait_for_build(ix, st));
    // the largest chunk of queries whose scratch fits the array
    int64_t lo = 1, hi = nq;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (noalloc_chunk_bytes(ix, mid, cap) <= (size_t)NRLSH_NOALLOC_SCRATCH_BYTES)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int64_t chunk = lo;
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t qc = std::min(chunk, nq - q0);
        const float* Qc = queries + q0 * ix->d;
        Arena a{(char*)base, 0};
        float* qnorm = a.take<float>(qc);
        unsigned* qamb = a.take<unsigned>(1);
        const size_t qamb_cap = ambiguity_capacity(qc, ix->L);
        unsigned long long* qamb_list = a.take<unsigned long long>(qamb_cap);
        char* qcodes = a.take<char>((size_t)qc * ix->code_bytes);
        uint32_t* H = a.take<uint32_t>((size_t)qc * ix->ncls);
        uint32_t* cand = a.take<uint32_t>((size_t)qc * cap);
        float* lo_s = a.take<float>((size_t)qc * cap);
        float* hi_s = a.take<float>((size_t)qc * cap);
        uint32_t* cont = a.take<uint32_t>((size_t)qc * cap);
        double* cont_s = a.take<double>((size_t)qc * cap);
        // everything that must start at zero is cleared: the array keeps the
        // previous call's contents
        NRLSH_CK(cudaMemsetAsync(H, 0, sizeof(uint32_t) * qc * ix->ncls, st));
        NRLSH_CK(launch_hash_queries(Qc, qc, ix->d, ix->L, ix->Lp, ix->A_pad, ix->anorm, qnorm,
                                     qcodes, ix->code_bytes, qamb_list, qamb, (unsigned)qamb_cap, ix->At32, st));
        NRLSH_CK(launch_hist(ix->codes, qcodes, ix->code_bytes, qc, ix->m, ix->L, ix->tiles,
                             ix->ntiles, H, st));
        NRLSH_CK(launch_probe_rerank(H, ix->order, ix->m, ix->L, ix->n, ix->seg, qc, probe_budget, nullptr, 0u,
                                     ix->codes, qcodes, ix->code_bytes, ix->Xp, ix->dtype, ix->dp,
                                     ix->d, Qc, ix->xnorm, qnorm, ix->perm, k, nullptr, cand, lo_s,
                                     hi_s, cont, cont_s, cap, ids + q0 * k, scores + q0 * k, k, st));
    }
    return NRLSH_OK;
}
