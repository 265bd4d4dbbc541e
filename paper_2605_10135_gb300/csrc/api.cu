// extern "C" entry points of libann.so: argument checks, workspace layout and
// the calls into the stage drivers.  Every stage runs in the CUDA kernels of
// this library; nothing falls back to the host.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdarg.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "stages.cuh"

namespace ann {

// ---- error state ---------------------------------------------------------------
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

// ---- launch counter and tile timing --------------------------------------------
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::mutex g_timing_mu;
static bool g_timing = false;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_tile_events;
static std::vector<cudaEvent_t> g_event_pool;

bool tile_timing_on() { return g_timing; }
static bool g_counters = false;
bool tile_counters_on() { return g_counters; }
cudaEvent_t tile_event() {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
void tile_timing_record(cudaEvent_t a, cudaEvent_t b) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_tile_events.emplace_back(a, b);
}

// ---- device status word ----------------------------------------------------------
__device__ int g_dev_status;

int* device_status_ptr() {
    static std::mutex mu;
    static int* ptrs[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dev_status) == cudaSuccess) ptrs[dev] = (int*)p;
    }
    return ptrs[dev];
}

static bool valid_dtype(int dt) { return dt >= ANN_F32 && dt <= ANN_U8; }

// Vector arrays (X, queries) may be device memory of the current device, managed
// memory, or page-locked host memory mapped into the device's address space at
// the same address (unified addressing): on a Grace-Blackwell node the kernels
// then read the vectors from host memory over NVLink-C2C, so X need not fit in
// HBM.  Anything else (pageable host memory, another device's memory) is refused
// here instead of being handed to a kernel.
static int check_readable(const void* p, const char* name) {
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ANN_ERR_INVALID_ARG, "%s: not a CUDA-visible pointer (%s)", name,
                    cudaGetErrorString(e));
    }
    int cur = -1;
    ANN_CHECK_CUDA(cudaGetDevice(&cur));
    if (a.type == cudaMemoryTypeDevice && a.device == cur) return ANN_OK;
    if (a.type == cudaMemoryTypeManaged) return ANN_OK;
    if (a.type == cudaMemoryTypeHost && a.devicePointer == p) return ANN_OK;
    return fail(ANN_ERR_INVALID_ARG,
                "%s must be memory of the current device or page-locked host memory mapped "
                "at the same address", name);
}

static int check_ws(void* ws, size_t have, size_t need) {
    if (need > 256 && (!ws || have < need))
        return fail(ANN_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, have);
    return ANN_OK;
}

// small per-device scratch for ann_recall / ann_search_eval hit counters
__device__ unsigned long long g_hits;
static unsigned long long* hits_ptr() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_hits) != cudaSuccess) return nullptr;
    return (unsigned long long*)p;
}

}  // namespace ann

using namespace ann;

extern "C" {

const char* ann_last_error(void) { return ann::g_err; }

int ann_version(void) { return 104; }  // 1.04: selective partition, tile skipping, scheduler

unsigned long long ann_launch_count(void) { return g_launches.load(); }

int ann_timing_enable(int on) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timing = on != 0;
    return ANN_OK;
}

int ann_tile_counters_enable(int on) {
    g_counters = on != 0;
    return ANN_OK;
}

int ann_tile_prune(int on) {
    tile_prune_set(on != 0);
    return ANN_OK;
}

int ann_tile_prune_stats(unsigned long long* out, int n) {
    ANN_REQUIRE(out && n >= 0, "bad arguments");
    return tile_prune_stats(out, n, true);
}

int ann_tile_counters_read(unsigned long long* out, int n) {
    ANN_REQUIRE(out && n >= 0, "bad arguments");
    return tile_counters_read(out, n, true);
}

int ann_timing_read(double* tile_ms, int* launches) {
    ANN_REQUIRE(tile_ms && launches, "NULL pointer");
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    {
        std::lock_guard<std::mutex> lk(g_timing_mu);
        ev.swap(g_tile_events);
    }
    double tot = 0.0;
    int rc = ANN_OK;
    for (auto& p : ev) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.second) != cudaSuccess ||
            cudaEventElapsedTime(&ms, p.first, p.second) != cudaSuccess)
            rc = fail(ANN_ERR_CUDA, "tile timing events failed");
        tot += ms;
    }
    {
        std::lock_guard<std::mutex> lk(g_timing_mu);
        for (auto& p : ev) {
            g_event_pool.push_back(p.first);
            g_event_pool.push_back(p.second);
        }
    }
    *tile_ms = tot;
    *launches = (int)ev.size();
    return rc;
}

int ann_device_status(int* out) {
    ANN_REQUIRE(out != nullptr, "ann_device_status: out is NULL");
    ANN_CHECK_CUDA(cudaDeviceSynchronize());
    int v = 0, zero = 0;
    ANN_CHECK_CUDA(cudaMemcpyFromSymbol(&v, g_dev_status, sizeof(int)));
    ANN_CHECK_CUDA(cudaMemcpyToSymbol(g_dev_status, &zero, sizeof(int)));
    *out = v;
    if (v & DEV_TIMEOUT) return fail(ANN_ERR_TIMEOUT, "a bounded device wait gave up");
    return ANN_OK;
}

// ---------------------------------------------------------------- wait self-test
// One warp waits on an mbarrier that nothing arrives on, through the same bounded
// wait the pipelined kernels use (globaltimer limit, abort flag).  mode 0: the
// limit runs out; mode 1: the abort flag is already set.  Either way the wait
// gives up, the kernel records DEV_TIMEOUT and returns.
__global__ void k_wait_selftest(int mode, uint64_t limit_ns, int* status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = mode == 1 ? 1 : 0;
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        // phase 0 never completes: no thread arrives and no copy is pending
        const bool ok = mbar_wait(smem_u32(&bar), 0, (volatile int*)&abort_flag, limit_ns);
        if (!ok) atomicOr(status, DEV_TIMEOUT);
    }
    __syncwarp();
}

int ann_wait_selftest(int mode, int64_t limit_us, void* stream) {
    ANN_REQUIRE(mode == 0 || mode == 1, "mode must be 0 or 1");
    ANN_REQUIRE(limit_us >= 1 && limit_us <= 2000000, "limit_us must be in [1, 2e6]");
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(mode, (uint64_t)limit_us * 1000ull,
                                                         device_status_ptr());
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

// ---------------------------------------------------------------- partition
int ann_partition_workspace(int64_t N, int d, int C, int r, int64_t S, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    ANN_REQUIRE(N >= 0 && N < (1ll << 32), "N out of range");
    ANN_REQUIRE(d >= 1 && d <= 4096, "d out of range");
    ANN_REQUIRE(C >= 1 && C <= 1024 && r >= 1 && r <= C, "need 1 <= r <= C <= 1024");
    ANN_REQUIRE(S >= 0 && S <= N, "S out of range");
    *bytes = partition_ws(N, d, C, r, S, nullptr, nullptr, 0);
    return ANN_OK;
}

int ann_partition(const void* X, int64_t N, int d, int dtype, int C, int r,
                  const float* init_centroids, const uint32_t* sample_idx, int64_t S, int iters,
                  float* centroids_out, uint32_t* members_out, int64_t* offsets_out, void* ws,
                  size_t ws_bytes, void* stream) {
    size_t need = 0;
    int rc = ann_partition_workspace(N, d, C, r, S, &need);
    if (rc) return rc;
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype %d", dtype);
    ANN_REQUIRE(iters >= 0, "iters < 0");
    ANN_REQUIRE(init_centroids && centroids_out && offsets_out, "NULL pointer");
    ANN_REQUIRE(N == 0 || (X && members_out), "NULL pointer");
    ANN_REQUIRE(S == 0 || iters == 0 || sample_idx, "sample_idx is NULL");
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    if (N > 0 && (rc = check_readable(X, "X"))) return rc;
    PartitionWs w;
    partition_ws(N, d, C, r, S, &w, ws, ws_bytes);
    if (N == 0) {
        ANN_CHECK_CUDA(cudaMemsetAsync(offsets_out, 0, sizeof(int64_t) * (C + 1), (cudaStream_t)stream));
        ANN_CHECK_CUDA(cudaMemcpyAsync(centroids_out, init_centroids, sizeof(float) * C * d,
                                       cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
        return ANN_OK;
    }
    return run_partition(X, N, d, dtype, C, r, init_centroids, sample_idx, S, iters, centroids_out,
                         members_out, offsets_out, w, (cudaStream_t)stream);
}

static int check_selective(int64_t N, int d, int C, int64_t S, const ann_selective_params* p) {
    ANN_REQUIRE(p, "params is NULL");
    ANN_REQUIRE(N >= 0 && N < (1ll << 32), "N out of range");
    ANN_REQUIRE(d >= 1 && d <= 4096, "d out of range");
    ANN_REQUIRE(C >= 1 && C <= 1024, "need 1 <= C <= 1024");
    ANN_REQUIRE(S >= 0 && S <= N, "S out of range");
    ANN_REQUIRE(p->cand >= 1 && p->cand <= (C < 32 ? C : 32), "need 1 <= cand <= min(C, 32)");
    ANN_REQUIRE(p->omega >= 1 && p->omega <= p->cand, "need 1 <= omega <= cand");
    ANN_REQUIRE(p->epsilon >= 0.0 && !isnan(p->epsilon), "epsilon must be >= 0 or +inf");
    ANN_REQUIRE(p->tau0 >= 0.0 && isfinite(p->tau0), "tau0 must be finite and >= 0");
    ANN_REQUIRE(p->block >= 1, "block must be >= 1");
    ANN_REQUIRE(p->capacity >= 0 && p->capacity < (1ll << 40), "capacity out of range");
    return ANN_OK;
}

int ann_partition_selective_workspace(int64_t N, int d, int C, int64_t S,
                                      const ann_selective_params* p, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    int rc = check_selective(N, d, C, S, p);
    if (rc) return rc;
    *bytes = selective_ws(N, d, C, S, p->cand, p->omega, p->block, nullptr, nullptr, 0);
    return ANN_OK;
}

int ann_partition_selective(const void* X, int64_t N, int d, int dtype, int C,
                            const float* init_centroids, const uint32_t* sample_idx, int64_t S,
                            int iters, const ann_selective_params* p, float* centroids_out,
                            uint32_t* assign_out, uint32_t* members_out, int64_t* offsets_out,
                            int64_t* stats_out, void* ws, size_t ws_bytes, void* stream) {
    size_t need = 0;
    int rc = ann_partition_selective_workspace(N, d, C, S, p, &need);
    if (rc) return rc;
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype %d", dtype);
    ANN_REQUIRE(iters >= 0, "iters < 0");
    ANN_REQUIRE(init_centroids && centroids_out && offsets_out, "NULL pointer");
    ANN_REQUIRE(N == 0 || (X && members_out), "NULL pointer");
    ANN_REQUIRE(S == 0 || iters == 0 || sample_idx, "sample_idx is NULL");
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    if (N > 0 && (rc = check_readable(X, "X"))) return rc;
    SelectiveWs w;
    selective_ws(N, d, C, S, p->cand, p->omega, p->block, &w, ws, ws_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0) {
        ANN_CHECK_CUDA(cudaMemsetAsync(offsets_out, 0, sizeof(int64_t) * (C + 1), st));
        if (stats_out) ANN_CHECK_CUDA(cudaMemsetAsync(stats_out, 0, 2 * sizeof(int64_t), st));
        ANN_CHECK_CUDA(cudaMemcpyAsync(centroids_out, init_centroids, sizeof(float) * C * d,
                                       cudaMemcpyDeviceToDevice, st));
        return ANN_OK;
    }
    SelectiveArgs a;
    a.eps = p->epsilon;
    a.tau0 = p->tau0;
    a.block = p->block;
    a.cap = p->capacity;
    a.omega = p->omega;
    a.M = p->cand;
    return run_partition_selective(X, N, d, dtype, C, init_centroids, sample_idx, S, iters, a,
                                   centroids_out, assign_out, members_out, offsets_out, stats_out,
                                   w, st);
}

// ---------------------------------------------------------------- autotuner
// Plans chosen by timing, per (d, dtype, k, precision, rerank_k, shard-size
// bucket = floor(log2(rows / C))); process-wide, guarded by a mutex.
struct TuneKey {
    int d, dtype, k, precision, rerank_k, bucket;
    bool operator<(const TuneKey& o) const {
        return std::tie(d, dtype, k, precision, rerank_k, bucket) <
               std::tie(o.d, o.dtype, o.k, o.precision, o.rerank_k, o.bucket);
    }
};
struct TuneEntry {
    KnnPlan plan;
    float ms;
    int tried;
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneEntry> g_tuned;
static std::atomic<bool> g_autotune{false};

static TuneKey tune_key(int d, int dtype, int k, int precision, int rerank_k, int64_t rows, int C) {
    int64_t per = rows / (C > 0 ? C : 1);
    int b = 0;
    while (per > 1) {
        per >>= 1;
        ++b;
    }
    return TuneKey{d, dtype, k, precision, rerank_k, b};
}

static bool tuned_plan(const TuneKey& key, KnnPlan* pl) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it == g_tuned.end()) return false;
    *pl = it->second.plan;
    return true;
}

static void store_tuned(const TuneKey& key, const KnnPlan& pl, float ms, int tried) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = TuneEntry{pl, ms, tried};
}

int ann_autotune(int on) {
    g_autotune.store(on != 0);
    if (on < 0) {  // forget every decision
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned.clear();
        g_autotune.store(false);
    }
    return ANN_OK;
}

int ann_autotune_lookup(int d, int dtype, int k, int precision, int rerank_k, int64_t rows, int C,
                        int* found, int* bn, int* nst, int* a_stream, float* ms, int* tried) {
    ANN_REQUIRE(found && bn && nst && a_stream && ms && tried, "NULL pointer");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(d, dtype, k, precision, rerank_k, rows, C));
    *found = it != g_tuned.end();
    if (*found) {
        *bn = it->second.plan.bn;
        *nst = it->second.plan.nst;
        *a_stream = it->second.plan.a_stream;
        *ms = it->second.ms;
        *tried = it->second.tried;
    }
    return ANN_OK;
}

// ---------------------------------------------------------------- shard kNN
static int knn_args(int64_t N, int d, int dtype, int C, int64_t rows, int k, int precision,
                    int rerank_k) {
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype %d", dtype);
    ANN_REQUIRE(N >= 0 && N < (1ll << 32), "N out of range");
    ANN_REQUIRE(C >= 1 && C <= 1024, "C must be in [1, 1024]");
    ANN_REQUIRE(rows >= 0 && rows < (1ll << 40), "rows out of range");
    ANN_REQUIRE(k >= 1 && k <= 240, "k must be in [1, 240]");
    ANN_REQUIRE(d >= 1, "d < 1");
    ANN_REQUIRE(rerank_k == 0 || (rerank_k >= k && rerank_k <= 256), "rerank_k must be 0 or in [k, 256]");
    if (precision != ANN_EXACT && precision != ANN_BF16_RERANK && precision != ANN_FP8_RERANK &&
        precision != ANN_F16_RERANK && precision != ANN_LEARNED)
        return fail(ANN_ERR_INVALID_ARG, "bad precision %d", precision);
    if (precision == ANN_LEARNED) {
        ANN_REQUIRE(d <= 4096, "learned form: d must be <= 4096");
        return ANN_OK;
    }
    ANN_REQUIRE(d <= 4096, "shard_knn: d must be <= 4096");
    if (dtype == ANN_U8 && d > 258)
        return fail(ANN_ERR_UNSUPPORTED, "uint8 with d > 258: the integer tiles are not exact");
    return ANN_OK;
}

// The learned form screens 32-dimensional FP32 embeddings with scaled FP16 tiles.
static int learned_plan(int k, int rerank_k, KnnPlan* pl) {
    return knn_plan(ml::OUT, ANN_F32, k, ANN_F16_RERANK, rerank_k, pl);
}

static size_t learned_knn_bytes(int64_t N, int d, int C, int64_t rows, const KnnPlan& pl) {
    return knn_ws(C, rows, pl, nullptr, nullptr, 0) + align_up((size_t)N * ml::OUT * 4, 256) +
           learned_embed_ws(N, d) + 512;
}

int ann_shard_knn_workspace(int64_t N, int d, int dtype, int C, int64_t rows, int k,
                            int precision, int rerank_k, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    int rc = knn_args(N, d, dtype, C, rows, k, precision, rerank_k);
    if (rc) return rc;
    KnnPlan pl;
    if (precision == ANN_LEARNED) {  // enough for the exact form too (no model given)
        if ((rc = learned_plan(k, rerank_k, &pl))) return rc;
        size_t b = learned_knn_bytes(N, d, C, rows, pl);
        KnnPlan pe;
        if (knn_plan(d, dtype, k, ANN_EXACT, rerank_k, &pe) == ANN_OK) {
            const size_t be = knn_ws(C, rows, pe, nullptr, nullptr, 0);
            if (be > b) b = be;
        }
        *bytes = b;
        return ANN_OK;
    }
    if ((rc = knn_plan(d, dtype, k, precision, rerank_k, &pl))) return rc;
    *bytes = knn_ws(C, rows, pl, nullptr, nullptr, 0);
    return ANN_OK;
}

int ann_shard_knn(const void* X, int64_t N, int d, int dtype, const uint32_t* members,
                  const int64_t* offsets, int C, int64_t rows, int k, int precision, int rerank_k,
                  const void* model, uint32_t* knn_id, float* knn_d, void* ws, size_t ws_bytes,
                  void* stream) {
    int rc = knn_args(N, d, dtype, C, rows, k, precision, rerank_k);
    if (rc) return rc;
    ANN_REQUIRE(offsets, "offsets is NULL");
    ANN_REQUIRE(rows == 0 || (X && members && knn_id && knn_d), "NULL pointer");
    KnnPlan pl;
    if (precision == ANN_LEARNED && !model) {  // no model: the exact form
        precision = ANN_EXACT;
        if ((rc = knn_args(N, d, dtype, C, rows, k, precision, rerank_k))) return rc;
    }
    if (precision == ANN_LEARNED) {
        if ((rc = learned_plan(k, rerank_k, &pl))) return rc;
        if ((rc = check_ws(ws, ws_bytes, learned_knn_bytes(N, d, C, rows, pl)))) return rc;
        if (rows == 0) return ANN_OK;
        if ((rc = check_readable(X, "X"))) return rc;
        Carver cv(ws, ws_bytes);
        const size_t kb = knn_ws(C, rows, pl, nullptr, nullptr, 0);
        uint8_t* kbase = cv.take<uint8_t>(kb);
        float* E = cv.take<float>((size_t)N * ml::OUT);
        const size_t eb = learned_embed_ws(N, d);
        uint8_t* ebase = cv.take<uint8_t>(eb);
        if (!cv.ok) return fail(ANN_ERR_WORKSPACE, "workspace too small");
        cudaStream_t st = (cudaStream_t)stream;
        if ((rc = run_learned_embed(X, N, d, dtype, (const float*)model, E, ebase, eb, st)))
            return rc;
        KnnWs w;
        knn_ws(C, rows, pl, &w, kbase, kb);
        return run_shard_knn(E, N, ml::OUT, ANN_F32, members, offsets, C, rows, k, pl, w, knn_id,
                             knn_d, st, X, d, dtype);
    }
    ANN_REQUIRE(model == nullptr, "model must be NULL unless precision is ANN_LEARNED");
    if ((rc = knn_plan(d, dtype, k, precision, rerank_k, &pl))) return rc;
    size_t need = knn_ws(C, rows, pl, nullptr, nullptr, 0);
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    if (rows == 0) return ANN_OK;
    if ((rc = check_readable(X, "X"))) return rc;
    KnnWs w;
    knn_ws(C, rows, pl, &w, ws, ws_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    const TuneKey key = tune_key(d, dtype, k, precision, rerank_k, rows, C);
    if (tuned_plan(key, &pl)) {
        return run_shard_knn(X, N, d, dtype, members, offsets, C, rows, k, pl, w, knn_id, knn_d,
                             st);
    }
    if (!g_autotune.load()) {
        return run_shard_knn(X, N, d, dtype, members, offsets, C, rows, k, pl, w, knn_id, knn_d,
                             st);
    }
    // Autotune: run the whole shard kNN once per plan, timed with events on the
    // stream; every run writes the same lists, so the last one is the result.
    KnnPlan vars[8];
    const int nv = knn_plan_variants(d, dtype, k, precision, rerank_k, vars, 8);
    if (nv <= 0) return -nv;
    cudaEvent_t e0, e1;
    ANN_CHECK_CUDA(cudaEventCreate(&e0));
    ANN_CHECK_CUDA(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 0.0f;
    for (int v = 0; v < nv && !rc; ++v) {
        ANN_CHECK_CUDA(cudaEventRecord(e0, st));
        rc = run_shard_knn(X, N, d, dtype, members, offsets, C, rows, k, vars[v], w, knn_id, knn_d,
                           st);
        ANN_CHECK_CUDA(cudaEventRecord(e1, st));
        ANN_CHECK_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        ANN_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (v == 0 || ms < best_ms) {
            best = v;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    store_tuned(key, vars[best], best_ms, nv);
    return ANN_OK;
}

// ---------------------------------------------------------------- learned form
static int learned_args(int64_t N, int d, int dtype, int64_t S, int kk, int kpos, int batch) {
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype %d", dtype);
    ANN_REQUIRE(d >= 1 && d <= 4096, "learned training: d must be in [1, 4096]");
    ANN_REQUIRE(kk >= 2 && kk <= 95, "kk must be in [2, 95]");
    ANN_REQUIRE(N >= kk + 2 && N < (1ll << 32), "N must be in [kk + 2, 2^32)");
    ANN_REQUIRE(kpos >= 1 && kpos < kk, "kpos must be in [1, kk)");
    ANN_REQUIRE(S >= 1 && S <= N, "S must be in [1, N]");
    ANN_REQUIRE(batch >= 1 && batch <= (1 << 16), "batch must be in [1, 65536]");
    return ANN_OK;
}

int ann_learned_train_workspace(int64_t N, int d, int dtype, int64_t S, int kk, int batch,
                                size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    int rc = learned_args(N, d, dtype, S, kk, 1, batch);
    if (rc) return rc;
    *bytes = learned_train_ws(N, d, dtype, S, kk, batch, nullptr, nullptr, 0);
    return *bytes ? ANN_OK : fail(ANN_ERR_UNSUPPORTED, "learned training: no plan for d=%d", d);
}

int ann_learned_train(const void* X, int64_t N, int d, int dtype, const uint32_t* sample,
                      int64_t S, int kk, int kpos, const uint32_t* draws, int steps, int batch,
                      float lr, float margin, float* params, float* losses, float* recall_est,
                      void* ws, size_t ws_bytes, void* stream) {
    int rc = learned_args(N, d, dtype, S, kk, kpos, batch);
    if (rc) return rc;
    ANN_REQUIRE(steps >= 0, "steps < 0");
    ANN_REQUIRE(X && sample && params && (steps == 0 || draws), "NULL pointer");
    ANN_REQUIRE(lr > 0.0f && margin >= 0.0f, "lr must be > 0 and margin >= 0");
    const size_t need = learned_train_ws(N, d, dtype, S, kk, batch, nullptr, nullptr, 0);
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    return run_learned_train(X, N, d, dtype, sample, S, kk, kpos, draws, steps, batch, lr, margin,
                             params, losses, recall_est, ws, ws_bytes, (cudaStream_t)stream);
}

int ann_learned_grad_workspace(int64_t N, int d, int dtype, int B, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype %d", dtype);
    ANN_REQUIRE(N >= 1 && N < (1ll << 32) && d >= 1 && d <= 4096, "N / d out of range");
    ANN_REQUIRE(B >= 1 && B <= (1 << 16), "B must be in [1, 65536]");
    *bytes = learned_grad_bytes(B, d);
    return ANN_OK;
}

int ann_learned_grad(const void* X, int64_t N, int d, int dtype, const float* params,
                     const uint32_t* rows, int B, float margin, float* grads, float* loss,
                     void* ws, size_t ws_bytes, void* stream) {
    size_t need = 0;
    int rc = ann_learned_grad_workspace(N, d, dtype, B, &need);
    if (rc) return rc;
    ANN_REQUIRE(X && params && rows && grads && loss, "NULL pointer");
    ANN_REQUIRE(margin >= 0.0f, "margin must be >= 0");
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    if ((rc = check_readable(X, "X"))) return rc;
    return run_learned_grad(X, N, d, dtype, params, rows, B, margin, grads, loss, ws, ws_bytes,
                            (cudaStream_t)stream);
}

int ann_learned_embed_workspace(int64_t N, int d, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    ANN_REQUIRE(N >= 0 && d >= 1 && d <= 4096, "N / d out of range");
    *bytes = learned_embed_ws(N, d);
    return ANN_OK;
}

int ann_learned_embed(const void* X, int64_t N, int d, int dtype, const float* params, float* E,
                      void* ws, size_t ws_bytes, void* stream) {
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype %d", dtype);
    ANN_REQUIRE(N >= 0 && N < (1ll << 32) && d >= 1 && d <= 4096, "N / d out of range");
    ANN_REQUIRE(N == 0 || (X && params && E), "NULL pointer");
    int rc = check_ws(ws, ws_bytes, learned_embed_ws(N, d));
    if (rc) return rc;
    return run_learned_embed(X, N, d, dtype, params, E, ws, ws_bytes, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- prune / merge
int ann_screen_width(int d, int dtype, int k, int precision, int rerank_k, int* kprime) {
    ANN_REQUIRE(kprime, "kprime is NULL");
    ANN_REQUIRE(precision != ANN_LEARNED, "the learned form screens in its embedding space");
    KnnPlan pl;
    int rc = knn_plan(d, dtype, k, precision, rerank_k, &pl);
    if (rc) return rc;
    *kprime = pl.rerank ? pl.kprime : k;
    return ANN_OK;
}

int ann_shard_knn_screen(const void* X, int64_t N, int d, int dtype, const uint32_t* members,
                         const int64_t* offsets, int C, int64_t rows, int k, int precision,
                         int rerank_k, uint32_t* cand_id, float* cand_d, void* ws,
                         size_t ws_bytes, void* stream) {
    int rc = knn_args(N, d, dtype, C, rows, k, precision, rerank_k);
    if (rc) return rc;
    ANN_REQUIRE(precision != ANN_LEARNED, "the learned form screens in its embedding space");
    ANN_REQUIRE(offsets, "offsets is NULL");
    ANN_REQUIRE(rows == 0 || (X && members && cand_id && cand_d), "NULL pointer");
    KnnPlan pl;
    if ((rc = knn_plan(d, dtype, k, precision, rerank_k, &pl))) return rc;
    if ((rc = check_ws(ws, ws_bytes, knn_ws(C, rows, pl, nullptr, nullptr, 0)))) return rc;
    if (rows == 0) return ANN_OK;
    if ((rc = check_readable(X, "X"))) return rc;
    KnnWs w;
    knn_ws(C, rows, pl, &w, ws, ws_bytes);
    return run_shard_knn(X, N, d, dtype, members, offsets, C, rows, k, pl, w, cand_id, cand_d,
                         (cudaStream_t)stream, nullptr, 0, 0, true);
}

int ann_prune_workspace(int64_t N, int64_t rows, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    ANN_REQUIRE(N >= 0 && N < (1ll << 32) && rows >= 0, "N / rows out of range");
    *bytes = rowlist_ws(N, rows, nullptr, nullptr, 0);
    return ANN_OK;
}

int ann_prune(const uint32_t* knn_id, const float* knn_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t rows, int64_t N, int k, int R, int rule,
              uint32_t* pr_id, float* pr_d, void* ws, size_t ws_bytes, void* stream) {
    ANN_REQUIRE(k >= 1 && k <= 256, "k must be in [1, 256]");
    ANN_REQUIRE(R >= 1 && R <= 256, "R must be in [1, 256]");
    ANN_REQUIRE(rule == ANN_PRUNE_RANK || rule == ANN_PRUNE_TRUNC, "bad rule %d", rule);
    ANN_REQUIRE(C >= 1 && rows >= 0, "bad C / rows");
    ANN_REQUIRE(N >= 0 && N < (1ll << 32), "N out of range");
    ANN_REQUIRE(offsets, "offsets is NULL");
    ANN_REQUIRE(rows == 0 || (knn_id && knn_d && members && pr_id && pr_d), "NULL pointer");
    size_t need = rowlist_ws(N, rows, nullptr, nullptr, 0);
    int rc = check_ws(ws, ws_bytes, need);
    if (rc) return rc;
    RowlistWs w;
    rowlist_ws(N, rows, &w, ws, ws_bytes);
    return run_prune(knn_id, knn_d, members, offsets, C, rows, N, k, R, rule, pr_id, pr_d, w,
                     (cudaStream_t)stream);
}

int ann_merge_workspace(int64_t N, int64_t rows, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    ANN_REQUIRE(N >= 0 && N < (1ll << 32) && rows >= 0, "N / rows out of range");
    *bytes = rowlist_ws(N, rows, nullptr, nullptr, 0);
    return ANN_OK;
}

int ann_merge(const uint32_t* pr_id, const float* pr_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t rows, int64_t N, int R, uint32_t* graph,
              float* gdist, uint32_t* degree, void* ws, size_t ws_bytes, void* stream) {
    size_t need = 0;
    int rc = ann_merge_workspace(N, rows, &need);
    if (rc) return rc;
    ANN_REQUIRE(R >= 1 && R <= 256, "R must be in [1, 256]");
    ANN_REQUIRE(C >= 1, "C < 1");
    ANN_REQUIRE(N == 0 || (graph && gdist && degree), "NULL pointer");
    ANN_REQUIRE(rows == 0 || (pr_id && pr_d && members), "NULL pointer");
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    RowlistWs w;
    rowlist_ws(N, rows, &w, ws, ws_bytes);
    return run_merge(pr_id, pr_d, members, offsets, C, rows, N, R, graph, gdist, degree, w,
                     (cudaStream_t)stream);
}

int ann_merge_reverse_workspace(int64_t N, int R, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    ANN_REQUIRE(N >= 0 && N < (1ll << 32), "N out of range");
    ANN_REQUIRE(R >= 1 && R <= 64, "R must be in [1, 64]");
    *bytes = merge_rev_ws(N, R, nullptr, nullptr, 0);
    return ANN_OK;
}

int ann_merge_reverse(const uint32_t* graph, const float* gdist, const uint32_t* degree,
                      int64_t N, int R, uint32_t* out_graph, float* out_gdist,
                      uint32_t* out_degree, void* ws, size_t ws_bytes, void* stream) {
    size_t need = 0;
    int rc = ann_merge_reverse_workspace(N, R, &need);
    if (rc) return rc;
    ANN_REQUIRE(N == 0 || (graph && gdist && degree && out_graph && out_gdist && out_degree),
                "NULL pointer");
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    MergeRevWs w;
    merge_rev_ws(N, R, &w, ws, ws_bytes);
    return run_merge_reverse(graph, gdist, degree, N, R, out_graph, out_gdist, out_degree, w,
                             (cudaStream_t)stream);
}

// ---------------------------------------------------------------- query side
int ann_medoid_workspace(int64_t N, int d, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    ANN_REQUIRE(N >= 1 && d >= 1, "N and d must be >= 1");
    *bytes = medoid_ws(N, d, nullptr, nullptr, nullptr, nullptr, 0);
    return ANN_OK;
}

int ann_medoid(const void* X, int64_t N, int d, int dtype, uint32_t* entry_out, void* ws,
               size_t ws_bytes, void* stream) {
    size_t need = 0;
    int rc = ann_medoid_workspace(N, d, &need);
    if (rc) return rc;
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype");
    ANN_REQUIRE(X && entry_out, "NULL pointer");
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    if ((rc = check_readable(X, "X"))) return rc;
    double* part;
    float* mean;
    unsigned long long* best;
    medoid_ws(N, d, &part, &mean, &best, ws, ws_bytes);
    return run_medoid(X, N, d, dtype, entry_out, part, mean, best, (cudaStream_t)stream);
}

int ann_medoid_noalloc(const void* X, int64_t N, int d, int dtype, uint32_t* entry_out,
                       void* stream) {
    ANN_REQUIRE(N >= 1 && N < (1ll << 32) && d >= 1, "N and d must be >= 1");
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype");
    ANN_REQUIRE(X && entry_out, "NULL pointer");
    int rc = medoid_noalloc_check(N, d);
    if (rc) return rc;
    if ((rc = check_readable(X, "X"))) return rc;
    return run_medoid_noalloc(X, N, d, dtype, entry_out, (cudaStream_t)stream);
}

int ann_knn_query_workspace(int64_t N, int64_t nq, int d, int dtype, int k, size_t* bytes) {
    ANN_REQUIRE(bytes, "bytes is NULL");
    int rc = knn_args(N, d, dtype, 1, nq, k, ANN_EXACT, 0);
    if (rc) return rc;
    ANN_REQUIRE(N < (1 << 24) && nq < (1 << 24), "N and nq must be < 2^24");
    KnnPlan pl;
    if ((rc = knn_plan(d, dtype, k, ANN_EXACT, 0, &pl))) return rc;
    *bytes = query_ws(N, nq, pl, nullptr, nullptr, 0);
    return ANN_OK;
}

int ann_knn_query(const void* X, int64_t N, const void* Q, int64_t nq, int d, int dtype, int k,
                  uint32_t* out_id, float* out_d, void* ws, size_t ws_bytes, void* stream) {
    size_t need = 0;
    int rc = ann_knn_query_workspace(N, nq, d, dtype, k, &need);
    if (rc) return rc;
    ANN_REQUIRE(nq == 0 || (X && Q && out_id && out_d), "NULL pointer");
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    if (nq == 0) return ANN_OK;
    if ((rc = check_readable(X, "X")) || (rc = check_readable(Q, "Q"))) return rc;
    KnnPlan pl;
    knn_plan(d, dtype, k, ANN_EXACT, 0, &pl);
    QueryWs w;
    query_ws(N, nq, pl, &w, ws, ws_bytes);
    return run_knn_query(X, N, Q, nq, d, dtype, k, pl, w, out_id, out_d, (cudaStream_t)stream);
}

static int search_args(int R, int64_t N, int d, int dtype, int64_t nq, uint32_t entry, int Ls,
                       int topk) {
    ANN_REQUIRE(valid_dtype(dtype), "bad dtype");
    ANN_REQUIRE(R >= 1 && R <= 64, "R must be in [1, 64]");
    ANN_REQUIRE(N >= 1 && N < (1ll << 32) && d >= 1 && d <= 4096, "N / d out of range");
    ANN_REQUIRE(nq >= 0 && nq < (1ll << 31), "nq out of range");
    ANN_REQUIRE(entry < N, "entry >= N");
    ANN_REQUIRE(Ls >= 1 && Ls <= 256, "Ls must be in [1, 256]");
    ANN_REQUIRE(topk >= 1 && topk <= Ls, "topk must be in [1, Ls]");
    return ANN_OK;
}

int ann_search(const uint32_t* graph, const uint32_t* degree, int R, const void* X, int64_t N,
               int d, int dtype, const void* Q, int64_t nq, uint32_t entry, int Ls, int topk,
               uint32_t* out_id, uint32_t* out_count, void* stream) {
    int rc = search_args(R, N, d, dtype, nq, entry, Ls, topk);
    if (rc) return rc;
    ANN_REQUIRE(nq == 0 || (graph && degree && X && Q && out_id && out_count), "NULL pointer");
    if (nq > 0 && ((rc = check_readable(X, "X")) || (rc = check_readable(Q, "Q")))) return rc;
    return run_search(graph, degree, R, X, N, d, dtype, Q, nq, entry, nullptr, 0, Ls, topk,
                      out_id, out_count, (cudaStream_t)stream);
}

int ann_search_entries(const uint32_t* graph, const uint32_t* degree, int R, const void* X,
                       int64_t N, int d, int dtype, const void* Q, int64_t nq,
                       const uint32_t* entries, int ne, int Ls, int topk, uint32_t* out_id,
                       uint32_t* out_count, void* stream) {
    int rc = search_args(R, N, d, dtype, nq, 0, Ls, topk);
    if (rc) return rc;
    ANN_REQUIRE(ne >= 1 && ne <= (1 << 20), "ne must be in [1, 2^20]");
    ANN_REQUIRE(nq == 0 || (graph && degree && X && Q && entries && out_id && out_count),
                "NULL pointer");
    if (nq > 0 && ((rc = check_readable(X, "X")) || (rc = check_readable(Q, "Q")))) return rc;
    return run_search(graph, degree, R, X, N, d, dtype, Q, nq, 0, entries, ne, Ls, topk, out_id,
                      out_count, (cudaStream_t)stream);
}

int ann_recall(const uint32_t* found, int found_stride, const uint32_t* truth, int truth_stride,
               int64_t nq, int kk, float* recall_out, void* stream) {
    ANN_REQUIRE(kk >= 1 && kk <= found_stride && kk <= truth_stride, "bad kk / strides");
    ANN_REQUIRE(nq >= 0 && recall_out, "bad nq / NULL recall_out");
    ANN_REQUIRE(nq == 0 || (found && truth), "NULL pointer");
    unsigned long long* h = hits_ptr();
    if (!h) return fail(ANN_ERR_CUDA, "hit counter unavailable");
    return run_recall(found, found_stride, truth, truth_stride, nq, kk, recall_out, h,
                      (cudaStream_t)stream);
}

int ann_search_eval(const uint32_t* graph, const uint32_t* degree, int R, const void* X,
                    int64_t N, int d, int dtype, const void* Q, int64_t nq, const uint32_t* gt,
                    uint32_t entry, int Ls, uint32_t* out_id, float* recall_out,
                    uint32_t* dist_count_out, void* stream) {
    ANN_REQUIRE(Ls >= 10, "Ls must be >= 10 for recall@10");
    ANN_REQUIRE(nq == 0 || gt, "gt is NULL");
    ANN_REQUIRE(recall_out, "recall_out is NULL");
    int rc = ann_search(graph, degree, R, X, N, d, dtype, Q, nq, entry, Ls, 10, out_id,
                        dist_count_out, stream);
    if (rc) return rc;
    return ann_recall(out_id, 10, gt, 10, nq, 10, recall_out, stream);
}

}  // extern "C"
