// Query-side evaluation of the merged graph (Sec. VI-B2: top-10 recall with a
// best-first search following DiskANN's strategy; Sec. VI-B2 also reports the
// number of distance computations as a proxy for latency).
//
//  k_search : one warp per query.  The candidate list (<= 256 entries, sorted
//             by (distance, id), with an "expanded" flag) and a visited hash
//             set live in shared memory.  Expanding a vertex lets lane j take
//             out-neighbour j: unseen neighbours are inserted into the visited
//             set (atomicCAS) and get their distance from one lane in FP32 with
//             terms added in index order, unfused (the same value a plain loop
//             gives), then enter the list in lane order.
//  medoid   : FP64 column sums (fixed-order two-pass reduction), mean rounded
//             to float, then argmin of (d32, id) with a 64-bit atomicMin.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "stages.cuh"

namespace ann {

__device__ __forceinline__ float d32_vec(const float* __restrict__ q, const void* X, int dtype,
                                         int64_t row, int d) {
    float s = 0.0f;
    const int64_t b = row * d;
    for (int t = 0; t < d; ++t) {
        const float df = __fsub_rn(q[t], load_elem(X, dtype, b + t));
        s = __fadd_rn(s, __fmul_rn(df, df));
    }
    return s;
}

__device__ __forceinline__ bool vis_insert(uint32_t* vis, int mask, uint32_t v) {
    uint32_t h = (v * 2654435761u) & (uint32_t)mask;
    for (int probe = 0; probe <= mask; ++probe) {
        const uint32_t prev = atomicCAS(vis + h, ANN_PAD, v);
        if (prev == ANN_PAD) return true;
        if (prev == v) return false;
        h = (h + 1) & (uint32_t)mask;
    }
    return false;  // table full: treated as seen (reported through the fill count)
}

constexpr int LSMAX = 256;

__global__ void k_search(const uint32_t* __restrict__ graph, const uint32_t* __restrict__ degree,
                         int R, const void* X, int64_t N, int d, int dtype, const void* Q, int64_t nq,
                         uint32_t entry, const uint32_t* __restrict__ entries, int ne, int Ls,
                         int topk, int vis_mask, uint32_t* __restrict__ out_id,
                         uint32_t* __restrict__ out_count, int* status) {
    extern __shared__ __align__(16) uint8_t sm[];
    float* qv = (float*)sm;                       // [d]
    uint32_t* lid = (uint32_t*)(qv + ((d + 3) & ~3));  // [LSMAX]
    float* ld = (float*)(lid + LSMAX);            // [LSMAX]
    uint32_t* lexp = (uint32_t*)(ld + LSMAX);     // [LSMAX]
    uint32_t* vis = lexp + LSMAX;                 // [vis_mask + 1]
    const int lane = threadIdx.x;
    const int64_t q = blockIdx.x;
    if (q >= nq) return;
    for (int t = lane; t < d; t += 32) qv[t] = load_elem(Q, dtype, q * d + t);
    for (int h = lane; h <= vis_mask; h += 32) vis[h] = ANN_PAD;
    __syncwarp();
    uint32_t count = 1, nvis = 1;
    if (entries) {
        // start from the listed entry of smallest (d32, id): lane-parallel, then a
        // warp argmin on the packed (distance bits, id) key
        unsigned long long best = ~0ull;
        uint32_t nvalid = 0;
        for (int e = lane; e < ne; e += 32) {
            uint32_t v = entries[e];
            if (v >= (uint32_t)N) continue;
            ++nvalid;
            const float dv = d32_vec(qv, X, dtype, v, d);
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(dv) << 32) | (unsigned long long)v;
            best = key < best ? key : best;
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, o);
            best = x < best ? x : best;
            nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
        }
        if (best == ~0ull) {  // no valid entry
            if (lane == 0) atomicOr(status, DEV_BAD_INPUT);
            for (int e = lane; e < topk; e += 32) out_id[q * topk + e] = ANN_PAD;
            if (lane == 0) out_count[q] = 0;
            return;
        }
        entry = (uint32_t)(best & 0xFFFFFFFFull);
        count += nvalid;
    }
    int n = 1;
    if (lane == 0) {
        lid[0] = entry;
        ld[0] = d32_vec(qv, X, dtype, entry, d);
        lexp[0] = 0;
        vis_insert(vis, vis_mask, entry);
    }
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1;
    for (int guard = 0; guard < (1 << 24); ++guard) {
        int cur = -1;
        for (int e0 = 0; e0 < n; e0 += 32) {
            const int e = e0 + lane;
            const uint32_t b = __ballot_sync(0xffffffffu, e < n && !lexp[e]);
            if (b) { cur = e0 + __ffs(b) - 1; break; }
        }
        if (cur < 0) break;
        const uint32_t u = lid[cur];
        __syncwarp();
        if (lane == 0) lexp[cur] = 1;
        __syncwarp();
        int deg = (int)degree[u];
        if (deg > R) deg = R;
        for (int j0 = 0; j0 < deg; j0 += 32) {
            const int j = j0 + lane;
            uint32_t v = j < deg ? graph[(int64_t)u * R + j] : ANN_PAD;
            if (v >= (uint32_t)N) v = ANN_PAD;
            const bool isnew = v != ANN_PAD && vis_insert(vis, vis_mask, v);
            const float dv = isnew ? d32_vec(qv, X, dtype, v, d) : INFINITY;
            uint32_t b = __ballot_sync(0xffffffffu, isnew);
            count += __popc(b);
            nvis += __popc(b);
            while (b) {
                const int src = __ffs(b) - 1;
                b &= b - 1;
                const uint32_t cv = __shfl_sync(0xffffffffu, v, src);
                const float cd = __shfl_sync(0xffffffffu, dv, src);
                int pos = 0;
                for (int e0 = 0; e0 < n; e0 += 32) {
                    const int e = e0 + lane;
                    const bool less = e < n && (ld[e] < cd || (ld[e] == cd && lid[e] < cv));
                    pos += __popc(__ballot_sync(0xffffffffu, less));
                }
                if (pos >= Ls) continue;
                const int last = n < Ls ? n : Ls - 1;  // entries [pos, last) move up by one
                uint32_t ti[LSMAX / 32], te[LSMAX / 32];
                float td[LSMAX / 32];
#pragma unroll
                for (int r = 0; r < LSMAX / 32; ++r) {
                    const int e = pos + r * 32 + lane;
                    if (e < last) { ti[r] = lid[e]; td[r] = ld[e]; te[r] = lexp[e]; }
                }
                __syncwarp();
#pragma unroll
                for (int r = 0; r < LSMAX / 32; ++r) {
                    const int e = pos + r * 32 + lane;
                    if (e < last) { lid[e + 1] = ti[r]; ld[e + 1] = td[r]; lexp[e + 1] = te[r]; }
                }
                if (lane == 0) { lid[pos] = cv; ld[pos] = cd; lexp[pos] = 0; }
                __syncwarp();
                if (n < Ls) ++n;
            }
        }
        (void)lt;
        if (nvis * 10 > (uint32_t)(vis_mask + 1) * 9) {
            if (lane == 0) atomicOr(status, DEV_OVERFLOW);
            break;
        }
    }
    for (int e = lane; e < topk; e += 32) out_id[q * topk + e] = e < n ? lid[e] : ANN_PAD;
    if (lane == 0) out_count[q] = count;
}

// ---- recall ------------------------------------------------------------------------
__global__ void k_recall_count(const uint32_t* __restrict__ found, int fs,
                               const uint32_t* __restrict__ truth, int ts, int64_t nq, int kk,
                               unsigned long long* hits) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long h = 0;
    if (q < nq) {
        for (int a = 0; a < kk; ++a) {
            const uint32_t f = found[q * fs + a];
            if (f == ANN_PAD) continue;
            for (int b = 0; b < kk; ++b)
                if (truth[q * ts + b] == f) { ++h; break; }
        }
    }
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0 && h) atomicAdd(hits, h);
}

__global__ void k_recall_finish(const unsigned long long* hits, int64_t nq, int kk, float* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *out = nq > 0 ? (float)((double)*hits / ((double)nq * kk)) : 0.0f;
}

// ---- medoid --------------------------------------------------------------------------
constexpr int MED_ROWS = 4096;  // rows per partial-sum chunk

// Chunk c (rows [c * MED_ROWS, ...)) of column t; chunks c = blockIdx.y,
// blockIdx.y + gridDim.y, ... (the grid's y extent is capped at 65535).
__global__ void k_col_partials(const void* X, int64_t N, int d, int dtype, int64_t nchunk,
                               double* __restrict__ part /* [nchunk][d] */) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d) return;
    for (int64_t c = blockIdx.y; c < nchunk; c += gridDim.y) {
        const int64_t r0 = c * (int64_t)MED_ROWS;
        double s = 0.0;
        const int64_t r1 = r0 + MED_ROWS < N ? r0 + MED_ROWS : N;
        for (int64_t r = r0; r < r1; ++r) s += (double)load_elem(X, dtype, r * d + t);
        part[c * (int64_t)d + t] = s;
    }
}

__global__ void k_col_mean(const double* __restrict__ part, int64_t nchunk, int64_t N, int d,
                           float* __restrict__ mean, unsigned long long* best) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *best = ~0ull;
    if (t >= d) return;
    double s = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) s += part[c * d + t];
    mean[t] = (float)(s / (double)N);
}

__global__ void k_nearest(const void* X, int64_t N, int d, int dtype, const float* __restrict__ mean,
                          unsigned long long* best) {
    unsigned long long b = ~0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float di = d32_vec(mean, X, dtype, i, d);
        const unsigned long long key = ((unsigned long long)f2ord(di) << 32) | (uint32_t)i;
        b = key < b ? key : b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
        b = y < b ? y : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(best, b);
}

__global__ void k_entry_out(const unsigned long long* best, uint32_t* entry) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *entry = (uint32_t)(*best & 0xFFFFFFFFull);
}

// ---- host drivers -----------------------------------------------------------------------
int search_vis_mask(int Ls, int R) {
    int64_t want = (int64_t)4 * Ls * R;
    int64_t cap = 2048;
    while (cap < want && cap < 16384) cap <<= 1;
    return (int)cap - 1;
}

int run_search(const uint32_t* graph, const uint32_t* degree, int R, const void* X, int64_t N, int d,
               int dtype, const void* Q, int64_t nq, uint32_t entry, const uint32_t* entries,
               int ne, int Ls, int topk, uint32_t* out_id, uint32_t* out_count, cudaStream_t st) {
    if (nq == 0) return ANN_OK;
    const int vis_mask = search_vis_mask(Ls, R);
    const size_t smem = (size_t)((d + 3) & ~3) * 4 + (size_t)LSMAX * 12 + (size_t)(vis_mask + 1) * 4;
    ANN_CHECK_CUDA(cudaFuncSetAttribute(k_search, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    k_search<<<(unsigned)nq, 32, smem, st>>>(graph, degree, R, X, N, d, dtype, Q, nq, entry,
                                             entries, ne, Ls, topk, vis_mask, out_id, out_count,
                                             device_status_ptr());
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

int run_recall(const uint32_t* found, int fs, const uint32_t* truth, int ts, int64_t nq, int kk,
               float* recall_out, unsigned long long* hits, cudaStream_t st) {
    ANN_CHECK_CUDA(cudaMemsetAsync(hits, 0, sizeof(unsigned long long), st));
    if (nq > 0) {
        k_recall_count<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(found, fs, truth, ts, nq, kk, hits);
        ANN_CHECK_LAUNCH();
    }
    k_recall_finish<<<1, 32, 0, st>>>(hits, nq, kk, recall_out);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

size_t medoid_ws(int64_t N, int d, double** part, float** mean, unsigned long long** best, void* base,
                 size_t cap) {
    Carver cv(base, cap);
    const int64_t nchunk = (N + MED_ROWS - 1) / MED_ROWS;
    double* p = cv.take<double>((size_t)(nchunk > 0 ? nchunk : 1) * d);
    float* m = cv.take<float>((size_t)d);
    unsigned long long* b = cv.take<unsigned long long>(1);
    if (part) *part = p;
    if (mean) *mean = m;
    if (best) *best = b;
    return cv.used + 256;
}

int run_medoid(const void* X, int64_t N, int d, int dtype, uint32_t* entry, double* part, float* mean,
               unsigned long long* best, cudaStream_t st) {
    const int64_t nchunk = (N + MED_ROWS - 1) / MED_ROWS;
    dim3 g1((unsigned)((d + 127) / 128), (unsigned)(nchunk < 65535 ? nchunk : 65535));
    k_col_partials<<<g1, 128, 0, st>>>(X, N, d, dtype, nchunk, part);
    ANN_CHECK_LAUNCH();
    k_col_mean<<<(unsigned)((d + 127) / 128), 128, 0, st>>>(part, nchunk, N, d, mean, best);
    ANN_CHECK_LAUNCH();
    int64_t want = (N + 255) / 256;
    k_nearest<<<(unsigned)(want < 152 * 16 ? want : 152 * 16), 256, 0, st>>>(X, N, d, dtype, mean, best);
    ANN_CHECK_LAUNCH();
    k_entry_out<<<1, 32, 0, st>>>(best, entry);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

// ---- medoid without allocation -----------------------------------------------------
// Scratch of ann_medoid_noalloc: per-chunk FP64 column sums, the float mean and
// the 64-bit argmin, in one array reserved for the lifetime of the process on
// every device that loads the library.
constexpr size_t NOALLOC_PART_DOUBLES = (size_t)1 << 19;  // 4 MiB of column sums
constexpr size_t NOALLOC_MEAN_FLOATS = 4096;               // d <= 4096
constexpr size_t NOALLOC_BYTES = NOALLOC_PART_DOUBLES * 8 + NOALLOC_MEAN_FLOATS * 4 + 256;
static __device__ __align__(256) unsigned char g_medoid_scratch[NOALLOC_BYTES];

// Device address of g_medoid_scratch in the current context, looked up once per
// context (with its device current) and cached.  The cache is keyed on the
// driver context, so a context created after a device reset gets its own
// lookup.  Host code must never hand the symbol itself to a kernel: on the host
// it names a stand-in, not device memory.
typedef int (*PFN_ctxGetCurrent)(void**);

static int current_context(void** ctx) {
    static PFN_ctxGetCurrent fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return fail(ANN_ERR_CUDA, "cuCtxGetCurrent unavailable");
        fn = (PFN_ctxGetCurrent)p;
    }
    *ctx = nullptr;
    if (fn(ctx) != 0) return fail(ANN_ERR_CUDA, "cuCtxGetCurrent failed");
    return ANN_OK;
}

static int medoid_scratch_ptr(unsigned char** out) {
    static std::mutex mu;
    constexpr int SLOTS = 64;
    static void* ctxs[SLOTS] = {nullptr};
    static unsigned char* ptrs[SLOTS] = {nullptr};
    void* ctx = nullptr;
    int rc = current_context(&ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(mu);
    int slot = -1;
    for (int i = 0; ctx && i < SLOTS; ++i)
        if (ctxs[i] == ctx) { slot = i; break; }
    if (slot < 0) {
        // The lookup also makes the current device's primary context current on
        // this thread when none was.
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_medoid_scratch);
        if (e != cudaSuccess || !p)
            return fail(ANN_ERR_CUDA, "cudaGetSymbolAddress(g_medoid_scratch): %s",
                        cudaGetErrorString(e));
        if (!ctx && (rc = current_context(&ctx))) return rc;
        slot = 0;
        for (int i = 0; i < SLOTS; ++i)
            if (!ctxs[i]) { slot = i; break; }
        // all slots taken (more than 64 contexts seen): reuse slot 0
        ctxs[slot] = ctx;
        ptrs[slot] = (unsigned char*)p;
    }
    *out = ptrs[slot];
    return ANN_OK;
}

// Size limits of ann_medoid_noalloc (checked before any pointer query or launch).
int medoid_noalloc_check(int64_t N, int d) {
    const int64_t nchunk = (N + MED_ROWS - 1) / MED_ROWS;
    if (d < 1 || d > (int)NOALLOC_MEAN_FLOATS)
        return fail(ANN_ERR_INVALID_ARG, "ann_medoid_noalloc: d must be in [1, %d]",
                    (int)NOALLOC_MEAN_FLOATS);
    if ((size_t)nchunk * (size_t)d > NOALLOC_PART_DOUBLES)
        return fail(ANN_ERR_INVALID_ARG,
                    "ann_medoid_noalloc: ceil(N / %d) * d = %lld exceeds the fixed scratch of "
                    "%zu column sums; use ann_medoid with a workspace",
                    MED_ROWS, (long long)nchunk * d, NOALLOC_PART_DOUBLES);
    return ANN_OK;
}

int run_medoid_noalloc(const void* X, int64_t N, int d, int dtype, uint32_t* entry,
                       cudaStream_t st) {
    int rc = medoid_noalloc_check(N, d);
    if (rc) return rc;
    unsigned char* base = nullptr;
    rc = medoid_scratch_ptr(&base);
    if (rc) return rc;
    // Every scratch byte read below is written first in the same call (partial
    // sums, then the mean and the argmin seed), so nothing needs clearing.
    double* part = (double*)base;
    float* mean = (float*)(base + NOALLOC_PART_DOUBLES * 8);
    unsigned long long* best =
        (unsigned long long*)(base + NOALLOC_PART_DOUBLES * 8 + NOALLOC_MEAN_FLOATS * 4);
    return run_medoid(X, N, d, dtype, entry, part, mean, best, st);
}

}  // namespace ann
