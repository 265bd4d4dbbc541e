// Exact per-shard kNN (Sec. IV Workflow (2): each shard's graph is built
// independently, with no exchange between shards).
//
// Distance tiles are dense contractions on the 5th-generation tensor cores:
//   dist(i, j) = |x_i|^2 + |y_j|^2 - 2 x_i . y_j = |x_i|^2 + 2 key(i, j),
//   key(i, j)  = |y_j|^2 / 2 - x_i . y_j.
// |x_i|^2 is constant along a row, so rows are ranked by key.  The key comes out
// of the tensor cores whole: the main MMAs run with A negated (-x . y) and one
// extra K=16 step adds [1, 1, 1, 0, ...] . [h, m, l, 0, ...], where h + m + l
// is |y_j|^2 / 2 split exactly into three BF16 values.
//
// Kernel k_knn_tiles: one CTA per 128-row block of one problem (a shard, or a
// query batch against all vectors); all problems in one launch, largest first.
// Warp roles:
//   warp 0   : TMA producer.  The CTA's A rows (all K) stay resident in shared
//              memory when they fit, else their K blocks stream beside the B
//              blocks (large d); B tiles of 256 (or 128) rows stream through a
//              ring of stages (one 128-byte K block, 128-byte swizzle) and their
//              16-element norm blocks through a second, small ring (32-byte
//              swizzle).
//   warp 1   : allocates 512 TMEM columns (two FP32 accumulators) and issues
//              tcgen05.mma (M=128, N=256 or 128, K=16; K=32 for E4M3) from one
//              thread.  The issue of an MMA waits for room in the tensor pipe, so
//              the thread does little else: one commit per stage and one per tile.
//   warps 2-9: epilogue, two warps per TMEM lane quarter (one thread per row,
//              one column half per warp).  32-column chunks are read with
//              tcgen05.ld (the next chunk's load overlaps the current chunk's
//              work) and reduced with 3-input minima; a chunk is skipped unless
//              some row of the warp has a key at or below its threshold (the
//              smaller of the bounds its two column halves have reached).
//              Survivors (key, column) are stashed in shared memory and, once
//              the tile's accumulator is back with the MMA warp, appended with
//              their global ids to the row's candidate pool for that half (in
//              global memory, no lock: each half has one writer).  A pool that
//              would overflow is compacted by its warp: a cooperative selection
//              finds a bound keeping between k' and k' plus an eighth of the
//              slack entries, the rest are dropped and the threshold lowered.
//              After the sweep k_pool_finalize selects each row's k' smallest
//              (key, global id) from its two pools, so ties go to the smaller
//              id whatever the order the candidates came in.
// Rows are ordered by cell, cells along a chain of nearby pivots (see
// run_shard_knn), and each sweep starts at the block's own tile and moves
// outward, so the thresholds are tight after the first few tiles and later
// chunks are almost always skipped.
// Every wait is bounded; on a timeout the CTA records DEV_TIMEOUT, drains its
// copies, frees TMEM and returns.
//
// Operand modes:
//   plain : A = B = one BF16/FP16 copy of the vectors.  uint8 values, their
//           products and all partial sums (integers or half-integers below
//           2^23 for d <= 128) are exact in BF16 x BF16 -> FP32.
//   split : float vectors stored as hi = bf16(x), lo = bf16(x - hi) in two
//           K sections; x.y ~ hi.hi + hi.lo + lo.hi (three products), used to
//           screen a widened list that k_rerank re-scores in FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "stages.cuh"

namespace ann {

namespace kt {
constexpr int BM = 128;
constexpr int BNMAX = 256;              // widest tile (N of one MMA)
constexpr int KB = 64;                  // 16-bit elements per 128-byte K block
constexpr int KB8 = 128;                // 8-bit elements per 128-byte K block
constexpr int KAUG = 16;                // norm block: 16 elements (32 bytes)
constexpr int A_BLK_BYTES = BM * 128;   // one K block of the 128 A rows
constexpr int A_AUG_BYTES = BM * 32;
constexpr int NAUG = 1;                 // norm-block slots (loaded first in each tile)
constexpr int NACC = 2;
constexpr int EPI_WARPS = 8;            // two warps per TMEM lane quarter
constexpr int PH_MAX = 320;             // candidate pool entries per row half, at most
constexpr int SC = 24;                  // survivors a thread stashes before a tile's release
constexpr int KS = 33;                  // floats per row of a warp's key scratch (32 + 1 pad)
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = NACC * BNMAX;
constexpr int MAX_NST = 6;
constexpr int CELL = 128;               // rows per pivot cell, short rows (at most 1024 a shard)
constexpr int CELL_WIDE = 1024;         // rows per pivot cell, rows over 512 bytes
constexpr int TL_MAX = 2048;            // tile-list entries per row block (shards of <= 2048 tiles)
}  // namespace kt

// Optional per-role cycle and event counters of k_knn_tiles (ann_tile_counters_*).
enum TileCounter {
    TC_EPI_CYCLES = 0,   // epilogue threads: cycles from first wait to the end of the sweep
    TC_EPI_WAIT,         // epilogue threads: cycles waiting for a finished accumulator
    TC_EPI_FLUSH,        // epilogue threads: cycles inside pool compactions
    TC_CHUNKS,           // warp-level: 32-column chunks examined
    TC_SLOW_CHUNKS,      // warp-level: chunks where some row had a candidate
    TC_FLUSHES,          // warp-level: compaction calls
    TC_FLUSH_ITERS,      // warp-level: rows compacted
    TC_INSERTS,          // thread-level: pool entries left after compactions (unused: 0)
    TC_APPENDS,          // thread-level: survivors appended to the pools
    TC_MMA_WAIT_FULL,    // MMA thread: cycles waiting for B stages
    TC_MMA_WAIT_ACC,     // MMA thread: cycles waiting for a free accumulator
    TC_PROD_WAIT,        // producer: cycles waiting for a free stage
    TC_CTA_CYCLES,       // thread 0: cycles from start to teardown
    TC_CTAS,             // CTAs that ran
    TC_LD_WAIT,          // epilogue threads: cycles blocked in tcgen05.wait::ld
    TC_FILTER,           // epilogue threads: cycles in the chunk filter (min + vote)
    TC_APPEND,           // epilogue threads: cycles appending survivors (incl. flush)
    TC_MMA_ISSUE,        // MMA thread: cycles issuing tcgen05.mma
    TC_MMA_COMMIT,       // MMA thread: cycles in tcgen05.commit
    TC_MMA_LOOP,         // MMA thread: cycles from the A wait to the end of the tile loop
    TC_STASH,            // epilogue threads: cycles writing survivors to the stash
    TC_DIRECT,           // epilogue threads: cycles appending a chunk straight to the pools
    TC_FLUSH_LOOP,       // epilogue threads: cycles moving stashed survivors to the pools
    TC_N
};
__device__ unsigned long long g_tile_counters[TC_N];

struct KnnParams {
    const int64_t* blk_off;  // [nprob+1] prefix sums of row blocks
    const KnnProblem* probs;
    int nprob;
    const float* na;          // |x|^2 per A row
    const uint32_t* gid;      // global id per B row (NULL: the column index itself)
    const int64_t* outrow;    // output row per A row (NULL: out_row0 + row index)
    int self_exclude;
    int local_first;          // sweep the columns near the row block first
    int mode;      // 0 plain, 1 split
    int nkb_a;     // A k-blocks (resident unless a_stream)
    int a_stream;  // A blocks per ring stage (0: A resident; large d: 1, or 2 for split)
    int nkb_b;     // B k-blocks per tile
    int kprime;    // list width k': candidates kept per row
    int k_out;     // entries written per row
    int nst;       // main pipeline stages
    int kbe;       // elements per 128-byte K block (64 for 16-bit, 128 for 8-bit operands)
    int kind8;     // 1: E4M3 operands (tcgen05.mma kind::f8f6f4, K = 32 per MMA)
    // K steps of 32 bytes (one MMA each) that hold data: steps at and beyond ksteps
    // are zero padding of the last K block and are not issued.  Split operands with
    // resident A (compact layout): steps [0, hs) are the hi section, [hs, 2 hs) the
    // lo section, both of B and of A.
    int ksteps, hs;
    uint32_t idesc_neg, idesc_aug;
    uint32_t* out_id;
    float* out_d;
    int* status;
    // Exact tile skipping (NULL: every tile of the row block's shard).  tlist:
    // TL_MAX entries per row block, the column tiles it sweeps in sweep order;
    // tcount: their number (-1: sweep every tile).  Used only where the shard has
    // at most TL_MAX tiles.
    const uint16_t* tlist;
    const int* tcount;
    // Candidate pools (global memory): A row a, column half h holds its survivors
    // at pool[(2 a + h) * ph ...], their number in pool_cnt[2 a + h] after the sweep.
    uint64_t* pool;
    int* pool_cnt;
    int ph;
    // Optional upper bound of every A row's k'-th squared distance (rowub[a]; NULL:
    // none): the sweep starts with that threshold.  Keys of split operands carry an
    // error, covered by the relative margin ub_margin (0 for exact keys).
    const float* rowub;
    float ub_margin;
};

// Entries of a row half's candidate pool, whole warps: 256 (what a compaction holds
// in registers) for list widths 32 to 128, the list width plus 64 above; always at
// least 32 more than k' (a chunk's survivors fit after a compaction).  A larger pool
// compacts less often at the same cost per compaction.
__host__ __device__ inline int pool_half(int kprime) {
    int ph = kprime < 32 ? 2 * kprime : kprime <= 128 ? 256 : kprime + 64;
    if (ph < kprime + 32) ph = kprime + 32;
    ph = (ph + 31) / 32 * 32;
    return ph > kt::PH_MAX ? kt::PH_MAX : ph;
}

struct KnnSmemLayout {
    uint32_t a, aaug, b, baug, tau, stash, kscr, bars, tmem_slot, abort_flag, total;
};

// a_stream = 0: the CTA's A rows stay resident (nkb_a K blocks) and a ring stage
// holds one B block; a_stream > 0 (large d): nothing resident, a stage holds one
// B block followed by the a_stream A blocks it multiplies (split operands: the hi
// and lo blocks against a hi B block, the hi block against a lo B block).
__host__ __device__ inline uint32_t knn_stage_bytes(int bn, int a_stream) {
    return (uint32_t)bn * 128 + a_stream * kt::A_BLK_BYTES;
}

__host__ __device__ inline KnnSmemLayout knn_smem_layout(int bn, int nkb_a, int nst, int a_stream) {
    KnnSmemLayout L;
    uint32_t o = 0;
    L.a = o;
    o += (a_stream ? 0 : nkb_a) * kt::A_BLK_BYTES;
    L.aaug = o;
    o += 1024 * ((kt::A_AUG_BYTES + 1023) / 1024);
    L.b = o;
    o += nst * knn_stage_bytes(bn, a_stream);
    L.baug = o;
    o += kt::NAUG * bn * 32;
    L.tau = o;  // [2][BM] floats: each column half's current k'-th key per row
    o += 2 * kt::BM * 4;
    L.stash = o;  // [EPI_WARPS][SC][32] survivors (key bits << 32 | column), lane-minor
    o += kt::EPI_WARPS * kt::SC * 32 * 8;
    L.kscr = o;   // [EPI_WARPS][32][KS] a chunk's keys, one row per thread
    o += kt::EPI_WARPS * 32 * kt::KS * 4;
    L.bars = o;
    o += (2 * kt::MAX_NST + 2 * kt::NAUG + 2 * kt::NACC + 2) * 8;
    L.tmem_slot = o;
    o += 4;
    L.abort_flag = o;
    o += 4;
    L.total = o + 1024;  // slack for 1024-byte alignment of the base
    return L;
}

// Wait for outstanding tcgen05.ld; the registers are tied to the wait so that no
// use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused when swizzled)
    d |= (uint64_t)(256 >> 4) << 32;        // stride byte offset: 8 rows x 32 B
    d |= (uint64_t)1 << 46;                 // descriptor version (sm_100 family)
    d |= (uint64_t)6 << 61;                 // layout: SWIZZLE_32B
    return d;
}

__device__ __forceinline__ float min32(const float (&k)[32]) {
    float a[11];
#pragma unroll
    for (int q = 0; q < 10; ++q) a[q] = min3f(k[3 * q], k[3 * q + 1], k[3 * q + 2]);
    a[10] = fminf(k[30], k[31]);
    const float b0 = min3f(a[0], a[1], a[2]), b1 = min3f(a[3], a[4], a[5]);
    const float b2 = min3f(a[6], a[7], a[8]), b3 = fminf(a[9], a[10]);
    return fminf(min3f(b0, b1, b2), b3);
}

// ---- per-row candidate pools ----------------------------------------------------
// The smallest `kp` composite values (key bits << 32 | global id) among a warp's
// entries, E per lane (UINT64_MAX = no entry), n valid in all: returns the kp-th
// smallest valid value (the largest valid one when n <= kp).  Bisection first on
// the key bits, then on the ids of the entries tied at the k-th key; every count is
// a warp-wide sum (redux.sync), so all lanes return the same value.
template <int E>
__device__ __forceinline__ uint64_t warp_select_kth(const uint64_t (&v)[E], int n, int kp) {
    const uint32_t FULL = 0xffffffffu;
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (v[e] != ~0ull) {
            const uint32_t h = (uint32_t)(v[e] >> 32);
            kmin = h < kmin ? h : kmin;
            kmax = h > kmax ? h : kmax;
        }
    }
    kmin = __reduce_min_sync(FULL, kmin);
    kmax = __reduce_max_sync(FULL, kmax);
    if (n <= kp) {  // every entry stays: the largest one
        uint32_t imax = 0;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (v[e] != ~0ull && (uint32_t)(v[e] >> 32) == kmax) {
                const uint32_t id = (uint32_t)v[e];
                imax = id > imax ? id : imax;
            }
        imax = __reduce_max_sync(FULL, imax);
        return ((uint64_t)kmax << 32) | imax;
    }
    // least key K with #{key <= K} >= kp: each step counts at three pivots that
    // split [lo, hi] in four (independent warp sums) and keeps one quarter
    uint32_t lo = kmin, hi = kmax;
    while (lo < hi) {
        const uint32_t q = (hi - lo) >> 2;
        const uint32_t p1 = lo + q, p2 = lo + ((hi - lo) >> 1), p3 = hi - q - 1 > p2 ? hi - q - 1 : p2;
        uint32_t c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t h = (uint32_t)(v[e] >> 32);
            c1 += h <= p1 ? 1u : 0u;
            c2 += h <= p2 ? 1u : 0u;
            c3 += h <= p3 ? 1u : 0u;
        }
        c1 = __reduce_add_sync(FULL, c1);
        c2 = __reduce_add_sync(FULL, c2);
        c3 = __reduce_add_sync(FULL, c3);
        if (c1 >= (uint32_t)kp) hi = p1;
        else if (c2 >= (uint32_t)kp) { lo = p1 + 1; hi = p2; }
        else if (c3 >= (uint32_t)kp) { lo = p2 + 1; hi = p3; }
        else lo = p3 + 1;
    }
    const uint32_t K = lo;
    uint32_t below = 0, tied = 0, imin = 0xFFFFFFFFu, imax = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t h = (uint32_t)(v[e] >> 32), id = (uint32_t)v[e];
        below += h < K ? 1u : 0u;
        if (h == K && v[e] != ~0ull) {
            ++tied;
            imin = id < imin ? id : imin;
            imax = id > imax ? id : imax;
        }
    }
    below = __reduce_add_sync(FULL, below);
    tied = __reduce_add_sync(FULL, tied);
    imin = __reduce_min_sync(FULL, imin);
    imax = __reduce_max_sync(FULL, imax);
    const uint32_t need = (uint32_t)kp - below;  // 1 <= need <= tied
    if (need >= tied) return ((uint64_t)K << 32) | imax;
    uint32_t ilo = imin, ihi = imax;  // least id I with #{key == K, id <= I} >= need
    while (ilo < ihi) {
        const uint32_t mid = ilo + ((ihi - ilo) >> 1);
        uint32_t c = 0;
#pragma unroll
        for (int e = 0; e < E; ++e)
            c += ((uint32_t)(v[e] >> 32) == K && v[e] != ~0ull && (uint32_t)v[e] <= mid) ? 1u : 0u;
        c = __reduce_add_sync(FULL, c);
        if (c >= need) ihi = mid; else ilo = mid + 1;
    }
    return ((uint64_t)K << 32) | ilo;
}

// A bound T with kp <= #{entries <= T} <= maxkeep (n > maxkeep valid entries, E per
// lane): the same search on the key bits as warp_select_kth, stopped as soon as the
// keys at or below the upper end of the range number at most maxkeep; only when
// more than maxkeep entries share the kp-th key are the ids of those entries
// searched (then exactly kp stay).  Every entry at or below T is kept by the
// caller, so the bound tightens by whole keys without an exact selection.
template <int E>
__device__ __forceinline__ uint64_t warp_select_bound(const uint64_t (&v)[E], int n, int kp,
                                                      int maxkeep) {
    const uint32_t FULL = 0xffffffffu;
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (v[e] != ~0ull) {
            const uint32_t h = (uint32_t)(v[e] >> 32);
            kmin = h < kmin ? h : kmin;
            kmax = h > kmax ? h : kmax;
        }
    }
    kmin = __reduce_min_sync(FULL, kmin);
    kmax = __reduce_max_sync(FULL, kmax);
    // invariant: #{key <= hi} = chi >= kp, #{key < lo} < kp
    uint32_t lo = kmin, hi = kmax, chi = (uint32_t)n;
    while (chi > (uint32_t)maxkeep && lo < hi) {
        const uint32_t q = (hi - lo) >> 2;
        const uint32_t p1 = lo + q, p2 = lo + ((hi - lo) >> 1), p3 = hi - q - 1 > p2 ? hi - q - 1 : p2;
        uint32_t c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t h = (uint32_t)(v[e] >> 32);
            c1 += h <= p1 ? 1u : 0u;
            c2 += h <= p2 ? 1u : 0u;
            c3 += h <= p3 ? 1u : 0u;
        }
        c1 = __reduce_add_sync(FULL, c1);
        c2 = __reduce_add_sync(FULL, c2);
        c3 = __reduce_add_sync(FULL, c3);
        if (c1 >= (uint32_t)kp) { hi = p1; chi = c1; }
        else if (c2 >= (uint32_t)kp) { lo = p1 + 1; hi = p2; chi = c2; }
        else if (c3 >= (uint32_t)kp) { lo = p2 + 1; hi = p3; chi = c3; }
        else lo = p3 + 1;
    }
    if (chi <= (uint32_t)maxkeep) return ((uint64_t)hi << 32) | 0xFFFFFFFFull;
    // more than maxkeep entries at or below the kp-th key K = hi: the ties at K are
    // split by id so that exactly kp entries stay
    const uint32_t K = hi;
    uint32_t below = 0, imin = 0xFFFFFFFFu, imax = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t h = (uint32_t)(v[e] >> 32), id = (uint32_t)v[e];
        below += h < K ? 1u : 0u;
        if (h == K && v[e] != ~0ull) {
            imin = id < imin ? id : imin;
            imax = id > imax ? id : imax;
        }
    }
    below = __reduce_add_sync(FULL, below);
    imin = __reduce_min_sync(FULL, imin);
    imax = __reduce_max_sync(FULL, imax);
    const uint32_t need = (uint32_t)kp - below;
    uint32_t ilo = imin, ihi = imax;
    while (ilo < ihi) {
        const uint32_t mid = ilo + ((ihi - ilo) >> 1);
        uint32_t c = 0;
#pragma unroll
        for (int e = 0; e < E; ++e)
            c += ((uint32_t)(v[e] >> 32) == K && v[e] != ~0ull && (uint32_t)v[e] <= mid) ? 1u : 0u;
        c = __reduce_add_sync(FULL, c);
        if (c >= need) ihi = mid; else ilo = mid + 1;
    }
    return ((uint64_t)K << 32) | ilo;
}

// Per-row top-k state of one epilogue thread (lane = row, one column half).
// Survivors of the threshold test are appended to the row half's pool in global
// memory (no lock: each half has its own pool); a pool about to overflow is
// compacted by the whole warp to its kp smallest entries, which makes the kp-th
// of them the half's new threshold tau.  A column half's entries above the other
// half's tau cannot be among the row's kp smallest either, so the test uses
// teff = min(tau, other half's tau) (read from shared memory; it only decreases,
// so a stale value is still a valid bound).  With kp = 1 the pool is the running
// minimum in a register.
struct EpiState {
    uint64_t* pool;       // this thread's row half
    uint64_t* pool0;      // row 0 of the warp, same half (row r at pool0 + 2 r ph)
    float* tau_own;       // shared [BM]: this half's tau per row
    const volatile float* tau_other;
    uint64_t* stash;      // shared: this warp's stash, entry e of lane l at [e * 32 + l]
    const uint32_t* gidrow;  // global id of each column of the shard (NULL: the column)
    uint32_t kscr;        // shared address of this thread's row of the key scratch
    int row, kp, ph, c, sn;
    float tau, teff;
    uint64_t best;        // kp == 1
    // counters (used only by the profiling instantiation)
    unsigned long long c_flush_cyc, c_chunks, c_slow, c_flushes, c_iters, c_app;
    unsigned long long c_ldw, c_filter, c_append, c_stash, c_direct, c_floop;
};

// Compact the pools of the rows in `mask` (lanes of this warp) to their kp
// smallest entries and lower those rows' tau.  Each lane passes its row's count
// and tau and gets them back (changed only for the rows compacted).  Kept out of
// line: it is rare, and the sweep loop keeps two chunks of keys in registers.
struct PoolState {
    int c;
    float tau;
};
template <int EM>  // EM * 32 >= ph
__device__ __noinline__ PoolState epi_compact(uint64_t* pool0, int ph, int kp, int c, float tau,
                                              uint32_t mask, float* tau_own, int row) {
    __syncwarp();  // every lane's appends are visible to the warp
    const int lane = threadIdx.x & 31;
    const int E = ph >> 5;
    while (mask) {
        const int r = __ffs(mask) - 1;
        mask &= mask - 1;
        const int cr = __shfl_sync(0xffffffffu, c, r);
        uint64_t* pr = pool0 + (int64_t)r * 2 * ph;
        uint64_t v[EM];
#pragma unroll
        for (int e = 0; e < EM; ++e) {
            const int idx = lane + 32 * e;
            v[e] = (e < E && idx < cr) ? pr[idx] : ~0ull;
        }
        // keep between kp and maxkeep entries: an eighth of the slack may stay
        // above the kp-th, which lets the bound stop early
        int maxkeep = kp + ((ph - kp) >> 3);
        if (maxkeep > ph - 32) maxkeep = ph - 32;
        if (maxkeep < kp) maxkeep = kp;
        const uint64_t T = cr > maxkeep ? warp_select_bound(v, cr, kp, maxkeep) : ~0ull - 1;
        __syncwarp();  // every load done before the pool is rewritten in place
        int base = 0;
#pragma unroll
        for (int e = 0; e < EM; ++e) {
            const bool keep = v[e] <= T && v[e] != ~0ull;
            const uint32_t b = __ballot_sync(0xffffffffu, keep);
            if (keep) pr[base + __popc(b & ((1u << lane) - 1u))] = v[e];
            base += __popc(b);
        }
        __syncwarp();
        if (lane == r) {
            c = base;
            if (cr > maxkeep) {
                tau = fminf(tau, ord2f((uint32_t)(T >> 32)));
                tau_own[row] = tau;
            }
        }
    }
    __syncwarp();
    PoolState o;
    o.c = c;
    o.tau = tau;
    return o;
}

// Compact the pools of the rows whose count would pass ph with `add` more entries.
template <bool PROF, int EMX>
__device__ __forceinline__ void epi_make_room(EpiState& s, int add) {
    const uint32_t over = __ballot_sync(0xffffffffu, s.c + add > s.ph);
    if (over) {
        long long t0 = 0;
        if (PROF) t0 = clock64();
        // one call site: a dispatch on ph here costs the sweep loop registers
        const PoolState o =
            epi_compact<EMX>(s.pool0, s.ph, s.kp, s.c, s.tau, over, s.tau_own, s.row);
        s.c = o.c;
        s.tau = o.tau;
        s.teff = fminf(s.tau, s.tau_other[s.row]);
        if (PROF) {
            s.c_flush_cyc += clock64() - t0;
            ++s.c_flushes;
            s.c_iters += __popc(over);
        }
    }
}

// Move every thread's stashed survivors (key bits << 32 | shard column) into its
// pool as (key bits << 32 | global id), after a tile's accumulator is released.
template <bool PROF, int EMX>
__device__ __forceinline__ void epi_flush_stash(EpiState& s) {
    if (!__any_sync(0xffffffffu, s.sn > 0)) return;
    long long f0 = 0;
    if (PROF) f0 = clock64();
    epi_make_room<PROF, EMX>(s, s.sn);
    long long fl0 = 0;
    if (PROF) fl0 = clock64();
    const int lane = threadIdx.x & 31;
    const int mx = __reduce_max_sync(0xffffffffu, (uint32_t)s.sn);
    for (int e0 = 0; e0 < mx; e0 += 4) {
        uint64_t v[4];
        uint32_t g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = e0 + q < s.sn ? s.stash[(e0 + q) * 32 + lane] : ~0ull;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t col = (uint32_t)v[q];
            g[q] = (v[q] != ~0ull && s.gidrow) ? __ldg(s.gidrow + col) : col;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (v[q] != ~0ull && ord2f((uint32_t)(v[q] >> 32)) <= s.teff) {
                s.pool[s.c] = (v[q] & 0xFFFFFFFF00000000ull) | g[q];
                ++s.c;
                if (PROF) ++s.c_app;
            }
        }
    }
    s.sn = 0;
    __syncwarp();
    if (PROF) {
        const long long f1 = clock64();
        s.c_floop += f1 - fl0;
        s.c_append += f1 - f0;
    }
}

// One 32-column chunk: keys come straight from TMEM; masked columns become NaN
// (every comparison with NaN is false, and the minimum skips NaN).  A chunk with
// survivors stashes them (shared memory, no global id yet) so the accumulator can
// go back to the MMA warp soon; a thread whose stash cannot take them has the
// stashes emptied first, and a chunk with more survivors than a stash holds (the
// first tiles of a sweep) goes straight to the pools.
template <bool PROF, int EMX>
__device__ __forceinline__ void epi_chunk(EpiState& s, const uint32_t (&v)[32], int j0, int i,
                                          int n_cols, int self_exclude, bool edge) {
    long long f0 = 0;
    if (PROF) {
        ++s.c_chunks;
        f0 = clock64();
    }
    float key[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) key[u] = __uint_as_float(v[u]);
    if (edge) {  // warp-uniform
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int j = j0 + u;
            if (j >= n_cols || (self_exclude && j == i)) key[u] = __uint_as_float(0x7fc00000u);
        }
    }
    const float m = min32(key);
    // "<=": a key equal to the current k-th may still win on the global id
    const bool any = __any_sync(0xffffffffu, m <= s.teff);
    if (PROF) {
        const long long f1 = clock64();
        s.c_filter += f1 - f0;
        f0 = f1;
    }
    if (!any) return;
    if (PROF) ++s.c_slow;
    const int lane = threadIdx.x & 31;
    if (s.kp == 1) {  // the running minimum
        uint32_t g_l = (uint32_t)(j0 + lane);  // global id of column j0 + lane
        if (s.gidrow && j0 + lane < n_cols) g_l = __ldg(s.gidrow + j0 + lane);
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const uint32_t gid = __shfl_sync(0xffffffffu, g_l, u);
            const uint64_t x = ((uint64_t)f2ord(key[u]) << 32) | gid;
            if (key[u] <= s.teff && x < s.best) s.best = x;
        }
        if (s.best != ~0ull) {
            s.tau = ord2f((uint32_t)(s.best >> 32));
            s.teff = s.tau;
        }
        if (PROF) s.c_append += clock64() - f0;
        return;
    }
    s.teff = fminf(s.tau, s.tau_other[s.row]);
    uint32_t surv = 0;  // bit u: column j0 + u survives for this row
#pragma unroll
    for (int u = 0; u < 32; ++u) surv |= (key[u] <= s.teff ? 1u : 0u) << u;
    if (__any_sync(0xffffffffu, s.sn + __popc(surv) > kt::SC)) {
        epi_flush_stash<PROF, EMX>(s);
        surv = 0;
#pragma unroll
        for (int u = 0; u < 32; ++u) surv |= (key[u] <= s.teff ? 1u : 0u) << u;
        if (__any_sync(0xffffffffu, __popc(surv) > kt::SC)) {
            // straight to the pools, global ids shuffled from the lanes that hold them
            uint32_t g_l = (uint32_t)(j0 + lane);
            if (s.gidrow && j0 + lane < n_cols) g_l = __ldg(s.gidrow + j0 + lane);
            epi_make_room<PROF, EMX>(s, __popc(surv));
            long long d0 = 0;
            if (PROF) d0 = clock64();
            const uint32_t any_col = __reduce_or_sync(0xffffffffu, surv);
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                if ((any_col >> u) & 1u) {
                    const uint32_t gid = __shfl_sync(0xffffffffu, g_l, u);
                    if (key[u] <= s.teff) {
                        s.pool[s.c] = ((uint64_t)f2ord(key[u]) << 32) | gid;
                        ++s.c;
                        if (PROF) ++s.c_app;
                    }
                }
            }
            if (PROF) {
                const long long f1 = clock64();
                s.c_direct += f1 - d0;
                s.c_append += f1 - f0;
            }
            return;
        }
    }
    long long w0 = 0;
    if (PROF) w0 = clock64();
    // the chunk's keys to this thread's scratch row (a fixed number of stores, rows
    // padded so the warp's stores hit distinct banks), then only the survivors
    // into the stash (a loop as long as the thread's survivor count)
    if (surv) {
#pragma unroll
        for (int u = 0; u < 32; ++u) sts_u32(s.kscr + 4 * u, v[u]);
        for (uint32_t m = surv; m; m &= m - 1) {
            const int u = __ffs(m) - 1;
            const float kv = __uint_as_float(lds_u32(s.kscr + 4 * u));
            s.stash[s.sn * 32 + lane] = ((uint64_t)f2ord(kv) << 32) | (uint32_t)(j0 + u);
            ++s.sn;
        }
    }
    if (PROF) {
        const long long f1 = clock64();
        s.c_stash += f1 - w0;
        s.c_append += f1 - f0;
    }
}

__device__ __forceinline__ void prof_add(int which, unsigned long long v) {
    if (v) atomicAdd(&g_tile_counters[which], v);
}
__device__ __forceinline__ void prof_add_warp(int which, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) prof_add(which, v);
}

// D (+)= A * B^T with E4M3 operands (kind::f8f6f4), FP32 accumulator.
__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The tt-th tile of a sweep that starts at t0 and moves outward: t0, t0+1, t0-1,
// t0+2, t0-2, ... while both sides have tiles, then the rest of the longer side.
__device__ __forceinline__ int tile_at(int tt, int t0, int ntiles) {
    const int left = t0, right = ntiles - 1 - t0;
    const int m = left < right ? left : right;
    if (tt <= 2 * m) {
        const int k = (tt + 1) >> 1;
        return (tt & 1) ? t0 + k : t0 - k;
    }
    const int extra = tt - 2 * m;
    return right > left ? t0 + m + extra : t0 - m - extra;
}

// EMX: pool entries per row half / 32 that the compaction holds in registers
// (ph <= 32 EMX); a larger EMX costs the sweep loop registers, so the common
// pools (ph <= 256) use their own instantiation.
template <int BN, bool PROF, int EMX>
__global__ void __launch_bounds__(kt::THREADS, 1)
    k_knn_tiles(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const __grid_constant__ CUtensorMap tmAaug,
                const __grid_constant__ CUtensorMap tmBaug, const KnnParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // Find this CTA's problem and row block.
    const int64_t bid = blockIdx.x;
    if (bid >= P.blk_off[P.nprob]) return;
    int lo = 0, hi = P.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.blk_off[mid] <= bid) lo = mid; else hi = mid - 1;
    }
    const KnnProblem pr = P.probs[lo];
    const int rb = (int)(bid - P.blk_off[lo]);
    const int ntiles = (pr.n_cols + BN - 1) / BN;
    constexpr int B_BLK_BYTES = BN * 128, B_AUG_BYTES = BN * 32;
    // Sweep order (tile_at): with local_first the sweep starts at the tile holding
    // the block's first row and moves outward, alternating forward and backward;
    // rows are ordered by cell and cells along a chain of nearby pivots, so each
    // row's k-th key tightens early and far cells come last.
    int t0 = 0;
    if (P.local_first) {
        t0 = rb * kt::BM / BN;
        if (t0 >= ntiles) t0 = ntiles - 1;
    }
    // Tiles this block sweeps (nrun of them): with exact skipping, those of its tile
    // list in list order (nearest first); else all, in tile_at order.
    const uint16_t* tlist =
        (P.tlist && ntiles <= kt::TL_MAX && P.tcount[bid] >= 0) ? P.tlist + bid * kt::TL_MAX
                                                               : nullptr;
    const int nrun = tlist ? P.tcount[bid] : ntiles;

    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const KnnSmemLayout L = knn_smem_layout(BN, P.nkb_a, P.nst, P.a_stream);
    const uint32_t STG = knn_stage_bytes(BN, P.a_stream);
    const uint32_t sA = smem_u32(base + L.a);
    const uint32_t sAaug = smem_u32(base + L.aaug);
    const uint32_t sB = smem_u32(base + L.b);
    const uint32_t sBaug = smem_u32(base + L.baug);
    const uint32_t bars = smem_u32(base + L.bars);
    const uint32_t full_bar = bars, empty_bar = bars + kt::MAX_NST * 8;
    const uint32_t afull_bar = bars + 2 * kt::MAX_NST * 8, aempty_bar = afull_bar + kt::NAUG * 8;
    const uint32_t accf_bar = aempty_bar + kt::NAUG * 8;
    const uint32_t acce_bar = accf_bar + kt::NACC * 8;
    const uint32_t a_bar = acce_bar + kt::NACC * 8, done_bar = a_bar + 8;
    volatile uint32_t* tmem_slot = (volatile uint32_t*)(base + L.tmem_slot);
    volatile int* abort_flag = (volatile int*)(base + L.abort_flag);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long cta_t0 = 0;
    if (PROF) cta_t0 = clock64();
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.nst; ++s) {
            mbar_init(full_bar + 8 * s, 1);
            mbar_init(empty_bar + 8 * s, 1);
        }
        for (int s = 0; s < kt::NAUG; ++s) {
            mbar_init(afull_bar + 8 * s, 1);
            mbar_init(aempty_bar + 8 * s, 1);
        }
        for (int a = 0; a < kt::NACC; ++a) {
            mbar_init(accf_bar + 8 * a, 1);
            mbar_init(acce_bar + 8 * a, kt::EPI_WARPS);
        }
        mbar_init(a_bar, 1);
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32((const void*)tmem_slot), kt::TMEM_COLS);
        tmem_relinquish();
    }
    if (warp >= 2) {  // thresholds of both column halves: the window bound, or +inf
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        const int i = rb * kt::BM + row;
        float t = INFINITY;
        if (P.rowub && i < pr.n_rows) {
            const float ub = P.rowub[pr.a_row0 + i];
            if (ub < INFINITY) {
                // key = (dist - |x|^2) / 2, rounded up; split keys get the margin
                const float nx = P.na[pr.a_row0 + i];
                const float d = __fmaf_ru(P.ub_margin, 3.0f * nx + 2.0f * ub, ub);
                t = 0.5f * __fsub_ru(d, nx);
            }
        }
        ((float*)(base + L.tau))[h * kt::BM + row] = t;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            tma_prefetch_desc(&tmAaug);
            tma_prefetch_desc(&tmBaug);
            const int a_y = (int)(pr.a_row0 + (int64_t)rb * kt::BM);
            const int nres = P.a_stream ? 0 : P.nkb_a;
            mbar_expect_tx(a_bar, nres * kt::A_BLK_BYTES + kt::A_AUG_BYTES);
            for (int b = 0; b < nres; ++b)
                tma_load_2d(sA + b * kt::A_BLK_BYTES, &tmA, a_bar, b * P.kbe, a_y);
            tma_load_2d(sAaug, &tmAaug, a_bar, 0, 0);
            uint32_t last_par = 0, used = 0, alast_par = 0, aused = 0;
            int st = 0, sa = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true;
            unsigned long long prod_wait = 0;
            for (int run = 0; run < nrun && ok;) {
                const int t = tlist ? (int)tlist[run] : tile_at(run, t0, ntiles);
                ++run;
                const int b_y = (int)(pr.b_row0 + (int64_t)t * BN);
                // the norm block first: its MMA opens the tile, so the slot frees early
                if (!mbar_wait(aempty_bar + 8 * sa, aph ^ 1, abort_flag)) { ok = false; break; }
                mbar_expect_tx(afull_bar + 8 * sa, B_AUG_BYTES);
                tma_load_2d(sBaug + sa * B_AUG_BYTES, &tmBaug, afull_bar + 8 * sa, 0, b_y);
                aused |= 1u << sa;
                alast_par = (alast_par & ~(1u << sa)) | (aph << sa);
                if (++sa == kt::NAUG) { sa = 0; aph ^= 1; }
                for (int j = 0; j < P.nkb_b; ++j) {
                    long long w0 = 0;
                    if (PROF) w0 = clock64();
                    if (!mbar_wait(empty_bar + 8 * st, ph ^ 1, abort_flag)) { ok = false; break; }
                    if (PROF) prod_wait += clock64() - w0;
                    // streamed A blocks of this B block (see knn_stage_bytes)
                    int as0 = j, na = 0;
                    if (P.a_stream) {
                        na = 1;
                        if (P.mode == 1) {
                            const int H2 = P.nkb_b >> 1;
                            if (j < H2) na = 2; else as0 = j - H2;
                        }
                    }
                    mbar_expect_tx(full_bar + 8 * st, B_BLK_BYTES + na * kt::A_BLK_BYTES);
                    tma_load_2d(sB + st * STG, &tmB, full_bar + 8 * st, j * P.kbe, b_y);
                    if (na >= 1)
                        tma_load_2d(sB + st * STG + B_BLK_BYTES, &tmA, full_bar + 8 * st,
                                    as0 * P.kbe, a_y);
                    if (na == 2)  // the lo block of the same columns
                        tma_load_2d(sB + st * STG + B_BLK_BYTES + kt::A_BLK_BYTES, &tmA,
                                    full_bar + 8 * st, (as0 + (P.nkb_b >> 1)) * P.kbe, a_y);
                    used |= 1u << st;
                    last_par = (last_par & ~(1u << st)) | (ph << st);
                    if (++st == P.nst) { st = 0; ph ^= 1; }
                }
            }
            // Drain: every issued copy must land before the CTA may exit.
            int dummy = 0;
            for (int s = 0; s < P.nst; ++s)
                if (used >> s & 1)
                    mbar_wait(full_bar + 8 * s, (last_par >> s) & 1, &dummy, 200000000ull);
            for (int s = 0; s < kt::NAUG; ++s)
                if (aused >> s & 1)
                    mbar_wait(afull_bar + 8 * s, (alast_par >> s) & 1, &dummy, 200000000ull);
            mbar_wait(a_bar, 0, &dummy, 200000000ull);
            if (!ok) atomicOr(P.status, DEV_TIMEOUT);
            if (PROF) prof_add(TC_PROD_WAIT, prod_wait);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------- MMA
        if (lane == 0) {
            bool ok = mbar_wait(a_bar, 0, abort_flag);
            tc_fence_after();
            int st = 0, sa = 0;
            uint32_t ph = 0, aph = 0;
            const int H2 = P.nkb_b >> 1;
            unsigned long long w_full = 0, w_acc = 0, c_iss = 0, c_com = 0;
            long long loop0 = 0;
            if (PROF) loop0 = clock64();
            for (int t = 0; t < nrun && ok; ++t) {
                const int a = t % kt::NACC;
                long long w0 = 0;
                if (PROF) w0 = clock64();
                if (!mbar_wait(acce_bar + 8 * a, ((t / kt::NACC) & 1) ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                if (PROF) w_acc += clock64() - w0;
                tc_fence_after();
                const uint32_t d_tmem = tmem + a * BN;
                // D = [1,1,1,0..] . [h,m,l,0..] (= |y|^2 / 2), then D -= x . y
                if (PROF) w0 = clock64();
                if (!mbar_wait(afull_bar + 8 * sa, aph, abort_flag)) { ok = false; break; }
                if (PROF) w_full += clock64() - w0;
                tc_fence_after();
                umma_f16(d_tmem, sdesc_sw32(sAaug), sdesc_sw32(sBaug + sa * B_AUG_BYTES),
                         P.idesc_aug, 0);
                umma_commit(aempty_bar + 8 * sa);
                if (++sa == kt::NAUG) { sa = 0; aph ^= 1; }
                const uint32_t accum = 1;
                for (int j = 0; j < P.nkb_b; ++j) {
                    if (PROF) w0 = clock64();
                    if (!mbar_wait(full_bar + 8 * st, ph, abort_flag)) { ok = false; break; }
                    if (PROF) w_full += clock64() - w0;
                    tc_fence_after();
                    if (PROF) w0 = clock64();
                    const uint32_t bsm = sB + st * STG;
                    if (P.mode == 1 && !P.a_stream) {
                        // compact split sections (A resident): B step sb < hs (hi)
                        // meets A steps sb (hi . hi) and sb + hs (lo . hi); B step
                        // sb >= hs (lo) meets A step sb - hs (hi . lo).  A step a sits
                        // in block a / 4 at byte 32 (a % 4).
                        for (int u = 0; u < 4 && 4 * j + u < P.ksteps; ++u) {
                            const int sb = 4 * j + u;
                            const int a0 = sb < P.hs ? sb : sb - P.hs;
                            umma_f16(d_tmem,
                                     sdesc_sw128(sA + (a0 >> 2) * kt::A_BLK_BYTES + (a0 & 3) * 32),
                                     sdesc_sw128(bsm + u * 32), P.idesc_neg, accum);
                            if (sb < P.hs) {
                                const int a1 = sb + P.hs;
                                umma_f16(d_tmem,
                                         sdesc_sw128(sA + (a1 >> 2) * kt::A_BLK_BYTES +
                                                     (a1 & 3) * 32),
                                         sdesc_sw128(bsm + u * 32), P.idesc_neg, accum);
                            }
                        }
                    } else {
                        int ablk[2];
                        int na = 1;
                        if (P.mode == 0) {
                            ablk[0] = j;
                        } else if (j < H2) {
                            ablk[0] = j;       // hi . hi
                            ablk[1] = H2 + j;  // lo . hi
                            na = 2;
                        } else {
                            ablk[0] = j - H2;  // hi . lo
                        }
                        // K steps of the block that hold data: the last block of plain
                        // operands may end in zero steps, which are not issued
                        const bool full = P.mode == 1 || 4 * j + 4 <= P.ksteps;
                        for (int q = 0; q < na; ++q) {
                            const uint32_t asm_ = P.a_stream
                                                      ? bsm + B_BLK_BYTES + q * kt::A_BLK_BYTES
                                                      : sA + ablk[q] * kt::A_BLK_BYTES;
                            // four K steps of 32 bytes per 128-byte block (K = 16 for
                            // 16-bit operands, K = 32 for E4M3)
                            if (full) {
#pragma unroll
                                for (int s = 0; s < 4; ++s) {
                                    if (P.kind8)
                                        umma_f8(d_tmem, sdesc_sw128(asm_ + s * 32),
                                                sdesc_sw128(bsm + s * 32), P.idesc_neg, accum);
                                    else
                                        umma_f16(d_tmem, sdesc_sw128(asm_ + s * 32),
                                                 sdesc_sw128(bsm + s * 32), P.idesc_neg, accum);
                                }
                            } else {
                                for (int s = 0; 4 * j + s < P.ksteps; ++s) {
                                    if (P.kind8)
                                        umma_f8(d_tmem, sdesc_sw128(asm_ + s * 32),
                                                sdesc_sw128(bsm + s * 32), P.idesc_neg, accum);
                                    else
                                        umma_f16(d_tmem, sdesc_sw128(asm_ + s * 32),
                                                 sdesc_sw128(bsm + s * 32), P.idesc_neg, accum);
                                }
                            }
                        }
                    }
                    long long w1 = 0;
                    if (PROF) {
                        w1 = clock64();
                        c_iss += w1 - w0;
                    }
                    umma_commit(empty_bar + 8 * st);
                    if (PROF) c_com += clock64() - w1;
                    if (++st == P.nst) { st = 0; ph ^= 1; }
                }
                if (!ok) break;
                umma_commit(accf_bar + 8 * a);
            }
            if (PROF) {
                prof_add(TC_MMA_LOOP, (unsigned long long)(clock64() - loop0));
                prof_add(TC_MMA_ISSUE, c_iss);
                prof_add(TC_MMA_COMMIT, c_com);
            }
            umma_commit(done_bar);  // every issued MMA completes before TMEM is released
            int dummy = 0;
            mbar_wait(done_bar, 0, &dummy, 200000000ull);
            if (!ok) atomicOr(P.status, DEV_TIMEOUT);
            if (PROF) {
                prof_add(TC_MMA_WAIT_FULL, w_full);
                prof_add(TC_MMA_WAIT_ACC, w_acc);
            }
        }
    } else {
        // -------------------------------------------------------- epilogue
        // Warp (q, h): TMEM lane quarter q (rows 32q..32q+31), columns
        // [128h, 128h + 128) of every tile.
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        EpiState s;
        s.row = q * 32 + lane;
        const int i = rb * kt::BM + s.row;     // row index inside the problem
        const int i0 = rb * kt::BM + q * 32;   // first row of this warp
        const int64_t arow0 = pr.a_row0 + i0;  // gathered A row of lane 0
        s.ph = P.ph;
        s.kp = P.kprime;
        s.pool0 = P.pool + (arow0 * 2 + h) * (int64_t)P.ph;
        s.pool = s.pool0 + (int64_t)lane * 2 * P.ph;
        s.tau_own = (float*)(base + L.tau) + h * kt::BM;
        s.tau_other = (const volatile float*)((float*)(base + L.tau) + (1 - h) * kt::BM);
        s.c = 0;
        s.sn = 0;
        s.stash = (uint64_t*)(base + L.stash) + (warp - 2) * kt::SC * 32;
        s.kscr = smem_u32(base + L.kscr) + ((warp - 2) * 32 + lane) * kt::KS * 4;
        s.gidrow = P.gid ? P.gid + pr.b_row0 : nullptr;
        s.best = ~0ull;
        s.tau = s.tau_own[s.row];
        s.teff = fminf(s.tau, s.tau_other[s.row]);
        s.c_flush_cyc = s.c_chunks = s.c_slow = s.c_flushes = s.c_iters = s.c_app = 0;
        s.c_ldw = s.c_filter = s.c_append = s.c_stash = s.c_direct = s.c_floop = 0;
        unsigned long long e_wait = 0;
        long long e_t0 = 0;
        if (PROF) e_t0 = clock64();
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        bool ok = true;
        constexpr int HALF = BN / 2;
        for (int run = 0; run < nrun;) {
            const int t = tlist ? (int)tlist[run] : tile_at(run, t0, ntiles);
            const int a = run % kt::NACC;
            const int par = (run / kt::NACC) & 1;
            ++run;
            long long w0 = 0;
            if (PROF) w0 = clock64();
            if (!mbar_wait(accf_bar + 8 * a, par, abort_flag)) { ok = false; break; }
            if (PROF) e_wait += clock64() - w0;
            tc_fence_after();
            {
                const uint32_t tb = tmem + lane_addr + a * BN + h * HALF;
                const int jt = t * BN + h * HALF;

                const bool edge = (jt + HALF > pr.n_cols) ||
                                  (P.self_exclude && i0 + 32 > jt && i0 < jt + HALF);
                uint32_t va[32], vb[32];
                __syncwarp();
                tmem_ld32(tb, va);
#pragma unroll 1
                for (int c = 0; c < HALF / 32; c += 2) {
                    long long l0 = 0;
                    if (PROF) l0 = clock64();
                    tmem_wait_ld32(va);
                    if (PROF) s.c_ldw += clock64() - l0;
                    tmem_ld32(tb + (c + 1) * 32, vb);
                    if (jt + c * 32 < pr.n_cols)
                        epi_chunk<PROF, EMX>(s, va, jt + c * 32, i, pr.n_cols, P.self_exclude, edge);
                    __syncwarp();
                    if (PROF) l0 = clock64();
                    tmem_wait_ld32(vb);
                    if (PROF) s.c_ldw += clock64() - l0;
                    if (c + 2 < HALF / 32) {
                        tmem_ld32(tb + (c + 2) * 32, va);
                    } else {
                        // the tile's last chunk is in registers: hand the accumulator
                        // back to the MMA warp before working on it
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acce_bar + 8 * a);
                    }
                    if (jt + (c + 1) * 32 < pr.n_cols)
                        epi_chunk<PROF, EMX>(s, vb, jt + (c + 1) * 32, i, pr.n_cols, P.self_exclude,
                                        edge);
                    __syncwarp();
                }
                // the accumulator is back with the MMA warp: the tile's stashed
                // survivors join the pools while the next tile is computed
                epi_flush_stash<PROF, EMX>(s);
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (PROF) {
            prof_add_warp(TC_EPI_CYCLES, (unsigned long long)(clock64() - e_t0));
            prof_add_warp(TC_EPI_WAIT, e_wait);
            prof_add_warp(TC_EPI_FLUSH, s.c_flush_cyc);
            prof_add_warp(TC_APPENDS, s.c_app);
            prof_add_warp(TC_LD_WAIT, s.c_ldw);
            prof_add_warp(TC_FILTER, s.c_filter);
            prof_add_warp(TC_APPEND, s.c_append);
            prof_add_warp(TC_STASH, s.c_stash);
            prof_add_warp(TC_DIRECT, s.c_direct);
            prof_add_warp(TC_FLUSH_LOOP, s.c_floop);
            if (lane == 0) {
                prof_add(TC_CHUNKS, s.c_chunks);
                prof_add(TC_SLOW_CHUNKS, s.c_slow);
                prof_add(TC_FLUSHES, s.c_flushes);
                prof_add(TC_FLUSH_ITERS, s.c_iters);
            }
        }
        if (!ok || *abort_flag) {
            if (lane == 0) atomicOr(P.status, DEV_TIMEOUT);
        } else if (i < pr.n_rows) {
            // the pool's size (k_pool_finalize merges the two halves)
            if (s.kp == 1) {
                if (s.best != ~0ull) s.pool[0] = s.best;
                s.c = s.best != ~0ull ? 1 : 0;
            }
            P.pool_cnt[(pr.a_row0 + i) * 2 + h] = s.c;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (PROF && threadIdx.x == 0) {
        prof_add(TC_CTA_CYCLES, (unsigned long long)(clock64() - cta_t0));
        prof_add(TC_CTAS, 1);
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kt::TMEM_COLS);
    }
}

// ---- problem tables, gather and norms ------------------------------------------
// probs[s] for the C shards: a/b rows at the 128-padded offsets, out rows at offsets.
// One block of 1024 threads, thread s = shard s (C <= 1024).  Gathered rows stay
// in shard order (pad_off: 128-padded row offsets); the problem table lists the
// shards by decreasing size (order[j] = shard of problem j), so the CTAs of the
// largest shards start first and the launch ends on short CTAs.
__global__ void __launch_bounds__(1024)
    k_shard_tables(const int64_t* __restrict__ offsets, int C, int64_t rows,
                   int64_t* __restrict__ blk_off, int64_t* __restrict__ pad_off,
                   KnnProblem* __restrict__ probs, int32_t* __restrict__ order_out, int* status) {
    __shared__ int64_t nbk[1024], scan[1024], psh[1024];
    __shared__ int order[1024];
    __shared__ int bad;
    const int s = threadIdx.x;
    if (blockIdx.x) return;
    if (s == 0) bad = (offsets[0] != 0 || offsets[C] != rows) ? 1 : 0;
    __syncthreads();
    int64_t n = 0;
    if (s < C) {
        n = offsets[s + 1] - offsets[s];
        if (n < 0 || n >= (1ll << 24)) {
            bad = 1;
            n = 0;
        }
    }
    nbk[s] = (n + kt::BM - 1) / kt::BM;
    scan[s] = nbk[s];
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive prefix sum (Hillis-Steele)
        const int64_t v = s >= o ? scan[s - o] : 0;
        __syncthreads();
        scan[s] += v;
        __syncthreads();
    }
    psh[s] = (scan[s] - nbk[s]) * kt::BM;
    if (s < C) pad_off[s] = psh[s];
    if (s == C - 1) pad_off[C] = scan[s] * kt::BM;
    if (s < C) {  // rank by (size descending, shard ascending)
        int r = 0;
        for (int t = 0; t < C; ++t) {
            int64_t m = offsets[t + 1] - offsets[t];
            if (m < 0 || m >= (1ll << 24)) m = 0;
            r += (m > n || (m == n && t < s)) ? 1 : 0;
        }
        order[r] = s;
    }
    __syncthreads();
    const int sh = s < C ? order[s] : 0;
    const int64_t mine = s < C ? nbk[sh] : 0;
    __syncthreads();
    scan[s] = mine;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = s >= o ? scan[s - o] : 0;
        __syncthreads();
        scan[s] += v;
        __syncthreads();
    }
    if (s < C) {
        const int64_t ns = nbk[sh] ? offsets[sh + 1] - offsets[sh] : 0;
        blk_off[s] = scan[s] - mine;
        order_out[s] = sh;
        KnnProblem q;
        q.a_row0 = psh[sh];
        q.b_row0 = psh[sh];
        q.out_row0 = offsets[sh];
        q.mem_row0 = offsets[sh];
        q.n_rows = (int32_t)ns;
        q.n_cols = (int32_t)ns;
        probs[s] = q;
    }
    if (s == C - 1) {
        blk_off[C] = bad ? 0 : scan[s];  // nothing runs on inconsistent input
        if (bad) atomicOr(status, DEV_BAD_INPUT);
    }
}

// [1, 1, 1, 0 x 13] in every one of 128 rows: the A side of the norm K step.
__global__ void k_ones_tile(__nv_bfloat16* __restrict__ t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 128 * kt::KAUG) t[i] = __float2bfloat16_rn((i % kt::KAUG) < 3 ? 1.0f : 0.0f);
}

template <typename T>
__device__ __forceinline__ T cvt_from_float(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_float(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half cvt_from_float(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_fp8_e4m3 cvt_from_float(float v) {
    __nv_fp8_e4m3 r;
    r.__x = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);  // round to nearest even
    return r;
}
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_float(__nv_fp8_e4m3 v) { return (float)v; }

// Largest |x| over n elements (for the E4M3 scale), as float bits in *out (init 0).
__global__ void k_absmax(const void* X, int dtype, int64_t n, unsigned int* out) {
    float m = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(load_elem(X, dtype, i)));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Gather rows into the tile layout: row p' of G (pitch Kp elements) holds the
// operand copy of vector src[p'] (zeros when src[p'] < 0); norms[p'] = |x|^2
// and aug[p'] = |x|^2 / 2 split exactly into three BF16 values (hi, mid, lo)
// followed by zeros.
// mode 0: element t = cvt(x_t).  mode 1: [hi | lo] sections of Kh elements.
// scale (E4M3 only): every element is multiplied by 448 / *amax_bits, and the
// norms by its square, so keys keep their order.
template <typename T>
__global__ void k_gather(const void* X, int dtype, int d, const int64_t* __restrict__ srcrow,
                         int64_t rows_cap, int mode, int Kp, int Kh, T* __restrict__ G,
                         float* __restrict__ norms, __nv_bfloat16* __restrict__ aug,
                         const unsigned int* __restrict__ amax_bits) {
    // Global operand scale: E4M3 maps max|x| to 448 (the largest finite value);
    // scaled FP16 multiplies by the power of two that puts max|x| in [2^13, 2^14)
    // (exact, and far from both overflow and the subnormal range).
    float scale = 1.0f;
    if (amax_bits) {
        const float am = __uint_as_float(*amax_bits);
        if (am > 0.0f && am <= 3.0e38f) {
            if (sizeof(T) == 1) {
                scale = 448.0f / am;
            } else {
                int ex;
                frexpf(am, &ex);
                scale = ldexpf(1.0f, 14 - ex);
            }
        }
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp_g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t pr = warp_g; pr < rows_cap; pr += nwarps) {
        const int64_t src = srcrow[pr];
        T* g = G + pr * Kp;
        float nrm = 0.0f;
        for (int t = lane; t < Kp; t += 32) {
            float v = 0.0f;
            if (mode == 0) {
                if (src >= 0 && t < d) {
                    v = load_elem(X, dtype, src * d + t) * scale;
                    nrm = fmaf(v, v, nrm);
                }
                g[t] = cvt_from_float<T>(v);
            } else {
                const int tt = t < Kh ? t : t - Kh;
                T out = cvt_from_float<T>(0.0f);
                if (src >= 0 && tt < d) {
                    v = load_elem(X, dtype, src * d + tt);
                    const T h = cvt_from_float<T>(v);
                    if (t < Kh) {
                        out = h;
                        nrm = fmaf(v, v, nrm);
                    } else {
                        out = cvt_from_float<T>(v - to_float(h));
                    }
                }
                g[t] = out;
            }
        }
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if (lane == 0) norms[pr] = nrm;
        if (lane < kt::KAUG) {
            const float half = 0.5f * nrm;
            const __nv_bfloat16 h = __float2bfloat16_rn(half);
            const float r1 = half - __bfloat162float(h);
            const __nv_bfloat16 m = __float2bfloat16_rn(r1);
            const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
            __nv_bfloat16 o = __float2bfloat16_rn(0.0f);
            if (lane == 0) o = h;
            if (lane == 1) o = m;
            if (lane == 2) o = l;
            aug[pr * kt::KAUG + lane] = o;
        }
    }
}

// ---- row maps: which vector each gathered row holds ----------------------------
__device__ __forceinline__ int shard_of_padded(const int64_t* __restrict__ pad_off, int C,
                                               int64_t pr) {
    int lo = 0, hi = C - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pad_off[mid] <= pr) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Shard order as given: row pad_off[s] + li holds member offsets[s] + li.
__global__ void k_rowmap_plain(const uint32_t* __restrict__ members,
                               const int64_t* __restrict__ offsets,
                               const int64_t* __restrict__ pad_off, int C, int64_t rows_cap,
                               int64_t* __restrict__ src) {
    for (int64_t pr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pr < rows_cap;
         pr += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = -1;
        if (pr < pad_off[C]) {
            const int s = shard_of_padded(pad_off, C, pr);
            const int64_t li = pr - pad_off[s];
            if (li < offsets[s + 1] - offsets[s]) {
                const int64_t p = offsets[s] + li;
                v = members ? (int64_t)members[p] : p;
            }
        }
        src[pr] = v;
    }
}

// Pivots of every shard: P_s = ceil(n_s / cell) evenly spaced members (cells of
// about `cell` rows).  Tables for the pivot-assignment launch: A = the shard's
// rows, B = its pivots, listed in the same order as the shard problems
// (order[j] = shard of problem j) so that both launches share blk_off.
__global__ void k_pivot_tables(const int64_t* __restrict__ offsets, int C, int cell,
                               const int64_t* __restrict__ pad_off, const int32_t* __restrict__ order,
                               int64_t* __restrict__ ppad_off, int32_t* __restrict__ npiv,
                               KnnProblem* __restrict__ pprobs) {
    if (threadIdx.x || blockIdx.x) return;
    int64_t p = 0;
    for (int s = 0; s < C; ++s) {
        int64_t n = offsets[s + 1] - offsets[s];
        if (n < 0) n = 0;
        int64_t P = (n + cell - 1) / cell;
        if (P < 1) P = 1;
        if (P > 1024) P = 1024;
        npiv[s] = (int32_t)P;
        ppad_off[s] = p;
        p += (P + kt::BM - 1) / kt::BM * kt::BM;
    }
    ppad_off[C] = p;
    for (int j = 0; j < C; ++j) {
        const int s = order[j];
        int64_t n = offsets[s + 1] - offsets[s];
        if (n < 0) n = 0;
        KnnProblem pr;
        pr.a_row0 = pad_off[s];
        pr.b_row0 = ppad_off[s];
        pr.out_row0 = offsets[s];
        pr.mem_row0 = 0;
        pr.n_rows = (int32_t)n;
        pr.n_cols = n > 0 ? npiv[s] : 0;
        pprobs[j] = pr;
    }
}

__global__ void k_rowmap_pivots(const uint32_t* __restrict__ members,
                                const int64_t* __restrict__ offsets,
                                const int64_t* __restrict__ ppad_off,
                                const int32_t* __restrict__ npiv, int C, int64_t rows_cap,
                                int64_t* __restrict__ src) {
    for (int64_t pr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pr < rows_cap;
         pr += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = -1;
        if (pr < ppad_off[C]) {
            const int s = shard_of_padded(ppad_off, C, pr);
            const int64_t q = pr - ppad_off[s];
            const int64_t n = offsets[s + 1] - offsets[s];
            if (q < npiv[s] && n > 0) v = (int64_t)members[offsets[s] + q * n / npiv[s]];
        }
        src[pr] = v;
    }
}

// 16 bytes of a row as floats (V elements of type DT).
template <int DT>
struct Chunk16 {
    static constexpr int V = DT == ANN_F32 ? 4 : (DT == ANN_U8 ? 16 : 8);
    __device__ static void unpack(const uint4& w, float (&f)[V]) {
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (DT == ANN_F32) {
                f[i] = __uint_as_float(u[i]);
            } else if (DT == ANN_F16) {
                const float2 t = __half22float2(*(const __half2*)&u[i]);
                f[2 * i] = t.x;
                f[2 * i + 1] = t.y;
            } else if (DT == ANN_BF16) {
                const float2 t = __bfloat1622float2(*(const __nv_bfloat162*)&u[i]);
                f[2 * i] = t.x;
                f[2 * i + 1] = t.y;
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b) f[4 * i + b] = (float)((u[i] >> (8 * b)) & 0xFFu);
            }
        }
    }
};

// Order the pivots of each shard along a greedy chain (start at pivot 0, always
// step to the nearest pivot not yet taken; FP32 distances from the vectors), so
// that cells adjacent in the row order are near in space.  crank[ppad_off[s] + q]
// = chain position of pivot q.  One block per shard: the current pivot's row is
// staged in shared memory, every thread scores its pivots with 16-byte loads
// (VEC) or element loads, and warp shuffles plus one shared-memory pass pick the
// nearest.  Only the sweep order depends on it, never a result.
template <int DT, bool VEC>
__global__ void __launch_bounds__(1024)
    k_pivot_chain(const void* X, int d, const int64_t* __restrict__ psrc,
                  const int64_t* __restrict__ ppad_off, const int32_t* __restrict__ npiv,
                  uint32_t* __restrict__ crank) {
    extern __shared__ float cur_row[];  // d floats
    __shared__ uint8_t taken[1024];
    __shared__ float wbd[32];
    __shared__ int wbq[32];
    __shared__ int cur;
    constexpr int V = Chunk16<DT>::V;
    const int s = blockIdx.x;
    const int P = npiv[s];
    const int64_t base = ppad_off[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < P; q += blockDim.x) taken[q] = 0;
    if (threadIdx.x == 0) {
        cur = 0;
        taken[0] = 1;
        crank[base] = 0;
    }
    __syncthreads();
    for (int step = 1; step < P; ++step) {
        const int64_t rc = psrc[base + cur];
        for (int t = threadIdx.x; t < d; t += blockDim.x)
            cur_row[t] = rc >= 0 ? load_elem(X, DT, rc * d + t) : 0.0f;
        __syncthreads();
        float best = INFINITY;
        int bi = P;
        for (int q = threadIdx.x; q < P; q += blockDim.x) {
            if (taken[q]) continue;
            const int64_t rq = psrc[base + q];
            float acc = 0.0f;
            if (rq >= 0) {
                if (VEC) {
                    const uint4* row = (const uint4*)X + rq * (d / V);
                    for (int c = 0; c < d / V; ++c) {
                        float f[V];
                        Chunk16<DT>::unpack(__ldg(row + c), f);
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            const float df = f[e] - cur_row[c * V + e];
                            acc = fmaf(df, df, acc);
                        }
                    }
                } else {
                    for (int t = 0; t < d; ++t) {
                        const float df = load_elem(X, DT, rq * d + t) - cur_row[t];
                        acc = fmaf(df, df, acc);
                    }
                }
            }
            if (acc < best || (acc == best && q < bi)) {
                best = acc;
                bi = q;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float a = __shfl_xor_sync(0xffffffffu, best, o);
            const int aq = __shfl_xor_sync(0xffffffffu, bi, o);
            if (a < best || (a == best && aq < bi)) {
                best = a;
                bi = aq;
            }
        }
        if (lane == 0) {
            wbd[wid] = best;
            wbq[wid] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float b0 = wbd[0];
            int nx = wbq[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (wbd[w] < b0 || (wbd[w] == b0 && wbq[w] < nx)) {
                    b0 = wbd[w];
                    nx = wbq[w];
                }
            if (nx >= P) nx = 0;  // unreachable while pivots remain
            taken[nx] = 1;
            crank[base + nx] = (uint32_t)step;
            cur = nx;
        }
        __syncthreads();
    }
}

static int launch_pivot_chain(const void* X, int dtype, int d, const KnnWs& w, int C,
                              cudaStream_t st) {
    const bool vec = ((size_t)d * dtype_bytes(dtype)) % 16 == 0 && (uintptr_t)X % 16 == 0;
    const size_t sm = (size_t)d * sizeof(float);
#define ANN_CHAIN(DT)                                                                          \
    (vec ? k_pivot_chain<DT, true><<<C, 1024, sm, st>>>(X, d, w.psrc, w.ppad_off, w.npiv, w.crank)  \
         : k_pivot_chain<DT, false><<<C, 1024, sm, st>>>(X, d, w.psrc, w.ppad_off, w.npiv, w.crank))
    switch (dtype) {
    case ANN_F32: ANN_CHAIN(ANN_F32); break;
    case ANN_F16: ANN_CHAIN(ANN_F16); break;
    case ANN_BF16: ANN_CHAIN(ANN_BF16); break;
    default: ANN_CHAIN(ANN_U8); break;
    }
#undef ANN_CHAIN
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

// Counting sort of each shard's rows by cell (the nearest pivot), cells taken in
// chain order (crank): perm[off_s + pos] = local index.  The order inside a cell
// does not affect any result.
__global__ void k_cell_sort(const uint32_t* __restrict__ cellid,
                            const int64_t* __restrict__ offsets, const int32_t* __restrict__ npiv,
                            const uint32_t* __restrict__ crank,
                            const int64_t* __restrict__ ppad_off, uint32_t* __restrict__ perm) {
    __shared__ int32_t cnt[1024];
    __shared__ int32_t base[1024];
    const int s = blockIdx.x;
    const int64_t o = offsets[s], n = offsets[s + 1] - o;
    const int P = npiv[s];
    for (int c = threadIdx.x; c < P; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    const uint32_t* rk = crank + ppad_off[s];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        uint32_t c = cellid[o + i];
        c = c < (uint32_t)P ? rk[c] : 0;
        if (c >= (uint32_t)P) c = 0;
        atomicAdd(&cnt[c], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int c = 0; c < P; ++c) {
            base[c] = acc;
            acc += cnt[c];
        }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        uint32_t c = cellid[o + i];
        c = c < (uint32_t)P ? rk[c] : 0;
        if (c >= (uint32_t)P) c = 0;
        const int32_t pos = atomicAdd(&base[c], 1);
        perm[o + pos] = (uint32_t)i;
    }
}

// Cell order: row pad_off[s] + pos holds member offsets[s] + perm[...]; also the
// global id of each row and the output row it belongs to.
__global__ void k_rowmap_cells(const uint32_t* __restrict__ members,
                               const int64_t* __restrict__ offsets,
                               const int64_t* __restrict__ pad_off,
                               const uint32_t* __restrict__ perm, int C, int64_t rows_cap,
                               int64_t* __restrict__ src, uint32_t* __restrict__ gid,
                               int64_t* __restrict__ outrow) {
    for (int64_t pr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pr < rows_cap;
         pr += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = -1, orow = -1;
        if (pr < pad_off[C]) {
            const int s = shard_of_padded(pad_off, C, pr);
            const int64_t pos = pr - pad_off[s];
            if (pos < offsets[s + 1] - offsets[s]) {
                orow = offsets[s] + perm[offsets[s] + pos];
                v = (int64_t)members[orow];
            }
        }
        src[pr] = v;
        gid[pr] = v >= 0 ? (uint32_t)v : ANN_PAD;
        outrow[pr] = orow;
    }
}

// ---- exact re-rank (FP32 direct form) -------------------------------------------
// Row p: candidates cand[p][0..kc) (global ids) scored by sum_t (x_t - y_t)^2,
// each lane summing dims lane, lane+32, ... in order, then a fixed xor-tree, so
// d(u, v) and d(v, u) are the same bits.  Sorted by (distance, id); first k kept.
template <int E>
__device__ __forceinline__ void warp_bitonic_u64(uint64_t (&v)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= E) {
                const int lp = j / E;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = lane * E + e;
                    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v[e], lp);
                    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v[e] >> 32), lp);
                    const uint64_t o = ((uint64_t)hi << 32) | lo;
                    const bool up = (i & k) == 0, lower = (i & j) == 0;
                    const uint64_t mn = v[e] < o ? v[e] : o, mx = v[e] < o ? o : v[e];
                    v[e] = (lower == up) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int pe = e ^ j;
                    if (pe > e) {
                        const int i = lane * E + e;
                        const bool up = (i & k) == 0;
                        const uint64_t a = v[e], b = v[pe];
                        if ((a > b) == up) { v[e] = b; v[pe] = a; }
                    }
                }
            }
        }
    }
}

// ---- pool finalisation ---------------------------------------------------------------
// Every valid A row of the tile launch's problems: the kprime smallest entries of
// the union of its two column halves' pools, sorted by (key, global id), written as
// (global id, |x|^2 + 2 key) to the first k_out slots of its output row, then ANN_PAD
// / +inf.  One warp per row: the row's entries are selected with warp_select_kth,
// gathered into shared memory in ballot order, then sorted with a warp bitonic sort
// of KE entries per lane.
template <int KE, int EH>  // KE: sorted entries per lane; EH = ph / 32
__global__ void __launch_bounds__(256)
k_pool_finalize(const KnnParams P) {
    __shared__ uint64_t stage[8][32 * KE];
    const int64_t bid = blockIdx.x;
    if (bid >= P.blk_off[P.nprob]) return;
    int lo = 0, hi = P.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.blk_off[mid] <= bid) lo = mid; else hi = mid - 1;
    }
    const KnnProblem pr = P.probs[lo];
    const int rb = (int)(bid - P.blk_off[lo]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* stg = stage[warp];
    for (int r = warp; r < kt::BM; r += 8) {
        const int i = rb * kt::BM + r;
        if (i >= pr.n_rows) break;
        const int64_t arow = pr.a_row0 + i;
        // counts clamped to the pool (an aborted sweep leaves them unwritten)
        const int c0 = min(max(P.pool_cnt[arow * 2], 0), P.ph);
        const int c1 = min(max(P.pool_cnt[arow * 2 + 1], 0), P.ph);
        const uint64_t* h0 = P.pool + arow * 2 * (int64_t)P.ph;
        const uint64_t* h1 = h0 + P.ph;
        uint64_t v[2 * EH];
#pragma unroll
        for (int e = 0; e < EH; ++e) {
            const int idx = lane + 32 * e;
            v[e] = idx < c0 ? h0[idx] : ~0ull;
            v[EH + e] = idx < c1 ? h1[idx] : ~0ull;
        }
        const int n = c0 + c1;
        const int kp = P.kprime;
        const uint64_t T = n > 0 ? warp_select_kth(v, n, kp) : 0ull;
        // the kept entries (kp of them, or all n) into the staging array
        for (int e = lane; e < 32 * KE; e += 32) stg[e] = ~0ull;
        __syncwarp();
        int base = 0;
#pragma unroll
        for (int e = 0; e < 2 * EH; ++e) {
            const bool keep = n > 0 && v[e] != ~0ull && v[e] <= T;
            const uint32_t b = __ballot_sync(0xffffffffu, keep);
            const int pos = base + __popc(b & ((1u << lane) - 1u));
            if (keep && pos < 32 * KE) stg[pos] = v[e];
            base += __popc(b);
        }
        __syncwarp();
        uint64_t w[KE];
#pragma unroll
        for (int e = 0; e < KE; ++e) w[e] = stg[lane * KE + e];
        __syncwarp();
        warp_bitonic_u64<KE>(w);
        const float nx = P.na[arow];
        const int64_t orow = P.outrow ? P.outrow[arow] : pr.out_row0 + i;
#pragma unroll
        for (int e = 0; e < KE; ++e) {
            const int slot = lane * KE + e;
            if (slot < P.k_out) {
                uint32_t id = ANN_PAD;
                float dd = INFINITY;
                if (w[e] != ~0ull) {
                    id = (uint32_t)w[e];
                    dd = fmaf(2.0f, ord2f((uint32_t)(w[e] >> 32)), nx);
                }
                P.out_id[orow * P.k_out + slot] = id;
                P.out_d[orow * P.k_out + slot] = dd;
            }
        }
    }
}

// k' = 1 (the pivot assignment): a thread per row takes the smaller of the two
// halves' entries.
__global__ void __launch_bounds__(kt::BM) k_pool_finalize1(const KnnParams P) {
    const int64_t bid = blockIdx.x;
    if (bid >= P.blk_off[P.nprob]) return;
    int lo = 0, hi = P.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.blk_off[mid] <= bid) lo = mid; else hi = mid - 1;
    }
    const KnnProblem pr = P.probs[lo];
    const int i = (int)(bid - P.blk_off[lo]) * kt::BM + (int)threadIdx.x;
    if (i >= pr.n_rows) return;
    const int64_t arow = pr.a_row0 + i;
    const uint64_t* h0 = P.pool + arow * 2 * (int64_t)P.ph;
    const uint64_t a = P.pool_cnt[arow * 2] > 0 ? h0[0] : ~0ull;
    const uint64_t b = P.pool_cnt[arow * 2 + 1] > 0 ? h0[P.ph] : ~0ull;
    const uint64_t w = a < b ? a : b;
    const int64_t orow = P.outrow ? P.outrow[arow] : pr.out_row0 + i;
    uint32_t id = ANN_PAD;
    float dd = INFINITY;
    if (w != ~0ull) {
        id = (uint32_t)w;
        dd = fmaf(2.0f, ord2f((uint32_t)(w >> 32)), P.na[arow]);
    }
    P.out_id[orow * P.k_out] = id;
    P.out_d[orow * P.k_out] = dd;
    for (int slot = 1; slot < P.k_out; ++slot) {
        P.out_id[orow * P.k_out + slot] = ANN_PAD;
        P.out_d[orow * P.k_out + slot] = INFINITY;
    }
}

template <int E>
__global__ void k_rerank(const void* X, const void* Xrow, int dtype, int d,
                         const uint32_t* __restrict__ row_ids, int64_t nrows,
                         const uint32_t* __restrict__ cand, int kc, int k,
                         uint32_t* __restrict__ out_id, float* __restrict__ out_d,
                         const int64_t* __restrict__ order) {
    const int lane = threadIdx.x & 31;
    int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= nrows) return;
    if (order && (p = order[p]) < 0) return;
    const int64_t u = row_ids ? (int64_t)row_ids[p] : p;
    uint64_t keys[E];
#pragma unroll
    for (int e = 0; e < E; ++e) keys[e] = ~0ull;
    for (int c = 0; c < kc; ++c) {
        const uint32_t v = cand[p * kc + c];
        if (v == ANN_PAD) continue;  // uniform
        float s = 0.0f;
        for (int t = lane; t < d; t += 32) {
            const float df = __fsub_rn(load_elem(Xrow, dtype, u * d + t),
                                       load_elem(X, dtype, (int64_t)v * d + t));
            s = __fadd_rn(s, __fmul_rn(df, df));
        }
        for (int o = 16; o > 0; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
        if ((c & 31) == lane) {  // candidate c held by lane c % 32, slot c / 32
            const int e = c >> 5;
#pragma unroll
            for (int q = 0; q < E; ++q)
                if (q == e) keys[q] = ((uint64_t)f2ord(s) << 32) | v;
        }
    }
    warp_bitonic_u64<E>(keys);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = lane * E + e;
        if (idx < k) {
            const uint64_t x = keys[e];
            const bool pad = (x == ~0ull);
            out_id[p * k + idx] = pad ? ANN_PAD : (uint32_t)x;
            out_d[p * k + idx] = pad ? INFINITY : ord2f((uint32_t)(x >> 32));
        }
    }
}

// The same re-rank with 16-byte loads (rows 16-byte aligned, d * element size a
// multiple of 16): lane l sums the squared differences of 16-byte chunks
// l, l + 32, ... in order, then a fixed xor tree adds the 32 partial sums.  Two
// candidates are scored per pass so that their loads overlap.
template <int E, int DT>
__global__ void k_rerank_vec(const void* X, const void* Xrow, int d,
                             const uint32_t* __restrict__ row_ids, int64_t nrows,
                             const uint32_t* __restrict__ cand, int kc, int k,
                             uint32_t* __restrict__ out_id, float* __restrict__ out_d,
                             const int64_t* __restrict__ order) {
    constexpr int V = Chunk16<DT>::V;
    const int lane = threadIdx.x & 31;
    int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= nrows) return;
    if (order && (p = order[p]) < 0) return;
    const int64_t u = row_ids ? (int64_t)row_ids[p] : p;
    const int nch = d / V;
    const uint4* xu = (const uint4*)Xrow + u * nch;
    uint64_t keys[E];
#pragma unroll
    for (int e = 0; e < E; ++e) keys[e] = ~0ull;
    for (int c = 0; c < kc; c += 2) {
        const uint32_t v0 = cand[p * kc + c];
        const uint32_t v1 = c + 1 < kc ? cand[p * kc + c + 1] : ANN_PAD;
        if (v0 == ANN_PAD && v1 == ANN_PAD) continue;  // uniform
        const uint4* x0 = (const uint4*)X + (int64_t)(v0 == ANN_PAD ? 0 : v0) * nch;
        const uint4* x1 = (const uint4*)X + (int64_t)(v1 == ANN_PAD ? 0 : v1) * nch;
        float s0 = 0.0f, s1 = 0.0f;
        for (int q = lane; q < nch; q += 32) {
            const uint4 wa = __ldg(xu + q), w0 = __ldg(x0 + q), w1 = __ldg(x1 + q);
            float fa[V], f0[V], f1[V];
            Chunk16<DT>::unpack(wa, fa);
            Chunk16<DT>::unpack(w0, f0);
            Chunk16<DT>::unpack(w1, f1);
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const float d0 = __fsub_rn(fa[t], f0[t]), d1 = __fsub_rn(fa[t], f1[t]);
                s0 = __fadd_rn(s0, __fmul_rn(d0, d0));
                s1 = __fadd_rn(s1, __fmul_rn(d1, d1));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 = __fadd_rn(s0, __shfl_xor_sync(0xffffffffu, s0, o));
            s1 = __fadd_rn(s1, __shfl_xor_sync(0xffffffffu, s1, o));
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int cc = c + h;
            const uint32_t v = h ? v1 : v0;
            if (v != ANN_PAD && (cc & 31) == lane) {
                const int e = cc >> 5;
#pragma unroll
                for (int q = 0; q < E; ++q)
                    if (q == e) keys[q] = ((uint64_t)f2ord(h ? s1 : s0) << 32) | v;
            }
        }
    }
    warp_bitonic_u64<E>(keys);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = lane * E + e;
        if (idx < k) {
            const uint64_t x = keys[e];
            const bool pad = (x == ~0ull);
            out_id[p * k + idx] = pad ? ANN_PAD : (uint32_t)x;
            out_d[p * k + idx] = pad ? INFINITY : ord2f((uint32_t)(x >> 32));
        }
    }
}

// Rows of at most 32 16-byte chunks (d <= 128 for FP32, 256 for 16-bit types): a
// group of 8 lanes per candidate, four candidates at a time.  Lane g of a group
// holds chunks g, g + 8, g + 16, g + 24 of the row in registers (loaded once), sums
// its chunks' squared differences in order and the group adds its 8 partial sums by
// an xor tree (4, 2, 1): a fixed order, the same in every lane.  Three shuffles per
// four candidates instead of five per candidate.
template <int E, int DT>
__global__ void k_rerank_g8(const void* X, const void* Xrow, int d,
                            const uint32_t* __restrict__ row_ids, int64_t nrows,
                            const uint32_t* __restrict__ cand, int kc, int k,
                            uint32_t* __restrict__ out_id, float* __restrict__ out_d,
                            const int64_t* __restrict__ order) {
    constexpr int V = Chunk16<DT>::V;
    const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
    int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= nrows) return;
    if (order && (p = order[p]) < 0) return;
    const int64_t u = row_ids ? (int64_t)row_ids[p] : p;
    const int nch = d / V;  // <= 32
    const uint4* xu = (const uint4*)Xrow + u * nch;
    float fa[4][V];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ch = gl + 8 * q;
        if (ch < nch) {
            Chunk16<DT>::unpack(__ldg(xu + ch), fa[q]);
        } else {
#pragma unroll
            for (int t = 0; t < V; ++t) fa[q][t] = 0.0f;
        }
    }
    uint64_t keys[E];
#pragma unroll
    for (int e = 0; e < E; ++e) keys[e] = ~0ull;
    for (int c0 = 0; c0 < kc; c0 += 4) {
        const int c = c0 + grp;
        const uint32_t v = c < kc ? cand[p * kc + c] : ANN_PAD;
        const uint4* xv = (const uint4*)X + (int64_t)(v == ANN_PAD ? 0 : v) * nch;
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ch = gl + 8 * q;
            if (ch < nch) {
                float f[V];
                Chunk16<DT>::unpack(__ldg(xv + ch), f);
#pragma unroll
                for (int t = 0; t < V; ++t) {
                    const float df = __fsub_rn(fa[q][t], f[t]);
                    s = __fadd_rn(s, __fmul_rn(df, df));
                }
            }
        }
        s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, 4));
        s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, 2));
        s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, 1));
        // candidate c0 + q goes to lane (c0 + q) % 32, register c0 / 32 (c0 is a
        // multiple of 4): lane L takes group (L - c0) % 32 when that is below 4
        const int qL = (lane - c0) & 31;
        const float sq = __shfl_sync(0xffffffffu, s, (qL & 3) * 8);
        const uint32_t vq = __shfl_sync(0xffffffffu, v, (qL & 3) * 8);
        const bool mine = qL < 4 && c0 + qL < kc && vq != ANN_PAD;
        const uint64_t key = ((uint64_t)f2ord(sq) << 32) | vq;
        const int eit = c0 >> 5;
#pragma unroll
        for (int e = 0; e < E; ++e) keys[e] = (mine && e == eit) ? key : keys[e];
    }
    warp_bitonic_u64<E>(keys);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = lane * E + e;
        if (idx < k) {
            const uint64_t x = keys[e];
            const bool pad = (x == ~0ull);
            out_id[p * k + idx] = pad ? ANN_PAD : (uint32_t)x;
            out_d[p * k + idx] = pad ? INFINITY : ord2f((uint32_t)(x >> 32));
        }
    }
}

// ---- host side -------------------------------------------------------------------
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

// 2-D tensor map over a [rows x inner] matrix of 16-bit (esize 2) or 8-bit (esize 1)
// elements with box {box_inner, box_rows}.
int make_tmap(CUtensorMap* m, const void* G, int64_t rows, int inner, int box_inner, int box_rows,
              CUtensorMapSwizzle swz, int esize) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return fail(ANN_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)inner * esize};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapDataType dt =
        esize == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(m, dt, 2, (void*)G, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ANN_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ANN_OK;
}

// Operand layout, tile width and pipeline depth for a dtype / precision.
//   ANN_EXACT      : uint8 -> BF16 copy (exact integer keys, no re-rank);
//                    float -> BF16 hi/lo split (FP32 data) or the data's own
//                    16-bit type, screening k + 16 (or rerank_k) for the re-rank.
//   ANN_BF16_RERANK: one BF16 copy, screening rerank_k (default 128).
//   ANN_FP8_RERANK : one E4M3 copy (all values scaled by 448 / max|x|), screening
//                    rerank_k (default 128).
int knn_plan(int d, int dtype, int k, int precision, int rerank_k, KnnPlan* pl) {
    KnnPlan p;
    p.elem8 = 0;
    p.scaled = 0;
    if (precision == ANN_FP8_RERANK) {
        p.mode = 0;
        p.Kh = 0;
        p.elem8 = 1;
        p.scaled = 1;
        p.Kp = (int)align_up((size_t)d, kt::KB8);
        p.ab_fmt = 0;  // E4M3
        p.rerank = true;
    } else if (precision == ANN_F16_RERANK) {
        p.mode = 0;
        p.Kh = 0;
        p.scaled = 1;
        p.Kp = (int)align_up((size_t)d, kt::KB);
        p.ab_fmt = 0;  // FP16
        p.rerank = true;
    } else if (precision == ANN_BF16_RERANK) {
        p.mode = 0;
        p.Kh = 0;
        p.Kp = (int)align_up((size_t)d, kt::KB);
        p.ab_fmt = 1;
        p.rerank = true;
    } else if (dtype == ANN_F32) {
        // compact split layout (A resident): sections of align(d, 16) elements,
        // the row padded to whole K blocks after the lo section
        p.mode = 1;
        p.Kh = (int)align_up((size_t)d, 16);
        p.Kp = (int)align_up((size_t)(2 * p.Kh), kt::KB);
        p.ab_fmt = 1;
        p.rerank = true;
    } else {
        p.mode = 0;
        p.Kh = 0;
        p.Kp = (int)align_up((size_t)d, kt::KB);
        p.ab_fmt = dtype == ANN_F16 ? 0 : 1;
        p.rerank = dtype != ANN_U8;
    }
    p.kbe = p.elem8 ? kt::KB8 : kt::KB;
    const int wide = precision == ANN_EXACT ? k + 16 : 128;
    p.kprime = p.rerank ? (rerank_k > 0 ? rerank_k : wide) : k;
    if (p.kprime < k) p.kprime = k;
    if (p.kprime > 256) return fail(ANN_ERR_UNSUPPORTED, "list width k' > 256");
    // Resident A rows if they fit: the widest tile with a 3-stage ring, else with
    // 2 stages (an N = 256 MMA does twice the work of an N = 128 one for about the
    // same issue cost), else the narrow tile.  Otherwise (large d) the A blocks
    // stream through the ring beside the B blocks; split operands then use
    // sections of whole K blocks (the streamed pairing is by block).
    const size_t cap = 227 * 1024;
    p.nst = 0;
    p.a_stream = 0;
    const int tries[4][2] = {{256, 3}, {256, 2}, {128, 3}, {128, 2}};
    for (int as = 0; as <= (p.mode ? 2 : 1) && !p.nst; as += (p.mode ? 2 : 1)) {
        if (as && p.mode == 1) {
            p.Kh = (int)align_up((size_t)d, kt::KB);
            p.Kp = 2 * p.Kh;
        }
        p.nkb_a = p.Kp / p.kbe;
        p.nkb_b = p.nkb_a;
        for (int q = 0; q < 4 && !p.nst; ++q) {
            const int bn = tries[q][0];
            for (int nst = kt::MAX_NST; nst >= tries[q][1]; --nst)
                if (knn_smem_layout(bn, p.nkb_a, nst, as).total <= cap) {
                    p.nst = nst;
                    p.bn = bn;
                    p.a_stream = as;
                    break;
                }
        }
    }
    // K steps holding data (32 bytes each): see KnnParams::ksteps
    const int step_elems = p.kbe / 4;
    p.hs = p.mode == 1 ? p.Kh / step_elems : 0;
    p.ksteps = p.mode == 1 ? 2 * p.hs : (int)((d + step_elems - 1) / step_elems);
    if (!p.nst)
        return fail(ANN_ERR_UNSUPPORTED, "shard_knn: d=%d with k'=%d does not fit shared memory",
                    d, p.kprime);
    p.smem = knn_smem_layout(p.bn, p.nkb_a, p.nst, p.a_stream).total;
    *pl = p;
    return ANN_OK;
}

// Every shared-memory plan of the same problem (same operand form and list width)
// that the autotuner may time: for each tile width the two deepest rings that
// fit, A resident if any plan with resident A fits, else streamed.  out[0] is
// the default plan.  Results never depend on the plan (same per-pair arithmetic,
// ties by id), only the speed does.
int knn_plan_variants(int d, int dtype, int k, int precision, int rerank_k, KnnPlan* out,
                      int max_out) {
    KnnPlan base;
    int rc = knn_plan(d, dtype, k, precision, rerank_k, &base);
    if (rc) return -rc;
    int n = 0;
    out[n++] = base;
    const size_t cap = 227 * 1024;
    for (int bn = 256; bn >= 128 && n < max_out; bn -= 128) {
        int found = 0;
        for (int nst = kt::MAX_NST; nst >= 2 && found < 2 && n < max_out; --nst) {
            if (knn_smem_layout(bn, base.nkb_a, nst, base.a_stream).total > cap)
                continue;
            ++found;
            if (bn == base.bn && nst == base.nst) continue;
            KnnPlan v = base;
            v.bn = bn;
            v.nst = nst;
            v.smem = knn_smem_layout(bn, base.nkb_a, nst, base.a_stream).total;
            out[n++] = v;
        }
    }
    return n;
}

// Operand bytes per gathered row.
static inline size_t row_bytes(const KnnPlan& pl) { return (size_t)pl.Kp * (pl.elem8 ? 1 : 2); }

// ---- exact tile skipping ------------------------------------------------------------
// For a row block A (128 gathered rows) and a column group G (128 gathered rows of
// the same shard), with centres c_A, c_G and radii r_A >= max |x - c_A|, r_G, every
// pair satisfies |x - y| >= |c_A - c_G| - r_A - r_G (triangle inequality).  The k-th
// distance of each row among the other rows of its 256-row window bounds its final
// k-th squared distance from above (k_ub_own); a column tile whose
// groups all lie beyond the block's largest bound cannot hold a neighbour of any of
// its rows, so the sweep skips it (its copies, products and epilogue).  Ties stay
// exact: a skipped column is strictly farther than the bound.  Used for plain
// (single-product) operands of integer data, whose tile keys are exact; every
// rounding in the bound is pushed outward by a relative margin far above FP32's
// error on these sums.
static bool g_tile_prune = true;
void tile_prune_set(bool on) { g_tile_prune = on; }
bool tile_prune_on() { return g_tile_prune; }
__device__ unsigned long long g_prune_stats[3];  // tiles, tiles swept, pairs swept

static bool prunable(const KnnPlan& pl) {
    return !pl.elem8 && !pl.a_stream;
}

// Centre (mean of the valid rows) and radius bound of every 128-row group of the
// gathered layout; src[row] = the vector of a gathered row, -1 = padding.
__global__ void __launch_bounds__(128)
k_group_geom(const void* X, int dtype, int d, const int64_t* __restrict__ src, int64_t ngroups,
             int ldc, float* __restrict__ gcent, float* __restrict__ grad,
             float* __restrict__ gmaxn) {
    extern __shared__ float cs[];  // [d]
    __shared__ int nvalid;
    __shared__ float rmax[4], nmax[4];
    const int64_t g = blockIdx.x;
    if (g >= ngroups) return;
    const int64_t r0 = g * kt::BM;
    const int tid = threadIdx.x;
    __shared__ int64_t rs[kt::BM];
    if (tid == 0) nvalid = 0;
    __syncthreads();
    const int64_t my = src[r0 + tid];
    rs[tid] = my;
    if (my >= 0) atomicAdd(&nvalid, 1);
    __syncthreads();
    const int n = nvalid;
    if (n == 0) {
        if (tid == 0) {
            grad[g] = -1.0f;
            gmaxn[g] = 0.0f;
        }
        return;
    }
    for (int t = tid; t < d; t += blockDim.x) {
        float sum = 0.0f;
#pragma unroll 8
        for (int i = 0; i < kt::BM; ++i) {
            const int64_t v = rs[i];
            if (v >= 0) sum += load_elem(X, dtype, v * d + t);
        }
        const float c = sum / (float)n;
        cs[t] = c;
        gcent[g * ldc + t] = c;
    }
    __syncthreads();
    // radius: one warp per row, lanes over the dimensions (coalesced row reads)
    const int warp = tid >> 5, lane = tid & 31;
    float rw = 0.0f, nw = 0.0f;
    for (int i = warp; i < kt::BM; i += 4) {
        const int64_t v = rs[i];
        if (v < 0) continue;
        float r2 = 0.0f, n2 = 0.0f;
        for (int t = lane; t < d; t += 32) {
            const float x = load_elem(X, dtype, v * d + t);
            const float df = x - cs[t];
            r2 = fmaf(df, df, r2);
            n2 = fmaf(x, x, n2);
        }
        for (int o = 16; o; o >>= 1) {
            r2 += __shfl_xor_sync(0xffffffffu, r2, o);
            n2 += __shfl_xor_sync(0xffffffffu, n2, o);
        }
        rw = fmaxf(rw, r2);
        nw = fmaxf(nw, n2);
    }
    if (lane == 0) {
        rmax[warp] = rw;
        nmax[warp] = nw;
    }
    __syncthreads();
    if (tid == 0) {
        gmaxn[g] = fmaxf(fmaxf(nmax[0], nmax[1]), fmaxf(nmax[2], nmax[3])) * (1.0f + 0x1p-16f);
        const float m = fmaxf(fmaxf(rmax[0], rmax[1]), fmaxf(rmax[2], rmax[3]));
        // FP32 sums of d squares: relative error below (d + 2) 2^-24; pushed up
        grad[g] = sqrtf(m * (1.0f + (float)(d + 4) * 0x1p-22f)) * (1.0f + 0x1p-20f);
    }
}

__device__ __forceinline__ int block_problem(const int64_t* __restrict__ blk_off, int nprob,
                                             int64_t bid) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk_off[mid] <= bid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// bub[bid] = the largest, over the block's rows, k-th smallest squared distance
// from the row to the other valid rows of its 256-row window of the shard (the
// window holding the block), or +inf where a row has fewer than k others there:
// an upper bound of every row's final k-th distance.  uint8 vectors with d a
// multiple of 4, NW4 = d / 4 words at most; exact integer arithmetic
// (|x|^2 + |y|^2 - 2 x.y with dp4a).  One block of 256 threads per row block; the
// window's vectors are staged in shared memory, each row's words held in registers.
template <int NW4>
__global__ void __launch_bounds__(256)
k_ub_own(const uint8_t* __restrict__ X, int d, const int64_t* __restrict__ src,
         const int64_t* __restrict__ blk_off, const KnnProblem* __restrict__ probs, int nprob,
         int k, int64_t nblocks, float* __restrict__ bub, float* __restrict__ rowub) {
    extern __shared__ uint32_t wv[];  // [256][ws] packed vectors, then [256] norms
    __shared__ unsigned int bmax;
    const int64_t bid = blockIdx.x;
    if (bid >= nblocks) return;
    if (bid >= blk_off[nprob]) {
        if (threadIdx.x == 0) bub[bid] = INFINITY;
        return;
    }
    const int p = block_problem(blk_off, nprob, bid);
    const KnnProblem pr = probs[p];
    const int rb = (int)(bid - blk_off[p]);
    const int nw4 = d / 4;
    const int ws = nw4 + 1;  // padded row stride (words): no bank conflicts across lanes
    uint32_t* nrm = wv + 256 * ws;
    const int c0 = (rb >> 1) * 256;  // first column of the window (shard-relative)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) bmax = 0;
    // stage: warp w loads columns w, w + 8, ...; lane q loads word q (coalesced)
    for (int c = warp; c < 256; c += 8) {
        const bool valid = c0 + c < pr.n_cols;
        const int64_t v = valid ? src[pr.b_row0 + c0 + c] : -1;
        uint32_t n2 = 0;
        for (int q = lane; q < nw4; q += 32) {
            const uint32_t word = v >= 0 ? ((const uint32_t*)(X + v * d))[q] : 0u;
            wv[c * ws + q] = word;
            n2 = __dp4a(word, word, n2);
        }
        for (int o = 16; o; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
        if (lane == 0) nrm[c] = v >= 0 ? n2 : 0xFFFFFFFFu;  // all ones: not a column
    }
    __syncthreads();
    unsigned int wmax = 0;
    for (int r = warp; r < kt::BM; r += 8) {
        const int i = rb * kt::BM + r;  // row index in the shard
        if (i >= pr.n_rows) continue;
        const int cr = i - c0;          // the row's own column in the window
        const uint32_t nr = nrm[cr];
        uint32_t rw[NW4];
#pragma unroll
        for (int w = 0; w < NW4; ++w) rw[w] = w < nw4 ? wv[cr * ws + w] : 0u;
        uint32_t dv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = lane + 32 * q;
            const uint32_t nc = nrm[c];
            const uint32_t* cw = wv + c * ws;
            uint32_t dot = 0;
#pragma unroll
            for (int w = 0; w < NW4; ++w)
                if (w < nw4) dot = __dp4a(rw[w], cw[w], dot);
            dv[q] = (nc == 0xFFFFFFFFu || c == cr) ? 0xFFFFFFFFu : nr + nc - 2u * dot;
        }
        // k-th smallest of the window's distances: least v with #{dist <= v} >= k
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) cnt += dv[q] != 0xFFFFFFFFu;
        for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        unsigned int ub = 0xFFFFFFFFu;
        if (cnt >= k) {
            unsigned int lo = 0, hi = 1u << 24;  // squared distances of uint8 rows, d <= 256
            while (lo < hi) {
                const unsigned int mid = lo + (hi - lo) / 2;
                int c = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) c += dv[q] <= mid;
                for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                if (c >= k) hi = mid; else lo = mid + 1;
            }
            ub = lo;
        }
        if (rowub && lane == 0) rowub[pr.a_row0 + i] = ub == 0xFFFFFFFFu ? INFINITY : (float)ub;
        wmax = ub > wmax ? ub : wmax;
    }
    if (lane == 0) atomicMax(&bmax, wmax);
    __syncthreads();
    if (tid == 0) bub[bid] = bmax == 0xFFFFFFFFu ? INFINITY : (float)bmax;
}

// As k_ub_own for float vectors (d <= 200): FP32 direct-form squared distances
// (x - y)^2 summed in index order, the k-th smallest found by a search on the bit
// patterns of the non-negative floats.  Register tiles: a warp takes 8 rows at a
// time and each lane 8 window columns (lane + 32 q), so one pass over the
// dimensions reads 8 broadcast row values and 8 column values from shared memory
// for 64 products.
__global__ void __launch_bounds__(256)
k_ub_own_f32(const float* __restrict__ X, int d, const int64_t* __restrict__ src,
             const int64_t* __restrict__ blk_off, const KnnProblem* __restrict__ probs, int nprob,
             int k, int64_t nblocks, float* __restrict__ bub, float* __restrict__ rowub) {
    extern __shared__ float wf[];  // [256][d + 1]
    __shared__ unsigned int bmax;
    const int64_t bid = blockIdx.x;
    if (bid >= nblocks) return;
    if (bid >= blk_off[nprob]) {
        if (threadIdx.x == 0) bub[bid] = INFINITY;
        return;
    }
    const int p = block_problem(blk_off, nprob, bid);
    const KnnProblem pr = probs[p];
    const int rb = (int)(bid - blk_off[p]);
    const int ws = d + 1;
    const int c0 = (rb >> 1) * 256;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ unsigned char cvalid[256];
    if (tid == 0) bmax = 0;
    for (int c = warp; c < 256; c += 8) {
        const bool valid = c0 + c < pr.n_cols;
        const int64_t v = valid ? src[pr.b_row0 + c0 + c] : -1;
        for (int t = lane; t < d; t += 32) wf[c * ws + t] = v >= 0 ? X[v * d + t] : 0.0f;
        if (lane == 0) cvalid[c] = v >= 0;
    }
    __syncthreads();
    const uint32_t NONE = 0x7F800000u;  // +inf: not a column
    unsigned int wmax = 0;
    for (int g = 0; g < 2; ++g) {
        const int r0 = warp * 16 + g * 8;  // rows r0 .. r0 + 7 of the block
        const int i0 = rb * kt::BM + r0;   // their row index in the shard
        if (i0 >= pr.n_rows) break;
        float acc[8][8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[j][q] = 0.0f;
        const float* xr = wf + (i0 - c0) * ws;  // row r0's own window column
        const float* xc = wf + lane * ws;
        for (int t = 0; t < d; ++t) {
            float a[8], b[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = xr[j * ws + t];
#pragma unroll
            for (int q = 0; q < 8; ++q) b[q] = xc[32 * q * ws + t];
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float df = a[j] - b[q];
                    acc[j][q] = fmaf(df, df, acc[j][q]);
                }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = i0 + j;
            if (i >= pr.n_rows) break;  // warp-uniform
            const int cr = i - c0;       // the row's own column in the window
            uint32_t dv[8];
            int cnt = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = lane + 32 * q;
                dv[q] = (!cvalid[c] || c == cr) ? NONE : __float_as_uint(acc[j][q]);
                cnt += dv[q] != NONE;
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            unsigned int ub = NONE;
            if (cnt >= k) {
                unsigned int lo = 0, hi = NONE;
                while (lo < hi) {
                    const unsigned int mid = lo + (hi - lo) / 2;
                    unsigned int c = 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) c += dv[q] <= mid;
                    c = __reduce_add_sync(0xffffffffu, c);
                    if (c >= (unsigned int)k) hi = mid; else lo = mid + 1;
                }
                ub = lo;
            }
            // FP32 sums of d squares: relative error below (d + 2) 2^-24; pushed up
            if (rowub && lane == 0)
                rowub[pr.a_row0 + i] =
                    ub >= NONE ? INFINITY : __uint_as_float(ub) * (1.0f + (float)(d + 4) * 0x1p-22f);
            wmax = ub > wmax ? ub : wmax;
        }
    }
    if (lane == 0) atomicMax(&bmax, wmax);
    __syncthreads();
    // FP32 sums of d squares: relative error below (d + 2) 2^-24; pushed up
    if (tid == 0)
        bub[bid] = bmax >= NONE ? INFINITY
                                : __uint_as_float(bmax) * (1.0f + (float)(d + 4) * 0x1p-22f);
}

// tlist[bid]: the column tiles a row block sweeps, nearest first.  A tile is left
// out when every one of its groups is provably farther than the block's bound;
// the kept ones are ordered by the smallest distance from the block's centre to
// a group ball of the tile, (|c_A - c_G| - r_G), so the thresholds tighten on the
// first tiles of the sweep and fewer candidates pass them later.  tcount[bid]:
// the number kept (-1 where the shard has more than TL_MAX tiles: the block then
// sweeps every tile).
//
// One CTA of 256 threads per TLB consecutive row blocks: those of one problem share
// the column groups, which are staged in shared memory 64 at a time (row stride
// d | 1, so a warp's 32 groups fall in distinct banks) and each thread takes two
// (row block, group) pairs, summing (c_A - c_G)^2 over the dimensions in order;
// then each row block's kept tiles are sorted in shared memory.
constexpr int TLB = 8, TLG = 64;

struct TileListSmem {
    size_t ca, cg, gnear, gflag, tkey, tkeep, sk, total;
};
__host__ __device__ inline TileListSmem tile_list_smem(int d) {
    const int sd = d | 1;
    TileListSmem L;
    size_t o = 0;
    L.sk = o;      o += (size_t)kt::TL_MAX * 8;          // sort buffer
    L.tkey = o;    o += (size_t)TLB * kt::TL_MAX * 4;    // order bits of each tile's key
    L.tkeep = o;   o += (size_t)TLB * (kt::TL_MAX / 32) * 4;
    L.ca = o;      o += (size_t)TLB * sd * 4;
    L.cg = o;      o += (size_t)TLG * sd * 4;
    L.gnear = o;   o += (size_t)TLB * TLG * 4;
    L.gflag = o;   o += (size_t)TLB * TLG;
    L.total = (o + 15) / 16 * 16;
    return L;
}

__global__ void __launch_bounds__(256)
k_tile_list(const int64_t* __restrict__ blk_off, const KnnProblem* __restrict__ probs, int nprob,
            int bn, int d, int ldc, const float* __restrict__ gcent, const float* __restrict__ grad,
            const float* __restrict__ gmaxn, float kslack, const float* __restrict__ bub,
            int64_t nblocks, uint16_t* __restrict__ tlist, int* __restrict__ tcount) {
    extern __shared__ __align__(16) uint8_t tsm[];
    const TileListSmem L = tile_list_smem(d);
    uint64_t* sk = (uint64_t*)(tsm + L.sk);
    uint32_t* tkey = (uint32_t*)(tsm + L.tkey);
    uint32_t* tkeep = (uint32_t*)(tsm + L.tkeep);
    float* ca = (float*)(tsm + L.ca);
    float* cg = (float*)(tsm + L.cg);
    float* gnear = (float*)(tsm + L.gnear);
    uint8_t* gflag = tsm + L.gflag;  // bit 0: a valid group; bit 1: it may hold a neighbour
    __shared__ int s_n;
    __shared__ unsigned long long s_pairs;
    const int sd = d | 1;
    const int64_t nb = nblocks < blk_off[nprob] ? nblocks : blk_off[nprob];
    const int gpt = bn / kt::BM;  // groups per tile
    for (int64_t r0 = (int64_t)blockIdx.x * TLB; r0 < (int64_t)(blockIdx.x + 1) * TLB && r0 < nb;) {
        // a run of row blocks of one problem
        const int p = block_problem(blk_off, nprob, r0);
        int64_t r1 = (int64_t)(blockIdx.x + 1) * TLB;
        if (r1 > nb) r1 = nb;
        if (r1 > blk_off[p + 1]) r1 = blk_off[p + 1];
        const int na = (int)(r1 - r0);
        const KnnProblem pr = probs[p];
        const int ntiles = (pr.n_cols + bn - 1) / bn;
        if (ntiles > kt::TL_MAX) {  // no list: these blocks sweep every tile
            if (threadIdx.x < na) {
                const int rb = (int)(r0 + threadIdx.x - blk_off[p]);
                const int rows_here = min(kt::BM, pr.n_rows - rb * kt::BM);
                tcount[r0 + threadIdx.x] = -1;
                atomicAdd(&g_prune_stats[0], (unsigned long long)ntiles);
                atomicAdd(&g_prune_stats[1], (unsigned long long)ntiles);
                atomicAdd(&g_prune_stats[2], (unsigned long long)rows_here * pr.n_cols);
            }
            r0 = r1;
            continue;
        }
        // the run's centres and bounds
        for (int x = threadIdx.x; x < na * d; x += blockDim.x) {
            const int a = x / d, u = x - a * d;
            const int64_t gA = pr.a_row0 / kt::BM + (r0 + a - blk_off[p]);
            ca[a * sd + u] = gcent[gA * ldc + u];
        }
        for (int x = threadIdx.x; x < TLB * (kt::TL_MAX / 32); x += blockDim.x) tkeep[x] = 0;
        // (c_A - c_G)^2 sums of the run against the shard's groups, TLG groups at a time
        const int ngroups = (pr.n_cols + kt::BM - 1) / kt::BM;
        const int64_t g0s = pr.b_row0 / kt::BM;
        for (int c0 = 0; c0 < ngroups; c0 += TLG) {
            const int nc = min(TLG, ngroups - c0);
            __syncthreads();  // the previous chunk's reads are done
            for (int x = threadIdx.x; x < nc * d; x += blockDim.x) {
                const int g = x / d, u = x - g * d;
                cg[g * sd + u] = __ldg(gcent + (g0s + c0 + g) * ldc + u);
            }
            __syncthreads();
            for (int pi = threadIdx.x; pi < TLB * TLG; pi += blockDim.x) {
                const int a = pi / TLG, g = pi - a * TLG;
                if (a >= na || g >= nc) continue;
                const int64_t gA = pr.a_row0 / kt::BM + (r0 + a - blk_off[p]);
                const float rA = grad[gA];
                const float rg = grad[g0s + c0 + g];
                uint8_t fl = 0;
                float near = INFINITY;
                if (rA >= 0.0f && rg >= 0.0f) {
                    fl = 1;
                    const float* xa = ca + a * sd;
                    const float* xg = cg + g * sd;
                    float d2 = 0.0f;
                    for (int u = 0; u < d; ++u) {
                        const float df = xa[u] - xg[u];
                        d2 = fmaf(df, df, d2);
                    }
                    near = sqrtf(d2) - rg;
                    const float ub = bub[r0 + a];
                    if (ub < INFINITY) {
                        const float D =
                            sqrtf(d2 * (1.0f - (float)(d + 4) * 0x1p-22f)) * (1.0f - 0x1p-20f);
                        // kslack (float data): twice the largest error of a tile key's
                        // squared distance, which scales with |x|^2 + |y|^2
                        const float lbg = (D - rA - rg) * (1.0f - 0x1p-20f);
                        const float need =
                            ub * (1.0f + 0x1p-18f) + kslack * (gmaxn[gA] + gmaxn[g0s + c0 + g]);
                        if (!(lbg > 0.0f && lbg * lbg > need)) fl |= 2;  // may hold one
                    } else {
                        fl |= 2;
                    }
                }
                gnear[a * TLG + g] = near;
                gflag[a * TLG + g] = fl;
            }
            __syncthreads();
            // per (row block, tile) of the chunk: keep, and the ordering key
            const int t0 = c0 / gpt, nt = (c0 + nc + gpt - 1) / gpt - t0;
            for (int x = threadIdx.x; x < na * nt; x += blockDim.x) {
                const int a = x / nt, t = t0 + (x - a * nt);
                float near = INFINITY;
                bool any = false, may = false;
                for (int q = 0; q < gpt; ++q) {
                    const int g = t * gpt + q - c0;
                    if (t * gpt + q >= ngroups) break;
                    const uint8_t fl = gflag[a * TLG + g];
                    any = any || (fl & 1);
                    may = may || (fl & 2);
                    near = fminf(near, gnear[a * TLG + g]);
                }
                const bool keep = !any || may;
                tkey[a * kt::TL_MAX + t] = f2ord(near);
                if (keep) atomicOr(&tkeep[a * (kt::TL_MAX / 32) + (t >> 5)], 1u << (t & 31));
            }
        }
        __syncthreads();
        // each row block: its kept tiles, sorted by key
        for (int a = 0; a < na; ++a) {
            const int64_t bid = r0 + a;
            const int rb = (int)(bid - blk_off[p]);
            const int rows_here = min(kt::BM, pr.n_rows - rb * kt::BM);
            if (threadIdx.x == 0) {
                s_n = 0;
                s_pairs = 0;
            }
            __syncthreads();
            unsigned long long pairs = 0;
            for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
                if ((tkeep[a * (kt::TL_MAX / 32) + (t >> 5)] >> (t & 31)) & 1u) {
                    const int idx = atomicAdd(&s_n, 1);
                    sk[idx] = ((uint64_t)tkey[a * kt::TL_MAX + t] << 32) | (uint32_t)t;
                    pairs += (unsigned long long)rows_here * min(bn, pr.n_cols - t * bn);
                }
            }
            if (pairs) atomicAdd(&s_pairs, pairs);
            __syncthreads();
            const int n = s_n;
            int p2 = 1;
            while (p2 < n) p2 <<= 1;
            for (int x = n + threadIdx.x; x < p2; x += blockDim.x) sk[x] = ~0ull;
            __syncthreads();
            for (int k = 2; k <= p2; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int x = threadIdx.x; x < p2; x += blockDim.x) {
                        const int l = x ^ j;
                        if (l > x) {
                            const uint64_t va = sk[x], vb = sk[l];
                            if ((va > vb) == ((x & k) == 0)) {
                                sk[x] = vb;
                                sk[l] = va;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            uint16_t* tl = tlist + bid * kt::TL_MAX;
            for (int x = threadIdx.x; x < n; x += blockDim.x) tl[x] = (uint16_t)(sk[x] & 0xFFFFu);
            if (threadIdx.x == 0) {
                tcount[bid] = n;
                atomicAdd(&g_prune_stats[0], (unsigned long long)ntiles);
                atomicAdd(&g_prune_stats[1], (unsigned long long)n);
                atomicAdd(&g_prune_stats[2], s_pairs);
            }
            __syncthreads();
        }
        r0 = r1;
    }
}

int tile_prune_stats(unsigned long long* out, int n, bool reset) {
    unsigned long long tmp[3];
    ANN_CHECK_CUDA(cudaDeviceSynchronize());
    ANN_CHECK_CUDA(cudaMemcpyFromSymbol(tmp, g_prune_stats, sizeof(tmp)));
    for (int i = 0; i < n && i < 3; ++i) out[i] = tmp[i];
    if (reset) {
        unsigned long long z[3] = {0, 0, 0};
        ANN_CHECK_CUDA(cudaMemcpyToSymbol(g_prune_stats, z, sizeof(z)));
    }
    return ANN_OK;
}

size_t knn_ws(int C, int64_t rows, const KnnPlan& pl, KnnWs* out, void* base, size_t cap) {
    Carver cv(base, cap);
    KnnWs w;
    w.rows_cap = rows + (int64_t)kt::BM * C + kt::BNMAX;
    w.blk_off = cv.take<int64_t>(C + 1);
    w.pad_off = cv.take<int64_t>(C + 1);
    w.probs = cv.take<KnnProblem>(C);
    w.G = (__nv_bfloat16*)cv.take<uint8_t>((size_t)w.rows_cap * row_bytes(pl));
    w.aug = cv.take<__nv_bfloat16>((size_t)w.rows_cap * kt::KAUG);
    w.ones = cv.take<__nv_bfloat16>((size_t)128 * kt::KAUG);
    w.norms = cv.take<float>((size_t)w.rows_cap + 512);
    w.cand_id = pl.rerank ? cv.take<uint32_t>((size_t)rows * pl.kprime) : nullptr;
    w.cand_d = pl.rerank ? cv.take<float>((size_t)rows * pl.kprime) : nullptr;
    w.pool = cv.take<uint64_t>((size_t)w.rows_cap * 2 * pool_half(pl.kprime));
    w.pool_cnt = cv.take<int>((size_t)w.rows_cap * 2);
    w.src = cv.take<int64_t>((size_t)w.rows_cap);
    w.gid = cv.take<uint32_t>((size_t)w.rows_cap);
    w.outrow = cv.take<int64_t>((size_t)w.rows_cap);
    w.prows_cap = rows / kt::CELL + (int64_t)(kt::BM + 1) * C + kt::BNMAX;
    w.ppad_off = cv.take<int64_t>(C + 1);
    w.npiv = cv.take<int32_t>(C);
    w.order = cv.take<int32_t>(C);
    w.pprobs = cv.take<KnnProblem>(C);
    w.psrc = cv.take<int64_t>((size_t)w.prows_cap);
    w.GP = (__nv_bfloat16*)cv.take<uint8_t>((size_t)w.prows_cap * row_bytes(pl));
    w.paug = cv.take<__nv_bfloat16>((size_t)w.prows_cap * kt::KAUG);
    w.pnorms = cv.take<float>((size_t)w.prows_cap + 512);
    w.cell = cv.take<uint32_t>((size_t)rows);
    w.cell_d = cv.take<float>((size_t)rows);
    w.perm = cv.take<uint32_t>((size_t)rows);
    w.crank = cv.take<uint32_t>((size_t)w.prows_cap);
    w.amax = cv.take<float>(4);
    w.nblocks = rows / kt::BM + C + 1;
    if (prunable(pl)) {
        const int64_t ng = w.rows_cap / kt::BM + 1;
        w.gcent = cv.take<float>((size_t)ng * pl.Kp);
        w.grad = cv.take<float>((size_t)ng);
        w.gmaxn = cv.take<float>((size_t)ng);
        w.bub = cv.take<float>((size_t)w.nblocks);
        w.tlist = cv.take<uint16_t>((size_t)w.nblocks * kt::TL_MAX);
        w.tcount = cv.take<int>((size_t)w.nblocks);
        w.rowub = cv.take<float>((size_t)w.rows_cap);
    } else {
        w.rowub = nullptr;
        w.gcent = nullptr;
        w.grad = nullptr;
        w.gmaxn = nullptr;
        w.bub = nullptr;
        w.tlist = nullptr;
        w.tcount = nullptr;
    }
    if (out) *out = w;
    return cv.used + 256;
}

static int launch_tiles(const KnnPlan& pl, const void* GA, int64_t rowsA, const void* ones,
                        const void* GB, const void* augB, int64_t rowsB, const KnnParams& P,
                        int64_t grid, cudaStream_t st, bool timed) {
    CUtensorMap ta, tb, taa, tba;
    const int es = pl.elem8 ? 1 : 2;
    int rc = make_tmap(&ta, GA, rowsA, pl.Kp, pl.kbe, kt::BM, CU_TENSOR_MAP_SWIZZLE_128B, es);
    if (!rc) rc = make_tmap(&tb, GB, rowsB, pl.Kp, pl.kbe, pl.bn, CU_TENSOR_MAP_SWIZZLE_128B, es);
    if (!rc) rc = make_tmap(&taa, ones, 128, kt::KAUG, kt::KAUG, kt::BM, CU_TENSOR_MAP_SWIZZLE_32B);
    if (!rc)
        rc = make_tmap(&tba, augB, rowsB, kt::KAUG, kt::KAUG, pl.bn, CU_TENSOR_MAP_SWIZZLE_32B);
    if (rc) return rc;
    const bool prof = timed && tile_counters_on();
    constexpr int EBIG = kt::PH_MAX / 32;
    const bool big = P.ph > 256;
    auto kern = pl.bn == 256
                    ? (prof ? k_knn_tiles<256, true, EBIG>
                            : big ? k_knn_tiles<256, false, EBIG> : k_knn_tiles<256, false, 8>)
                    : (prof ? k_knn_tiles<128, true, EBIG>
                            : big ? k_knn_tiles<128, false, EBIG> : k_knn_tiles<128, false, 8>);
    ANN_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)pl.smem));
    if (grid <= 0) return ANN_OK;
    if (!P.pool || !P.pool_cnt || P.ph < P.kprime + (P.kprime > 1 ? 32 : 0))
        return fail(ANN_ERR_UNSUPPORTED, "tile launch: candidate pools missing or too small");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed && tile_timing_on()) {
        e0 = tile_event();
        e1 = tile_event();
        ANN_CHECK_CUDA(cudaEventRecord(e0, st));
    }
    kern<<<(unsigned)grid, kt::THREADS, pl.smem, st>>>(ta, tb, taa, tba, P);
    ANN_CHECK_LAUNCH();
    if (e0) {
        ANN_CHECK_CUDA(cudaEventRecord(e1, st));
        tile_timing_record(e0, e1);
    }
    // merge the two column halves' pools of every row into its sorted list
    const unsigned g = (unsigned)grid;
    if (P.kprime == 1) {
        k_pool_finalize1<<<g, kt::BM, 0, st>>>(P);
        ANN_CHECK_LAUNCH();
        return ANN_OK;
    }
    const int ke = P.kprime <= 32 ? 1 : P.kprime <= 64 ? 2 : P.kprime <= 128 ? 4 : 8;
    const int eh = P.ph >> 5;
#define ANN_FINALIZE(KE, EH)                                  \
    if (ke == KE && eh == EH) {                               \
        k_pool_finalize<KE, EH><<<g, 256, 0, st>>>(P);        \
        ANN_CHECK_LAUNCH();                                   \
        return ANN_OK;                                        \
    }
    ANN_FINALIZE(1, 2)
    ANN_FINALIZE(1, 8)

    ANN_FINALIZE(2, 3)
    ANN_FINALIZE(2, 4)
    ANN_FINALIZE(2, 6)
    ANN_FINALIZE(2, 8)

    ANN_FINALIZE(4, 5)
    ANN_FINALIZE(4, 6)
    ANN_FINALIZE(4, 7)
    ANN_FINALIZE(4, 8)
    ANN_FINALIZE(8, 7)
    ANN_FINALIZE(8, 8)
    ANN_FINALIZE(8, 9)
    ANN_FINALIZE(8, 10)
#undef ANN_FINALIZE
    return fail(ANN_ERR_UNSUPPORTED, "tile launch: no finalize for k' = %d, pool %d", P.kprime,
                P.ph);
}

// order (optional, norder entries): warp q re-ranks row order[q] (-1: none), e.g.
// the rows in cell order, whose candidates are near one another in space, so
// consecutive warps read many of the same candidate vectors (L2 reuse).
static int launch_rerank(const void* X, const void* Xrow, int dtype, int d, const uint32_t* row_ids,
                         int64_t nrows, const uint32_t* cand, int kc, int k, uint32_t* out_id,
                         float* out_d, cudaStream_t st, const int64_t* order = nullptr,
                         int64_t norder = 0) {
    const int threads = 128;
    if (nrows == 0) return ANN_OK;
    const int64_t nwarps = order ? norder : nrows;
    const unsigned grid = (unsigned)((nwarps * 32 + threads - 1) / threads);
    const int es = dtype_bytes(dtype);
    const bool vec = ((size_t)d * es) % 16 == 0 && (uintptr_t)X % 16 == 0 &&
                     (uintptr_t)Xrow % 16 == 0;
    const bool narrow = (d * es) / 16 <= 32;  // whole row in 4 chunks per lane of 8
#define ANN_RERANK_VEC(E, DT)                                                                  \
    if (narrow)                                                                                \
        k_rerank_g8<E, DT><<<grid, threads, 0, st>>>(X, Xrow, d, row_ids, nwarps, cand, kc, k, \
                                                     out_id, out_d, order);                     \
    else                                                                                       \
        k_rerank_vec<E, DT><<<grid, threads, 0, st>>>(X, Xrow, d, row_ids, nwarps, cand, kc,   \
                                                      k, out_id, out_d, order)
#define ANN_RERANK_VEC_W(DT)                                                                   \
    if (kc <= 64) ANN_RERANK_VEC(2, DT); else if (kc <= 128) ANN_RERANK_VEC(4, DT);              \
    else ANN_RERANK_VEC(8, DT);
    if (vec) {
        switch (dtype) {
        case ANN_F32: ANN_RERANK_VEC_W(ANN_F32) break;
        case ANN_F16: ANN_RERANK_VEC_W(ANN_F16) break;
        case ANN_BF16: ANN_RERANK_VEC_W(ANN_BF16) break;
        default: ANN_RERANK_VEC_W(ANN_U8) break;
        }
    } else if (kc <= 64) {
        k_rerank<2><<<grid, threads, 0, st>>>(X, Xrow, dtype, d, row_ids, nwarps, cand, kc, k,
                                              out_id, out_d, order);
    } else if (kc <= 128) {
        k_rerank<4><<<grid, threads, 0, st>>>(X, Xrow, dtype, d, row_ids, nwarps, cand, kc, k,
                                              out_id, out_d, order);
    } else {
        k_rerank<8><<<grid, threads, 0, st>>>(X, Xrow, dtype, d, row_ids, nwarps, cand, kc, k,
                                              out_id, out_d, order);
    }
#undef ANN_RERANK_VEC_W
#undef ANN_RERANK_VEC
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

static KnnParams base_params(const KnnPlan& pl, int k, const int64_t* blk_off,
                             const KnnProblem* probs, int nprob, const float* na,
                             const uint32_t* gid, const int64_t* outrow, int self_exclude,
                             int local_first, uint32_t* out_id, float* out_d) {
    KnnParams P;
    P.blk_off = blk_off;
    P.probs = probs;
    P.nprob = nprob;
    P.na = na;
    P.gid = gid;
    P.outrow = outrow;
    P.self_exclude = self_exclude;
    P.local_first = local_first;
    P.mode = pl.mode;
    P.nkb_a = pl.nkb_a;
    P.a_stream = pl.a_stream;
    P.nkb_b = pl.nkb_b;
    P.kprime = pl.kprime;
    P.k_out = pl.rerank ? pl.kprime : k;
    P.nst = pl.nst;
    P.kbe = pl.kbe;
    P.kind8 = pl.elem8;
    P.ksteps = pl.ksteps;
    P.hs = pl.hs;
    // same descriptor layout for kind::f16 and kind::f8f6f4 (format 0 = FP16 / E4M3)
    P.idesc_neg = idesc_f16(kt::BM, pl.bn, pl.ab_fmt) | (1u << 13);  // negate A
    P.idesc_aug = idesc_f16(kt::BM, pl.bn, 1);                       // BF16 norm step
    P.out_id = out_id;
    P.out_d = out_d;
    P.status = device_status_ptr();
    P.tlist = nullptr;
    P.tcount = nullptr;
    P.pool = nullptr;
    P.pool_cnt = nullptr;
    P.ph = pool_half(pl.kprime);
    P.rowub = nullptr;
    P.ub_margin = 0.0f;
    return P;
}

static int launch_gather(const void* X, int dtype, int d, const int64_t* src, int64_t rows_cap,
                         const KnnPlan& pl, void* G, float* norms, __nv_bfloat16* aug,
                         const unsigned int* amax, cudaStream_t st) {
    const int threads = 256;
    const int64_t want = (rows_cap * 32 + threads - 1) / threads;
    const unsigned grid = (unsigned)(want < 152 * 64 ? want : 152 * 64);
    if (pl.elem8)
        k_gather<__nv_fp8_e4m3><<<grid, threads, 0, st>>>(X, dtype, d, src, rows_cap, pl.mode,
                                                          pl.Kp, pl.Kh, (__nv_fp8_e4m3*)G, norms,
                                                          aug, amax);
    else if (pl.ab_fmt == 1)
        k_gather<__nv_bfloat16><<<grid, threads, 0, st>>>(X, dtype, d, src, rows_cap, pl.mode,
                                                          pl.Kp, pl.Kh, (__nv_bfloat16*)G, norms,
                                                          aug, nullptr);
    else
        k_gather<__half><<<grid, threads, 0, st>>>(X, dtype, d, src, rows_cap, pl.mode, pl.Kp,
                                                  pl.Kh, (__half*)G, norms, aug,
                                                  pl.scaled ? amax : nullptr);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

// Scaled plans (E4M3, FP16): the largest |x| over the given arrays into amax
// (float bits).
int launch_absmax(const void* X, int dtype, int64_t n, const void* Q, int64_t nq_elems,
                  unsigned int* amax, cudaStream_t st) {
    ANN_CHECK_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned int), st));
    k_absmax<<<152 * 8, 256, 0, st>>>(X, dtype, n, amax);
    ANN_CHECK_LAUNCH();
    if (Q && nq_elems > 0) {
        k_absmax<<<152 * 2, 256, 0, st>>>(Q, dtype, nq_elems, amax);
        ANN_CHECK_LAUNCH();
    }
    return ANN_OK;
}

static unsigned grid_rows(int64_t rows, int threads) {
    const int64_t want = (rows + threads - 1) / threads;
    return (unsigned)(want < 152 * 32 ? (want > 0 ? want : 1) : 152 * 32);
}

// Rows of a shard are first grouped into cells around evenly spaced pivot
// members (the pivot assignment is itself a k = 1 launch of the tile kernel), so
// that each row block sweeps its own cell first; results do not depend on the
// order (ties are broken by global id), only the amount of top-k work does.
// One non-blocking side stream and a pair of fork / join events per device and
// host thread, created on first use and kept for the life of the process (so that
// a build can also be captured as a CUDA graph: the fork and join are events).
static int side_stream(cudaStream_t* s, cudaEvent_t* fork_ev, cudaEvent_t* join_ev) {
    struct Side {
        int dev = -1;
        cudaStream_t s = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
    };
    static thread_local Side cache[8];
    int dev = 0;
    ANN_CHECK_CUDA(cudaGetDevice(&dev));
    Side& c = cache[dev & 7];
    if (c.dev != dev) {
        ANN_CHECK_CUDA(cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking));
        ANN_CHECK_CUDA(cudaEventCreateWithFlags(&c.a, cudaEventDisableTiming));
        ANN_CHECK_CUDA(cudaEventCreateWithFlags(&c.b, cudaEventDisableTiming));
        c.dev = dev;
    }
    *s = c.s;
    *fork_ev = c.a;
    *join_ev = c.b;
    return ANN_OK;
}

// Screening distances of scaled operands back in the data's units: divided by the
// square of the operand scale (448 / max|x| for E4M3, a power of two for FP16).
__global__ void k_unscale_dist(float* __restrict__ dist, int64_t n, const unsigned int* amax_bits,
                               int e4m3) {
    const float am = __uint_as_float(*amax_bits);
    if (!(am > 0.0f && am <= 3.0e38f)) return;
    float scale;
    if (e4m3) {
        scale = 448.0f / am;
    } else {
        int ex;
        frexpf(am, &ex);
        scale = ldexpf(1.0f, 14 - ex);
    }
    const float inv = 1.0f / scale;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dist[i] = (dist[i] * inv) * inv;
}

int run_shard_knn(const void* X, int64_t N, int d, int dtype, const uint32_t* members,
                  const int64_t* offsets, int C, int64_t rows, int k, const KnnPlan& pl,
                  const KnnWs& w, uint32_t* knn_id, float* knn_d, cudaStream_t st,
                  const void* Xr, int dr, int dtype_r, bool screen_only) {
    if (!Xr) {
        Xr = X;
        dr = d;
        dtype_r = dtype;
    }
    (void)N;
    int* status = device_status_ptr();
    k_shard_tables<<<1, 1024, 0, st>>>(offsets, C, rows, w.blk_off, w.pad_off, w.probs, w.order,
                                       status);
    ANN_CHECK_LAUNCH();
    k_ones_tile<<<(128 * kt::KAUG + 255) / 256, 256, 0, st>>>(w.ones);
    ANN_CHECK_LAUNCH();
    int rc;
    // 1. pivots and the cell of every row
    KnnPlan pp = pl;
    pp.kprime = 1;
    pp.rerank = false;
    pp.smem = knn_smem_layout(pp.bn, pp.nkb_a, pp.nst, pp.a_stream).total;
    const unsigned int* amax = nullptr;
    if (pl.scaled) {
        int rc8 = launch_absmax(X, dtype, N * d, nullptr, 0, (unsigned int*)w.amax, st);
        if (rc8) return rc8;
        amax = (const unsigned int*)w.amax;
    }
    // Fine cells pay off where the top-k epilogue bounds the sweep (short rows);
    // with long rows the contraction dominates and coarse cells keep the pivot
    // launch (rows x pivots x d) and the chain (pivots^2 x d) cheap.
    const int cell = row_bytes(pl) <= 512 ? kt::CELL : kt::CELL_WIDE;
    k_pivot_tables<<<1, 32, 0, st>>>(offsets, C, cell, w.pad_off, w.order, w.ppad_off, w.npiv,
                                     w.pprobs);
    ANN_CHECK_LAUNCH();
    k_rowmap_plain<<<grid_rows(w.rows_cap, 256), 256, 0, st>>>(members, offsets, w.pad_off, C,
                                                               w.rows_cap, w.src);
    ANN_CHECK_LAUNCH();
    k_rowmap_pivots<<<grid_rows(w.prows_cap, 256), 256, 0, st>>>(members, offsets, w.ppad_off,
                                                                 w.npiv, C, w.prows_cap, w.psrc);
    ANN_CHECK_LAUNCH();
    // The pivot chain needs only the pivots and runs on one SM per shard: it goes
    // to a side stream, beside the gathers and the pivot-assignment launch.
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    if ((rc = side_stream(&side, &fork_ev, &join_ev))) return rc;
    ANN_CHECK_CUDA(cudaEventRecord(fork_ev, st));
    ANN_CHECK_CUDA(cudaStreamWaitEvent(side, fork_ev, 0));
    if ((rc = launch_pivot_chain(X, dtype, d, w, C, side))) return rc;
    ANN_CHECK_CUDA(cudaEventRecord(join_ev, side));
    if ((rc = launch_gather(X, dtype, d, w.src, w.rows_cap, pl, w.G, w.norms, w.aug, amax, st)))
        return rc;
    if ((rc = launch_gather(X, dtype, d, w.psrc, w.prows_cap, pl, w.GP, w.pnorms, w.paug, amax,
                            st)))
        return rc;
    KnnParams PP = base_params(pp, 1, w.blk_off, w.pprobs, C, w.norms, nullptr, nullptr, 0, 0,
                               w.cell, w.cell_d);
    PP.k_out = 1;
    PP.pool = w.pool;
    PP.pool_cnt = w.pool_cnt;
    rc = launch_tiles(pp, w.G, w.rows_cap, w.ones, w.GP, w.paug, w.prows_cap, PP,
                      rows / kt::BM + C + 1, st, false);
    if (rc) return rc;
    // 2. cell order
    ANN_CHECK_CUDA(cudaStreamWaitEvent(st, join_ev, 0));
    k_cell_sort<<<C, 512, 0, st>>>(w.cell, offsets, w.npiv, w.crank, w.ppad_off, w.perm);
    ANN_CHECK_LAUNCH();
    k_rowmap_cells<<<grid_rows(w.rows_cap, 256), 256, 0, st>>>(members, offsets, w.pad_off, w.perm,
                                                               C, w.rows_cap, w.src, w.gid,
                                                               w.outrow);
    ANN_CHECK_LAUNCH();
    if ((rc = launch_gather(X, dtype, d, w.src, w.rows_cap, pl, w.G, w.norms, w.aug, amax, st)))
        return rc;
    // 3. the kNN sweep
    const bool to_cand = pl.rerank && !screen_only;
    KnnParams P = base_params(pl, k, w.blk_off, w.probs, C, w.norms, w.gid, w.outrow, 1, 1,
                              to_cand ? w.cand_id : knn_id, to_cand ? w.cand_d : knn_d);
    P.pool = w.pool;
    P.pool_cnt = w.pool_cnt;
    const int64_t grid = rows / kt::BM + C + 1;
    const bool skip_u8 = dtype == ANN_U8 && pl.mode == 0 && !pl.rerank && d <= 256 &&
                         d % 4 == 0 && ((uintptr_t)X & 3) == 0;
    // FP32 data: the split keys of the exact form, or the BF16 screening form (plain
    // BF16 operands, no scale), or the scaled FP16 form; each with the margin of its
    // key error below
    const bool split_keys = pl.mode == 1;
    const bool bf16_keys = pl.mode == 0 && pl.ab_fmt == 1 && !pl.scaled && !pl.elem8;
    const bool f16_keys = pl.mode == 0 && pl.ab_fmt == 0 && pl.scaled && !pl.elem8;
    const bool skip_f32 =
        dtype == ANN_F32 && pl.rerank && d <= 200 && (split_keys || bf16_keys || f16_keys);
    if (w.tlist && tile_prune_on() && (skip_u8 || skip_f32)) {
        // 3a. bounds: each row's k'-th distance within its 256-row window (k' = the
        // list width), the centre and radius of every 128-row group, and each block's
        // list of the tiles that may hold a neighbour, nearest first
        const int64_t ng = w.rows_cap / kt::BM;
        k_group_geom<<<(unsigned)ng, 128, (size_t)d * sizeof(float), st>>>(
            X, dtype, d, w.src, ng, pl.Kp, w.gcent, w.grad, w.gmaxn);
        ANN_CHECK_LAUNCH();
        float kslack = 0.0f;
        if (skip_u8) {
            const size_t ubs = ((size_t)256 * (d / 4 + 1) + 256) * sizeof(uint32_t);
            if (d <= 128) {
                ANN_CHECK_CUDA(cudaFuncSetAttribute(
                    k_ub_own<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ubs));
                k_ub_own<32><<<(unsigned)grid, 256, ubs, st>>>(
                    (const uint8_t*)X, d, w.src, w.blk_off, w.probs, C, pl.kprime, grid, w.bub, w.rowub);
            } else {
                ANN_CHECK_CUDA(cudaFuncSetAttribute(
                    k_ub_own<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ubs));
                k_ub_own<64><<<(unsigned)grid, 256, ubs, st>>>(
                    (const uint8_t*)X, d, w.src, w.blk_off, w.probs, C, pl.kprime, grid, w.bub, w.rowub);
            }
        } else {
            // Split BF16 keys (three products, FP32 accumulation): the error of a
            // squared distance stays below (2^-16 + (d + 4) 2^-24)(|x|^2 + |y|^2);
            // BF16 operands (each rounded once, relative 2^-9; the norms in FP32):
            // below (2^-8 + (d + 8) 2^-24)(|x|^2 + |y|^2); FP16 operands after an
            // exact power-of-two scale (relative 2^-11 each): below (2^-10 + (d + 8)
            // 2^-24)(|x|^2 + |y|^2) in the data's units.  A skipped column must
            // clear the bound by twice that, taken 4x larger.
            kslack = split_keys  ? 8.0f * (0x1p-16f + (float)(d + 4) * 0x1p-24f)
                     : bf16_keys ? 8.0f * (0x1p-8f + (float)(d + 8) * 0x1p-24f)
                                 : 8.0f * (0x1p-10f + (float)(d + 8) * 0x1p-24f);
            const size_t ubs = (size_t)256 * (d + 1) * sizeof(float);
            ANN_CHECK_CUDA(cudaFuncSetAttribute(
                k_ub_own_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ubs));
            k_ub_own_f32<<<(unsigned)grid, 256, ubs, st>>>(
                (const float*)X, d, w.src, w.blk_off, w.probs, C, pl.kprime, grid, w.bub, w.rowub);
        }
        ANN_CHECK_LAUNCH();
        const size_t tls = tile_list_smem(d).total;
        ANN_CHECK_CUDA(cudaFuncSetAttribute(k_tile_list, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)tls));
        k_tile_list<<<(unsigned)((grid + TLB - 1) / TLB), 256, tls, st>>>(
            w.blk_off, w.probs, C, pl.bn, d, pl.Kp, w.gcent, w.grad, w.gmaxn, kslack, w.bub, grid,
            w.tlist, w.tcount);
        ANN_CHECK_LAUNCH();
        P.tlist = w.tlist;
        P.tcount = w.tcount;
        // each row's window bound starts its threshold (keys in the data's units:
        // not for scaled operands, whose keys carry the square of the scale)
        P.rowub = pl.scaled ? nullptr : w.rowub;
        P.ub_margin = kslack;
    }
    rc = launch_tiles(pl, w.G, w.rows_cap, w.ones, w.G, w.aug, w.rows_cap, P, grid, st, true);
    if (rc) return rc;
    if (screen_only) {  // the screened list as it stands: k' entries per row
        if (pl.scaled) {
            k_unscale_dist<<<grid_rows(rows * P.k_out, 256), 256, 0, st>>>(
                knn_d, rows * P.k_out, (const unsigned int*)w.amax, pl.elem8);
            ANN_CHECK_LAUNCH();
        }
        return ANN_OK;
    }
    if (pl.rerank)
        return launch_rerank(Xr, Xr, dtype_r, dr, members, rows, w.cand_id, pl.kprime, k, knn_id,
                             knn_d, st, w.outrow, w.rows_cap);
    return ANN_OK;
}

// Query side: A = queries, B = all N vectors (one problem, no self exclusion).
size_t query_ws(int64_t N, int64_t nq, const KnnPlan& pl, QueryWs* out, void* base, size_t cap) {
    Carver cv(base, cap);
    QueryWs w;
    w.capA = nq + kt::BM + kt::BNMAX;
    w.capB = N + kt::BM + kt::BNMAX;
    w.blk_off = cv.take<int64_t>(4);
    w.pad_off = cv.take<int64_t>(4);
    w.offs = cv.take<int64_t>(4);
    w.prob = cv.take<KnnProblem>(1);
    w.GA = (__nv_bfloat16*)cv.take<uint8_t>((size_t)w.capA * row_bytes(pl));
    w.GB = (__nv_bfloat16*)cv.take<uint8_t>((size_t)w.capB * row_bytes(pl));
    w.augA = cv.take<__nv_bfloat16>((size_t)w.capA * kt::KAUG);
    w.augB = cv.take<__nv_bfloat16>((size_t)w.capB * kt::KAUG);
    w.ones = cv.take<__nv_bfloat16>((size_t)128 * kt::KAUG);
    w.na = cv.take<float>((size_t)w.capA + 512);
    w.nb = cv.take<float>((size_t)w.capB + 512);
    w.cand_id = pl.rerank ? cv.take<uint32_t>((size_t)nq * pl.kprime) : nullptr;
    w.cand_d = pl.rerank ? cv.take<float>((size_t)nq * pl.kprime) : nullptr;
    w.pool = cv.take<uint64_t>((size_t)w.capA * 2 * pool_half(pl.kprime));
    w.pool_cnt = cv.take<int>((size_t)w.capA * 2);
    w.srcA = cv.take<int64_t>((size_t)w.capA);
    w.srcB = cv.take<int64_t>((size_t)w.capB);
    w.amax = cv.take<float>(4);
    if (out) *out = w;
    return cv.used + 256;
}

__global__ void k_query_tables(int64_t N, int64_t nq, int64_t* blk_off, int64_t* pad4,
                               int64_t* offs4, KnnProblem* prob) {
    if (threadIdx.x || blockIdx.x) return;
    blk_off[0] = 0;
    blk_off[1] = (nq + kt::BM - 1) / kt::BM;
    offs4[0] = 0;  // A side (queries): offsets {0, nq}, padded {0, nq rounded up}
    offs4[1] = nq;
    offs4[2] = 0;  // B side (all vectors): offsets {0, N}
    offs4[3] = N;
    pad4[0] = 0;
    pad4[1] = blk_off[1] * kt::BM;
    pad4[2] = 0;
    pad4[3] = (N + kt::BM - 1) / kt::BM * kt::BM;
    KnnProblem p;
    p.a_row0 = 0;
    p.b_row0 = 0;
    p.out_row0 = 0;
    p.mem_row0 = 0;
    p.n_rows = (int32_t)nq;
    p.n_cols = (int32_t)N;
    prob[0] = p;
}

int run_knn_query(const void* X, int64_t N, const void* Q, int64_t nq, int d, int dtype, int k,
                  const KnnPlan& pl, const QueryWs& w, uint32_t* out_id, float* out_d,
                  cudaStream_t st) {
    k_query_tables<<<1, 32, 0, st>>>(N, nq, w.blk_off, w.pad_off, w.offs, w.prob);
    ANN_CHECK_LAUNCH();
    k_ones_tile<<<(128 * kt::KAUG + 255) / 256, 256, 0, st>>>(w.ones);
    ANN_CHECK_LAUNCH();
    k_rowmap_plain<<<grid_rows(w.capA, 256), 256, 0, st>>>(nullptr, w.offs, w.pad_off, 1, w.capA,
                                                           w.srcA);
    ANN_CHECK_LAUNCH();
    k_rowmap_plain<<<grid_rows(w.capB, 256), 256, 0, st>>>(nullptr, w.offs + 2, w.pad_off + 2, 1,
                                                           w.capB, w.srcB);
    ANN_CHECK_LAUNCH();
    const unsigned int* amax = nullptr;
    if (pl.scaled) {
        int rc8 = launch_absmax(X, dtype, N * d, Q, nq * d, (unsigned int*)w.amax, st);
        if (rc8) return rc8;
        amax = (const unsigned int*)w.amax;
    }
    int rc = launch_gather(Q, dtype, d, w.srcA, w.capA, pl, w.GA, w.na, w.augA, amax, st);
    if (!rc) rc = launch_gather(X, dtype, d, w.srcB, w.capB, pl, w.GB, w.nb, w.augB, amax, st);
    if (rc) return rc;
    KnnParams P = base_params(pl, k, w.blk_off, w.prob, 1, w.na, nullptr, nullptr, 0, 0,
                              pl.rerank ? w.cand_id : out_id, pl.rerank ? w.cand_d : out_d);
    P.pool = w.pool;
    P.pool_cnt = w.pool_cnt;
    const int64_t grid = (nq + kt::BM - 1) / kt::BM;
    rc = launch_tiles(pl, w.GA, w.capA, w.ones, w.GB, w.augB, w.capB, P, grid, st, true);
    if (rc) return rc;
    if (pl.rerank)
        return launch_rerank(X, Q, dtype, d, nullptr, nq, w.cand_id, pl.kprime, k, out_id, out_d,
                             st);
    return ANN_OK;
}

int tile_counters_read(unsigned long long* out, int n, bool reset) {
    unsigned long long tmp[TC_N];
    ANN_CHECK_CUDA(cudaDeviceSynchronize());
    ANN_CHECK_CUDA(cudaMemcpyFromSymbol(tmp, g_tile_counters, sizeof(tmp)));
    for (int i = 0; i < n && i < TC_N; ++i) out[i] = tmp[i];
    if (reset) {
        unsigned long long z[TC_N] = {0};
        ANN_CHECK_CUDA(cudaMemcpyToSymbol(g_tile_counters, z, sizeof(z)));
    }
    return ANN_OK;
}

// ---- screening query: tile keys only, exact decisions taken by the caller ---------
// For every A row p (row rowsel[p0 + p] of Xa, or p0 + p when rowsel is NULL) the
// ks rows of Xb with the smallest tile key |y|^2/2 - x.y (ties to the smaller
// index), written as indices into Xb.  Both sides use the FP32 split operand form
// (three BF16 products), whatever their element types.

static int screen_plan(int d, int ks, KnnPlan* pl) {
    int rc = knn_plan(d, ANN_F32, ks, ANN_EXACT, 0, pl);
    if (rc) return rc;
    pl->rerank = false;
    pl->kprime = ks;
    pl->smem = knn_smem_layout(pl->bn, pl->nkb_a, pl->nst, pl->a_stream).total;
    return ANN_OK;
}

size_t screen_ws(int64_t na, int64_t nb, int d, int ks) {
    KnnPlan pl;
    if (screen_plan(d, ks, &pl)) return 0;
    Carver cv(nullptr, ~(size_t)0);
    cv.take<uint8_t>(query_ws(nb, na, pl, nullptr, nullptr, 0));
    cv.take<float>((size_t)na * ks);
    return cv.used + 256;
}

__global__ void k_rowmap_sel(const uint32_t* __restrict__ rowsel, int64_t p0, int64_t n,
                             int64_t cap, int64_t* __restrict__ src) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < cap;
         p += (int64_t)gridDim.x * blockDim.x)
        src[p] = p < n ? (rowsel ? (int64_t)rowsel[p0 + p] : p0 + p) : -1;
}

int run_screen(const void* Xa, int dta, const uint32_t* rowsel, int64_t p0, int64_t na,
               const void* Xb, int dtb, int64_t nb, int d, int ks, uint32_t* out_id, void* ws,
               size_t ws_bytes, cudaStream_t st) {
    KnnPlan pl;
    int rc = screen_plan(d, ks, &pl);
    if (rc) return rc;
    if (screen_ws(na, nb, d, ks) > ws_bytes) return fail(ANN_ERR_WORKSPACE, "screen: workspace");
    if (na == 0) return ANN_OK;
    Carver cv(ws, ws_bytes);
    const size_t qb = query_ws(nb, na, pl, nullptr, nullptr, 0);
    uint8_t* qbase = cv.take<uint8_t>(qb);
    float* out_d = cv.take<float>((size_t)na * ks);
    QueryWs w;
    query_ws(nb, na, pl, &w, qbase, qb);
    k_query_tables<<<1, 32, 0, st>>>(nb, na, w.blk_off, w.pad_off, w.offs, w.prob);
    ANN_CHECK_LAUNCH();
    k_ones_tile<<<(128 * kt::KAUG + 255) / 256, 256, 0, st>>>(w.ones);
    ANN_CHECK_LAUNCH();
    k_rowmap_sel<<<grid_rows(w.capA, 256), 256, 0, st>>>(rowsel, p0, na, w.capA, w.srcA);
    ANN_CHECK_LAUNCH();
    k_rowmap_plain<<<grid_rows(w.capB, 256), 256, 0, st>>>(nullptr, w.offs + 2, w.pad_off + 2, 1,
                                                           w.capB, w.srcB);
    ANN_CHECK_LAUNCH();
    if ((rc = launch_gather(Xa, dta, d, w.srcA, w.capA, pl, w.GA, w.na, w.augA, nullptr, st)))
        return rc;
    if ((rc = launch_gather(Xb, dtb, d, w.srcB, w.capB, pl, w.GB, w.nb, w.augB, nullptr, st)))
        return rc;
    KnnParams P = base_params(pl, ks, w.blk_off, w.prob, 1, w.na, nullptr, nullptr, 0, 0, out_id,
                              out_d);
    P.pool = w.pool;
    P.pool_cnt = w.pool_cnt;
    const int64_t grid = (na + kt::BM - 1) / kt::BM;
    return launch_tiles(pl, w.GA, w.capA, w.ones, w.GB, w.augB, w.capB, P, grid, st, false);
}

}  // namespace ann
