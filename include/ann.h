/*
 * ann.h - C-ABI of the GB300 (sm_103a) divide-and-merge graph-index build.
 *
 * The method is ScaleGANN's (arxiv 2605.10135), Sec. IV "Workflow": (1) data
 * partitioning by k-means with replication of each vector into its nearest
 * shards, (2) an independent graph build per shard, (3) merging the shard
 * graphs into one graph by edge union, with the replicated vectors as links
 * (Sec. II-B).  Here the per-shard graph is the exact k-nearest-neighbour
 * graph of intermediate degree k (the paper's L), pruned to degree R.
 *
 * Conventions shared by every call
 *  - Every pointer argument is a DEVICE pointer (cudaMalloc / PyTorch CUDA
 *    tensor) owned by the caller, unless the argument says "host".  The
 *    library never frees or retains caller memory.
 *  - The vectors X of ann_partition, ann_partition_selective, ann_shard_knn,
 *    ann_medoid, ann_medoid_noalloc, ann_knn_query, ann_search and
 *    ann_search_entries, and their
 *    queries Q, may instead be page-locked
 *    host memory mapped into the device's address space at the same address
 *    (cudaHostAlloc / cudaHostRegister with unified addressing, a pinned
 *    PyTorch CPU tensor): the kernels then read the vectors over the host link
 *    (NVLink-C2C on Grace-Blackwell), so X need not fit in device memory.
 *    Pageable host memory or another device's memory is refused with
 *    ANN_ERR_INVALID_ARG before any launch (the check runs once the workspace
 *    checks, or ann_medoid_noalloc's size checks, have passed).
 *  - Scratch memory comes from a caller-supplied workspace of at least the
 *    size the matching *_workspace() call reports; it may be reused after the
 *    call's work on the stream has completed.
 *  - Calls are asynchronous on the CUDA stream passed as `stream` (a
 *    cudaStream_t; NULL = legacy default stream).  Results are valid once the
 *    stream's work has completed.
 *  - Row-major layouts throughout.  Vector ids are uint32 global row indices;
 *    ANN_PAD (0xFFFFFFFF) marks an empty neighbour slot, whose distance is +inf.
 *  - Distances are squared Euclidean distances stored as float32.  For uint8
 *    vectors they are exact integers.
 *  - Return value: ANN_OK or an ANN_ERR_* code; ann_last_error() gives a
 *    message (thread-local).  Calls never abort the process.  Conditions found
 *    on the device (a bounded wait that gave up, inconsistent offsets) are
 *    recorded in a device status word read by ann_device_status().
 */
#ifndef ANN_GB300_H
#define ANN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ANN_PAD 0xFFFFFFFFu

enum ann_status {
    ANN_OK = 0,
    ANN_ERR_INVALID_ARG = 1,  /* a size, pointer or enum outside its documented range */
    ANN_ERR_UNSUPPORTED = 2,  /* a valid combination the library does not implement */
    ANN_ERR_CUDA = 3,         /* a CUDA runtime/driver call failed */
    ANN_ERR_TIMEOUT = 4,      /* a device-side bounded wait gave up (see ann_device_status) */
    ANN_ERR_WORKSPACE = 5     /* workspace missing or smaller than reported */
};

/* Element type of the input vectors (Table 3: uint8 and float datasets). */
enum ann_dtype { ANN_F32 = 0, ANN_F16 = 1, ANN_BF16 = 2, ANN_U8 = 3 };

/* How shard distance tiles are computed.
 *  ANN_EXACT: uint8 -> BF16 tiles with FP32 accumulation (exact integers);
 *             float -> BF16 hi/lo split tiles (three products) screening a
 *             widened list, then an FP32 direct-form re-rank.
 *  ANN_BF16_RERANK: float vectors rounded once to BF16 (one product per
 *             pair, FP32 accumulation) screen a list of rerank_k (default
 *             128) candidates per row, then the FP32 direct-form re-rank
 *             picks the k of smallest (distance, id); on uint8 it equals
 *             ANN_EXACT (BF16 holds 0..255 exactly).
 *  ANN_FP8_RERANK: as ANN_BF16_RERANK with E4M3 screening tiles
 *             (tcgen05 kind::f8f6f4): every element is multiplied by one
 *             global scale 448 / max|x| before rounding, and the norm terms
 *             use the same scaled values.  E4M3 keeps 3 mantissa bits, so
 *             the screened list misses more true neighbours than BF16's.
 *  ANN_F16_RERANK: as ANN_BF16_RERANK with FP16 screening tiles: every
 *             element is multiplied by the power of two that puts max|x| in
 *             [2^13, 2^14) (exact), then rounded to FP16 (11 significant bits
 *             against BF16's 8, same tensor-core rate).  Exact on uint8.
 *  ANN_LEARNED: candidates proposed by a learned 32-dimensional embedding,
 *             re-ranked exactly (see ann_learned_train below). */
enum ann_precision {
    ANN_EXACT = 0,
    ANN_BF16_RERANK = 1,
    ANN_FP8_RERANK = 2,
    ANN_LEARNED = 3,
    ANN_F16_RERANK = 4
};

/* Prune rule for L -> R (Sec. III, Sec. VI-B2 use L = 2R; the rule itself is
 * not printed in the paper).  ANN_PRUNE_RANK: rank-based detour count
 * c_j = #{ i < j : pos_{v_i}(v_j) < j } over u's sorted list, keep the R
 * entries of smallest (c_j, j) in list order.  ANN_PRUNE_TRUNC: first R. */
enum ann_prune_rule { ANN_PRUNE_RANK = 0, ANN_PRUNE_TRUNC = 1 };

/* Message of the last failed call on this host thread ("" if none). */
const char* ann_last_error(void);

/* Library ABI version (major*100 + minor); 103 adds ANN_F16_RERANK, the learned
 * form, the autotuner and the wait self-test to 100; 104 adds
 * ann_partition_selective, ann_search_entries, host-resident vectors, the tile
 * skipping switch and statistics, and the scheduler calls. */
int ann_version(void);

/* Number of kernels this library has launched in this process (host counter). */
unsigned long long ann_launch_count(void);

/* Measurement hooks.  ann_timing_enable(1) makes every later launch of the
 * distance-tile kernel (ann_shard_knn, ann_knn_query) record a pair of CUDA
 * events on the launching stream.  ann_timing_read() waits for the recorded
 * events, returns the summed kernel time in milliseconds (host tile_ms) and the
 * number of launches timed (host launches), and forgets them. */
int ann_timing_enable(int on);
int ann_timing_read(double* tile_ms, int* launches);

/* Profiling hook.  ann_tile_counters_enable(1) switches later distance-tile
 * launches to a variant that accumulates per-role clock64() cycle counts and
 * event counts into a device array; ann_tile_counters_read() synchronises the
 * device, copies up to n counters to host out[] and clears them.  Order:
 * epilogue cycles, epilogue wait cycles, pool compaction cycles, chunks, chunks
 * with survivors, compactions, rows compacted, (unused, 0), appended survivors,
 * MMA wait-for-data cycles, MMA wait-for-accumulator cycles, producer wait
 * cycles, CTA cycles, CTAs, TMEM-load wait cycles, filter cycles, append cycles
 * (everything after the filter, compactions included), MMA issue cycles, MMA
 * commit cycles, MMA loop cycles, stash-write cycles, cycles appending chunks
 * straight to the pools, cycles moving the stash to the pools. */
int ann_tile_counters_enable(int on);
int ann_tile_counters_read(unsigned long long* out, int n);

/* Exact skipping of distance tiles (on by default).  For ANN_EXACT on uint8
 * vectors of d <= 256 (d a multiple of 4, X 4-byte aligned) and on float32 vectors
 * of d <= 200, each
 * row's k'-th squared distance among the rows of its 256-row window of the shard
 * (k' = the screened list width) bounds its final one from above; for float32 the
 * bound also carries a margin for the error of the tile keys.  A column tile is then
 * skipped (no copy, no product, no epilogue) when the triangle inequality over
 * 128-row groups (centre and radius bound of each group) shows that every column
 * in it is strictly farther than the block's largest bound.  The lists do not
 * change (ties included).  ann_tile_prune(0) sweeps every tile.
 * ann_tile_prune_stats synchronises the device, writes up to n counters to host
 * out[] and clears them: column tiles of the blocks, tiles swept, (row, column)
 * pairs swept. */
int ann_tile_prune(int on);
int ann_tile_prune_stats(unsigned long long* out, int n);


/* Self-test of the bounded device waits (no fault, no hang): one warp waits on
 * an mbarrier that nothing completes, through the bounded wait that every
 * pipelined kernel uses; mode 0 lets the limit (limit_us microseconds, at most
 * 2 s) run out, mode 1 starts with the abort flag set.  The kernel records the
 * timeout bit in the device status word and returns, so a following
 * ann_device_status() returns ANN_ERR_TIMEOUT and the context stays usable. */
int ann_wait_selftest(int mode, int64_t limit_us, void* stream);

/* Autotuner of the distance-tile plan.  ann_autotune(1): every later
 * ann_shard_knn call (not ANN_LEARNED) whose key (d, dtype, k, precision,
 * rerank_k, floor(log2(rows / C))) has no decision yet runs the whole shard kNN
 * once with each candidate plan - tile width 256 or 128, the two deepest TMA
 * rings that fit shared memory - timing each with CUDA events on its stream
 * (the call synchronises that stream), and keeps the fastest for the key.  The
 * lists do not depend on the plan, so the call's output is the same as
 * untuned.  Decided keys use their plan whether tuning is on or off.
 * ann_autotune(0) stops tuning new keys; ann_autotune(-1) also forgets every
 * decision.  ann_autotune_lookup: host out found (0/1) and, if found, the
 * chosen tile width bn, ring depth nst, streamed-A flag, its time in ms and the
 * number of plans tried. */
int ann_autotune(int on);
int ann_autotune_lookup(int d, int dtype, int k, int precision, int rerank_k, int64_t rows, int C,
                        int* found, int* bn, int* nst, int* a_stream, float* ms, int* tried);

/* Reads (host out) and clears the device status word of the current device:
 * bit 1 = a bounded device wait gave up, bit 2 = inconsistent input found on
 * the device (e.g. offsets[C] != rows), bit 4 = a fixed-capacity buffer
 * overflowed.  Synchronises the device.  Returns ANN_OK, or ANN_ERR_TIMEOUT
 * if bit 1 was set. */
int ann_device_status(int* out);

/* ---------------------------------------------------------------------------
 * ann_partition - Sec. IV Workflow (1) and Sec. II-B: k-means shard centroids,
 * then each vector replicated into its r nearest shards ("typically two";
 * Sec. VI-B2: one replication, r = 2).
 *
 *  X               [N x d] vectors of type dtype.
 *  init_centroids  [C x d] float32 starting centroids.
 *  sample_idx      [S] uint32 rows of X used for k-means (any order; the FP64
 *                  centroid sums follow this order).
 *  iters           Lloyd iterations (>= 0).  Each assigns every sample row
 *                  to the centroid of smallest (d32, id) - d32 being the FP32
 *                  squared distance with terms added in index order, unfused -
 *                  then sets each centroid to the FP64 mean of its rows,
 *                  rounded to float; an empty cluster keeps its centroid.
 *  centroids_out   [C x d] float32 final centroids.
 *  members_out     [N*r] uint32: shard c's members are
 *                  members_out[offsets_out[c] .. offsets_out[c+1]), ids in
 *                  increasing order.  A vector goes to the r centroids of
 *                  smallest (d32, id).
 *  offsets_out     [C+1] int64.
 * Limits: 1 <= r <= C <= 1024, 1 <= d <= 4096, N < 2^32.
 * ------------------------------------------------------------------------- */
int ann_partition_workspace(int64_t N, int d, int C, int r, int64_t S, size_t* bytes);
int ann_partition(const void* X, int64_t N, int d, int dtype, int C, int r,
                  const float* init_centroids, const uint32_t* sample_idx, int64_t S, int iters,
                  float* centroids_out, uint32_t* members_out, int64_t* offsets_out, void* ws,
                  size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ann_partition_selective - Sec. V: k-means centroids as in ann_partition,
 * then the blockwise-adaptive assignment with selective replication (Sec.
 * V-A, Sec. V-B, Algorithm 1).  Vectors are taken once, in id order, in blocks
 * of `block` vectors.  Vector v considers its `cand` (M) centroids of smallest
 * (d32, id).  Per cluster c the call tracks its members (tot), originals,
 * replicas, and squared radius rad2 = the largest d32 of its originals so far.
 * For block b (1-based):
 *   1. originals: each v, in id order, joins its nearest candidate with
 *      tot < capacity (capacity 0: no limit); with none of the M free it
 *      joins its nearest one anyway (counted in stats_out[1]);
 *   2. per cluster, replica threshold theta = max(0, capacity -
 *      ceil(originals * N / processed)), processed = vectors in blocks 1..b
 *      (room kept for the originals still to come; no threshold without a
 *      capacity), and rad2 updated with the block's originals;
 *   3. replicas: each v, in id order, walks its candidates nearest first and
 *      joins c' (not its original c) while it is in fewer than omega shards,
 *      if replicas(c') < theta(c'), tot(c') < capacity, and
 *         d32(v,c') < (eps*eps) * d32(v,c)                 (distance test)
 *         d32(v,c') < ((eps*tau)*(eps*tau)) * rad2(c')     (radius test),
 *      tau = 1 + (tau0 - 1) / b, both right-hand sides in FP64 (the paper's
 *      d' < eps d and d' < eps tau R[c'] on squared distances).  epsilon =
 *      +INFINITY drops both tests.
 * With epsilon = +INFINITY and capacity 0 the result is ann_partition's with
 * r = omega.
 *
 *  params        host pointer to the parameters below.
 *  assign_out    [N x omega] uint32 or NULL: v's original shard first, then
 *                its replicas nearest first, then ANN_PAD.
 *  members_out   room for N*omega uint32; shard c's members (ids ascending)
 *                are members_out[offsets_out[c] .. offsets_out[c+1]).
 *  offsets_out   [C+1] int64; offsets_out[C] = N + replicas.
 *  stats_out     [2] int64 or NULL: replicas, originals that found no room.
 * Limits: 1 <= omega <= cand <= min(C, 32), C <= 1024, epsilon >= 0 (or
 * +inf), tau0 finite >= 0, block >= 1, capacity < 2^40.  Without a capacity
 * every stage runs over all vectors in parallel; with one, the dependence of
 * each vector on the earlier ones is resolved by one thread block.
 * ------------------------------------------------------------------------- */
typedef struct ann_selective_params {
    double epsilon;    /* eps of Sec. V-B (Table 4: 1.1 .. 1.5); +inf: no test */
    double tau0;       /* tau of the first block (Sec. V-B: large, then falling) */
    int64_t block;     /* vectors per block (Sec. V-A) */
    int64_t capacity;  /* members per shard, 0 = unlimited */
    int omega;         /* most shards a vector joins (omega = 2: one replica) */
    int cand;          /* candidate centroids per vector (M) */
} ann_selective_params;

int ann_partition_selective_workspace(int64_t N, int d, int C, int64_t S,
                                      const ann_selective_params* params, size_t* bytes);
int ann_partition_selective(const void* X, int64_t N, int d, int dtype, int C,
                            const float* init_centroids, const uint32_t* sample_idx, int64_t S,
                            int iters, const ann_selective_params* params, float* centroids_out,
                            uint32_t* assign_out, uint32_t* members_out, int64_t* offsets_out,
                            int64_t* stats_out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ann_shard_knn - Sec. IV Workflow (2): the graph of every shard, built
 * independently.  For shard member u (row p = its position in members), the
 * k other members of the same shard with the smallest (distance, id), self
 * excluded by id; fewer than k others -> trailing ANN_PAD / +inf.
 *
 *  members, offsets  as produced by ann_partition (C shards, rows = offsets[C]
 *                    total members; each shard's ids sorted increasingly).
 *  knn_id / knn_d    [rows x k] output, row p for members[p].
 *  precision         ANN_EXACT, ANN_BF16_RERANK, ANN_F16_RERANK or
 *                    ANN_FP8_RERANK (see enum).  uint8 results are bit-exact
 *                    under ANN_EXACT, ANN_BF16_RERANK and ANN_F16_RERANK; float
 *                    results carry FP32 direct-form distances of the ids
 *                    returned.
 *  rerank_k          width of the screened list before the re-rank: 0 =
 *                    k + 16 (ANN_EXACT) or 128 (the screening forms); else
 *                    k <= rerank_k <= 128.  Ignored for uint8 under ANN_EXACT.
 *  model             ANN_LEARNED: the device parameter array of the MLP (see
 *                    ann_learned_train); NULL makes ANN_LEARNED the exact form
 *                    (ANN_EXACT).  Other precisions: NULL.
 * Limits: d <= 4096 (uint8: d <= 258, which keeps the integer tiles exact),
 * 1 <= k <= 240, rerank_k <= 256, 1 <= C <= 1024, every shard smaller than 2^24
 * members.  When
 * the 128 rows of a block do not fit shared memory (large d) their K blocks
 * stream through the ring beside the B blocks instead of staying resident.
 * ------------------------------------------------------------------------- */
int ann_shard_knn_workspace(int64_t N, int d, int dtype, int C, int64_t rows, int k,
                            int precision, int rerank_k, size_t* bytes);
int ann_shard_knn(const void* X, int64_t N, int d, int dtype, const uint32_t* members,
                  const int64_t* offsets, int C, int64_t rows, int k, int precision, int rerank_k,
                  const void* model, uint32_t* knn_id, float* knn_d, void* ws, size_t ws_bytes,
                  void* stream);

/* ann_shard_knn_screen: the screened lists of ann_shard_knn before its FP32
 *   re-rank, for measuring a precision form's screening error: per shard row
 *   the k' smallest screening keys (ann_screen_width gives k'), written as
 *   (global id, |x|^2 + 2 key) in the data's units (scaled operands divided by
 *   the scale squared), sorted by (distance, id); cand_id / cand_d [rows x k'].
 *   Forms without a re-rank (uint8 ANN_EXACT) return the final lists (k' = k).
 *   Same workspace as ann_shard_knn; ANN_LEARNED is not accepted. */
int ann_screen_width(int d, int dtype, int k, int precision, int rerank_k, int* kprime);
int ann_shard_knn_screen(const void* X, int64_t N, int d, int dtype, const uint32_t* members,
                         const int64_t* offsets, int C, int64_t rows, int k, int precision,
                         int rerank_k, uint32_t* cand_id, float* cand_d, void* ws,
                         size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ann_prune - intermediate degree k (L) to final degree R per shard row, by
 * `rule` (enum ann_prune_rule).  The paper builds each shard graph with an
 * intermediate degree L and a final index degree R (Sec. III "Motivation",
 * the (R, L) = (32, 64) and (64, 128) settings; Sec. VI-B2, default R = 64,
 * L = 128) and takes the reduction from its shard builder, CAGRA (Sec. II-A);
 * it prints no rule.  ANN_PRUNE_RANK is the reading used here: for row u with
 * list v_0 .. v_{k-1}, c_j counts the i < j whose own list ranks v_j before
 * position j (a two-hop path with both hops ranked ahead of the direct edge),
 * and the R entries of smallest (c_j, j) are kept.  Integer logic on the lists only: the output
 * depends on knn_id alone (knn_d is carried), so identical lists give
 * identical results.  pr_id / pr_d: [rows x R], kept entries in list order
 * then ANN_PAD / +inf.  N = number of vectors (ids < N).  The workspace holds
 * the inverse of the member lists (the rows of every id).
 * Limits: 1 <= R, k <= 256.
 * ------------------------------------------------------------------------- */
int ann_prune_workspace(int64_t N, int64_t rows, size_t* bytes);
int ann_prune(const uint32_t* knn_id, const float* knn_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t rows, int64_t N, int k, int R, int rule,
              uint32_t* pr_id, float* pr_d, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ann_merge - Sec. IV Workflow (3), Sec. II-B "edge union": for every vector
 * g the union of its pruned lists over the shards holding g, duplicates
 * removed by id (smaller distance kept), then the R entries of smallest
 * (distance, id), sorted.  graph / gdist: [N x R]; degree: [N] uint32.
 * The result does not depend on the order of the shards.
 * Limits: (copies of one vector) * R <= 256.
 * ------------------------------------------------------------------------- */
int ann_merge_workspace(int64_t N, int64_t rows, size_t* bytes);
int ann_merge(const uint32_t* pr_id, const float* pr_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t rows, int64_t N, int R, uint32_t* graph,
              float* gdist, uint32_t* degree, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ann_merge_reverse - a variant of the merge with reverse edges (CAGRA adds
 * them after its rank-based prune, Sec. II-A; the paper merges by edge union
 * only, Sec. II-B, so this is an alternative, not a step of the method).  For
 * every vertex v of a merged graph: the first ceil(R/2) entries of v's list,
 * then the vertices u whose lists hold v, with the distance of that edge, in
 * (distance, id) order, skipping ids already taken, then the rest of v's own
 * list skipping ids already taken, up to R entries; the result sorted by
 * (distance, id).  graph / gdist / degree: a merged graph as ann_merge writes
 * it ([N x R], [N x R], [N]; ids < N, no self-loops, entries past degree
 * ignored); out_graph / out_gdist / out_degree the same shapes, caller-owned,
 * not overlapping the inputs.  A list entry >= N or equal to its own vertex
 * sets ANN_DEV_BAD_INPUT in ann_device_status and is skipped.
 * Limits: 1 <= R <= 64, N < 2^32.
 * ------------------------------------------------------------------------- */
int ann_merge_reverse_workspace(int64_t N, int R, size_t* bytes);
int ann_merge_reverse(const uint32_t* graph, const float* gdist, const uint32_t* degree,
                      int64_t N, int R, uint32_t* out_graph, float* out_gdist,
                      uint32_t* out_degree, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Query-side evaluation (Sec. VI-B2: top-10 recall with a best-first search
 * of the merged graph following DiskANN's strategy).
 *
 * ann_medoid: entry_out (device uint32[1]) = the vector nearest (d32) to the
 *   FP64 mean of X rounded to float, ties to the smaller id.
 * ann_knn_query: exact top-k of each of nq queries Q [nq x d] (type dtype)
 *   over all N vectors by (distance, id), same tile kernels and precision
 *   rules as ann_shard_knn; out_id / out_d [nq x k].
 * ann_search: best-first beam search from `entry`, list size Ls; expanding a
 *   vertex computes d32 to each unseen out-neighbour; stops when every listed
 *   vertex is expanded.  out_id [nq x topk]; out_count [nq] uint32 = distance
 *   computations.  Limits: Ls <= 256, R <= 64, topk <= Ls.
 * ann_recall: recall_out (device float[1]) = mean over queries of
 *   |first kk of found  intersect  first kk of truth| / kk.
 * ------------------------------------------------------------------------- */
int ann_medoid_workspace(int64_t N, int d, size_t* bytes);
int ann_medoid(const void* X, int64_t N, int d, int dtype, uint32_t* entry_out, void* ws,
               size_t ws_bytes, void* stream);
/* ann_medoid_noalloc: the same result as ann_medoid (same kernels, same order),
 * for callers that cannot allocate device memory - e.g. code running inside
 * a framework that owns the device's memory pool, or a pipeline stage where a
 * cudaMalloc could synchronise the device or fail part-way.  It takes no
 * workspace and calls no allocating routine: its scratch is a fixed array of
 * 4 MiB + 16 KiB inside the library, reserved on every device that loads the
 * library until the process exits.  Limits: d <= 4096 and
 * ceil(N / 4096) * d <= 524288 (e.g. N <= 2^21 at d = 1024); larger inputs are
 * rejected with ANN_ERR_INVALID_ARG (use ann_medoid with a workspace).  The
 * first call in a CUDA context looks up the array's device address (with that
 * context's device current) and caches it per context, so a context created
 * again after a device reset gets a fresh lookup; make the first call in a
 * context before any stream capture.  All calls share
 * the one array: calls whose work overlaps on the GPU (different streams, or
 * several host threads) race and must be serialised by the caller.  The paper
 * has no counterpart: this entry point exists only for such callers. */
int ann_medoid_noalloc(const void* X, int64_t N, int d, int dtype, uint32_t* entry_out,
                       void* stream);
int ann_knn_query_workspace(int64_t N, int64_t nq, int d, int dtype, int k, size_t* bytes);
int ann_knn_query(const void* X, int64_t N, const void* Q, int64_t nq, int d, int dtype, int k,
                  uint32_t* out_id, float* out_d, void* ws, size_t ws_bytes, void* stream);
int ann_search(const uint32_t* graph, const uint32_t* degree, int R, const void* X, int64_t N,
               int d, int dtype, const void* Q, int64_t nq, uint32_t entry, int Ls, int topk,
               uint32_t* out_id, uint32_t* out_count, void* stream);
/* ann_search_entries: ann_search, except that each query starts from the vector
 *   of smallest (d32(q, x), id) among the ne ids in entries (device uint32[ne];
 *   ids >= N are skipped; a query with no valid entry returns ANN_PAD ids and
 *   sets the bad-input bit of the device status).  out_count includes the
 *   distances to the valid entries.  Not in the paper, which searches from the medoid: an exact
 *   kNN graph of well-separated clusters has no edges between them, so one
 *   entry reaches only its own cluster.  Limits: 1 <= ne <= 2^20. */
int ann_search_entries(const uint32_t* graph, const uint32_t* degree, int R, const void* X,
                       int64_t N, int d, int dtype, const void* Q, int64_t nq,
                       const uint32_t* entries, int ne, int Ls, int topk, uint32_t* out_id,
                       uint32_t* out_count, void* stream);
int ann_recall(const uint32_t* found, int found_stride, const uint32_t* truth, int truth_stride,
               int64_t nq, int kk, float* recall_out, void* stream);

/* ann_search_eval: ann_search followed by ann_recall against gt [nq x 10]
 * (recall@10); recall_out (device float[1]), dist_count_out [nq] uint32. */
int ann_search_eval(const uint32_t* graph, const uint32_t* degree, int R, const void* X,
                    int64_t N, int d, int dtype, const void* Q, int64_t nq, const uint32_t* gt,
                    uint32_t entry, int Ls, uint32_t* out_id, float* recall_out,
                    uint32_t* dist_count_out, void* stream);

/* ---------------------------------------------------------------------------
 * Learned candidate form (ANN_LEARNED).  Not part of the paper, which builds
 * every shard graph from exact distances (Sec. II-B, Sec. IV Workflow (2)): a
 * small MLP embeds every vector in 32 dimensions, each shard row's nearest
 * members in that space are its candidates, and the candidates are re-ranked
 * with exact FP32 distances in the original space (the kernel of
 * ANN_F16_RERANK screens the FP32 embeddings).  Its error is its recall against
 * the exact graph; the plain exact ann_shard_knn is the fallback.
 *
 * model (parameters): one device float32 array of 256 d + 256 + 32 * 256 + 32
 *   values [W1 (256 x d, row-major) | b1 | W2 (32 x 256, row-major) | b2];
 *   f(x) = W2 relu(W1 (x / s) + b1) + b2 with s = max |x| over all N vectors.
 *
 * ann_learned_train: Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected, FP32)
 *   on the triplet margin loss (1/B) sum_i max(0, |f(a)-f(p)|^2 - |f(a)-f(n)|^2
 *   + margin), `steps` steps of `batch` triplets.  First the exact kk nearest
 *   vectors (all N, by (distance, id), the row itself excluded) of each of the
 *   S rows sample[] are found with the tile query kernel.  Triplet i of step t
 *   takes draws[(t * batch + i) * 3 + {0, 1, 2}] = (u, r1, r2): anchor
 *   a = sample[u mod S] with list L, positive L[r1 mod kpos], negative
 *   L[kpos + (r2 >> 1) mod (kk - kpos)] for even r2, else row (r2 >> 1) mod N.
 *   params: in = initial parameters, out = trained (updated in place).
 *   losses: NULL or device float[steps], the mean loss of each step.
 *   recall_est: NULL or device float[1]: the fraction of each sampled row's
 *   exact 10 nearest vectors found among its 64 nearest in embedding space
 *   (all N) - an estimate of the form's recall@10 before any shard is built.
 *   Ids in sample[] at or above N are replaced by 0 and set status bit 2.
 *   Limits: d <= 4096, 2 <= kk <= 95,
 *   1 <= kpos < kk, N >= kk + 2, 1 <= S <= N, batch <= 65536.
 * ann_learned_embed: E [N x 32] float32 = f(X) for all rows.  Layer 1 runs on
 *   the tensor cores with FP16 operands (x / s and W1 rounded to FP16, FP32
 *   accumulation), layer 2 in FP32; training uses FP32 throughout.
 *   Limits: d <= 4096.
 * ann_shard_knn with precision ANN_LEARNED: model = the parameters; the
 *   screened list has rerank_k (0 = 128) entries; any d <= 4096.
 * ------------------------------------------------------------------------- */
int ann_learned_train_workspace(int64_t N, int d, int dtype, int64_t S, int kk, int batch,
                                size_t* bytes);
int ann_learned_train(const void* X, int64_t N, int d, int dtype, const uint32_t* sample,
                      int64_t S, int kk, int kpos, const uint32_t* draws, int steps, int batch,
                      float lr, float margin, float* params, float* losses, float* recall_est,
                      void* ws, size_t ws_bytes, void* stream);
/* ann_learned_grad: the loss and gradient of one batch of B triplets, computed
 *   by the same kernels as a step of ann_learned_train (before its Adam update).
 *   rows [3B] uint32: anchors rows[0, B), positives rows[B, 2B), negatives
 *   rows[2B, 3B) (row ids of X, which is scaled by s = max|x| as in training);
 *   grads: device float32 array with the layout of model (n_params values);
 *   loss: device float32[1] = the batch's mean hinge loss.  Ids >= N are replaced
 *   by 0 and flagged in the device status word. */
int ann_learned_grad_workspace(int64_t N, int d, int dtype, int B, size_t* bytes);
int ann_learned_grad(const void* X, int64_t N, int d, int dtype, const float* params,
                     const uint32_t* rows, int B, float margin, float* grads, float* loss,
                     void* ws, size_t ws_bytes, void* stream);
int ann_learned_embed_workspace(int64_t N, int d, size_t* bytes);
int ann_learned_embed(const void* X, int64_t N, int d, int dtype, const float* params, float* E,
                      void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Shard-task scheduling over GPU instances that may leave (Sec. IV "Cloud
 * Instance Task Scheduler" and "Spot instance cost analysis").  Host code; no
 * device memory involved (every pointer here is a host pointer).
 *
 * ann_sched_decide: one decision at time `now`.  Pending tasks (ids, estimated
 *   durations in seconds, data transfers included) are taken longest first (ties:
 *   smaller id).  Availability-based scheduling (always on): only the n_idle idle
 *   instances (ids) can receive a task.  With ANN_SCHED_TIME in `policy`
 *   (time-based scheduling), an instance whose end time is announced (idle_end
 *   finite; +INFINITY when unknown) receives a task only if idle_end - now covers
 *   the estimate, and a task goes to the fitting instance with the least
 *   remaining time (ties: smaller id); otherwise to the idle instance of smallest
 *   id.  A task that fits nowhere stays pending while smaller ones are tried.
 *   task_of_idle[j] = the task given to idle instance j, or -1.
 * ann_sched_simulate: discrete-event run of the scheduler.  Instance j is up in
 *   [inst_start[j], inst_end[j]) (+INFINITY: never leaves); inst_notice[j] = 1
 *   when its end is announced to the scheduler (NULL: never).  Decisions use est;
 *   a task occupies its instance for actual[t] (NULL: est).  A task still
 *   running when its instance leaves is lost and goes back to the pending list
 *   (reallocation).  At one instant: completions, then departures, then
 *   arrivals, then one decision.  Outputs per task: the instance that completed
 *   it (-1 if none), first start, completion time, attempts.  summary[6] =
 *   makespan, GPU active seconds (lost runs included), lost seconds,
 *   reallocations, unfinished tasks, cost = makespan x cpu_price + GPU active
 *   seconds x gpu_price.  Returns ANN_ERR_UNSUPPORTED if a task was left
 *   unfinished (no instance could take it).
 * ann_sched_estimate: build-time model fitted by least squares on timed samples,
 *   t = a + b s (model 0: linear in the shard size, the paper's assumption) or
 *   t = a + b s^2 (model 1: the exact kNN graph's n^2 d work); est_out[i] for
 *   task_size[i].  Needs two distinct sample sizes. */
enum ann_sched_policy { ANN_SCHED_AVAIL = 0, ANN_SCHED_TIME = 1 };
int ann_sched_decide(double now, int n_pending, const int* pending_ids, const double* pending_est,
                     int n_idle, const int* idle_ids, const double* idle_end, int policy,
                     int* task_of_idle);
int ann_sched_simulate(int n_tasks, const double* est, const double* actual, int n_inst,
                       const double* inst_start, const double* inst_end, const int* inst_notice,
                       int policy, double cpu_price, double gpu_price, int* task_inst,
                       double* task_start, double* task_end, int* task_tries, double* summary);
int ann_sched_estimate(int n_samples, const double* sample_size, const double* sample_time,
                       int model, int n_tasks, const double* task_size, double* est_out);

#ifdef __cplusplus
}
#endif
#endif /* ANN_GB300_H */
