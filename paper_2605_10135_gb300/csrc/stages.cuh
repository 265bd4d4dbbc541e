// Internal interface between the C-ABI entry points (api.cu) and the stage
// drivers (partition.cu, knn.cu, graph.cu, search.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace ann {

// ---- partition ----------------------------------------------------------------
struct PartitionWs {
    float* cent;       // [C*d] working centroids
    float* centT;      // [d*C] transposed copy read by the distance kernel
    float* dist;       // [chunk*C] (full scan) or [chunk*ks] d32 of the screened candidates
    uint32_t* cand;    // [chunk*ks] screened centroid ids
    uint8_t* sws;      // screening workspace
    size_t sws_bytes;
    int ks;            // screened centroids per vector (final assignment)
    int32_t* lab;      // [S]
    double* sums;      // [C*d]
    int64_t* cnt;      // [C]
    int64_t* loff;     // [C+1] offsets of the per-label sample lists
    uint32_t* llist;   // [S] sample rows grouped by label, sample order inside a label
    uint32_t* assign;  // [N*r]
    int32_t* hist;     // [C*nblk]
    int64_t* tot;      // [C]
    int64_t chunk;
};
size_t partition_ws(int64_t N, int d, int C, int r, int64_t S, PartitionWs* out, void* base,
                    size_t cap);
int run_partition(const void* X, int64_t N, int d, int dtype, int C, int r, const float* init,
                  const uint32_t* sample_idx, int64_t S, int iters, float* cent_out,
                  uint32_t* members_out, int64_t* offsets_out, const PartitionWs& w,
                  cudaStream_t st);

// Blockwise-adaptive assignment with selective replication (Sec. V).
struct SelectiveArgs {
    double eps;    // +inf: no distance / radius test
    double tau0;   // tau of the first block
    int64_t block; // vectors per block
    int64_t cap;   // members per shard, 0 = no limit
    int omega;     // most shards per vector
    int M;         // candidate centroids per vector
};
struct SelectiveWs {
    PartitionWs p;      // k-means state; p.assign holds the [N x M] candidate lists
    float* cdd;         // [N x M] d32 of the candidates
    uint32_t* sel;      // [N x omega] assignment (when the caller passes none)
    uint8_t* oj;        // [N] candidate index of each original
    uint32_t* rad2b;    // [nb x C] squared radius per block (float bits)
    float* rthr;        // [nb x C] radius-test thresholds
    unsigned long long* stats;  // [2] replicas, overflowed originals
    int64_t nb;
};
size_t selective_ws(int64_t N, int d, int C, int64_t S, int M, int omega, int64_t block,
                    SelectiveWs* out, void* base, size_t cap);
int run_partition_selective(const void* X, int64_t N, int d, int dtype, int C,
                            const float* init_centroids, const uint32_t* sample_idx, int64_t S,
                            int iters, const SelectiveArgs& a, float* centroids_out,
                            uint32_t* assign_out, uint32_t* members_out, int64_t* offsets_out,
                            int64_t* stats_out, const SelectiveWs& w, cudaStream_t st);

// ---- kNN tiles --------------------------------------------------------------------
struct KnnProblem {
    int64_t a_row0;    // first row of the problem in the A buffer (padded index space)
    int64_t b_row0;    // first row in the B buffer
    int64_t out_row0;  // first output row
    int64_t mem_row0;  // members[] offset of column 0 (global id lookup)
    int32_t n_rows, n_cols;
};

struct KnnPlan {
    int mode;         // 0 plain, 1 split (hi/lo BF16 sections)
    int Kp;           // elements per gathered row
    int Kh;           // split: elements per section
    int nkb_a, nkb_b;
    int ksteps, hs;   // K steps (32 bytes) holding data; split: steps per section
    int elem8;        // 1: E4M3 operands (kind::f8f6f4)
    int scaled;       // 1: operands carry one global scale from max|x| (E4M3, scaled FP16)
    int kbe;          // elements per 128-byte K block
    int bn;           // tile width (N of one MMA): 256 or 128
    int a_stream;     // 1: A blocks stream through the ring (d too large to keep resident)
    uint32_t ab_fmt;  // 16-bit operands: 0 fp16, 1 bf16 (E4M3: 0)
    bool rerank;
    int kprime;
    int nst;
    size_t smem;
};
int knn_plan(int d, int dtype, int k, int precision, int rerank_k, KnnPlan* pl);
// Plans the autotuner may time (default first); returns their number, or minus
// the error code when no plan exists.
int knn_plan_variants(int d, int dtype, int k, int precision, int rerank_k, KnnPlan* out,
                      int max_out);

struct KnnWs {
    int64_t* blk_off;
    int64_t* pad_off;
    KnnProblem* probs;
    __nv_bfloat16* G;     // [rows_cap x Kp] (fp16 bits when ab_fmt == 0)
    __nv_bfloat16* aug;   // [rows_cap x 16]: |y|^2 / 2 as three BF16 values, then zeros
    __nv_bfloat16* ones;  // [128 x 16]: 1, 1, 1, then zeros
    float* norms;         // [rows_cap + 512]
    uint32_t* cand_id;  // [rows x kprime] when re-ranking
    float* cand_d;
    uint64_t* pool;     // [rows_cap x 2 x pool_half(kprime)] candidate pools of the sweeps
    int* pool_cnt;      // [rows_cap x 2]
    int64_t rows_cap;
    // cell ordering
    int64_t* src;       // [rows_cap] vector held by each gathered row (-1: padding)
    uint32_t* gid;      // [rows_cap] its global id
    int64_t* outrow;    // [rows_cap] the output row it belongs to
    int64_t prows_cap;  // pivot rows (padded per shard)
    int64_t* ppad_off;  // [C+1]
    int32_t* npiv;      // [C]
    int32_t* order;     // [C] shard of problem j (shards by decreasing size)
    KnnProblem* pprobs; // [C]
    int64_t* psrc;      // [prows_cap]
    __nv_bfloat16* GP;  // [prows_cap x Kp]
    __nv_bfloat16* paug;
    float* pnorms;
    uint32_t* cell;     // [rows] nearest pivot of each member row
    float* cell_d;
    uint32_t* perm;     // [rows] local index of the row at each cell-ordered position
    uint32_t* crank;    // [prows_cap] chain position of each pivot (cell order)
    float* amax;        // E4M3 plans: largest |x| (float bits)
    // exact tile skipping (plain operands only; NULL otherwise)
    float* gcent;       // [rows_cap / 128 x Kp] centre of every 128-row group
    float* grad;        // [rows_cap / 128] radius bound of the group (-1: empty)
    float* gmaxn;       // [rows_cap / 128] largest |y|^2 of the group
    float* bub;         // [blocks] bound on the k-th squared distance of a row block
    uint16_t* tlist;    // [blocks x 2048] tiles each row block sweeps, nearest first
    int* tcount;        // [blocks] their number (-1: every tile)
    float* rowub;       // [rows_cap] bound on each row's k'-th squared distance
    int64_t nblocks;
};
// Exact skipping of distance tiles (switch, statistics of the last launches).
void tile_prune_set(bool on);
bool tile_prune_on();
int tile_prune_stats(unsigned long long* out, int n, bool reset);
size_t knn_ws(int C, int64_t rows, const KnnPlan& pl, KnnWs* out, void* base, size_t cap);
// X [N x d] screens the candidates; the re-rank (float plans) scores them on Xr
// [N x dr] (type dtype_r), which defaults to X itself.
int run_shard_knn(const void* X, int64_t N, int d, int dtype, const uint32_t* members,
                  const int64_t* offsets, int C, int64_t rows, int k, const KnnPlan& pl,
                  const KnnWs& w, uint32_t* knn_id, float* knn_d, cudaStream_t st,
                  const void* Xr = nullptr, int dr = 0, int dtype_r = 0,
                  bool screen_only = false);

struct QueryWs {
    int64_t* blk_off;
    int64_t* pad_off;  // {0, padded nq, 0, padded N}
    int64_t* offs;     // {0, nq, 0, N}
    KnnProblem* prob;
    __nv_bfloat16* GA;
    __nv_bfloat16* GB;
    __nv_bfloat16* augA;
    __nv_bfloat16* augB;
    __nv_bfloat16* ones;
    float* na;
    float* nb;
    uint32_t* cand_id;
    float* cand_d;
    uint64_t* pool;     // [capA x 2 x pool_half(kprime)] candidate pools of the sweep
    int* pool_cnt;      // [capA x 2]
    int64_t capA, capB;
    int64_t* srcA;
    int64_t* srcB;
    float* amax;
};
size_t query_ws(int64_t N, int64_t nq, const KnnPlan& pl, QueryWs* out, void* base, size_t cap);
int run_knn_query(const void* X, int64_t N, const void* Q, int64_t nq, int d, int dtype, int k,
                  const KnnPlan& pl, const QueryWs& w, uint32_t* out_id, float* out_d,
                  cudaStream_t st);

// ---- prune / merge ---------------------------------------------------------------
// Inverse of the member lists: start[g] .. start[g+1] index rowlist[], the rows
// holding vector g.  Shared by prune (to find a neighbour's row in the same shard)
// and merge (to gather a vector's lists from all its shards).
struct RowlistWs {
    int32_t* cnt;
    int64_t* start;
    int64_t* bsum;
    int64_t* rowlist;
};
size_t rowlist_ws(int64_t N, int64_t rows, RowlistWs* out, void* base, size_t cap);
int run_prune(const uint32_t* knn_id, const float* knn_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t rows, int64_t N, int k, int R, int rule,
              uint32_t* pr_id, float* pr_d, const RowlistWs& w, cudaStream_t st);
int run_merge(const uint32_t* pr_id, const float* pr_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t rows, int64_t N, int R, uint32_t* graph,
              float* gdist, uint32_t* degree, const RowlistWs& w, cudaStream_t st);
struct MergeRevWs {
    int32_t* cnt;
    int64_t* start;
    int64_t* bsum;
    uint64_t* rkey;
};
size_t merge_rev_ws(int64_t N, int R, MergeRevWs* out, void* base, size_t cap);
int run_merge_reverse(const uint32_t* graph, const float* gdist, const uint32_t* degree, int64_t N,
                      int R, uint32_t* out_g, float* out_d, uint32_t* out_deg, const MergeRevWs& w,
                      cudaStream_t st);

// ---- query side ------------------------------------------------------------------
int search_vis_mask(int Ls, int R);
int run_search(const uint32_t* graph, const uint32_t* degree, int R, const void* X, int64_t N,
               int d, int dtype, const void* Q, int64_t nq, uint32_t entry,
               const uint32_t* entries, int ne, int Ls, int topk, uint32_t* out_id,
               uint32_t* out_count, cudaStream_t st);
int run_recall(const uint32_t* found, int fs, const uint32_t* truth, int ts, int64_t nq, int kk,
               float* recall_out, unsigned long long* hits, cudaStream_t st);

// Screening query (tile keys only): for A rows p0 .. p0+na-1 (through rowsel when
// given) of Xa, the ks rows of Xb [nb x d] of smallest tile key, as indices.
size_t screen_ws(int64_t na, int64_t nb, int d, int ks);
int run_screen(const void* Xa, int dta, const uint32_t* rowsel, int64_t p0, int64_t na,
               const void* Xb, int dtb, int64_t nb, int d, int ks, uint32_t* out_id, void* ws,
               size_t ws_bytes, cudaStream_t st);

// 2-D tensor map over a [rows x inner] matrix of 16-bit (esize 2) or 8-bit
// (esize 1) elements, box {box_inner, box_rows}.
int make_tmap(CUtensorMap* m, const void* G, int64_t rows, int inner, int box_inner, int box_rows,
              CUtensorMapSwizzle swz, int esize = 2);

// max |x| over X [n elements] and, if given, Q [nq_elems] into *amax (float bits;
// the word is zeroed first).
int launch_absmax(const void* X, int dtype, int64_t n, const void* Q, int64_t nq_elems,
                  unsigned int* amax, cudaStream_t st);

// ---- learned candidate form ---------------------------------------------------------
namespace ml {
constexpr int HID = 256;  // hidden width
constexpr int OUT = 32;   // embedding width
inline int64_t n_params(int d) { return (int64_t)HID * d + HID + (int64_t)OUT * HID + OUT; }
}  // namespace ml
struct LearnTrainWs;
size_t learned_train_ws(int64_t N, int d, int dtype, int64_t S, int kk, int batch,
                        LearnTrainWs* out, void* base, size_t cap);
int run_learned_train(const void* X, int64_t N, int d, int dtype, const uint32_t* sample,
                      int64_t S, int kk, int kpos, const uint32_t* draws, int steps, int batch,
                      float lr, float margin, float* params, float* losses, float* recall_est,
                      void* ws, size_t ws_bytes, cudaStream_t st);
size_t learned_grad_bytes(int64_t B, int d);
int run_learned_grad(const void* X, int64_t N, int d, int dtype, const float* params,
                     const uint32_t* rows, int B, float margin, float* grads, float* loss,
                     void* ws, size_t ws_bytes, cudaStream_t st);
size_t learned_embed_ws(int64_t N, int d);
int run_learned_embed(const void* X, int64_t N, int d, int dtype, const float* params,
                      float* E, void* ws, size_t ws_bytes, cudaStream_t st);
size_t medoid_ws(int64_t N, int d, double** part, float** mean, unsigned long long** best,
                 void* base, size_t cap);
int run_medoid(const void* X, int64_t N, int d, int dtype, uint32_t* entry, double* part,
               float* mean, unsigned long long* best, cudaStream_t st);
int medoid_noalloc_check(int64_t N, int d);
int run_medoid_noalloc(const void* X, int64_t N, int d, int dtype, uint32_t* entry,
                       cudaStream_t st);

}  // namespace ann
