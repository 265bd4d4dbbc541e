// Replicated k-means partitioning (Sec. IV Workflow (1); Sec. II-B: k-means
// shards, each vector replicated into its nearest shards).
//
//  distances         : d32 = FP32 squared distance with the terms added in index
//                      order, unfused (the oracle's definition).  Up to 32
//                      centroids every d32 is computed (thread per pair); with
//                      more, the tensor cores screen them first: a tile query keeps the
//                      min(C, r + 6) centroids of smallest tile key per vector,
//                      and d32 is computed for those only.  The result equals the
//                      full d32 scan unless more than 6 other centroids lie within
//                      the screen's rounding (about 1e-6 relative) of the r-th.
//  kmeans iterations : nearest centroid by (d32, id) for every sample row, FP64
//                      centroid sums accumulated in sample order, mean rounded to
//                      float; empty clusters keep their centroid.
//  assignment        : the r centroids of smallest (d32, id) for every vector.
//  shard lists       : block histograms, per-shard scan over blocks, and a
//                      stable scatter (warp match_any ranks) so each shard's
//                      member ids come out in increasing order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "stages.cuh"

namespace ann {

// d32 between row `row` of X and centroid c (FP32, index order, unfused).
__device__ __forceinline__ float d32_row_centroid(const void* X, int dtype, int64_t row, int d,
                                                  const float* __restrict__ centT, int C, int c) {
    float s = 0.0f;
    const int64_t base = row * d;
    for (int t = 0; t < d; ++t) {
        float df = __fsub_rn(load_elem(X, dtype, base + t), __ldg(centT + (int64_t)t * C + c));
        s = __fadd_rn(s, __fmul_rn(df, df));
    }
    return s;
}

// dist[p][c] for p in [p0, p0+np): rows are rowsel[p] (or p itself when NULL).
__global__ void k_dist_centroids(const void* X, int dtype, int d, const uint32_t* rowsel,
                                 int64_t p0, int64_t np, const float* __restrict__ centT, int C,
                                 float* __restrict__ dist) {
    int64_t total = np * C;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = q / C;
        int c = (int)(q - p * C);
        int64_t row = rowsel ? (int64_t)rowsel[p0 + p] : p0 + p;
        dist[q] = d32_row_centroid(X, dtype, row, d, centT, C, c);
    }
}

// The r entries of smallest (dist, c) per point, in that order (full scan).
__global__ void k_topr(const float* __restrict__ dist, int64_t np, int C, int r,
                       uint32_t* __restrict__ out, int32_t* __restrict__ lab_out) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const float* dp = dist + p * C;
    float prev_d = -INFINITY;
    int prev_c = -1;
    for (int q = 0; q < r; ++q) {
        float bd = INFINITY;
        int bc = -1;
        for (int c = 0; c < C; ++c) {
            float v = dp[c];
            // strictly after (prev_d, prev_c) in (d, c) order
            bool after = (v > prev_d) || (v == prev_d && c > prev_c);
            if (!after) continue;
            if (bc < 0 || v < bd) { bd = v; bc = c; }
        }
        if (bc < 0) bc = 0;  // unreachable for finite distances
        if (out) out[p * r + q] = (uint32_t)bc;
        if (lab_out && q == 0) lab_out[p] = bc;
        prev_d = bd;
        prev_c = bc;
    }
}

// d32 of the screened candidates: dist[p * ks + j] for centroid cand[p * ks + j]
// (centroids row-major [C x d]).
__global__ void k_d32_cand(const void* X, int dtype, int d, const uint32_t* rowsel, int64_t p0,
                           int64_t np, const float* __restrict__ cent,
                           const uint32_t* __restrict__ cand, int ks, float* __restrict__ dist) {
    const int64_t total = np * ks;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = q / ks;
        const int64_t row = rowsel ? (int64_t)rowsel[p0 + p] : p0 + p;
        const float* c = cent + (int64_t)cand[q] * d;
        float s = 0.0f;
        for (int t = 0; t < d; ++t) {
            const float df = __fsub_rn(load_elem(X, dtype, row * d + t), __ldg(c + t));
            s = __fadd_rn(s, __fmul_rn(df, df));
        }
        dist[q] = s;
    }
}

// The r candidates of smallest (d32, centroid id) per point, in that order.
__global__ void k_topr_cand(const float* __restrict__ dist, const uint32_t* __restrict__ cand,
                            int64_t np, int ks, int r, uint32_t* __restrict__ out,
                            int32_t* __restrict__ lab_out) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const float* dp = dist + p * ks;
    const uint32_t* cp = cand + p * ks;
    float prev_d = -INFINITY;
    int64_t prev_c = -1;
    for (int q = 0; q < r; ++q) {
        float bd = INFINITY;
        int64_t bc = -1;
        for (int j = 0; j < ks; ++j) {
            const float v = dp[j];
            const int64_t c = cp[j];
            const bool after = (v > prev_d) || (v == prev_d && c > prev_c);
            if (!after) continue;
            if (bc < 0 || v < bd || (v == bd && c < bc)) {
                bd = v;
                bc = c;
            }
        }
        if (bc < 0) bc = 0;  // unreachable: ks >= r distinct candidates
        if (out) out[p * r + q] = (uint32_t)bc;
        if (lab_out && q == 0) lab_out[p] = (int32_t)bc;
        prev_d = bd;
        prev_c = bc;
    }
}

// FP64 centroid sums in sample order (so each (c, t) sum is the plain sequential
// one).  list[off[c] .. off[c] + cnt[c]) holds the rows of the samples labelled c
// in sample order; one warp per (c, 32 consecutive dimensions) keeps a register
// accumulator per lane, visits only its own samples, loads 8 rows ahead, and only
// the FP64 adds are serial.  The C x d/32 warps are independent.
__global__ void k_kmeans_sums_lists(const void* X, int dtype, int d,
                                    const uint32_t* __restrict__ list,
                                    const int64_t* __restrict__ off,
                                    const int64_t* __restrict__ cnt, int C,
                                    double* __restrict__ sums) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int nt = (d + 31) / 32;
    if (w >= (int64_t)C * nt) return;
    const int c = (int)(w / nt);
    const int t = (int)(w % nt) * 32 + lane;
    const bool active = t < d;
    const uint32_t* lc = list + off[c];
    const int64_t n = cnt[c];
    double acc = 0.0;
    for (int64_t i0 = 0; i0 < n; i0 += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = (active && i0 + u < n) ? load_elem(X, dtype, (int64_t)__ldg(lc + i0 + u) * d + t)
                                          : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (i0 + u < n) acc = __dadd_rn(acc, (double)v[u]);
    }
    if (active) sums[(int64_t)c * d + t] = acc;
}

// Exclusive prefix of the label counts (C <= 1024; one thread).
__global__ void k_label_offsets(const int64_t* __restrict__ cnt, int C, int64_t* __restrict__ off) {
    if (threadIdx.x || blockIdx.x) return;
    int64_t a = 0;
    for (int c = 0; c < C; ++c) {
        off[c] = a;
        a += cnt[c];
    }
    off[C] = a;
}

// Rows of the samples labelled c in sample order (one block of 256 per c).
__global__ void __launch_bounds__(256)
    k_label_lists(const int32_t* __restrict__ lab, const uint32_t* __restrict__ sample,
                  int64_t S, const int64_t* __restrict__ off, uint32_t* __restrict__ list) {
    __shared__ int wcnt[8];
    __shared__ int64_t run;
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) run = 0;
    __syncthreads();
    for (int64_t s0 = 0; s0 < S; s0 += 256) {
        const int64_t s = s0 + threadIdx.x;
        const bool f = s < S && lab[s] == c;
        const uint32_t b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wcnt[wid] = __popc(b);
        __syncthreads();
        int before = 0, total = 0;
        for (int q = 0; q < 8; ++q) {
            if (q < wid) before += wcnt[q];
            total += wcnt[q];
        }
        if (f) list[off[c] + run + before + __popc(b & ((1u << lane) - 1))] = sample[s];
        __syncthreads();
        if (threadIdx.x == 0) run += total;
        __syncthreads();
    }
}

__global__ void k_count_labels(const int32_t* __restrict__ lab, int64_t S, int64_t* cnt) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long*)(cnt + lab[s]), 1ull);
}

__global__ void k_kmeans_update(const double* __restrict__ sums, const int64_t* __restrict__ cnt,
                                int C, int d, float* __restrict__ cent, float* __restrict__ centT) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)C * d) return;
    int c = (int)(q / d), t = (int)(q - (int64_t)c * d);
    float v = cent[q];
    if (cnt[c] > 0) v = (float)__ddiv_rn(sums[q], (double)cnt[c]);
    cent[q] = v;
    centT[(int64_t)t * C + c] = v;
}

__global__ void k_transpose_cent(const float* __restrict__ cent, int C, int d, float* cent_out,
                                 float* __restrict__ centT) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)C * d) return;
    int c = (int)(q / d), t = (int)(q - (int64_t)c * d);
    float v = cent[q];
    if (cent_out) cent_out[q] = v;
    centT[(int64_t)t * C + c] = v;
}

// ---- shard lists ------------------------------------------------------------
constexpr int SB = 256;  // points per scatter block

__global__ void k_block_hist(const uint32_t* __restrict__ assign, int64_t N, int r, int C,
                             int64_t nblk, int32_t* __restrict__ hist /* [C][nblk] */) {
    extern __shared__ int32_t h[];
    for (int i = threadIdx.x; i < C; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t g0 = blockIdx.x * (int64_t)SB;
    for (int i = threadIdx.x; i < SB * r; i += blockDim.x) {
        int64_t g = g0 + i / r;
        if (g < N) atomicAdd(&h[assign[g * r + (i % r)]], 1);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) hist[(int64_t)c * nblk + blockIdx.x] = h[c];
}

// One block per shard: exclusive scan of its block counts; total in tot[c].
__global__ void k_scan_blocks(int32_t* __restrict__ hist, int64_t nblk, int64_t* __restrict__ tot) {
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    int32_t* hc = hist + (int64_t)blockIdx.x * nblk;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t b0 = 0; b0 < nblk; b0 += blockDim.x) {
        int64_t b = b0 + threadIdx.x;
        int64_t v = b < nblk ? hc[b] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int64_t w = lane < nw ? warp_sum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) warp_sum[lane] = w;
        }
        __syncthreads();
        int64_t excl = carry + x - v + (wid > 0 ? warp_sum[wid - 1] : 0);
        if (b < nblk) hc[b] = (int32_t)excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

__global__ void k_offsets(const int64_t* __restrict__ tot, int C, int64_t* __restrict__ offsets) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t s = 0;
        offsets[0] = 0;
        for (int c = 0; c < C; ++c) {
            s += tot[c];
            offsets[c + 1] = s;
        }
    }
}

// One warp per block of SB points: entries (point, q) in order, ranked per
// shard with match_any so the scatter is stable (ids ascending per shard).
__global__ void k_scatter(const uint32_t* __restrict__ assign, int64_t N, int r, int C,
                          int64_t nblk, const int32_t* __restrict__ base /* [C][nblk] */,
                          const int64_t* __restrict__ offsets, uint32_t* __restrict__ members) {
    extern __shared__ int32_t run[];  // [C]
    for (int i = threadIdx.x; i < C; i += blockDim.x) run[i] = 0;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int64_t g0 = blockIdx.x * (int64_t)SB;
    const int64_t nent = (min((int64_t)SB, N - g0)) * r;
    for (int64_t e0 = 0; e0 < nent; e0 += 32) {
        int64_t e = e0 + lane;
        bool valid = e < nent;
        uint32_t c = valid ? assign[g0 * r + e] : 0xFFFFFFFFu;
        uint32_t peers = __match_any_sync(0xffffffffu, c);
        int rank = __popc(peers & ((1u << lane) - 1));
        int r0 = valid ? run[c] : 0;
        __syncwarp();
        if (valid) {
            int64_t pos = offsets[c] + base[(int64_t)c * nblk + blockIdx.x] + r0 + rank;
            members[pos] = (uint32_t)(g0 + e / r);
            if (rank == 0) run[c] = r0 + __popc(peers);
        }
        __syncwarp();
    }
}

// ---- host driver --------------------------------------------------------------
static constexpr int64_t ASSIGN_CHUNK = 131072;  // rows per assignment launch
static constexpr int FULL_SCAN_C = 32;            // up to this many centroids: no screen
static int screen_width(int C, int r) { return C < r + 6 ? C : r + 6; }

size_t partition_ws(int64_t N, int d, int C, int r, int64_t S, PartitionWs* out, void* base,
                    size_t cap) {
    Carver cv(base, cap);
    PartitionWs w;
    const int64_t nmax = N > S ? N : S;
    w.chunk = nmax < ASSIGN_CHUNK ? (nmax > 0 ? nmax : 1) : ASSIGN_CHUNK;
    w.ks = screen_width(C, r);
    const int ks1 = screen_width(C, 1);
    const size_t sw1 = screen_ws(w.chunk, C, d, w.ks), sw2 = screen_ws(w.chunk, C, d, ks1);
    w.sws_bytes = sw1 > sw2 ? sw1 : sw2;
    int64_t nblk = (N + SB - 1) / SB;
    w.cent = cv.take<float>((size_t)C * d);
    w.centT = cv.take<float>((size_t)C * d);
    const bool full = C <= FULL_SCAN_C;
    if (full) w.sws_bytes = 0;
    w.dist = cv.take<float>((size_t)w.chunk * (full ? C : w.ks));
    w.cand = cv.take<uint32_t>((size_t)w.chunk * w.ks);
    w.sws = cv.take<uint8_t>(w.sws_bytes + 1);
    w.lab = cv.take<int32_t>((size_t)(S > 0 ? S : 1));
    w.sums = cv.take<double>((size_t)C * d);
    w.cnt = cv.take<int64_t>((size_t)C);
    w.loff = cv.take<int64_t>((size_t)C + 1);
    w.llist = cv.take<uint32_t>((size_t)(S > 0 ? S : 1));
    w.assign = cv.take<uint32_t>((size_t)N * r);
    w.hist = cv.take<int32_t>((size_t)C * nblk);
    w.tot = cv.take<int64_t>((size_t)C);
    if (out) *out = w;
    return cv.used + 256;
}

// The r centroids of smallest (d32, id) for rows p0 .. p0+np-1 (through rowsel
// when given): tensor-core screen, then d32 of the candidates.
static int assign_chunk(const void* X, int dtype, int d, const uint32_t* rowsel, int64_t p0,
                        int64_t np, int C, int r, const PartitionWs& w, uint32_t* out,
                        int32_t* lab, cudaStream_t st) {
    if (C <= FULL_SCAN_C) {
        const int64_t tot = np * C;
        const unsigned g = (unsigned)((tot + 255) / 256 < 65535 * 8 ? (tot + 255) / 256 : 65535 * 8);
        k_dist_centroids<<<g, 256, 0, st>>>(X, dtype, d, rowsel, p0, np, w.centT, C, w.dist);
        ANN_CHECK_LAUNCH();
        k_topr<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(w.dist, np, C, r, out, lab);
        ANN_CHECK_LAUNCH();
        return ANN_OK;
    }
    const int ks = screen_width(C, r);
    int rc = run_screen(X, dtype, rowsel, p0, np, w.cent, ANN_F32, C, d, ks, w.cand, w.sws,
                        w.sws_bytes, st);
    if (rc) return rc;
    const int64_t tot = np * ks;
    const unsigned g = (unsigned)((tot + 255) / 256 < 65535 * 8 ? (tot + 255) / 256 : 65535 * 8);
    k_d32_cand<<<g, 256, 0, st>>>(X, dtype, d, rowsel, p0, np, w.cent, w.cand, ks, w.dist);
    ANN_CHECK_LAUNCH();
    k_topr_cand<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(w.dist, w.cand, np, ks, r, out, lab);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

int run_partition(const void* X, int64_t N, int d, int dtype, int C, int r,
                  const float* init_centroids, const uint32_t* sample_idx, int64_t S, int iters,
                  float* centroids_out, uint32_t* members_out, int64_t* offsets_out,
                  const PartitionWs& w, cudaStream_t st) {
    const int64_t cd = (int64_t)C * d;
    const int tpb = 256;
    auto nb = [](int64_t n, int t) { return (unsigned)((n + t - 1) / t); };
    k_transpose_cent<<<nb(cd, tpb), tpb, 0, st>>>(init_centroids, C, d, w.cent, w.centT);
    ANN_CHECK_LAUNCH();
    for (int it = 0; it < iters && S > 0; ++it) {
        for (int64_t p0 = 0; p0 < S; p0 += w.chunk) {
            int64_t np = S - p0 < w.chunk ? S - p0 : w.chunk;
            int rc = assign_chunk(X, dtype, d, sample_idx, p0, np, C, 1, w, nullptr,
                                  w.lab + p0, st);
            if (rc) return rc;
        }
        ANN_CHECK_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int64_t) * C, st));
        k_count_labels<<<nb(S, tpb) < 4096u ? nb(S, tpb) : 4096u, tpb, 0, st>>>(w.lab, S, w.cnt);
        ANN_CHECK_LAUNCH();
        k_label_offsets<<<1, 32, 0, st>>>(w.cnt, C, w.loff);
        ANN_CHECK_LAUNCH();
        k_label_lists<<<C, 256, 0, st>>>(w.lab, sample_idx, S, w.loff, w.llist);
        ANN_CHECK_LAUNCH();
        {
            const int64_t warps = (int64_t)C * ((d + 31) / 32);
            k_kmeans_sums_lists<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(
                X, dtype, d, w.llist, w.loff, w.cnt, C, w.sums);
        }
        ANN_CHECK_LAUNCH();
        k_kmeans_update<<<nb(cd, tpb), tpb, 0, st>>>(w.sums, w.cnt, C, d, w.cent, w.centT);
        ANN_CHECK_LAUNCH();
    }
    ANN_CHECK_CUDA(cudaMemcpyAsync(centroids_out, w.cent, sizeof(float) * cd,
                                   cudaMemcpyDeviceToDevice, st));
    for (int64_t p0 = 0; p0 < N; p0 += w.chunk) {
        int64_t np = N - p0 < w.chunk ? N - p0 : w.chunk;
        int rc = assign_chunk(X, dtype, d, nullptr, p0, np, C, r, w, w.assign + p0 * r, nullptr,
                              st);
        if (rc) return rc;
    }
    int64_t nblk = (N + SB - 1) / SB;
    k_block_hist<<<(unsigned)nblk, 256, C * sizeof(int32_t), st>>>(w.assign, N, r, C, nblk, w.hist);
    ANN_CHECK_LAUNCH();
    k_scan_blocks<<<C, 1024, 0, st>>>(w.hist, nblk, w.tot);
    ANN_CHECK_LAUNCH();
    k_offsets<<<1, 32, 0, st>>>(w.tot, C, offsets_out);
    ANN_CHECK_LAUNCH();
    k_scatter<<<(unsigned)nblk, 32, C * sizeof(int32_t), st>>>(w.assign, N, r, C, nblk, w.hist,
                                                               offsets_out, members_out);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

}  // namespace ann
