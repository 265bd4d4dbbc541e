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
                       uint32_t* __restrict__ out, int32_t* __restrict__ lab_out,
                       float* __restrict__ dout) {
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
        if (dout) dout[p * r + q] = bd;
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

// FP32 vectors with d a multiple of 4 and 16-byte aligned rows: the same sums
// (elements in index order, unfused), read 4 at a time.
__global__ void k_d32_cand_f4(const float* __restrict__ X, int d, const uint32_t* rowsel,
                              int64_t p0, int64_t np, const float* __restrict__ cent,
                              const uint32_t* __restrict__ cand, int ks,
                              float* __restrict__ dist) {
    const int64_t total = np * ks;
    const int d4 = d >> 2;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = q / ks;
        const int64_t row = rowsel ? (int64_t)rowsel[p0 + p] : p0 + p;
        const float4* x = (const float4*)(X + row * d);
        const float4* c = (const float4*)(cent + (int64_t)cand[q] * d);
        float s = 0.0f;
        for (int t = 0; t < d4; ++t) {
            const float4 a = __ldg(x + t), b = __ldg(c + t);
            float df = __fsub_rn(a.x, b.x);
            s = __fadd_rn(s, __fmul_rn(df, df));
            df = __fsub_rn(a.y, b.y);
            s = __fadd_rn(s, __fmul_rn(df, df));
            df = __fsub_rn(a.z, b.z);
            s = __fadd_rn(s, __fmul_rn(df, df));
            df = __fsub_rn(a.w, b.w);
            s = __fadd_rn(s, __fmul_rn(df, df));
        }
        dist[q] = s;
    }
}

// The r candidates of smallest (d32, centroid id) per point, in that order.
__global__ void k_topr_cand(const float* __restrict__ dist, const uint32_t* __restrict__ cand,
                            int64_t np, int ks, int r, uint32_t* __restrict__ out,
                            int32_t* __restrict__ lab_out, float* __restrict__ dout) {
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
        if (dout) dout[p * r + q] = bd;
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
        if (g < N) {
            const uint32_t c = assign[g * r + (i % r)];
            if (c < (uint32_t)C) atomicAdd(&h[c], 1);  // ANN_PAD: unused slot
        }
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
        uint32_t c = e < nent ? assign[g0 * r + e] : 0xFFFFFFFFu;
        if (c >= (uint32_t)C) c = 0xFFFFFFFFu;  // past the end, or an unused slot
        const bool valid = c != 0xFFFFFFFFu;
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
static constexpr int64_t ASSIGN_CHUNK = 1 << 20;  // rows per assignment launch
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
                        int32_t* lab, cudaStream_t st, float* dout = nullptr) {
    if (C <= FULL_SCAN_C) {
        const int64_t tot = np * C;
        const unsigned g = (unsigned)((tot + 255) / 256 < 65535 * 8 ? (tot + 255) / 256 : 65535 * 8);
        k_dist_centroids<<<g, 256, 0, st>>>(X, dtype, d, rowsel, p0, np, w.centT, C, w.dist);
        ANN_CHECK_LAUNCH();
        k_topr<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(w.dist, np, C, r, out, lab, dout);
        ANN_CHECK_LAUNCH();
        return ANN_OK;
    }
    const int ks = screen_width(C, r);
    int rc = run_screen(X, dtype, rowsel, p0, np, w.cent, ANN_F32, C, d, ks, w.cand, w.sws,
                        w.sws_bytes, st);
    if (rc) return rc;
    const int64_t tot = np * ks;
    const unsigned g = (unsigned)((tot + 255) / 256 < 65535 * 8 ? (tot + 255) / 256 : 65535 * 8);
    if (dtype == ANN_F32 && d % 4 == 0 && (uintptr_t)X % 16 == 0)
        k_d32_cand_f4<<<g, 256, 0, st>>>((const float*)X, d, rowsel, p0, np, w.cent, w.cand, ks,
                                          w.dist);
    else
        k_d32_cand<<<g, 256, 0, st>>>(X, dtype, d, rowsel, p0, np, w.cent, w.cand, ks, w.dist);
    ANN_CHECK_LAUNCH();
    k_topr_cand<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(w.dist, w.cand, np, ks, r, out, lab,
                                                               dout);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

// Lloyd iterations on the sample rows (centroids left in w.cent / w.centT and
// copied to centroids_out).
static int kmeans_stage(const void* X, int d, int dtype, int C, const float* init_centroids,
                        const uint32_t* sample_idx, int64_t S, int iters, float* centroids_out,
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
    return ANN_OK;
}

// Member lists from assign [N x r] (ANN_PAD slots skipped): ids ascending per shard.
static int shard_lists(const uint32_t* assign, int64_t N, int r, int C, const PartitionWs& w,
                       uint32_t* members_out, int64_t* offsets_out, cudaStream_t st) {
    int64_t nblk = (N + SB - 1) / SB;
    k_block_hist<<<(unsigned)nblk, 256, C * sizeof(int32_t), st>>>(assign, N, r, C, nblk, w.hist);
    ANN_CHECK_LAUNCH();
    k_scan_blocks<<<C, 1024, 0, st>>>(w.hist, nblk, w.tot);
    ANN_CHECK_LAUNCH();
    k_offsets<<<1, 32, 0, st>>>(w.tot, C, offsets_out);
    ANN_CHECK_LAUNCH();
    k_scatter<<<(unsigned)nblk, 32, C * sizeof(int32_t), st>>>(assign, N, r, C, nblk, w.hist,
                                                               offsets_out, members_out);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

int run_partition(const void* X, int64_t N, int d, int dtype, int C, int r,
                  const float* init_centroids, const uint32_t* sample_idx, int64_t S, int iters,
                  float* centroids_out, uint32_t* members_out, int64_t* offsets_out,
                  const PartitionWs& w, cudaStream_t st) {
    int rc = kmeans_stage(X, d, dtype, C, init_centroids, sample_idx, S, iters, centroids_out, w,
                          st);
    if (rc) return rc;
    for (int64_t p0 = 0; p0 < N; p0 += w.chunk) {
        int64_t np = N - p0 < w.chunk ? N - p0 : w.chunk;
        rc = assign_chunk(X, dtype, d, nullptr, p0, np, C, r, w, w.assign + p0 * r, nullptr, st);
        if (rc) return rc;
    }
    return shard_lists(w.assign, N, r, C, w, members_out, offsets_out, st);
}


// ---- blockwise-adaptive assignment with selective replication ------------------
// (Sec. V-A, Sec. V-B, Algorithm 1.)  Vectors are taken once, in id order, in
// blocks; per block: originals to their nearest candidate with room, then the
// cluster statistics (squared radius, replica threshold theta), then replicas.
// Candidates of vector v: cand[v*M + j], j < M, its M centroids of smallest
// (d32, id) in that order, with d32 in cdd[v*M + j].
//
// The paper's tests d' < eps d and d' < eps tau R[c'] are taken on squared d32
// values in FP64: dd' < (eps*eps)*dd and dd' < ((eps*tau)*(eps*tau))*rad2.  For
// a float x and a double rhs, x < rhs holds exactly when x < the smallest float
// >= rhs (no float lies strictly between rhs and that float), so each double
// right-hand side is turned into one float threshold (rounded up) once, and the
// per-candidate comparisons are FP32.
__device__ __forceinline__ double sel_et2(double eps, double tau0, int64_t beta) {
    const double tau = __dadd_rn(1.0, __ddiv_rn(__dsub_rn(tau0, 1.0), (double)beta));
    const double et = __dmul_rn(eps, tau);
    return __dmul_rn(et, et);
}

// No capacity limit: each original is the vector's nearest candidate.  Writes
// slot 0 of assign and folds the block's squared radii into rad2b[b*C + c]
// (float bits; non-negative floats order like their bit patterns).
__global__ void k_sel_orig(const uint32_t* __restrict__ cand, const float* __restrict__ cdd,
                           int64_t N, int M, int omega, int64_t block, int C,
                           uint32_t* __restrict__ rad2b, uint32_t* __restrict__ assign) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool in = v < N;
    const unsigned act = __ballot_sync(0xffffffffu, in);
    if (!in) return;
    const uint32_t c = cand[v * M];
    const uint32_t bits = __float_as_uint(cdd[v * M]);
    assign[v * omega] = c;
    const uint64_t key = (uint64_t)(v / block) * (uint64_t)C + c;
    const unsigned peers = __match_any_sync(act, key);
    const uint32_t mx = __reduce_max_sync(peers, bits);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(rad2b + key, mx);
}

// Per cluster: running maximum of the squared radius over blocks, turned into
// the radius-test threshold of each block (tau of block b = 1 + (tau0-1)/b).
__global__ void k_sel_thresholds(const uint32_t* __restrict__ rad2b, int64_t nb, int C,
                                 double eps, double tau0, float* __restrict__ rthr) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    uint32_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const uint32_t x = rad2b[b * C + c];
        run = x > run ? x : run;
        const double et2 = sel_et2(eps, tau0, b + 1);
        rthr[b * C + c] = __double2float_ru(__dmul_rn(et2, (double)__uint_as_float(run)));
    }
}

// No capacity limit: replicas of every vector in parallel (no size check).
__global__ void k_sel_rep(const uint32_t* __restrict__ cand, const float* __restrict__ cdd,
                          int64_t N, int M, int omega, int64_t block, int C, int test, double e2,
                          const float* __restrict__ rthr, uint32_t* __restrict__ assign,
                          unsigned long long* __restrict__ stats) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool in = v < N;
    const unsigned act = __ballot_sync(0xffffffffu, in);
    if (!in) return;
    const uint32_t* cv = cand + v * M;
    const float* dv = cdd + v * M;
    const float* rt = rthr + (v / block) * C;
    const float dthr = test ? __double2float_ru(__dmul_rn(e2, (double)dv[0])) : 0.0f;
    int assigned = 1;
    for (int j = 1; j < M && assigned < omega; ++j) {
        const uint32_t c2 = cv[j];
        if (test) {
            const float x = dv[j];
            if (!(x < dthr && x < rt[c2])) continue;
        }
        assign[v * omega + assigned++] = c2;
    }
    for (int q = assigned; q < omega; ++q) assign[v * omega + q] = ANN_PAD;
    const unsigned nrep = __reduce_add_sync(act, (unsigned)(assigned - 1));
    if ((threadIdx.x & 31) == __ffs(act) - 1 && nrep) atomicAdd(stats, (unsigned long long)nrep);
}

// With a capacity limit the blocks' vectors depend on one another in id order,
// so one CTA walks them: all warps stage SEL_CH vectors' candidates into shared
// memory, then warp 0 takes them 32 at a time (lane = vector, in id order).  A
// group of 32 whose first choices all fit the rooms left is committed at once
// (the serial order would accept exactly those); otherwise its lanes go one by
// one.  Cluster counters live in shared memory.
constexpr int SEL_CH = 512;

__host__ __device__ constexpr size_t sel_seq_smem(int C, int M) {
    return (size_t)C * (4 * 8 + 4 + 4 + 4) + (size_t)SEL_CH * M * 8;
}

__global__ void __launch_bounds__(1024, 1)
k_sel_seq(const uint32_t* __restrict__ cand, const float* __restrict__ cdd, int64_t N, int M,
          int omega, int64_t block, int C, unsigned long long cap, int test, double e2,
          double eps, double tau0, uint32_t* __restrict__ assign, uint8_t* __restrict__ oj,
          unsigned long long* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long* tot = (unsigned long long*)sm;
    unsigned long long* org = tot + C;
    unsigned long long* rep = org + C;
    unsigned long long* theta = rep + C;
    uint32_t* rad2 = (uint32_t*)(theta + C);
    float* rthr = (float*)(rad2 + C);
    int32_t* demand = (int32_t*)(rthr + C);
    uint32_t* sK = (uint32_t*)(demand + C);
    float* sD = (float*)(sK + (size_t)SEL_CH * M);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c = tid; c < C; c += blockDim.x) {
        tot[c] = org[c] = rep[c] = theta[c] = 0;
        rad2[c] = 0;
        demand[c] = 0;
    }
    unsigned long long nrep = 0, novf = 0;
    const unsigned lt = (1u << lane) - 1;
    for (int64_t b0 = 0, beta = 1; b0 < N; b0 += block, ++beta) {
        const int64_t b1 = N - b0 < block ? N : b0 + block;
        for (int phase = 0; phase < 2; ++phase) {
            if (phase == 1) {  // statistics after the block's originals
                __syncthreads();
                const double et2 = sel_et2(eps, tau0, beta);
                for (int c = tid; c < C; c += blockDim.x) {
                    const unsigned long long proj =
                        (org[c] * (unsigned long long)N + (unsigned long long)b1 - 1) /
                        (unsigned long long)b1;
                    theta[c] = cap > proj ? cap - proj : 0;
                    rthr[c] = __double2float_ru(__dmul_rn(et2, (double)__uint_as_float(rad2[c])));
                }
            }
            for (int64_t q0 = b0; q0 < b1; q0 += SEL_CH) {
                const int n = (int)(b1 - q0 < SEL_CH ? b1 - q0 : SEL_CH);
                __syncthreads();
                for (int e = tid; e < n * M; e += blockDim.x) {
                    sK[e] = cand[q0 * M + e];
                    sD[e] = cdd[q0 * M + e];
                }
                __syncthreads();
                if (warp != 0) continue;
                for (int i0 = 0; i0 < n; i0 += 32) {
                    const int i = i0 + lane;
                    const bool in = i < n;
                    const int64_t v = q0 + i;
                    const uint32_t* kv = sK + (size_t)i * M;
                    const float* dv = sD + (size_t)i * M;
                    if (phase == 0) {
                        // ---- originals: nearest candidate with tot < cap
                        const uint32_t c0 = in ? kv[0] : 0xFFFFFFFFu;
                        const unsigned peers = __match_any_sync(0xffffffffu, c0);
                        const unsigned rank = __popc(peers & lt);
                        const bool ok = !in || tot[c0] + rank < cap;
                        const bool all = __all_sync(0xffffffffu, ok);
                        int jj = 0;
                        if (all) {
                            if (in) {
                                if (rank == 0) {
                                    tot[c0] += __popc(peers);
                                    org[c0] += __popc(peers);
                                }
                                atomicMax(rad2 + c0, __float_as_uint(dv[0]));
                            }
                        } else {
                            // Deferred acceptance within the group (lanes in id order):
                            // each lane proposes to its current candidate, a cluster
                            // keeps its proposers of smallest lane up to the room it had
                            // at the group's start, the others move on; a lane whose
                            // candidates are all full goes to its nearest one (an
                            // overflow, which takes no room from later lanes: that
                            // cluster was full for them too).  With one priority order
                            // for all clusters this is the result of taking the lanes
                            // one at a time.
                            int jp = 0;
                            bool ovf = false;
                            for (int round = 0; round <= 32 * M; ++round) {
                                const bool act = in && !ovf;
                                const uint32_t c = act ? kv[jp] : 0xFFFFFFFFu;
                                const unsigned pe = __match_any_sync(0xffffffffu, c);
                                const unsigned rk = __popc(pe & lt);
                                const bool rej = act && !(tot[c] + rk < cap);
                                if (!__any_sync(0xffffffffu, rej)) break;
                                if (rej && ++jp == M) ovf = true;
                            }
                            __syncwarp();
                            jj = ovf ? 0 : jp;
                            if (in) {
                                if (ovf) ++novf;
                                const uint32_t c = kv[jj];
                                atomicAdd(tot + c, 1ull);
                                atomicAdd(org + c, 1ull);
                                atomicMax(rad2 + c, __float_as_uint(dv[jj]));
                            }
                        }
                        if (in) {
                            assign[v * omega] = kv[jj];
                            oj[v] = (uint8_t)jj;
                        }
                        __syncwarp();
                    } else {
                        // ---- replicas (Algorithm 1)
                        const int jo = in ? oj[v] : 0;
                        const float dthr =
                            (in && test) ? __double2float_ru(__dmul_rn(e2, (double)dv[jo])) : 0.0f;
                        uint32_t elig = 0;
                        if (in)
                            for (int j = 0; j < M; ++j) {
                                if (j == jo) continue;
                                const float x = dv[j];
                                if (!test || (x < dthr && x < rthr[kv[j]])) elig |= 1u << j;
                            }
                        // first omega-1 eligible candidates, ignoring the size check
                        uint32_t prop = 0, m = elig;
                        for (int q = 1; q < omega && m; ++q) {
                            const uint32_t bit = m & (0u - m);
                            prop |= bit;
                            m ^= bit;
                        }
                        for (uint32_t t = prop; t; t &= t - 1) atomicAdd(demand + kv[__ffs(t) - 1], 1);
                        __syncwarp();
                        bool ok = true;
                        for (uint32_t t = prop; t; t &= t - 1) {
                            const uint32_t c2 = kv[__ffs(t) - 1];
                            const unsigned long long dm = (unsigned long long)demand[c2];
                            ok = ok && rep[c2] + dm <= theta[c2] && tot[c2] + dm <= cap;
                        }
                        const bool all = __all_sync(0xffffffffu, ok);
                        for (uint32_t t = prop; t; t &= t - 1) demand[kv[__ffs(t) - 1]] = 0;
                        __syncwarp();
                        uint32_t took = 0;
                        if (all) {
                            took = prop;
                            for (uint32_t t = prop; t; t &= t - 1) {
                                const uint32_t c2 = kv[__ffs(t) - 1];
                                atomicAdd(rep + c2, 1ull);
                                atomicAdd(tot + c2, 1ull);
                            }
                        } else if (omega == 2) {
                            // one replica each: the same deferred acceptance over the
                            // eligible candidates, room = min(theta - rep, cap - tot)
                            // at the group's start
                            uint32_t rem = in ? elig : 0u;
                            for (int round = 0; round <= 32 * M; ++round) {
                                const bool act = rem != 0;
                                const uint32_t c = act ? kv[__ffs(rem) - 1] : 0xFFFFFFFFu;
                                const unsigned pe = __match_any_sync(0xffffffffu, c);
                                const unsigned rk = __popc(pe & lt);
                                const bool rej =
                                    act && !(rep[c] + rk < theta[c] && tot[c] + rk < cap);
                                if (!__any_sync(0xffffffffu, rej)) break;
                                if (rej) rem &= rem - 1;
                            }
                            __syncwarp();
                            took = rem & (0u - rem);
                            if (took) {
                                const uint32_t c2 = kv[__ffs(took) - 1];
                                atomicAdd(rep + c2, 1ull);
                                atomicAdd(tot + c2, 1ull);
                            }
                        } else {
                            for (int l = 0; l < 32; ++l) {
                                if (lane == l && in) {
                                    int assigned = 1;
                                    for (uint32_t t = elig; t && assigned < omega; t &= t - 1) {
                                        const uint32_t c2 = kv[__ffs(t) - 1];
                                        if (rep[c2] < theta[c2] && tot[c2] < cap) {
                                            rep[c2] += 1;
                                            tot[c2] += 1;
                                            took |= t & (0u - t);
                                            ++assigned;
                                        }
                                    }
                                }
                                __syncwarp();
                            }
                        }
                        if (in) {
                            int q = 1;
                            for (uint32_t t = took; t; t &= t - 1) assign[v * omega + q++] = kv[__ffs(t) - 1];
                            nrep += (unsigned long long)(q - 1);
                            for (; q < omega; ++q) assign[v * omega + q] = ANN_PAD;
                        }
                        __syncwarp();
                    }
                }
            }
        }
    }
    if (warp == 0) {
        for (int o = 16; o; o >>= 1) {
            nrep += __shfl_down_sync(0xffffffffu, nrep, o);
            novf += __shfl_down_sync(0xffffffffu, novf, o);
        }
        if (lane == 0) {
            stats[0] = nrep;
            stats[1] = novf;
        }
    }
}

size_t selective_ws(int64_t N, int d, int C, int64_t S, int M, int omega, int64_t block,
                    SelectiveWs* out, void* base, size_t cap) {
    Carver cv(base, cap);
    SelectiveWs w;
    const size_t pw = partition_ws(N, d, C, M, S, nullptr, nullptr, 0);
    uint8_t* pbase = cv.take<uint8_t>(pw);
    if (out) partition_ws(N, d, C, M, S, &w.p, pbase, pw);
    const int64_t nb = N > 0 ? (N + block - 1) / block : 1;
    w.cdd = cv.take<float>((size_t)(N > 0 ? N : 1) * M);
    w.sel = cv.take<uint32_t>((size_t)(N > 0 ? N : 1) * omega);
    w.oj = cv.take<uint8_t>((size_t)(N > 0 ? N : 1));
    w.rad2b = cv.take<uint32_t>((size_t)nb * C);
    w.rthr = cv.take<float>((size_t)nb * C);
    w.stats = cv.take<unsigned long long>(2);
    w.nb = nb;
    if (out) *out = w;
    return cv.used + 256;
}

int run_partition_selective(const void* X, int64_t N, int d, int dtype, int C,
                            const float* init_centroids, const uint32_t* sample_idx, int64_t S,
                            int iters, const SelectiveArgs& a, float* centroids_out,
                            uint32_t* assign_out, uint32_t* members_out, int64_t* offsets_out,
                            int64_t* stats_out, const SelectiveWs& w, cudaStream_t st) {
    const PartitionWs& pw = w.p;
    int rc = kmeans_stage(X, d, dtype, C, init_centroids, sample_idx, S, iters, centroids_out, pw,
                          st);
    if (rc) return rc;
    const int M = a.M, omega = a.omega;
    uint32_t* cand = pw.assign;  // [N x M]
    for (int64_t p0 = 0; p0 < N; p0 += pw.chunk) {
        const int64_t np = N - p0 < pw.chunk ? N - p0 : pw.chunk;
        rc = assign_chunk(X, dtype, d, nullptr, p0, np, C, M, pw, cand + p0 * M, nullptr, st,
                          w.cdd + p0 * M);
        if (rc) return rc;
    }
    uint32_t* sel = assign_out ? assign_out : w.sel;
    const int test = isinf(a.eps) ? 0 : 1;
    const double e2 = a.eps * a.eps;
    ANN_CHECK_CUDA(cudaMemsetAsync(w.stats, 0, 2 * sizeof(unsigned long long), st));
    if (a.cap == 0) {
        ANN_CHECK_CUDA(cudaMemsetAsync(w.rad2b, 0, sizeof(uint32_t) * (size_t)w.nb * C, st));
        const unsigned g = (unsigned)((N + 255) / 256);
        k_sel_orig<<<g, 256, 0, st>>>(cand, w.cdd, N, M, omega, a.block, C, w.rad2b, sel);
        ANN_CHECK_LAUNCH();
        k_sel_thresholds<<<(C + 127) / 128, 128, 0, st>>>(w.rad2b, w.nb, C,
                                                          test ? a.eps : 0.0, a.tau0, w.rthr);
        ANN_CHECK_LAUNCH();
        k_sel_rep<<<g, 256, 0, st>>>(cand, w.cdd, N, M, omega, a.block, C, test, e2, w.rthr, sel,
                                     w.stats);
        ANN_CHECK_LAUNCH();
    } else {
        const size_t smem = sel_seq_smem(C, M);
        ANN_CHECK_CUDA(cudaFuncSetAttribute(k_sel_seq, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        k_sel_seq<<<1, 1024, smem, st>>>(cand, w.cdd, N, M, omega, a.block, C,
                                         (unsigned long long)a.cap, test, e2,
                                         test ? a.eps : 0.0, a.tau0, sel, w.oj, w.stats);
        ANN_CHECK_LAUNCH();
    }
    if (stats_out)
        ANN_CHECK_CUDA(cudaMemcpyAsync(stats_out, w.stats, 2 * sizeof(int64_t),
                                       cudaMemcpyDeviceToDevice, st));
    return shard_lists(sel, N, omega, C, pw, members_out, offsets_out, st);
}

}  // namespace ann
