// Prune (intermediate degree L = k to final degree R; Sec. III and Sec. VI-B2
// use L = 2R) and merge of the replicated shard graphs by edge union (Sec. II-B,
// Sec. IV Workflow (3)).
//
// Prune, one warp per shard row u: the row's list is staged in shared memory
// with an id -> position hash; the lists of u's neighbours are read with
// coalesced 128-byte warp loads; each entry that is also in L_u at a later
// position j with a shorter detour rank increments c_j (shared atomics).  The
// R entries of smallest (c_j, j) are chosen by a warp bitonic sort and written
// in list order with a ballot/popc compaction.  Integer logic only.
//
// Merge, one warp per vector g: its pruned lists (one per shard holding g) are
// gathered, sorted by (id, distance) to drop duplicate ids (the smaller
// distance survives), re-sorted by (distance, id), and the first R written.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "stages.cuh"

namespace ann {

template <int E, typename T>
__device__ __forceinline__ T shfl_xor_any(T v, int m) {
    if constexpr (sizeof(T) == 8) {
        uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
        uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)((uint64_t)v >> 32), m);
        return (T)(((uint64_t)hi << 32) | lo);
    } else {
        return (T)__shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    }
}

// Ascending bitonic sort of 32*E keys held E per lane (element index lane*E + e).
template <int E, typename T>
__device__ __forceinline__ void warp_sort(T (&v)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= E) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = lane * E + e;
                    T o = shfl_xor_any<E, T>(v[e], j / E);
                    const bool up = (i & k) == 0, lower = (i & j) == 0;
                    const T mn = v[e] < o ? v[e] : o, mx = v[e] < o ? o : v[e];
                    v[e] = (lower == up) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int pe = e ^ j;
                    if (pe > e) {
                        const int i = lane * E + e;
                        const bool up = (i & k) == 0;
                        const T a = v[e], b = v[pe];
                        if ((a > b) == up) { v[e] = b; v[pe] = a; }
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ int shard_of(const int64_t* __restrict__ offsets, int C, int64_t p) {
    int lo = 0, hi = C - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(offsets + mid) <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Shared memory of one prune warp: table keys, list, overflow list, counts,
// overflow count, table positions, overflow positions, slot occupancy bits.
__host__ __device__ constexpr size_t prune_warp_smem(int KM) {
    return (size_t)1024 * 4 + (size_t)KM * 12 + 16 + 1024 + (size_t)KM + 128;
}

// ---- prune ------------------------------------------------------------------------
// start[g] .. start[g+1] index rowlist[], the rows p (all shards) with members[p] == g.
__device__ __forceinline__ int64_t row_in_range(const int64_t* __restrict__ start,
                                                const int64_t* __restrict__ rowlist, uint32_t v,
                                                int64_t m0, int64_t m1) {
    const int64_t a1 = start[v + 1];
    for (int64_t a = start[v]; a < a1; ++a) {
        const int64_t p = rowlist[a];
        if (p >= m0 && p < m1) return p;
    }
    return -1;
}

// Position of id x in the row's list: a direct-mapped table of TS slots keyed by
// the top bits of a multiplicative hash (one probe); ids that collide with an
// occupied slot go to a short overflow list, scanned only when the slot holds a
// different id and the overflow list is not empty.
constexpr int TS = 1024, TSHIFT = 22;  // 2^(32 - TSHIFT) = TS slots

__device__ __forceinline__ uint32_t tslot(uint32_t x) { return (x * 2654435761u) >> TSHIFT; }

__device__ __forceinline__ int table_find(const uint32_t* tkey, const uint8_t* tpos,
                                          const uint32_t* ovf, const uint8_t* ovf_pos, int novf,
                                          uint32_t x) {
    const uint32_t h = tslot(x);
    const uint32_t key = tkey[h];
    if (key == x) return tpos[h];
    if (key == ANN_PAD || novf == 0) return -1;
    for (int o = 0; o < novf; ++o)
        if (ovf[o] == x) return ovf_pos[o];
    return -1;
}

template <int E>  // 32*E >= k
__global__ void k_prune(const uint32_t* __restrict__ knn_id, const float* __restrict__ knn_d,
                        const int64_t* __restrict__ offsets, const int64_t* __restrict__ start,
                        const int64_t* __restrict__ rowlist, int C, int64_t rows, int k, int R,
                        int rule, uint32_t* __restrict__ pr_id, float* __restrict__ pr_d) {
    constexpr int KM = 32 * E;
    extern __shared__ __align__(16) uint8_t sm[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwb = blockDim.x >> 5;
    uint8_t* my = sm + (size_t)wib * prune_warp_smem(KM);
    uint32_t* tkey = (uint32_t*)my;              // [TS]
    uint32_t* list = tkey + TS;                  // [KM]
    uint32_t* ovf = list + KM;                   // [KM]
    int32_t* cnt = (int32_t*)(ovf + KM);         // [KM]
    int* novf_p = cnt + KM;                      // [1] (+pad)
    uint8_t* tpos = (uint8_t*)(novf_p + 4);      // [TS]
    uint8_t* ovf_pos = tpos + TS;                // [KM]
    uint32_t* occ_bits = (uint32_t*)(ovf_pos + KM);  // [TS / 32]: slot h used = bit h
    const uint32_t lt = (1u << lane) - 1;
    const bool vec = (k & 3) == 0;
    // the table starts empty once; after each row only the slots its ids used are
    // emptied again
    for (int h = lane; h < TS; h += 32) tkey[h] = ANN_PAD;
    occ_bits[lane] = 0;
    __syncwarp();

    for (int64_t p = blockIdx.x * (int64_t)nwb + wib; p < rows; p += (int64_t)gridDim.x * nwb) {
        const int s = shard_of(offsets, C, p);
        const int64_t m0 = __ldg(offsets + s), m1 = __ldg(offsets + s + 1);
        int m = 0;
        for (int t0 = 0; t0 < KM; t0 += 32) {
            const int t = t0 + lane;
            const uint32_t v = t < k ? __ldg(knn_id + p * k + t) : ANN_PAD;
            list[t] = v;
            m += __popc(__ballot_sync(0xffffffffu, v != ANN_PAD));
        }
        uint32_t sel[E];
        if (rule == ANN_PRUNE_TRUNC) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = lane * E + e;
                sel[e] = j < m ? (uint32_t)j : 0xFFFFFFFFu;
            }
        } else {
            for (int j = lane; j < KM; j += 32) cnt[j] = 0;
            if (lane == 0) *novf_p = 0;
            __syncwarp();
            for (int j = lane; j < m; j += 32) {
                const uint32_t id = list[j];
                const uint32_t h = tslot(id);
                if (atomicCAS(&tkey[h], ANN_PAD, id) == ANN_PAD) {
                    tpos[h] = (uint8_t)j;
                    atomicOr(&occ_bits[h >> 5], 1u << (h & 31));
                } else {
                    const int o = atomicAdd(novf_p, 1);
                    ovf[o] = id;
                    ovf_pos[o] = (uint8_t)j;
                }
            }
            __syncwarp();
            const int novf = *novf_p;
            // Each lane holds 32 of the table's occupancy bits: an id whose slot is
            // empty (most of a neighbour's list) is rejected with one shuffle,
            // without a shared-memory probe.
            const uint32_t occ = occ_bits[lane];
            // Lane-parallel over the neighbours v_i: each lane reads whole lists
            // (16-byte loads), so all of a row's list reads are in flight at once.
            // The neighbours' rows are looked up first, all lanes' loads together.
            int64_t wrow[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane + 32 * e;
                wrow[e] = i < m ? row_in_range(start, rowlist, list[i], m0, m1) : -1;
            }
            // every lane runs the same loops (the occupancy shuffles need the whole
            // warp); a lane without a neighbour row reads nothing
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane + 32 * e;
                const int64_t w = wrow[e];
                const bool has = w >= 0;
                const uint32_t* Lw = knn_id + (has ? w : 0) * k;
                if (vec) {
                    for (int t0 = 0; t0 < k; t0 += 16) {
                        uint4 q4[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            q4[r] = (has && t0 + 4 * r < k)
                                        ? __ldg((const uint4*)(Lw + t0) + r)
                                        : make_uint4(ANN_PAD, ANN_PAD, ANN_PAD, ANN_PAD);
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const uint32_t xs[4] = {q4[r].x, q4[r].y, q4[r].z, q4[r].w};
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int t = t0 + 4 * r + c;
                                const uint32_t h = tslot(xs[c]);
                                const uint32_t ow = __shfl_sync(0xffffffffu, occ, (int)(h >> 5));
                                if (has && ((ow >> (h & 31)) & 1u)) {
                                    const int j = table_find(tkey, tpos, ovf, ovf_pos, novf, xs[c]);
                                    if (j > i && t < j) atomicAdd(&cnt[j], 1);
                                }
                            }
                        }
                    }
                } else {
                    for (int t = 0; t < k; ++t) {
                        const uint32_t x = has ? __ldg(Lw + t) : ANN_PAD;
                        const uint32_t h = tslot(x);
                        const uint32_t ow = __shfl_sync(0xffffffffu, occ, (int)(h >> 5));
                        if (has && ((ow >> (h & 31)) & 1u)) {
                            const int j = table_find(tkey, tpos, ovf, ovf_pos, novf, x);
                            if (j > i && t < j) atomicAdd(&cnt[j], 1);
                        }
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = lane * E + e;
                sel[e] = j < m ? (((uint32_t)cnt[j] << 16) | (uint32_t)j) : 0xFFFFFFFFu;
            }
            for (int j = lane; j < m; j += 32) tkey[tslot(list[j])] = ANN_PAD;
            occ_bits[lane] = 0;
            warp_sort<E, uint32_t>(sel);
        }
        // sel[] (element index lane*E+e) now ranks positions; keep the first min(R, m).
        // Mark kept positions in cnt[] (reused as flags), then compact in list order.
        __syncwarp();
        for (int j = lane; j < KM; j += 32) cnt[j] = 0;
        __syncwarp();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = lane * E + e;
            if (idx < R && sel[e] != 0xFFFFFFFFu) cnt[sel[e] & 0xFFFFu] = 1;
        }
        __syncwarp();
        int outc = 0;
        for (int j0 = 0; j0 < m; j0 += 32) {
            const int j = j0 + lane;
            const bool f = j < m && cnt[j];
            const uint32_t b = __ballot_sync(0xffffffffu, f);
            if (f) {
                const int pos = outc + __popc(b & lt);
                pr_id[p * R + pos] = list[j];
                pr_d[p * R + pos] = __ldg(knn_d + p * k + j);
            }
            outc += __popc(b);
        }
        for (int o = outc + lane; o < R; o += 32) {
            pr_id[p * R + o] = ANN_PAD;
            pr_d[p * R + o] = INFINITY;
        }
        __syncwarp();
    }
}

// ---- merge ------------------------------------------------------------------------
__global__ void k_count_ids(const uint32_t* __restrict__ members, int64_t rows, int64_t N,
                            int32_t* __restrict__ cnt, int* status) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < rows;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = members[p];
        if (g < N) atomicAdd(cnt + g, 1); else atomicOr(status, DEV_BAD_INPUT);
    }
}

// Exclusive scan int32 -> int64 in three passes (block sums, scan of sums, apply).
constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_CHUNK = SCAN_T * SCAN_I;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* wsum, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    int64_t r = x - v + (wid > 0 ? wsum[wid - 1] : 0);
    if (total) *total = wsum[nw - 1];
    __syncthreads();
    return r;
}

__global__ void k_scan_sums(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ bsum) {
    __shared__ int64_t ws[32];
    const int64_t b0 = blockIdx.x * (int64_t)SCAN_CHUNK;
    int64_t s = 0;
    for (int q = 0; q < SCAN_I; ++q) {
        const int64_t i = b0 + (int64_t)q * SCAN_T + threadIdx.x;
        if (i < n) s += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        bsum[blockIdx.x] = t;
    }
}

__global__ void k_scan_bsums(int64_t* __restrict__ bsum, int64_t nb) {
    __shared__ int64_t ws[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t v = b < nb ? bsum[b] : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan(v, ws, &tot);
        if (b < nb) bsum[b] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t n,
                             const int64_t* __restrict__ bsum, int64_t* __restrict__ out) {
    __shared__ int64_t ws[32];
    const int64_t b0 = blockIdx.x * (int64_t)SCAN_CHUNK;
    int64_t v[SCAN_I];
    int64_t s = 0;
    for (int q = 0; q < SCAN_I; ++q) {
        const int64_t i = b0 + (int64_t)threadIdx.x * SCAN_I + q;
        v[q] = i < n ? in[i] : 0;
        s += v[q];
    }
    int64_t ex = block_excl_scan(s, ws, nullptr) + bsum[blockIdx.x];
    for (int q = 0; q < SCAN_I; ++q) {
        const int64_t i = b0 + (int64_t)threadIdx.x * SCAN_I + q;
        if (i < n) out[i] = ex;
        ex += v[q];
        if (i == n - 1) out[n] = ex;
    }
}

__global__ void k_fill_rowlist(const uint32_t* __restrict__ members, int64_t rows, int64_t N,
                               const int64_t* __restrict__ start, int32_t* __restrict__ fill,
                               int64_t* __restrict__ rowlist) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < rows;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = members[p];
        if (g >= N) continue;
        const int slot = atomicAdd(fill + g, 1);
        rowlist[start[g] + slot] = p;
    }
}

template <int E>
__device__ __forceinline__ void merge_one(const uint32_t* __restrict__ pr_id,
                                          const float* __restrict__ pr_d,
                                          const int64_t* __restrict__ rowlist, int64_t a0,
                                          int64_t ncand, int64_t g, int R,
                                          uint32_t* __restrict__ graph, float* __restrict__ gdist,
                                          uint32_t* __restrict__ degree) {
    const int lane = threadIdx.x & 31;
    uint64_t key[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t c = (int64_t)e * 32 + lane;  // candidate c: copy c / R, slot c % R
        key[e] = ~0ull;
        if (c < ncand) {
            const int64_t p = rowlist[a0 + c / R];
            const int j = (int)(c % R);
            const uint32_t v = pr_id[p * R + j];
            if (v != ANN_PAD) key[e] = ((uint64_t)v << 32) | f2ord(pr_d[p * R + j]);
        }
    }
    warp_sort<E, uint64_t>(key);  // by (id, distance)
    // drop every entry whose predecessor in this order has the same id
    const uint64_t prev_last = __shfl_up_sync(0xffffffffu, key[E - 1], 1);
    uint64_t k2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint64_t before = e > 0 ? key[e - 1] : prev_last;
        const bool dup = (e > 0 || lane > 0) && (before >> 32) == (key[e] >> 32);
        k2[e] = (key[e] == ~0ull || dup) ? ~0ull
                                          : (((key[e] & 0xFFFFFFFFull) << 32) | (key[e] >> 32));
    }
    warp_sort<E, uint64_t>(k2);  // by (distance, id)
    int valid = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane * E + e;
        if (i < R) {
            const bool ok = k2[e] != ~0ull;
            graph[g * R + i] = ok ? (uint32_t)k2[e] : ANN_PAD;
            gdist[g * R + i] = ok ? ord2f((uint32_t)(k2[e] >> 32)) : INFINITY;
            valid += ok;
        }
    }
    for (int o = 16; o > 0; o >>= 1) valid += __shfl_xor_sync(0xffffffffu, valid, o);
    if (lane == 0) degree[g] = (uint32_t)valid;
    for (int i = 32 * E + lane; i < R; i += 32) {
        graph[g * R + i] = ANN_PAD;
        gdist[g * R + i] = INFINITY;
    }
}

// One warp per vector; the candidate count picks the sort width (warp-uniform).
__global__ void k_merge(const uint32_t* __restrict__ pr_id, const float* __restrict__ pr_d,
                        const int64_t* __restrict__ start, const int64_t* __restrict__ rowlist,
                        int64_t N, int R, uint32_t* __restrict__ graph, float* __restrict__ gdist,
                        uint32_t* __restrict__ degree, int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (g >= N) return;
    const int64_t a0 = start[g], a1 = start[g + 1];
    int64_t ncand = (a1 - a0) * R;
    if (ncand > 256) {
        if (lane == 0) atomicOr(status, DEV_OVERFLOW);
        ncand = 256;
    }
    if (ncand <= 32) merge_one<1>(pr_id, pr_d, rowlist, a0, ncand, g, R, graph, gdist, degree);
    else if (ncand <= 64) merge_one<2>(pr_id, pr_d, rowlist, a0, ncand, g, R, graph, gdist, degree);
    else if (ncand <= 128) merge_one<4>(pr_id, pr_d, rowlist, a0, ncand, g, R, graph, gdist, degree);
    else merge_one<8>(pr_id, pr_d, rowlist, a0, ncand, g, R, graph, gdist, degree);
}

// ---- host drivers ----------------------------------------------------------------
size_t rowlist_ws(int64_t N, int64_t rows, RowlistWs* out, void* base, size_t cap) {
    Carver cv(base, cap);
    RowlistWs w;
    w.cnt = cv.take<int32_t>((size_t)N + 1);
    w.start = cv.take<int64_t>((size_t)N + 1);
    w.bsum = cv.take<int64_t>((size_t)(N / SCAN_CHUNK + 2));
    w.rowlist = cv.take<int64_t>((size_t)(rows > 0 ? rows : 1));
    if (out) *out = w;
    return cv.used + 256;
}

static unsigned grid_of(int64_t n, int t) {
    const int64_t g = (n + t - 1) / t;
    return (unsigned)(g < 152 * 64 ? (g > 0 ? g : 1) : 152 * 64);
}

// Inverse of members[]: for every id g the rows holding it (any order).
int build_rowlist(const uint32_t* members, int64_t rows, int64_t N, const RowlistWs& w,
                  cudaStream_t st) {
    const int tpb = 256;
    ANN_CHECK_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * (N + 1), st));
    k_count_ids<<<grid_of(rows, tpb), tpb, 0, st>>>(members, rows, N, w.cnt, device_status_ptr());
    ANN_CHECK_LAUNCH();
    const int64_t nb = (N + SCAN_CHUNK - 1) / SCAN_CHUNK;
    k_scan_sums<<<(unsigned)nb, SCAN_T, 0, st>>>(w.cnt, N, w.bsum);
    ANN_CHECK_LAUNCH();
    k_scan_bsums<<<1, 1024, 0, st>>>(w.bsum, nb);
    ANN_CHECK_LAUNCH();
    k_scan_apply<<<(unsigned)nb, SCAN_T, 0, st>>>(w.cnt, N, w.bsum, w.start);
    ANN_CHECK_LAUNCH();
    ANN_CHECK_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * (N + 1), st));
    k_fill_rowlist<<<grid_of(rows, tpb), tpb, 0, st>>>(members, rows, N, w.start, w.cnt, w.rowlist);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

int run_prune(const uint32_t* knn_id, const float* knn_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t rows, int64_t N, int k, int R, int rule,
              uint32_t* pr_id, float* pr_d, const RowlistWs& w, cudaStream_t st) {
    if (rows == 0) return ANN_OK;
    if (rule == ANN_PRUNE_RANK) {
        int rc = build_rowlist(members, rows, N, w, st);
        if (rc) return rc;
    }
    const int warps = 4;
    const int64_t want = (rows + warps - 1) / warps;
    const unsigned grid = (unsigned)(want < 152 * 32 ? want : 152 * 32);
#define ANN_PRUNE_CASE(EE)                                                                   \
    {                                                                                        \
        constexpr int KM = 32 * EE;                                                          \
        const size_t smem = (size_t)warps * prune_warp_smem(KM);                             \
        if (smem > 48 * 1024)                                                                \
            ANN_CHECK_CUDA(cudaFuncSetAttribute(k_prune<EE>,                                 \
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                (int)smem));                                 \
        k_prune<EE><<<grid, warps * 32, smem, st>>>(knn_id, knn_d, offsets, w.start,          \
                                                    w.rowlist, C, rows, k, R, rule, pr_id,   \
                                                    pr_d);                                   \
    }
    if (k <= 32) ANN_PRUNE_CASE(1)
    else if (k <= 64) ANN_PRUNE_CASE(2)
    else if (k <= 128) ANN_PRUNE_CASE(4)
    else ANN_PRUNE_CASE(8)
#undef ANN_PRUNE_CASE
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

int run_merge(const uint32_t* pr_id, const float* pr_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t rows, int64_t N, int R, uint32_t* graph,
              float* gdist, uint32_t* degree, const RowlistWs& w, cudaStream_t st) {
    (void)offsets;
    (void)C;
    if (N == 0) return ANN_OK;
    int rc = build_rowlist(members, rows, N, w, st);
    if (rc) return rc;
    const int tpb = 256;
    const unsigned mg = (unsigned)((N * 32 + tpb - 1) / tpb);
    k_merge<<<mg, tpb, 0, st>>>(pr_id, pr_d, w.start, w.rowlist, N, R, graph, gdist, degree,
                                device_status_ptr());
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

}  // namespace ann
